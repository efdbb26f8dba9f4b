// Measurement utility: the FP32 FMA throughput of the device, the
// denominator of the near-field roofline.  Each thread runs kChains
// independent FMA chains (enough in flight to cover the FMA latency) for
// `iters` steps; the grid is 8 blocks of 256 threads per multiprocessor.
#include "ankh_internal.cuh"

#include <string>

namespace ankh {

constexpr int kFfmaChains = 16;
constexpr int kFfmaThreads = 256;

__global__ void __launch_bounds__(kFfmaThreads) k_ffma(int iters, float a, float b, float *__restrict__ sink)
{
    float v[kFfmaChains];
#pragma unroll
    for (int k = 0; k < kFfmaChains; ++k) v[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kFfmaChains; ++k) v[k] = fmaf(v[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kFfmaChains; ++k) s += v[k];
    if (s == 12345.678f) sink[threadIdx.x] = s;   // keeps the chains live; never true for a = 1 - 2^-20, b = 1e-7
}

}  // namespace ankh

extern "C" int ankh_measure_fp32_peak(double *tflops, double *ms, void *cuda_stream)
{
    using namespace ankh;
    if (!tflops) {
        set_error("tflops is NULL");
        return ANKH_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        set_error("device query failed");
        return ANKH_ECUDA;
    }
    const int blocks = sms * 8, iters = 4096;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_error("cudaEventCreate");
        return ANKH_ECUDA;
    }
    const float a = 1.f - 9.5367431640625e-07f, b = 1e-7f;
    for (int w = 0; w < 3; ++w) k_ffma<<<blocks, kFfmaThreads, 0, s>>>(iters, a, b, nullptr);
    cudaEventRecord(e0, s);
    const int reps = 10;
    for (int r = 0; r < reps; ++r) k_ffma<<<blocks, kFfmaThreads, 0, s>>>(iters, a, b, nullptr);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(t > 0.f)) {
        set_error(std::string("FP32 peak measurement: ") + cudaGetErrorString(e));
        return ANKH_ECUDA;
    }
    const double flop = 2.0 * kFfmaChains * (double)iters * blocks * kFfmaThreads * reps;
    *tflops = flop / (t * 1e-3) / 1e12;
    if (ms) *ms = t / reps;
    return ANKH_OK;
}
