// Adjacent-leaf correction of the far field (plain FP32 form).
//
// The global circulant of k_far.cu keeps, for every pair of ADJACENT leaves
// (t, t+d), d in {-1,0,1}^3, the node pairs at |z|_inf >= h, while the paper's
// matrix A has zero blocks there (Eq. gtilde; those pairs belong to the near
// field).  They are removed by
//   E_corr = -1/2 sum_t sum_d M_t^T C_d M_{t+d},
//   (C_d)_{kl} = H((k - l - d (L_u-1)) delta) [ |k - l - d (L_u-1)|_inf >= L_u - 1 ],
// with the correction potential psi_t = sum_d C_d M_{t+d} (dE/dM_t = phi - psi_t).
// This is a dense batched contraction: for a tile of 64 target leaves,
//   Psi[ldm x 64] = sum_{d=0..26} C_d[ldm x ldm] . M_{.+d}[ldm x 64],
// one tile of 128 rows per block (blockIdx.y selects the row tile).
#include "ankh_internal.cuh"

namespace ankh {

constexpr int kCT = 64;    // target leaves per tile
constexpr int kKT = 128;   // rows (target nodes) per tile
constexpr int kLC = 32;    // contraction chunk

// leaf t + d (periodic), or -1 beyond a face of a non-periodic box
__device__ __forceinline__ int neighbour_leaf(int t, int d, int n, int nonperiodic)
{
    const int cx = t / (n * n), cy = (t / n) % n, cz = t % n;
    const int ax = cx + d / 9 - 1, ay = cy + (d / 3) % 3 - 1, az = cz + d % 3 - 1;
    if (nonperiodic && (ax < 0 || ax >= n || ay < 0 || ay >= n || az < 0 || az >= n)) return -1;
    return (((ax + n) % n) * n + (ay + n) % n) * n + (az + n) % n;
}

template <bool FORCES>
__global__ void __launch_bounds__(256)
k_corr_simt(Geo g, const float *__restrict__ M, const float *__restrict__ C, float *__restrict__ psi,
            double *__restrict__ part)
{
    // forces: all 27 offsets; energy alone: d = 0 and the 13 positive
    // offsets, the latter twice (C_(-d) = C_d^T)
    constexpr int d0 = FORCES ? 0 : 13;
    __shared__ __align__(16) float sA[kLC][kKT + 4];
    __shared__ __align__(16) float sB[kLC][kCT + 4];
    __shared__ double sh[32];
    const int ldm = g.ldm;
    const int t0 = blockIdx.x * kCT;
    const int k0 = blockIdx.y * kKT;
    const int tid = threadIdx.x;
    const int kg = tid & 31;          // rows k0 + 4 kg .. +3
    const int cg = tid >> 5;          // leaves t0 + 8 cg .. +7
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int d = d0; d < 27; ++d) {
        const float *Cd = C + (int64_t)d * ldm * ldm;
        const float wd = (d0 == 0 || d == 13) ? 1.f : 2.f;
        for (int l0 = 0; l0 < ldm; l0 += kLC) {
            __syncthreads();
            for (int e = tid; e < kKT * kLC; e += 256) {
                const int k = e / kLC, l = e % kLC;
                sA[l][k] = (k0 + k < ldm) ? wd * Cd[(int64_t)(k0 + k) * ldm + l0 + l] : 0.f;
            }
            for (int e = tid; e < kCT * kLC; e += 256) {
                const int j = e / kLC, l = e % kLC;
                const int t = t0 + j;
                float v = 0.f;
                if (t < g.ncell) {
                    const int nb = neighbour_leaf(t, d, g.n, g.nonperiodic);
                    if (nb >= 0) v = M[(int64_t)nb * ldm + l0 + l];
                }
                sB[l][j] = v;
            }
            __syncthreads();
#pragma unroll 8
            for (int l = 0; l < kLC; ++l) {
                const float4 a = *reinterpret_cast<const float4 *>(&sA[l][4 * kg]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&sB[l][8 * cg]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&sB[l][8 * cg + 4]);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
        }
    }
    double e = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int t = t0 + 8 * cg + j;
        if (t >= g.ncell) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + 4 * kg + i;
            if (k >= ldm) continue;
            if (FORCES) psi[(int64_t)t * ldm + k] = acc[i][j];
            e += (double)M[(int64_t)t * ldm + k] * (double)acc[i][j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0) sh[tid >> 5] = e;
    __syncthreads();
    if (tid == 0) {
        double u = 0.0;
        for (int w = 0; w < 8; ++w) u += sh[w];
        part[blockIdx.y * gridDim.x + blockIdx.x] = -0.5 * u;
    }
}

int corr_blocks(const Handle &H)
{
    const int gx = (H.g.ncell + kCT - 1) / kCT;
    const int gy = (H.g.ldm + kKT - 1) / kKT;
    return gx * gy;
}

cudaError_t launch_corr(Handle &H, bool forces, cudaStream_t s)
{
    dim3 grid((H.g.ncell + kCT - 1) / kCT, (H.g.ldm + kKT - 1) / kKT);
    double *part = H.d_part + H.part_off[kPartCorr];
    if (forces)
        k_corr_simt<true><<<grid, 256, 0, s>>>(H.g, H.d_M, H.d_C, H.d_psi, part);
    else
        k_corr_simt<false><<<grid, 256, 0, s>>>(H.g, H.d_M, H.d_C, H.d_psi, part);
    return cudaGetLastError();
}

}  // namespace ankh
