// Allocation-free variant of the leaf binning and stable sort.
//
// Some callers cannot call cudaMalloc: a molecular-dynamics engine that plans
// all device memory at start-up and treats any later allocation as an error,
// code that runs while its stream is being captured into a CUDA graph (where
// cudaMalloc is not allowed), or a host application whose device allocator
// belongs to another runtime.  For them, ankh_bin_sort_noalloc runs the same
// binning/sort kernels as the handle-based path, but its scratch (per-atom
// leaf ids and ranks, per-leaf counts, the error flag) lives in the
// file-scope device array below instead of in allocated memory.  The caller
// still passes the inputs (positions) and the outputs (permutation, leaf
// offsets).
#include "ankh_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace ankh {

constexpr int64_t kNoallocMaxAtoms = ANKH_NOALLOC_MAX_ATOMS;
constexpr int64_t kNoallocMaxLeaves = ANKH_NOALLOC_MAX_LEAVES;
constexpr size_t kNoallocBytes = (size_t)(2 * kNoallocMaxAtoms + kNoallocMaxLeaves) * sizeof(int) + 256;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of the array, looked up once per device.  In host code the
// symbol name is only a host-side stand-in, so it is never passed to a kernel.
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[256];

static int noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return ANKH_ECUDA;
    }
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal out of range");
        return ANKH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return ANKH_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return ANKH_OK;
}

}  // namespace ankh

extern "C" int ankh_bin_sort_noalloc(const float *x, int64_t N, double box_edge, int n_cells, int32_t *perm,
                                     int32_t *leaf_start, void *cuda_stream)
{
    using namespace ankh;
    if (!x || !perm || !leaf_start) {
        set_error("x, perm and leaf_start are required");
        return ANKH_EINVAL;
    }
    if (N < 1 || N > kNoallocMaxAtoms) {
        set_error("ankh_bin_sort_noalloc: N must be in [1, " + std::to_string(kNoallocMaxAtoms) +
                  "] (size of the static scratch array)");
        return ANKH_EINVAL;
    }
    if (!(box_edge > 0.0) || !std::isfinite(box_edge)) {
        set_error("box edge must be finite and > 0");
        return ANKH_EINVAL;
    }
    if (n_cells < 1 || (int64_t)n_cells * n_cells * n_cells > kNoallocMaxLeaves) {
        set_error("ankh_bin_sort_noalloc: n_cells^3 must be in [1, " + std::to_string(kNoallocMaxLeaves) +
                  "] (size of the static scratch array)");
        return ANKH_EINVAL;
    }
    void *base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc != ANKH_OK) return rc;
    int *cellid = reinterpret_cast<int *>(base);
    int *rank = cellid + kNoallocMaxAtoms;
    int *count = rank + kNoallocMaxAtoms;
    int *flag = count + kNoallocMaxLeaves;
    Geo g;
    std::memset(&g, 0, sizeof(g));
    g.n = n_cells;
    g.ncell = n_cells * n_cells * n_cells;
    g.box = box_edge;
    g.rB = box_edge / 2.0;
    g.inv_box = 1.0 / box_edge;
    g.h = box_edge / n_cells;
    cudaError_t e = launch_bin_sort_raw((int)N, x, g, cellid, rank, count, flag, leaf_start, perm,
                                        (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        set_error(std::string("ankh_bin_sort_noalloc: ") + cudaGetErrorString(e));
        return ANKH_ECUDA;
    }
    return ANKH_OK;
}
