// Allocation-free variant of the leaf binning and stable sort.
//
// Some callers cannot call cudaMalloc: a molecular-dynamics engine that plans
// all device memory at start-up and treats any later allocation as an error,
// or a host application whose device allocator belongs to another runtime and
// must not be bypassed.  For them, ankh_bin_sort_noalloc produces the
// output of the sort stage of the handle-based path (the leaf of every atom by
// the correctly rounded FP64 chain, then the stable radix sort by leaf), with
// its scratch (per-atom leaf ids, the values between radix passes, per-leaf
// counts, digit histograms and their scans, the error flag) in the file-scope
// device array below instead of in allocated memory.  The caller still passes
// the inputs (positions) and the outputs (permutation, leaf offsets).
#include "ankh_internal.cuh"

#include <cmath>
#include <cstring>
#include <string>

namespace ankh {

constexpr int64_t kNoallocMaxAtoms = ANKH_NOALLOC_MAX_ATOMS;
constexpr int64_t kNoallocMaxLeaves = ANKH_NOALLOC_MAX_LEAVES;
// Largest digit histogram of the radix sort within those limits: ids of at
// most 18 bits take one pass of <= 10 bits (1024 digits) or two of <= 9 bits,
// over at most 256 tiles of 4096 atoms.
constexpr int64_t kNoallocMaxHist = 1024 * 256;
constexpr int64_t kNoallocMaxBsum = 260;
constexpr int64_t kNoallocInts = 2 * kNoallocMaxAtoms + kNoallocMaxLeaves + 2 * kNoallocMaxHist + 1 +
                                 kNoallocMaxBsum + 4;
constexpr size_t kNoallocBytes = (size_t)kNoallocInts * sizeof(int) + 256;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of the array on the current device.  In host code the symbol
// name is only a host-side stand-in, so it is never passed to a kernel.  The
// address is looked up on every call (cheap once the module is loaded), so it
// stays right if the device's context is torn down and created again.
static int noalloc_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return ANKH_ECUDA;
    }
    *out = p;
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
    const int ncell = n_cells * n_cells * n_cells;
    const RadixPlan rp = radix_plan(N, ncell);
    if (rp.npass > 2 || rp.hist_len > kNoallocMaxHist || rp.bsum_len > kNoallocMaxBsum ||
        (ncell + 1023) / 1024 > kNoallocMaxBsum) {
        set_error("ankh_bin_sort_noalloc: sort plan exceeds the static scratch array");
        return ANKH_EINVAL;
    }
    void *base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc != ANKH_OK) return rc;
    int *cellid = reinterpret_cast<int *>(base);
    RadixBufs b;
    b.vtmp[0] = cellid + kNoallocMaxAtoms;
    b.vtmp[1] = nullptr;
    int *count = b.vtmp[0] + kNoallocMaxAtoms;
    b.hist = count + kNoallocMaxLeaves;
    b.goff = b.hist + kNoallocMaxHist;
    b.bsum = b.goff + kNoallocMaxHist + 1;
    int *flag = b.bsum + kNoallocMaxBsum;
    Geo g;
    std::memset(&g, 0, sizeof(g));
    g.n = n_cells;
    g.ncell = ncell;
    g.box = box_edge;
    g.rB = box_edge / 2.0;
    g.inv_box = 1.0 / box_edge;
    g.h = box_edge / n_cells;
    cudaError_t e = launch_bin_sort_raw((int)N, x, g, cellid, count, flag, rp, b, leaf_start, perm,
                                        (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        set_error(std::string("ankh_bin_sort_noalloc: ") + cudaGetErrorString(e));
        return ANKH_ECUDA;
    }
    return ANKH_OK;
}
