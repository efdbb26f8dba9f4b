// k = 0 far-field term and the FP64 energy reduction
// (Alg. 5 steps 4-5).  The self term of Eq. ewald (per atom in the gather
// kernel, k_sort.cu) is
// E_self = -(xi/sqrt(pi)) sum_i [q^2 + (2xi^2/3)|mu|^2 - (4xi^2/3) q tr(Theta)
//                                + (8xi^4/5) Theta:Theta + (4xi^4/5) tr(Theta)^2]
// (general symmetric Theta; for a traceless Theta this is the printed form).
// The k = 0 term of the far field is D_0 Q^2 / (2M) with Q = sum_i q_i exactly
// (partition of unity of the interpolation), evaluated in FP64; its
// potential D_0 Q / M is added to dE/dq by the gradient assembly (k_l2p).
#include "ankh_internal.cuh"

namespace ankh {

int self_blocks(const Handle &H) { return (int)((H.N + 255) / 256); }

// Sum of p[k] for k = b + tid, b + tid + nthr, ... < e in a fixed order.  The
// loads of eight consecutive strides are issued before they are added, so
// that their memory latencies overlap (one block reads tens of thousands of
// partials; a load-add chain per thread would wait for every load in turn).
__device__ __forceinline__ double strided_sum(const double *__restrict__ p, int b, int e, int tid, int nthr)
{
    double v = 0.0;
    int k = b + tid;
    for (; k + 7 * nthr < e; k += 8 * nthr) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = __ldg(&p[k + u * nthr]);
#pragma unroll
        for (int u = 0; u < 8; ++u) v += t[u];
    }
    for (; k < e; k += nthr) v += __ldg(&p[k]);
    return v;
}

static_assert(kReduceBlocks <= 32, "the last block adds the block sums within one warp");

// Fixed-order FP64 reduction of all energy partials, over kReduceBlocks
// blocks: block b sums the b-th contiguous share of every slot, and the last
// block to finish (ticket) adds the per-block sums in a fixed tree, so the
// result does not depend on which block finishes when.
// terms: [0] near [1] far (k != 0) [2] k = 0 [3] correction [4] self [5] total
//        [6] k = 0 potential [7] Q [8] error flag
__global__ void __launch_bounds__(256)
k_reduce(const double *__restrict__ part, const int *__restrict__ off_dev, double invM2, double D0,
         const int *__restrict__ flag, double *__restrict__ terms, double *__restrict__ scr,
         unsigned *__restrict__ ticket)
{
    __shared__ double sh[8];
    __shared__ bool last;
    for (int slot = 0; slot < kPartQ; ++slot) {   // near, far, correction, self (Q: the gather's last block)
        const int b = off_dev[slot], len = off_dev[slot + 1] - b;
        const int per = (len + (int)gridDim.x - 1) / (int)gridDim.x;
        const int lo = b + min(len, (int)blockIdx.x * per), hi = b + min(len, ((int)blockIdx.x + 1) * per);
        double v = strided_sum(part, lo, hi, (int)threadIdx.x, (int)blockDim.x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += sh[w];
            scr[blockIdx.x * kPartCount + slot] = u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    // lane l loads block l's sums (all loads in flight at once) and the warp
    // adds them in a fixed shuffle tree (kReduceBlocks <= 32)
    double res[kPartQ];
#pragma unroll
    for (int slot = 0; slot < kPartQ; ++slot)
        res[slot] = threadIdx.x < gridDim.x ? __ldcg(&scr[threadIdx.x * kPartCount + slot]) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int slot = 0; slot < kPartQ; ++slot) res[slot] += __shfl_down_sync(0xffffffffu, res[slot], o);
    if (threadIdx.x != 0) return;
    *ticket = 0u;
    const double Q = terms[7];
    const double near = res[kPartNear];
    const double glob = res[kPartGlob] * invM2;
    const double dc = D0 * Q * Q * invM2;
    const double corr = res[kPartCorr];
    const double self = res[kPartSelf];
    terms[0] = near;
    terms[1] = glob;
    terms[2] = dc;
    terms[3] = corr;
    terms[4] = self;
    terms[5] = near + glob + dc + corr + self;
    terms[8] = (double)(*flag);
    if (*flag) terms[5] = __longlong_as_double(0x7ff8000000000000LL);
}

// the self term and Q partials are produced by the gather kernel (k_sort.cu)
cudaError_t launch_self_dc(Handle &H, cudaStream_t s)
{
    (void)H;
    (void)s;
    return cudaSuccess;   // the gather's last block forms Q and the k = 0 potential
}

cudaError_t launch_reduce(Handle &H, cudaStream_t s)
{
    // ANKH-FMM: the far slot holds the root term itself and there is no k = 0 grid term
    const double invM2 = H.fmm.enabled ? 1.0 : 0.5 / (double)H.g.M;
    const double D0 = H.fmm.enabled ? 0.0 : H.D0;
    k_reduce<<<kReduceBlocks, 256, 0, s>>>(H.d_part, H.d_partoff, invM2, D0, H.d_flag, H.d_terms, H.d_rscr,
                                           H.d_ticket);
    return cudaGetLastError();
}

}  // namespace ankh
