// Leaf binning and stable sort of the atoms by leaf (step 1 of the ANKH
// method, Sec. 3.2: the leaves of a perfect octree form a uniform n^3 grid).
//
// Bit-exact contract: the leaf of atom i is computed in correctly rounded
// FP64 without fused operations,
//     s = (x + r_B) * (1/L);  s = s - floor(s);  c = min(floor(s * n), n - 1),
// and the atoms are ordered by (leaf, original index).  Counting uses
// atomics (any order), then each leaf's slots are sorted by atom index, so the
// final permutation is deterministic.
#include "ankh_internal.cuh"

namespace ankh {

__device__ __forceinline__ int leaf_coord(double xv, const Geo &g, double *frac_times_n)
{
    double s = __dmul_rn(__dadd_rn(xv, g.rB), g.inv_box);
    s = __dadd_rn(s, -floor(s));
    double sn = __dmul_rn(s, (double)g.n);
    int c = (int)floor(sn);
    if (c > g.n - 1) c = g.n - 1;
    *frac_times_n = sn;
    return c;
}

__global__ void k_bin(int N, const float *__restrict__ x, Geo g, int *__restrict__ cellid,
                      int *__restrict__ rank, int *__restrict__ count, int *__restrict__ flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double xv = (double)x[3 * (int64_t)i + a];
        if (!isfinite(xv)) { bad = true; xv = 0.0; }
        double sn;
        c[a] = leaf_coord(xv, g, &sn);
    }
    if (bad) atomicOr(flag, 1);
    int cell = (c[0] * g.n + c[1]) * g.n + c[2];
    cellid[i] = cell;
    rank[i] = atomicAdd(&count[cell], 1);
}

// FP32 screen in front of the FP64 chain (GB300's FP64 rate made the chain
// the largest cost of the sort).  a = fl32(x K + n/2), K = fl32(n / L), lies
// within 4.5 n 2^-24 of S = (x + r_B) n / L for a in [-n, 2n) (one rounding
// of K, one of the fused multiply-add).  When no integer lies within
// n 2^-20 of a, floor(S) = floor(a), and the FP64 chain (error below
// 2^-50 |S|) also returns floor(S) mod n: the leaf is the same bit for bit.
// The leaf-relative coordinate is x minus the centre of the unwrapped leaf,
// the centre carried as FP32 hi + lo (within one FP32 ulp of the FP64
// chain's value).  Returns false where the FP64 chain must decide: a close
// to a leaf face, more than one box length outside the box, or not finite.
__device__ __forceinline__ bool leaf_coord_fast(float x, const Geo &g, const float2 *__restrict__ ctr, int *c,
                                                float *loc)
{
    const float nf = (float)g.n;
    const float a = fmaf(x, g.Kf, 0.5f * nf);
    if (!(a >= -nf && a < 2.f * nf)) return false;
    const float fa = floorf(a);
    const float fr = a - fa;                        // exact: |a| < 2^23
    const float err = nf * 9.5367431640625e-07f;    // n 2^-20
    if (!(fr > err && fr < 1.f - err)) return false;
    const int cs = (int)fa;                         // -n .. 2n-1
    *c = cs < 0 ? cs + g.n : (cs >= g.n ? cs - g.n : cs);
    const float2 ce = __ldg(&ctr[cs + g.n]);
    *loc = (x - ce.x) - ce.y;
    return true;
}

// Same, and the coordinates relative to the leaf centre, loc = (s n - c - 1/2) h
// (FP64, rounded once to FP32; x - centre in FP32 on the fast path), for the
// move into leaf order.
__global__ void k_bin_loc(int N, const float *__restrict__ x, Geo g, const float2 *__restrict__ ctr,
                          int *__restrict__ cellid, int *__restrict__ rank, int *__restrict__ count,
                          int *__restrict__ flag, float4 *__restrict__ loc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c[3];
    float l[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xf = x[3 * (int64_t)i + a];
        if (leaf_coord_fast(xf, g, ctr, &c[a], &l[a])) continue;
        double xv = (double)xf;
        if (!isfinite(xv)) { bad = true; xv = 0.0; }
        double sn;
        c[a] = leaf_coord(xv, g, &sn);
        l[a] = (float)__dmul_rn(__dadd_rn(sn, -((double)c[a] + 0.5)), g.h);
    }
    if (bad) atomicOr(flag, 1);
    int cell = (c[0] * g.n + c[1]) * g.n + c[2];
    cellid[i] = cell;
    loc[i] = make_float4(l[0], l[1], l[2], 0.f);
    rank[i] = atomicAdd(&count[cell], 1);
}

// Non-periodic box (no wrapping): s = (x + r_B) * (1/L) must lie in [0, 1);
// c = min(floor(s * n), n - 1); an atom outside the box sets bit 8 of the
// error flag (its leaf is clamped so that the call completes).
__device__ __forceinline__ int leaf_coord_np(double xv, const Geo &g, double *frac_times_n, bool *outside)
{
    const double s = __dmul_rn(__dadd_rn(xv, g.rB), g.inv_box);
    *outside = !(s >= 0.0 && s < 1.0);
    const double sn = __dmul_rn(s, (double)g.n);
    int c = (int)floor(sn);
    c = c < 0 ? 0 : (c > g.n - 1 ? g.n - 1 : c);
    *frac_times_n = sn;
    return c;
}

__global__ void k_bin_np(int N, const float *__restrict__ x, Geo g, const float2 *__restrict__ ctr,
                         int *__restrict__ cellid, int *__restrict__ rank, int *__restrict__ count,
                         int *__restrict__ flag, float4 *__restrict__ loc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c[3];
    float l[3];
    bool bad = false, out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xf = x[3 * (int64_t)i + a];
        // the FP32 screen of the periodic binning; inside the box (leaf in
        // [0, n), away from every face) the clamped chain gives the same leaf
        int cf;
        float lf;
        const float af = fmaf(xf, g.Kf, 0.5f * (float)g.n);   // the screen's a
        if (af > 0.f && af < (float)g.n && leaf_coord_fast(xf, g, ctr, &cf, &lf)) {
            c[a] = cf;
            l[a] = lf;
            continue;
        }
        double xv = (double)xf;
        if (!isfinite(xv)) { bad = true; xv = 0.0; }
        double sn;
        bool o;
        c[a] = leaf_coord_np(xv, g, &sn, &o);
        out |= o;
        l[a] = (float)__dmul_rn(__dadd_rn(sn, -((double)c[a] + 0.5)), g.h);
    }
    if (bad) atomicOr(flag, 1);
    if (out) atomicOr(flag, 8);
    int cell = (c[0] * g.n + c[1]) * g.n + c[2];
    cellid[i] = cell;
    loc[i] = make_float4(l[0], l[1], l[2], 0.f);
    rank[i] = atomicAdd(&count[cell], 1);
}

// Exclusive scan of the per-leaf counts (single block, 1024 threads).
__global__ void k_scan(int ncell, const int *__restrict__ count, int *__restrict__ start)
{
    __shared__ int warp_tot[32];
    const int nt = blockDim.x;
    const int tid = threadIdx.x;
    const int chunk = (ncell + nt - 1) / nt;
    const int b = min(tid * chunk, ncell), e = min(b + chunk, ncell);
    int sum = 0;
    for (int k = b; k < e; ++k) sum += count[k];
    // inclusive warp scan
    int v = sum;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (nt >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    int excl = v - sum + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (int k = b; k < e; ++k) {
        start[k] = excl;
        excl += count[k];
    }
    if (tid == nt - 1) start[ncell] = excl;
}

// Multi-block exclusive scan: (1) per-block totals, (2) every block adds the
// totals of the blocks before it and scans its own 1024 counts.
__device__ __forceinline__ int block_excl_scan_1024(int v, int *warp_tot, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    *total = warp_tot[31];
    return x - v + (wid > 0 ? warp_tot[wid - 1] : 0);
}

__global__ void __launch_bounds__(1024) k_scan_totals(int ncell, const int *__restrict__ count, int *__restrict__ bsum)
{
    __shared__ int wt[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    int tot;
    block_excl_scan_1024(i < ncell ? count[i] : 0, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_apply(int ncell, const int *__restrict__ count,
                                                     const int *__restrict__ bsum, int *__restrict__ start)
{
    __shared__ int wt[32];
    __shared__ int base;
    if (threadIdx.x < 32) {
        int s = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += 32) s += bsum[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) base = s;
    }
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int c = i < ncell ? count[i] : 0;
    int tot;
    const int ex = block_excl_scan_1024(c, wt, &tot);
    __syncthreads();
    if (i < ncell) start[i] = base + ex;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 1023) start[ncell] = base + tot;
}

__global__ void k_scatter(int N, const int *__restrict__ cellid, const int *__restrict__ rank,
                          const int *__restrict__ start, int *__restrict__ perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    perm[start[cellid[i]] + rank[i]] = i;
}

// One thread per leaf: insertion sort of its slots by original atom index.
__global__ void k_leafsort(int ncell, const int *__restrict__ start, int *__restrict__ perm)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = start[c], e = start[c + 1];
    for (int k = b + 1; k < e; ++k) {
        int v = perm[k];
        int j = k - 1;
        while (j >= b && perm[j] > v) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = v;
    }
}

// Same, and the inverse permutation inv[perm[k]] = k (slot of each atom).
__global__ void k_leafsort_inv(int ncell, const int *__restrict__ start, int *__restrict__ perm,
                               int *__restrict__ inv)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = start[c], e = start[c + 1];
    for (int k = b + 1; k < e; ++k) {
        int v = perm[k];
        int j = k - 1;
        while (j >= b && perm[j] > v) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = v;
    }
    for (int k = b; k < e; ++k) inv[perm[k]] = k;
}

// Move the atoms into leaf order, one thread per atom in the caller's order
// (coalesced reads, one scattered write per sorted array); coordinates
// relative to the leaf centre (computed in FP64, rounded once to FP32).
// Self term of Eq. ewald per atom (general symmetric Theta), FP32:
//   -(xi/sqrt(pi)) [q^2 + (2xi^2/3)|mu|^2 - (4xi^2/3) q tr + (8xi^4/5) Theta:Theta + (4xi^4/5) tr^2]
__device__ __forceinline__ float self_energy_atom(float q, float mx, float my, float mz, const float *t, float xi)
{
    const float c = xi * 0.56418958354775628f, a2 = xi * xi, a4 = a2 * a2;
    const float tr = t[0] + t[3] + t[5];
    const float TT = t[0] * t[0] + t[3] * t[3] + t[5] * t[5] + 2.f * (t[1] * t[1] + t[2] * t[2] + t[4] * t[4]);
    return -c * (q * q + (2.f * a2 / 3.f) * (mx * mx + my * my + mz * mz) - (4.f * a2 / 3.f) * q * tr
                 + (8.f * a4 / 5.f) * TT + (4.f * a4 / 5.f) * tr * tr);
}

__global__ void __launch_bounds__(256)
k_gather(int N, const int *__restrict__ inv, const int *__restrict__ cellid, const float4 *__restrict__ loc,
         const float *__restrict__ q, const float *__restrict__ mu,
         const float *__restrict__ th, Geo g, int *__restrict__ scell,
         float4 *__restrict__ A0, float4 *__restrict__ A1, float4 *__restrict__ A2,
         float4 *__restrict__ A3, double *__restrict__ part_self, double *__restrict__ part_q)
{
    __shared__ double sh1[8], sh2[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double es = 0.0, qs = 0.0;
    if (i < N) {
    const int s = inv[i];
    const float4 lv = loc[i];
    const float l[3] = {lv.x, lv.y, lv.z};
    scell[s] = cellid[i];
    const float qi = q[i];
    A0[s] = make_float4(l[0], l[1], l[2], qi);
    float m3[3] = {0.f, 0.f, 0.f}, t6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (mu) {
        m3[0] = mu[3 * (int64_t)i]; m3[1] = mu[3 * (int64_t)i + 1]; m3[2] = mu[3 * (int64_t)i + 2];
    }
    if (th) {
        const float *t = th + 6 * (int64_t)i;
#pragma unroll
        for (int k = 0; k < 6; ++k) t6[k] = t[k];
    }
    A1[s] = make_float4(m3[0], m3[1], m3[2], 0.f);
    A2[s] = make_float4(t6[0], t6[1], t6[2], t6[3]);
    A3[s] = make_float4(t6[4], t6[5], 0.f, 0.f);
    es = (double)self_energy_atom(qi, m3[0], m3[1], m3[2], t6, g.xi);
    qs = (double)qi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        es += __shfl_down_sync(0xffffffffu, es, o);
        qs += __shfl_down_sync(0xffffffffu, qs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh1[threadIdx.x >> 5] = es;
        sh2[threadIdx.x >> 5] = qs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0, v = 0.0;
        for (int w = 0; w < 8; ++w) {
            u += sh1[w];
            v += sh2[w];
        }
        part_self[blockIdx.x] = u;
        part_q[blockIdx.x] = v;
    }
}

cudaError_t launch_bin(Handle &H, const float *x, cudaStream_t s)
{
    cudaMemsetAsync(H.d_count, 0, sizeof(int) * H.g.ncell, s);
    cudaMemsetAsync(H.d_flag, 0, sizeof(int), s);
    int N = (int)H.N;
    if (H.g.nonperiodic)
        k_bin_np<<<(N + 255) / 256, 256, 0, s>>>(N, x, H.g, H.d_ctr, H.d_cellid, H.d_rank, H.d_count,
                                                  H.d_flag, H.d_loc);
    else
        k_bin_loc<<<(N + 255) / 256, 256, 0, s>>>(N, x, H.g, H.d_ctr, H.d_cellid, H.d_rank, H.d_count,
                                                   H.d_flag, H.d_loc);
    return cudaGetLastError();
}

cudaError_t launch_scan(Handle &H, cudaStream_t s)
{
    const int nb = (H.g.ncell + 1023) / 1024;
    k_scan_totals<<<nb, 1024, 0, s>>>(H.g.ncell, H.d_count, H.d_bsum);
    k_scan_apply<<<nb, 1024, 0, s>>>(H.g.ncell, H.d_count, H.d_bsum, H.d_start);
    return cudaGetLastError();
}

cudaError_t launch_scatter_sort_gather(Handle &H, const float *x, const float *q, const float *mu,
                                       const float *theta, cudaStream_t s)
{
    int N = (int)H.N;
    k_scatter<<<(N + 255) / 256, 256, 0, s>>>(N, H.d_cellid, H.d_rank, H.d_start, H.d_perm);
    k_leafsort_inv<<<(H.g.ncell + 127) / 128, 128, 0, s>>>(H.g.ncell, H.d_start, H.d_perm, H.d_inv);
    (void)x;
    k_gather<<<(N + 255) / 256, 256, 0, s>>>(N, H.d_inv, H.d_cellid, H.d_loc, q, H.max_order >= 1 ? mu : nullptr,
                                              H.max_order >= 2 ? theta : nullptr, H.g, H.d_scell,
                                              H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_part + H.part_off[kPartSelf],
                                              H.d_part + H.part_off[kPartQ]);
    return cudaGetLastError();
}

// Same kernels on caller-provided buffers (used by the allocation-free entry
// point): count and flag are cleared here; start receives ncell + 1 offsets.
cudaError_t launch_bin_sort_raw(int N, const float *x, const Geo &g, int *cellid, int *rank, int *count,
                                int *flag, int *start, int *perm, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * g.ncell, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_bin<<<(N + 255) / 256, 256, 0, s>>>(N, x, g, cellid, rank, count, flag);
    k_scan<<<1, 1024, 0, s>>>(g.ncell, count, start);
    k_scatter<<<(N + 255) / 256, 256, 0, s>>>(N, cellid, rank, start, perm);
    k_leafsort<<<(g.ncell + 127) / 128, 128, 0, s>>>(g.ncell, start, perm);
    return cudaGetLastError();
}

}  // namespace ankh
