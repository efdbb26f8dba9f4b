// Leaf binning and stable sort of the atoms by leaf (step 1 of the ANKH
// method, Sec. 3.2: the leaves of a perfect octree form a uniform n^3 grid).
//
// Bit-exact contract: the leaf of atom i is computed in correctly rounded
// FP64 without fused operations,
//     s = (x + r_B) * (1/L);  s = s - floor(s);  c = min(floor(s * n), n - 1),
// and the atoms are ordered by (leaf, original index).  The leaf counts use
// atomics (sums: any order gives the same counts); the order is a stable LSD
// radix sort of the atom indices keyed on the leaf id, whose cost per atom is
// the same however the atoms are spread over the leaves (one leaf holding
// every atom included), and whose result is unique.
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
                      int *__restrict__ count, int *__restrict__ flag)
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
    atomicAdd(&count[cell], 1);
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
                          int *__restrict__ cellid, int *__restrict__ count, int *__restrict__ flag,
                          float4 *__restrict__ loc)
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
    atomicAdd(&count[cell], 1);
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
                         int *__restrict__ cellid, int *__restrict__ count, int *__restrict__ flag,
                         float4 *__restrict__ loc)
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
    atomicAdd(&count[cell], 1);
}

// Exclusive scan of a block of 1024 values; *total = the block's sum.
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

// Sum of bsum[0 .. nb) by the first warp (for the base of block nb).
__device__ __forceinline__ int warp_prefix_total(const int *__restrict__ bsum, int nb)
{
    int s = 0;
    for (int b = (int)(threadIdx.x & 31); b < nb; b += 32) s += bsum[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}

// Multi-block exclusive scan of len values: (1) per-block totals, (2) every
// block adds the totals of the blocks before it and scans its own 1024 values;
// out[len] = the total.
__global__ void __launch_bounds__(1024) k_scan_totals(int len, const int *__restrict__ v, int *__restrict__ bsum)
{
    __shared__ int wt[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    int tot;
    block_excl_scan_1024(i < len ? v[i] : 0, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_apply(int len, const int *__restrict__ v,
                                                     const int *__restrict__ bsum, int *__restrict__ out)
{
    __shared__ int wt[32];
    __shared__ int base;
    if (threadIdx.x < 32) {
        const int s = warp_prefix_total(bsum, (int)blockIdx.x);
        if (threadIdx.x == 0) base = s;
    }
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int c = i < len ? v[i] : 0;
    int tot;
    const int ex = block_excl_scan_1024(c, wt, &tot);
    if (i < len) out[i] = base + ex;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 1023) out[len] = base + tot;
}

// Single-block forms of the two scans for short inputs (one launch instead
// of two): thread t sums the contiguous chunk [t C, (t + 1) C), C =
// ceil(len / 1024), the chunk sums are scanned across the block, then each
// thread writes its chunk's prefixes.  Same integer results.
constexpr int kScanSmall = 1024 * 64;   // longest input scanned by one block

__global__ void __launch_bounds__(1024) k_scan_small(int len, const int *__restrict__ v, int *__restrict__ out)
{
    __shared__ int wt[32];
    const int C = (len + 1023) / 1024, b = threadIdx.x * C, e = min(len, b + C);
    int loc = 0;
    for (int i = b; i < e; ++i) loc += v[i];
    int tot;
    int run = block_excl_scan_1024(loc, wt, &tot);
    for (int i = b; i < e; ++i) {
        const int c = v[i];
        out[i] = run;
        run += c;
    }
    if (threadIdx.x == 1023) out[len] = tot;
}

// Scan of the leaf counts that also lays out the near-field work items: leaf
// t with c_t atoms gives ceil(c_t / kNearItemTargets) items (t, first target),
// in leaf order, so a leaf holding many atoms is spread over many warps.
// bsum holds the per-block count totals, then the per-block item totals.
__global__ void __launch_bounds__(1024) k_leafscan_totals(int ncell, const int *__restrict__ count,
                                                          int *__restrict__ bsum)
{
    __shared__ int wt[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int c = i < ncell ? count[i] : 0;
    int tc, ti;
    block_excl_scan_1024(c, wt, &tc);
    __syncthreads();
    block_excl_scan_1024((c + kNearItemTargets - 1) / kNearItemTargets, wt, &ti);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = tc;
        bsum[gridDim.x + blockIdx.x] = ti;
    }
}

__global__ void __launch_bounds__(1024) k_leafscan_small(int ncell, const int *__restrict__ count,
                                                         int *__restrict__ start, int2 *__restrict__ items,
                                                         int *__restrict__ nitems)
{
    __shared__ int wt[32];
    const int C = (ncell + 1023) / 1024, b = threadIdx.x * C, e = min(ncell, b + C);
    int lc = 0, li = 0;
    for (int i = b; i < e; ++i) {
        const int c = count[i];
        lc += c;
        li += (c + kNearItemTargets - 1) / kNearItemTargets;
    }
    int tc, ti;
    int rc = block_excl_scan_1024(lc, wt, &tc);
    __syncthreads();
    int ri = block_excl_scan_1024(li, wt, &ti);
    for (int i = b; i < e; ++i) {
        const int c = count[i], ch = (c + kNearItemTargets - 1) / kNearItemTargets;
        start[i] = rc;
        for (int j = 0; j < ch; ++j) items[ri + j] = make_int2(i, j * kNearItemTargets);
        rc += c;
        ri += ch;
    }
    if (threadIdx.x == 1023) {
        start[ncell] = tc;
        *nitems = ti;
    }
}

__global__ void __launch_bounds__(1024) k_leafscan_apply(int ncell, const int *__restrict__ count,
                                                         const int *__restrict__ bsum, int *__restrict__ start,
                                                         int2 *__restrict__ items, int *__restrict__ nitems)
{
    __shared__ int wt[32];
    __shared__ int base[2];
    if (threadIdx.x < 64) {
        const int w = threadIdx.x >> 5;
        const int s = warp_prefix_total(bsum + w * gridDim.x, (int)blockIdx.x);
        if ((threadIdx.x & 31) == 0) base[w] = s;
    }
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int c = i < ncell ? count[i] : 0;
    const int ch = (c + kNearItemTargets - 1) / kNearItemTargets;
    int tc, ti;
    const int exc = block_excl_scan_1024(c, wt, &tc);
    __syncthreads();
    const int exi = block_excl_scan_1024(ch, wt, &ti);
    if (i < ncell) {
        start[i] = base[0] + exc;
        const int io = base[1] + exi;
        for (int j = 0; j < ch; ++j) items[io + j] = make_int2(i, j * kNearItemTargets);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 1023) {
        start[ncell] = base[0] + tc;
        *nitems = base[1] + ti;
    }
}

// Stable LSD radix sort of the atom indices by leaf id.  Pass p orders by the
// digit (id >> shift_p) & (2^bits_p - 1), lowest digit first; each pass is
// stable, so the result is ordered by (leaf, atom index).  The input is cut
// into tiles of kRsTile consecutive elements:
//   k_rs_hist     per-tile digit counts, stored digit-major: hist[d][tile];
//   scan          exclusive scan of hist: the first output slot of each
//                 (digit, tile), all earlier tiles' elements of that digit first;
//   k_rs_scatter  the rank of each element among the tile's elements of its
//                 digit, in index order: each warp walks 32 consecutive
//                 elements at a time, groups equal digits with a match
//                 (lanes in order), and keeps per-warp digit counts in shared
//                 memory; the warps' counts are then prefixed in warp order.
// Keys are read as cellid[value] (the value is the atom index), so only the
// values move.  Every element costs the same whatever the leaf occupancy.
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;                          // 32-element rounds per warp
constexpr int kRsTile = kRsWarps * 32 * kRsRounds;     // 4096 elements per tile
constexpr int kRsMaxBits = 10;                         // <= 36 KB shared memory per scatter block
constexpr int kRsWideBits = 12;                        // one wide pass: 144 KB per scatter block

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(int N, const int *__restrict__ cellid,
                                                        const int *__restrict__ vin, int shift, int bits,
                                                        int ntiles, int *__restrict__ hist)
{
    extern __shared__ int sh[];
    const int nb = 1 << bits, mask = nb - 1;
    for (int d = threadIdx.x; d < nb; d += kRsThreads) sh[d] = 0;
    __syncthreads();
    const int base = blockIdx.x * kRsTile;
    for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
        const int i = base + k;
        if (i < N) {
            const int key = cellid[vin ? vin[i] : i];
            atomicAdd(&sh[(key >> shift) & mask], 1);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += kRsThreads) hist[(int64_t)d * ntiles + blockIdx.x] = sh[d];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(int N, const int *__restrict__ cellid,
                                                           const int *__restrict__ vin, int shift, int bits,
                                                           int ntiles, const int *__restrict__ goff,
                                                           int *__restrict__ vout, int *__restrict__ inv)
{
    extern __shared__ int sh[];   // [kRsWarps][nb] per-warp digit counts, then [nb] tile offsets
    const int nb = 1 << bits, mask = nb - 1;
    int *wcnt = sh, *toff = sh + kRsWarps * nb;
    for (int k = threadIdx.x; k < kRsWarps * nb; k += kRsThreads) wcnt[k] = 0;
    for (int d = threadIdx.x; d < nb; d += kRsThreads) toff[d] = goff[(int64_t)d * ntiles + blockIdx.x];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int *wc = wcnt + warp * nb;
    const int base = blockIdx.x * kRsTile + warp * 32 * kRsRounds;
    int rk[kRsRounds], dg[kRsRounds], val[kRsRounds];
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int i = base + r * 32 + lane;
        int v = 0, d = -1;   // lanes past the end carry digit -1 and touch nothing
        if (i < N) {
            v = vin ? vin[i] : i;
            d = (cellid[v] >> shift) & mask;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int c = d >= 0 ? wc[d] : 0;
        __syncwarp();
        if (d >= 0 && (peers & below) == 0) wc[d] = c + __popc(peers);   // lowest lane of the group
        __syncwarp();
        rk[r] = c + __popc(peers & below);
        dg[r] = d;
        val[r] = v;
    }
    __syncthreads();
    // first slot of every (warp, digit): the tile's offset plus the counts of the earlier warps
    for (int d = threadIdx.x; d < nb; d += kRsThreads) {
        int run = toff[d];
        for (int w = 0; w < kRsWarps; ++w) {
            const int t = wcnt[w * nb + d];
            wcnt[w * nb + d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        if (dg[r] >= 0) {
            const int pos = wc[dg[r]] + rk[r];
            vout[pos] = val[r];
            if (inv) inv[val[r]] = pos;
        }
    }
}

RadixPlan radix_plan(int64_t N, int ncell, int wide_tiles)
{
    RadixPlan rp;
    int B = 1;
    while (B < 31 && ((int64_t)1 << B) < ncell) ++B;   // ids 0 .. ncell - 1 fit in B bits
    rp.ntiles = (int)((N + kRsTile - 1) / kRsTile);
    // one pass of up to 12 bits where the tiles fit the wide_tiles blocks
    // (one 144 KB block per SM) instead of two: four launches fewer
    rp.npass = (B > kRsMaxBits && B <= kRsWideBits && rp.ntiles <= wide_tiles) ? 1
                                                                                : (B + kRsMaxBits - 1) / kRsMaxBits;
    const int base = B / rp.npass, rem = B % rp.npass;
    int sh = 0;
    for (int p = 0; p < 3; ++p) {
        rp.bits[p] = p < rp.npass ? base + (p < rem ? 1 : 0) : 0;
        rp.shift[p] = sh;
        sh += rp.bits[p];
    }
    int maxbits = 0;
    for (int p = 0; p < rp.npass; ++p) maxbits = rp.bits[p] > maxbits ? rp.bits[p] : maxbits;
    rp.hist_len = ((int64_t)1 << maxbits) * rp.ntiles;
    rp.bsum_len = (int)((rp.hist_len + 1023) / 1024) + 1;
    return rp;
}

// The scatter's dynamic shared memory for the wide pass (the attribute is the
// kernel's, process-wide: set to the largest need).
cudaError_t radix_prepare()
{
    return cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (kRsWarps + 1) * (1 << kRsWideBits) * (int)sizeof(int));
}

cudaError_t launch_radix(int N, const int *cellid, const RadixPlan &rp, const RadixBufs &b, int *perm, int *inv,
                         cudaStream_t s)
{
    const int *vin = nullptr;
    for (int p = 0; p < rp.npass; ++p) {
        const bool last = p == rp.npass - 1;
        int *vout = last ? perm : b.vtmp[p & 1];
        const int nb = 1 << rp.bits[p];
        const int len = nb * rp.ntiles;
        const int sb = (len + 1023) / 1024;
        k_rs_hist<<<rp.ntiles, kRsThreads, nb * sizeof(int), s>>>(N, cellid, vin, rp.shift[p], rp.bits[p],
                                                                  rp.ntiles, b.hist);
        if (len <= kScanSmall) {
            k_scan_small<<<1, 1024, 0, s>>>(len, b.hist, b.goff);
        } else {
            k_scan_totals<<<sb, 1024, 0, s>>>(len, b.hist, b.bsum);
            k_scan_apply<<<sb, 1024, 0, s>>>(len, b.hist, b.bsum, b.goff);
        }
        k_rs_scatter<<<rp.ntiles, kRsThreads, (kRsWarps + 1) * nb * sizeof(int), s>>>(
            N, cellid, vin, rp.shift[p], rp.bits[p], rp.ntiles, b.goff, vout, last ? inv : nullptr);
        vin = vout;
    }
    return cudaGetLastError();
}

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


// Gather into leaf order, one thread per sorted slot s (atom perm[s]), the
// coordinates relative to the leaf centre as binning computed them: the
// sorted arrays are written contiguously, the atom data read by atom index
// (an atom-major form, reading contiguously and writing at inv[i], took 50
// instead of about 15 us on 10^6 atoms); the self term and the total charge
// as per-block FP64 partials.
__global__ void __launch_bounds__(256)
k_gather_slot(int N, const int *__restrict__ perm, const int *__restrict__ cellid, const float4 *__restrict__ loc,
              const float *__restrict__ q, const float *__restrict__ mu, const float *__restrict__ th, Geo g,
              int *__restrict__ scell, float4 *__restrict__ A0, float4 *__restrict__ A1, float4 *__restrict__ A2,
              float4 *__restrict__ A3, double *__restrict__ part_self, double *__restrict__ part_q, double D0,
              double invM, double *__restrict__ terms, unsigned *__restrict__ ticket)
{
    __shared__ double sh1[8], sh2[8];
    __shared__ bool last;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double es = 0.0, qs = 0.0;
    if (s < N) {
        const int i = perm[s];
        const float4 lv = loc[i];
        scell[s] = cellid[i];
        const float qi = q[i];
        A0[s] = make_float4(lv.x, lv.y, lv.z, qi);
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
    // the last block to finish (ticket) forms the total charge from the
    // blocks' partials in a fixed order, and the k = 0 potential D0 Q / M
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double Q = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) Q += __ldcg(&part_q[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Q += __shfl_down_sync(0xffffffffu, Q, o);
    if ((threadIdx.x & 31) == 0) sh2[threadIdx.x >> 5] = Q;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < 8; ++w) u += sh2[w];
        terms[7] = u;
        terms[6] = D0 * u * invM;
        *ticket = 0u;
    }
}

cudaError_t launch_bin(Handle &H, const float *x, cudaStream_t s)
{
    // the leaf counts and the error flag (allocated right after them)
    cudaMemsetAsync(H.d_count, 0, sizeof(int) * (H.g.ncell + 1), s);
    int N = (int)H.N;
    if (H.g.nonperiodic)
        k_bin_np<<<(N + 255) / 256, 256, 0, s>>>(N, x, H.g, H.d_ctr, H.d_cellid, H.d_count, H.d_flag, H.d_loc);
    else
        k_bin_loc<<<(N + 255) / 256, 256, 0, s>>>(N, x, H.g, H.d_ctr, H.d_cellid, H.d_count, H.d_flag, H.d_loc);
    return cudaGetLastError();
}

// Kernels of the leaf sort as launch_bin, launch_scan and
// launch_scatter_sort_gather issue them: binning, the leaf scan (one or two),
// per digit pass a histogram, its scan (one or two) and the scatter, then
// the gather.
int sort_launches(const Handle &H)
{
    int k = 1 + (H.g.ncell <= kScanSmall ? 1 : 2);
    for (int p = 0; p < H.rs.npass; ++p) {
        const int64_t len = ((int64_t)1 << H.rs.bits[p]) * H.rs.ntiles;
        k += 2 + (len <= kScanSmall ? 1 : 2);
    }
    return k + 1;
}

cudaError_t launch_scan(Handle &H, cudaStream_t s)
{
    if (H.g.ncell <= kScanSmall) {
        k_leafscan_small<<<1, 1024, 0, s>>>(H.g.ncell, H.d_count, H.d_start, H.d_items, H.d_nitems);
        return cudaGetLastError();
    }
    const int nb = (H.g.ncell + 1023) / 1024;
    k_leafscan_totals<<<nb, 1024, 0, s>>>(H.g.ncell, H.d_count, H.d_bsum);
    k_leafscan_apply<<<nb, 1024, 0, s>>>(H.g.ncell, H.d_count, H.d_bsum, H.d_start, H.d_items, H.d_nitems);
    return cudaGetLastError();
}

cudaError_t launch_scatter_sort_gather(Handle &H, const float *x, const float *q, const float *mu,
                                       const float *theta, cudaStream_t s)
{
    int N = (int)H.N;
    (void)x;
    cudaError_t e = launch_radix(N, H.d_cellid, H.rs, H.rsb, H.d_perm, nullptr, s);
    if (e != cudaSuccess) return e;
    if (H.gather_wait && (e = cudaStreamWaitEvent(s, H.gather_wait, 0)) != cudaSuccess) return e;
    k_gather_slot<<<(N + 255) / 256, 256, 0, s>>>(N, H.d_perm, H.d_cellid, H.d_loc, q, H.max_order >= 1 ? mu : nullptr,
                                              H.max_order >= 2 ? theta : nullptr, H.g, H.d_scell,
                                              H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_part + H.part_off[kPartSelf],
                                              H.d_part + H.part_off[kPartQ], H.D0, 1.0 / (double)H.g.M, H.d_terms,
                                              H.d_ticket + 1);
    return cudaGetLastError();
}

// The same ordering on caller-provided buffers (the allocation-free entry
// point), with the FP64 binning chain alone (k_bin): count and flag are
// cleared here; start receives ncell + 1 offsets; b.bsum must hold
// max(ceil(ncell / 1024), rp.bsum_len) values.
cudaError_t launch_bin_sort_raw(int N, const float *x, const Geo &g, int *cellid, int *count, int *flag,
                                const RadixPlan &rp, const RadixBufs &b, int *start, int *perm, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * g.ncell, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_bin<<<(N + 255) / 256, 256, 0, s>>>(N, x, g, cellid, count, flag);
    const int nb = (g.ncell + 1023) / 1024;
    k_scan_totals<<<nb, 1024, 0, s>>>(g.ncell, count, b.bsum);
    k_scan_apply<<<nb, 1024, 0, s>>>(g.ncell, count, b.bsum, start);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_radix(N, cellid, rp, b, perm, nullptr, s);
}

}  // namespace ankh
