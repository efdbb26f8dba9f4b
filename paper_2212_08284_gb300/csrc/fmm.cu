// ANKH-FMM energy (Sec. 3, Alg. 3) on one GPU.
//
// Tree: a perfect octree of depth E over the box (n = 2^E leaves per axis);
// every cell of every level carries a tensor grid of L first-kind Chebyshev
// nodes r_k = cos((2k+1) pi / 2L) per axis (Sec. 3.5).
//
// Step 1 (multipole expansions).  The leaf modified charges Q_s are those of
// Alg. 2 at the Chebyshev nodes (the P2M kernel of k_interp.cu with
// W_p = (2/h)^p H D^p); M2M up the tree (Eq. M2M) with the separable
//   V_b[k][l] = S_k((2b - 1 + r_l) / 2),
// the parent's 1-D Lagrange basis at the nodes of its lower (b = 0) or upper
// (b = 1) child, applied axis by axis (k_m2m).
//
// Step 2 (mutual M2L, Sec. 3.6).  At every level e >= 1 the interaction list
// of a cell t holds the cells t + d (of the box or of a direct image) whose
// parent is adjacent to t's parent and which are not adjacent to t:
// d_a in [-2 - p_a, 3 - p_a], max_a |d_a| >= 2, p = t mod 2.  The relation is
// symmetric and C[t, t+d] = C[t+d, t]^T, so every pair is taken once, for the
// lexicographically positive d, with factor 1 in place of 1/2:
//   F_real = sum_e sum_t sum_{d in Lambda(p_t), d > 0} M_t^T C_e(d) M_{t+d},
//   C_e(d)[k][l] = H(h_e (o_k - o_l - d)),   o = r / 2 (cell units),
// with H = erfc(xi r) / r.  A cell of an image carries the expansion of its
// copy in the box (periodic wrap of t + d).
//   With the cells of a level stored parity-major (class p' = cell mod 2,
// parent coordinates X = cell div 2), the source t + d of a target of class p
// lies in class p' = (p + d) mod 2 at parent offset D = (p + d - p') / 2 in
// {-1, 0, 1}^3.  Each class is stored as X planes of m + 2 z-row blocks (a
// one-cell y halo) of S + 2 rows (a one-cell z halo), so the sources of one
// offset for a tile of R z-rows of one plane are one 3-D box of R blocks of S
// rows (one TMA copy for the levels with m >= 8).  The
// contraction then runs on the tensor cores like the adjacent-leaf correction
// (k_corr_tc.cu): one persistent launch over work items (level, class, tile of
// R z-rows of S cells, 128-row slice of the target nodes) of all levels; the
// stages of an item run over its class's offsets and K chunks with
// A = 2^eC C_e(d) and B = 2^eM rows of M, both split into fp16 hi + lo (three
// products, FP32 accumulation in tensor memory drained per stage with
// round-to-nearest additions), and the epilogue forms M_t . psi_t per item.
//
// Step 3 (near field) and step 5 (self term) are those of ANKH-FFT.
//
// Step 4 (periodicity, Sec. 3.3).  The images beyond the direct ones act on
// the root expansion M_B through F_per = 1/2 M_B^T K M_B,
//   K[k][l] = sum_{|I|_inf >= 2} H(x_k - x_l + L I),
// computed in FP64 at creation as the full lattice sum (a second Ewald split
// with eta = 12 / L: real images of erfc(eta r)/r, the band-limited reciprocal
// difference, separable over the axes, and the constant) minus the 27 nearest
// terms.  The constant pi / (V xi^2) multiplies Q^2 only (partition of unity)
// and cancels the tin-foil neutralising term: both are dropped.  The paper
// diagonalises this operator by a circulant embedding over an equispaced root
// grid; here the L^3 x L^3 matrix is applied directly (one block, FP64).
// With ANKH_INCLUDE_REC the smooth reciprocal part of the xi split is added to
// K (it is smooth over the box and is taken through the root expansion).
#include "tcgen05.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace ankh {

namespace {

constexpr int kBlk = 343;       // offsets d in [-3, 3]^3
constexpr int kBoxRows = 16;    // rows of one B copy

__host__ __device__ inline int blk_of(int dx, int dy, int dz) { return ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3); }

struct M2MTab {
    float v[2][8][8];
};

struct B3Maps {
    CUtensorMap hi[4], lo[4];   // levels e = 4 .. 7 (m >= 8)
};

// ---------------------------------------------------------------------------
// Step 1: M2M, one block per parent cell; children staged in shared memory,
// the three 1-D factors applied in turn (z, y, x).

template <int L>
__global__ void __launch_bounds__(128)
k_m2m(const float *__restrict__ Mc, float *__restrict__ Mp, int ne, int ldm, const __grid_constant__ M2MTab V,
      unsigned *__restrict__ mmax)
{
    constexpr int P = L * L * L;
    __shared__ float sA[8 * P], sB[8 * P];
    __shared__ float sV[2][L][L];   // lane-dependent indices: shared memory, not the constant bank
    __shared__ float smax[4];
    const int parent = blockIdx.x;
    const int X = parent / (ne * ne), Y = (parent / ne) % ne, Z = parent % ne, nc = 2 * ne;
    for (int i = threadIdx.x; i < 2 * L * L; i += blockDim.x) {
        const int b = i / (L * L), k = (i / L) % L, l = i % L;
        sV[b][k][l] = V.v[b][k][l];
    }
    for (int i = threadIdx.x; i < 8 * P; i += blockDim.x) {
        const int b = i / P, l = i - b * P;
        const int child = ((2 * X + (b >> 2)) * nc + 2 * Y + ((b >> 1) & 1)) * nc + 2 * Z + (b & 1);
        sA[i] = Mc[(int64_t)child * ldm + l];
    }
    __syncthreads();
    // z: sB[b][(l1 L + l2) L + k3] = sum_l3 V[bz][k3][l3] sA[b][(l1 L + l2) L + l3], one (b, l1, l2) row per thread
    for (int r = threadIdx.x; r < 8 * L * L; r += blockDim.x) {
        const int b = r / (L * L);
        float x[L];
#pragma unroll
        for (int l = 0; l < L; ++l) x[l] = sA[r * L + l];
#pragma unroll
        for (int k = 0; k < L; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int l = 0; l < L; ++l) acc = fmaf(sV[b & 1][k][l], x[l], acc);
            sB[r * L + k] = acc;
        }
    }
    __syncthreads();
    // y: sA[b][(l1 L + k2) L + k3] = sum_l2 V[by][k2][l2] sB[b][(l1 L + l2) L + k3], one (b, l1, k3) row per thread
    for (int r = threadIdx.x; r < 8 * L * L; r += blockDim.x) {
        const int b = r / (L * L), l1 = (r / L) % L, k3 = r % L;
        const int base = b * P + l1 * L * L + k3;
        float x[L];
#pragma unroll
        for (int l = 0; l < L; ++l) x[l] = sB[base + l * L];
#pragma unroll
        for (int k = 0; k < L; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int l = 0; l < L; ++l) acc = fmaf(sV[(b >> 1) & 1][k][l], x[l], acc);
            sA[base + k * L] = acc;
        }
    }
    __syncthreads();
    // x: M_parent[(k1 L + k2) L + k3] = sum_b sum_l1 V[bx][k1][l1] sA[b][(l1 L + k2) L + k3]
    float mx = 0.f;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const int k1 = k / (L * L), k23 = k - k1 * L * L;
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < 8; ++b)
#pragma unroll
            for (int l = 0; l < L; ++l) s = fmaf(sV[b >> 2][k1][l], sA[b * P + l * L * L + k23], s);
        Mp[(int64_t)parent * ldm + k] = s;
        mx = fmaxf(mx, fabsf(s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        const float m = fmaxf(fmaxf(smax[0], smax[1]), fmaxf(smax[2], smax[3]));
        atomicMax(mmax, __float_as_uint(m));
    }
}

// ---------------------------------------------------------------------------
// Step 2 operands.  B: every level's expansions, parity-major, with one-cell
// y and z halos: row (class, X, Yh, j) of a level holds the cell
// (2X + px, 2Y + py, 2Z + pz), Y = (Yh - 1) mod m, Z = (j - 1) mod m, scaled
// by 2^eM(level) and split into fp16 hi + lo.  One thread per 8 nodes of a
// row; the padding rows j > m + 1 stay zero.

__global__ void __launch_bounds__(256)
k_split_fmm(const __grid_constant__ FmmLevels lv, int E, int ldm, int ldk, int64_t rows,
            const unsigned *__restrict__ mmax, __half *__restrict__ Bhi, __half *__restrict__ Blo)
{
    const int per_row = ldk / 8;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * per_row) return;
    const int r = (int)(t / per_row);
    const int node0 = (int)(t % per_row) * 8;
    int e = 1;
    while (e < E && r >= lv.lv[e + 1].rowbase) ++e;
    const FmmLevel &L = lv.lv[e];
    const int m = L.m, rr = r - L.rowbase;
    const int j = rr % L.rowstride, q = rr / L.rowstride;
    if (j > m + 1) return;
    const int Yh = q % (m + 2), q2 = q / (m + 2);
    const int X = q2 % m, cls = q2 / m;
    const int Y = Yh == 0 ? m - 1 : (Yh == m + 1 ? 0 : Yh - 1);
    const int Z = j == 0 ? m - 1 : (j == m + 1 ? 0 : j - 1);
    const int ne = 2 * m;
    const int64_t cell = ((int64_t)(2 * X + (cls >> 2)) * ne + 2 * Y + ((cls >> 1) & 1)) * ne + 2 * Z + (cls & 1);
    const float scale = ldexpf(1.f, split_exponent_dev(__uint_as_float(mmax[e])));
    float v[8];
    if (node0 < ldm) {
        const float4 *src = reinterpret_cast<const float4 *>(L.M + cell * ldm + node0);
        const float4 a = src[0], b = src[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.f;
    }
    __align__(16) __half hi[8], lo[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float x = v[k] * scale;
        hi[k] = __float2half_rn(x);
        lo[k] = __float2half_rn(x - __half2float(hi[k]));
    }
    const int64_t o = (int64_t)r * ldk + node0;
    *reinterpret_cast<uint4 *>(Bhi + o) = *reinterpret_cast<const uint4 *>(hi);
    *reinterpret_cast<uint4 *>(Blo + o) = *reinterpret_cast<const uint4 *>(lo);
}

// A (creation time, FP64): [slices*128 rows (target node k)][E * 343 * ldk]
// with column (e - 1) 343 ldk + blk(d) ldk + l holding 2^eC_e C_e(d)[k][l]
// (zero for |d|_inf <= 1 and for padding nodes), split into fp16 hi + lo.
struct EcTab {
    int eC[kFmmMaxLevels];
};

__global__ void __launch_bounds__(256)
k_pre_m2l(int E, int L, int ldk, int64_t arows, double box, double xi, const __grid_constant__ EcTab ec,
          __half *__restrict__ Ahi, __half *__restrict__ Alo)
{
    const int64_t cols = (int64_t)E * kBlk * ldk;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= arows * cols) return;
    const int k = (int)(idx / cols);
    const int64_t c = idx % cols;
    const int e = (int)(c / ((int64_t)kBlk * ldk)) + 1;
    const int rem = (int)(c % ((int64_t)kBlk * ldk));
    const int blk = rem / ldk, l = rem % ldk;
    const int P = L * L * L;
    double v = 0.0;
    const int d[3] = {blk / 49 - 3, (blk / 7) % 7 - 3, blk % 7 - 3};
    const int dmax = max(abs(d[0]), max(abs(d[1]), abs(d[2])));
    if (k < P && l < P && dmax >= 2) {
        const double h = box / (double)(1 << e);
        const int kv[3] = {k / (L * L), (k / L) % L, k % L};
        const int lv[3] = {l / (L * L), (l / L) % L, l % L};
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double ok = 0.5 * cos((2 * kv[a] + 1) * M_PI / (2.0 * L));
            const double ol = 0.5 * cos((2 * lv[a] + 1) * M_PI / (2.0 * L));
            const double z = h * (ok - ol - d[a]);
            r2 += z * z;
        }
        const double r = sqrt(r2);
        v = (xi > 0.0 ? erfc(xi * r) : 1.0) / r;
    }
    const float x = (float)(v * ldexp(1.0, ec.eC[e]));
    const __half hi = __float2half_rn(x);
    Ahi[idx] = hi;
    Alo[idx] = __float2half_rn(x - __half2float(hi));
}

// ---------------------------------------------------------------------------
// Step 2: persistent tcgen05 M2L over the work items of all levels (energy).
// Warps 0-15 drain the tensor memory after every stage and finish the items
// (warp w: TMEM lanes 32 (w mod 4), columns 32 (w div 4) .. + 32: sixteen
// short drains in parallel keep the two large-product buffers turning over),
// warp 16 issues the TMA copies, warp 17 the MMAs.  Every wait is bounded; on
// a timeout the kernel raises bit 2 of the error flag, lets its own copies
// land, frees its tensor memory and returns.

__global__ void __launch_bounds__(576, 1)
k_m2l_tc(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
         const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
         const __grid_constant__ B3Maps b3, const FmmLevel *__restrict__ lvt, int ldm, int ldk, const int4 *__restrict__ items,
         const int *__restrict__ cta_off,
         const int *__restrict__ tab, const unsigned *__restrict__ mmax, uint32_t tmem_cols,
         double *__restrict__ part, int *__restrict__ errflag)
{
    using namespace tcg;
    constexpr int N = kMaxN;   // R S = 128 on every level
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t bbytes = (uint32_t)N * kRowBytes;
    constexpr uint32_t stage = 2 * kABytes + 2 * bbytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * stage);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;
    uint64_t *acc_empty = acc_full + kAccBufs;
    uint64_t *small_free = acc_empty + kAccBufs;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(small_free + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *issued = abort_flag + 1;
    __shared__ double red[16];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kch = ldk / kKc;
    // this CTA's work items: items[ibeg .. ibeg + nmine) (balanced on the host)
    const int ibeg = __ldg(&cta_off[blockIdx.x]), nmine = __ldg(&cta_off[blockIdx.x + 1]) - ibeg;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 16);
        }
        for (int p = 0; p < 2; ++p) mbar_init(&small_free[p], 16);
        *abort_flag = 0;
        *issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 17) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 16 && lane == 0) {
        // TMA producer.  A single thread issues every copy, so its per-stage
        // integer work sits on the critical path: the stage loop is nested over
        // (offset, K chunk) without divisions, the per-item leaf coordinates are
        // hoisted, and neighbours wrap by compare (m is a power of two).
        int gi = 0, s = 0;
        uint32_t ph = 0;
        bool stop = false;
        for (int j = 0; j < nmine && !stop; ++j) {
            const int4 item = __ldg(&items[ibeg + j]);
            const int lev = item.x & 15;
            const FmmLevel *L = lvt + lev;
            const int slice = item.x >> 8, m = L->m, nrow = m * m, lgm = __ffs(m) - 1;
            const int R = L->R, S = L->S, rowbase = L->rowbase, rowstride = L->rowstride, acol = L->acol;
            const int zrow0 = item.y * R, cx0 = zrow0 >> lgm, cy0 = zrow0 & (m - 1);
            for (int oi = 0; oi < item.w && !stop; ++oi) {
                const int ent = __ldg(&tab[item.z + oi]);
                const int blk = ent & 511, sc = (ent >> 9) & 7;
                const int Dx = ((ent >> 12) & 3) - 1, Dy = ((ent >> 14) & 3) - 1, Dz = ((ent >> 16) & 3) - 1;
                int ncx0 = cx0 + Dx;
                ncx0 += ncx0 < 0 ? m : 0;
                ncx0 -= ncx0 >= m ? m : 0;
                const int blk3 = ((sc << lgm) + ncx0) * (m + 2) + cy0 + Dy + 1;
                const int acol_d = acol + blk * ldk;
                for (int kc = 0; kc < kch; ++kc, ++gi, s = (s + 1 == kStages ? 0 : s + 1), ph ^= (s == 0 ? 1u : 0u)) {
                    // ring slot s = gi mod kStages, phase ph = (gi div kStages) mod 2
                    if (gi >= kStages && !mbar_wait(&empty[s], ph ^ 1u, kBudget)) {
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    if (*abort_flag) {
                        stop = true;
                        break;
                    }
                    unsigned char *st = smem + (size_t)s * stage;
                    mbar_expect_tx(&full[s], stage);
                    tma_2d(st, &tmAhi, &full[s], acol_d + kc * kKc, slice * kRows);
                    tma_2d(st + kABytes, &tmAlo, &full[s], acol_d + kc * kKc, slice * kRows);
                    if (m >= 8) {
                        // R divides m: the tile's z-rows lie in one X plane, and the
                        // sources are R consecutive y-halo blocks of class sc
                        tma_3d(st + 2 * kABytes, &b3.hi[lev - 4], &full[s], kc * kKc, 1 + Dz, blk3);
                        tma_3d(st + 2 * kABytes + bbytes, &b3.lo[lev - 4], &full[s], kc * kKc, 1 + Dz, blk3);
                    } else {
                        for (int r = 0; r < R; ++r) {
                            int zrow = zrow0 + r;
                            if (zrow >= nrow) zrow = nrow - 1;
                            int ncx = (zrow >> lgm) + Dx, ncy = (zrow & (m - 1)) + Dy;
                            ncx += ncx < 0 ? m : 0;
                            ncx -= ncx >= m ? m : 0;
                            ncy += ncy < 0 ? m : 0;
                            ncy -= ncy >= m ? m : 0;
                            const int brow = rowbase + (((sc << lgm) + ncx) * (m + 2) + ncy + 1) * rowstride + 1 + Dz;
                            for (int qb = 0; qb < S; qb += kBoxRows) {
                                const size_t so = ((size_t)r * S + qb) * kRowBytes;
                                tma_2d(st + 2 * kABytes + so, &tmBhi, &full[s], kc * kKc, brow + qb);
                                tma_2d(st + 2 * kABytes + bbytes + so, &tmBlo, &full[s], kc * kKc, brow + qb);
                            }
                        }
                    }
                    *issued = gi + 1;
                }
            }
        }
    } else if (warp == 17 && lane == 0) {
        // MMA issuer: large products into one of two buffers drained per stage,
        // small corrections into the item's accumulator (one per item parity)
        const uint32_t idesc = idesc_f16(kRows, N);
        int consumed = 0, gi = 0, s = 0;
        uint32_t ph = 0;
        bool stop = false;
        for (int j = 0; j < nmine && !stop; ++j) {
            const int4 item = __ldg(&items[ibeg + j]);
            const int nst = item.w * kch, par = j & 1;
            for (int it = 0; it < nst; ++it, ++gi, s = (s + 1 == kStages ? 0 : s + 1), ph ^= (s == 0 ? 1u : 0u)) {
                // ring slot s = gi mod kStages, phase ph = (gi div kStages) mod 2
                const int b = gi % kAccBufs, u = gi / kAccBufs;
                if (it == 0 && j >= 2 &&
                    !mbar_wait(&small_free[par], (uint32_t)(((j >> 1) - 1) & 1), kBudget)) {
                    *abort_flag = 1;
                    stop = true;
                    break;
                }
                if (gi >= kAccBufs && !mbar_wait(&acc_empty[b], (uint32_t)((u - 1) & 1), kBudget)) {
                    *abort_flag = 1;
                    stop = true;
                    break;
                }
                if (!mbar_wait(&full[s], ph, kBudget)) {
                    *abort_flag = 1;
                    stop = true;
                    break;
                }
                consumed = gi + 1;
                fence_after();
                const uint32_t big = tmem + (uint32_t)(b * N);
                const uint32_t small = tmem + (uint32_t)((kAccBufs + par) * N);
                const uint32_t base = su32(smem + (size_t)s * stage);
                const uint32_t ahi = base, alo = base + kABytes, bhi = base + 2 * kABytes, blo = bhi + bbytes;
                // descriptors built once per stage; a K step of 16 halves (32
                // bytes along the swizzled row) adds 2 to the encoded start address
                const uint64_t dah = desc_sw128(ahi), dal = desc_sw128(alo), dbh = desc_sw128(bhi), dbl = desc_sw128(blo);
#pragma unroll
                for (int k16 = 0; k16 < kKc / 16; ++k16) {
                    const uint64_t o = 2u * k16;
                    mma_f16(big, dah + o, dbh + o, idesc, k16 > 0 ? 1u : 0u);
                    mma_f16(small, dah + o, dbl + o, idesc, (it > 0 || k16 > 0) ? 1u : 0u);
                    mma_f16(small, dal + o, dbh + o, idesc, 1u);
                }
                mma_commit(&empty[s]);
                mma_commit(&acc_full[b]);
            }
        }
        if (*abort_flag) {
            for (int b = 0; b < kAccBufs; ++b) mma_commit(&acc_full[b]);
            const int nis = *issued;
            for (int g2 = consumed; g2 < nis; ++g2)
                mbar_wait(&full[g2 % kStages], (uint32_t)((g2 / kStages) & 1), kBudget);
        }
    }
    double e = 0.0;
    if (warp < 16) {
        // warp w drains TMEM lanes 32 (w mod 4) and columns 32 (w div 4) .. + 32
        const int qd = warp & 3, hf = warp >> 2;
        float acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0.f;
        bool ok = true;
        const uint32_t lanebase = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(hf * 32);
        int gi = 0;
        for (int j = 0; j < nmine && ok; ++j) {
            const int4 item = __ldg(&items[ibeg + j]);
            const int nst = item.w * kch;
            for (int it = 0; it < nst; ++it, ++gi) {
                const int b = gi % kAccBufs, u = gi / kAccBufs;
                const bool wok = mbar_wait(&acc_full[b], (uint32_t)(u & 1), 2 * kBudget);
                ok = __all_sync(0xffffffffu, wok && !*abort_flag);
                if (!ok) break;
                fence_after();
                const uint32_t ta = lanebase + (uint32_t)(b * N);
                uint32_t v[32];
                tmem_ld32_nowait(ta, v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[q] += __uint_as_float(v[q]);
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[b]);
            }
            if (!ok) break;
            // item complete: psi = (large + small) 2^-(eC + eM), folded into the
            // small accumulator, then e += M_t . psi, 8 columns at a time
            const int lev = item.x & 15, cls = (item.x >> 4) & 7, slice = item.x >> 8;
            const FmmLevel *L = lvt + lev;
            const float unscale = ldexpf(1.f, -(L->eC + split_exponent_dev(__uint_as_float(mmax[lev]))));
            const uint32_t ts = lanebase + (uint32_t)((kAccBufs + (j & 1)) * N);
#pragma unroll
            for (int c = 0; c < 1; ++c) {
                uint32_t v[32];
                tmem_ld32_nowait(ts + (uint32_t)(c * 32), v);
                tmem_wait_ld();
                float o[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    o[q] = (acc[c * 32 + q] + __uint_as_float(v[q])) * unscale;
                    acc[c * 32 + q] = 0.f;
                }
                tmem_st32(ts + (uint32_t)(c * 32), o);
            }
            tmem_wait_st();
            const int node = slice * kRows + qd * 32 + lane;
            const int m = L->m, S = L->S, R = L->R, ne = 2 * m, nrow = m * m;
            const float *Ml = L->M;
            const int px = cls >> 2, py = (cls >> 1) & 1, pz = cls & 1;
            float pe0 = 0.f, pe1 = 0.f;
            for (int c0 = 0; c0 < 32; c0 += 8) {
                float mv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int col = hf * 32 + c0 + q, slab = col / S, z = col - slab * S, zrow = item.y * R + slab;
                    mv[q] = 0.f;
                    if (node < ldm && z < m && zrow < nrow) {
                        const int X = zrow / m, Y = zrow - X * m;
                        const int64_t cell = ((int64_t)(2 * X + px) * ne + 2 * Y + py) * ne + 2 * z + pz;
                        mv[q] = __ldg(&Ml[cell * ldm + node]);
                    }
                }
                uint32_t v[8];
                tmem_ld8_nowait(ts + (uint32_t)c0, v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q & 1) pe1 = fmaf(mv[q], __uint_as_float(v[q]), pe1);
                    else pe0 = fmaf(mv[q], __uint_as_float(v[q]), pe0);
                }
            }
            e += (double)pe0 + (double)pe1;
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&small_free[j & 1]);
        }
        if (!ok) *abort_flag = 1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if (lane == 0) red[warp] = e;
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 16; ++w) t += red[w];
        part[blockIdx.x] = t;
        if (*abort_flag) atomicOr(errflag, 2);
    }
    if (warp == 17) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Step 4: F_per = 1/2 M_B^T K M_B (one block, FP64).

__global__ void __launch_bounds__(256)
k_root(const float *__restrict__ M0, const double *__restrict__ K, int P, double *__restrict__ part)
{
    __shared__ double sh[8];
    double e = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < P; ++l) s += K[(int64_t)k * P + l] * (double)M0[l];
        e += (double)M0[k] * s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[0] = 0.5 * t;
    }
}

// ---------------------------------------------------------------------------
// host tables

std::vector<double> cheb(int L)
{
    std::vector<double> r(L);
    for (int k = 0; k < L; ++k) r[k] = std::cos((2.0 * k + 1.0) * M_PI / (2.0 * L));
    return r;
}

// Lagrange basis of the Chebyshev nodes r at x (product form)
double lagrange(const std::vector<double> &r, int k, double x)
{
    double v = 1.0;
    for (int j = 0; j < (int)r.size(); ++j)
        if (j != k) v *= (x - r[j]) / (r[k] - r[j]);
    return v;
}

// K[(kx ky kz)][(lx ly lz)] = sum_{|I|_inf >= 2} H(x_k - x_l + L I) at the root
// nodes x = (L/2) r per axis, without the constant pi / (V xi^2).
std::vector<double> root_operator(int L, double box, double xi, bool include_rec)
{
    const int L2 = L * L, P = L * L * L;
    const std::vector<double> r = cheb(L);
    std::vector<double> d1(L2);
    for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l) d1[k * L + l] = 0.5 * box * (r[k] - r[l]);
    const double V = box * box * box, eta = 12.0 / box;
    const int mm = (int)std::ceil(12.6 * eta * box / (2.0 * M_PI));
    const int nm = 2 * mm + 1;
    const double tk = 2.0 * M_PI / box;
    // reciprocal coefficients (even in every component: cosine factors)
    std::vector<double> c((size_t)nm * nm * nm);
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b)
            for (int g = 0; g < nm; ++g) {
                const double m2 = (double)(a - mm) * (a - mm) + (double)(b - mm) * (b - mm) + (double)(g - mm) * (g - mm);
                double v = 0.0;
                if (m2 > 0.0) {
                    const double k2 = tk * tk * m2;
                    v = std::exp(-k2 / (4.0 * eta * eta));
                    if (!include_rec) v -= std::exp(-k2 / (4.0 * xi * xi));
                    v *= 4.0 * M_PI / (V * k2);
                }
                c[((size_t)a * nm + b) * nm + g] = v;
            }
    std::vector<double> cs((size_t)nm * L2);
    for (int a = 0; a < nm; ++a)
        for (int i = 0; i < L2; ++i) cs[(size_t)a * L2 + i] = std::cos(tk * (a - mm) * d1[i]);
    std::vector<double> T1((size_t)nm * nm * L2, 0.0), T2((size_t)nm * L2 * L2, 0.0);
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b)
            for (int kk = 0; kk < L2; ++kk) {
                double s = 0.0;
                for (int g = 0; g < nm; ++g) s += c[((size_t)a * nm + b) * nm + g] * cs[(size_t)g * L2 + kk];
                T1[((size_t)a * nm + b) * L2 + kk] = s;
            }
    for (int a = 0; a < nm; ++a)
        for (int jj = 0; jj < L2; ++jj)
            for (int kk = 0; kk < L2; ++kk) {
                double s = 0.0;
                for (int b = 0; b < nm; ++b) s += cs[(size_t)b * L2 + jj] * T1[((size_t)a * nm + b) * L2 + kk];
                T2[((size_t)a * L2 + jj) * L2 + kk] = s;
            }
    std::vector<double> K((size_t)P * P);
    const double cst = -M_PI / (V * eta * eta);   // (pi / V)(1/xi^2 - 1/eta^2) without pi / (V xi^2)
    for (int ii = 0; ii < L2; ++ii)
        for (int jj = 0; jj < L2; ++jj)
            for (int kk = 0; kk < L2; ++kk) {
                double g = cst;
                for (int a = 0; a < nm; ++a) g += cs[(size_t)a * L2 + ii] * T2[((size_t)a * L2 + jj) * L2 + kk];
                const double z[3] = {d1[ii], d1[jj], d1[kk]};
                const bool origin = (ii / L == ii % L) && (jj / L == jj % L) && (kk / L == kk % L);
                for (int mx = -1; mx <= 1; ++mx)
                    for (int my = -1; my <= 1; ++my)
                        for (int mz = -1; mz <= 1; ++mz) {
                            const double x = z[0] + box * mx, y = z[1] + box * my, w = z[2] + box * mz;
                            const double rr = std::sqrt(x * x + y * y + w * w);
                            if (origin && mx == 0 && my == 0 && mz == 0) {
                                // limit of (erfc(eta r) - erfc(xi r)) / r: the origin term of the
                                // lattice minus the (absent) self term H(0)
                                g += 2.0 / std::sqrt(M_PI) * (xi - eta);
                            } else {
                                g += std::erfc(eta * rr) / rr;        // lattice (real part)
                                g -= std::erfc(xi * rr) / rr;         // minus the direct region
                            }
                        }
                const int kx = ii / L, lx = ii % L, ky = jj / L, ly = jj % L, kz = kk / L, lz = kk % L;
                K[(size_t)((kx * L + ky) * L + kz) * P + (lx * L + ly) * L + lz] = g;
            }
    return K;
}

template <typename T>
cudaError_t falloc(Handle &H, T **p, size_t count)
{
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    const cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) H.device_bytes += (int64_t)bytes;
    return e;
}

size_t m2l_smem_bytes()
{
    const size_t stage = 2 * (size_t)tcg::kABytes + 2 * (size_t)tcg::kMaxN * tcg::kRowBytes;
    return (size_t)tcg::kStages * stage + 1024 + 256;
}

#define ANKH_FMM_L_SWITCH(Lv, ...)                                                                         \
    switch (Lv) {                                                                                          \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } break;                                                  \
    case 3: { constexpr int LL = 3; __VA_ARGS__; } break;                                                  \
    case 4: { constexpr int LL = 4; __VA_ARGS__; } break;                                                  \
    case 5: { constexpr int LL = 5; __VA_ARGS__; } break;                                                  \
    case 6: { constexpr int LL = 6; __VA_ARGS__; } break;                                                  \
    case 7: { constexpr int LL = 7; __VA_ARGS__; } break;                                                  \
    default: { constexpr int LL = 8; __VA_ARGS__; } break;                                                 \
    }

}  // namespace

// ---------------------------------------------------------------------------

void fmm_free(Handle &H)
{
    FmmPlan &F = H.fmm;
    for (int e = 0; e < kFmmMaxLevels; ++e)
        if (F.d_Mlev[e]) cudaFree(F.d_Mlev[e]);
    void *ptrs[] = {F.d_Bhi, F.d_Blo, F.d_Ahi, F.d_Alo, F.d_items, F.d_ctaoff, F.d_tab, F.d_K, F.d_lev};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    std::memset(&F, 0, sizeof(FmmPlan));
}

int fmm_prepare(Handle &H, double xi, bool include_rec, std::string &err)
{
    FmmPlan &F = H.fmm;
    const Geo &g = H.g;
    int E = 0;
    while ((1 << E) < g.n) ++E;
    if ((1 << E) != g.n || E < 2 || E >= kFmmMaxLevels) {
        err = "ANKH_FMM: n_cells must be 2^E with 2 <= E <= 7";
        return ANKH_EINVAL;
    }
    if (g.Lu != g.Lc || g.Lu > 8) {
        err = "ANKH_FMM: one Chebyshev order L = Lu = Lc <= 8";
        return ANKH_EINVAL;
    }
    const int L = g.Lu, P = g.P, ldm = g.ldm;
    F.E = E;
    F.L = L;
    F.ldk = tc_ldk(ldm);
    F.kch = F.ldk / tcg::kKc;
    F.slices = (ldm + tcg::kRows - 1) / tcg::kRows;
    F.tmem_cols = 512;   // two large-product buffers + two small accumulators of 128 columns
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess) err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaSuccess;
    };
    // expansions of the levels above the leaves
    for (int e = 0; e < E; ++e) {
        const int64_t nc = (int64_t)1 << (3 * e);
        if (!cu(falloc(H, &F.d_Mlev[e], (size_t)(nc * ldm)), "cudaMalloc level expansions")) return ANKH_ENOMEM;
        cudaMemset(F.d_Mlev[e], 0, sizeof(float) * nc * ldm);
    }
    if (!cu(falloc(H, &H.d_mmax, (size_t)(E + 1)), "cudaMalloc mmax")) return ANKH_ENOMEM;
    // level geometry: levels 1 .. E in increasing row order
    int rowbase = 0;
    const std::vector<double> r = cheb(L);
    EcTab ec{};
    for (int e = 1; e <= E; ++e) {
        FmmLevel &lv = F.lev.lv[e];
        lv.M = e == E ? H.d_M : F.d_Mlev[e];
        lv.m = 1 << (e - 1);
        lv.S = std::max(16, lv.m);
        lv.R = tcg::kMaxN / lv.S;
        lv.tiles = (lv.m * lv.m + lv.R - 1) / lv.R;
        lv.rowstride = lv.S + 2;
        lv.rowbase = rowbase;
        rowbase += 8 * lv.m * (lv.m + 2) * lv.rowstride;
        lv.acol = (e - 1) * kBlk * F.ldk;
        // largest |C_e|: the nearest node pair of an offset with |d|_inf = 2 is
        // h_e (2 - r_0) apart (o_k - o_l spans [-r_0, r_0])
        const double h = g.box / (double)(1 << e), rmin = h * (2.0 - r[0]);
        const double cmax = (xi > 0.0 ? std::erfc(xi * rmin) : 1.0) / rmin;
        lv.eC = split_exponent((float)cmax);
        ec.eC[e] = lv.eC;
    }
    F.brows = rowbase;
    const int64_t arows = (int64_t)F.slices * tcg::kRows, acols = (int64_t)E * kBlk * F.ldk;
    if (!cu(falloc(H, &F.d_Bhi, (size_t)(F.brows * F.ldk)), "cudaMalloc B") ||
        !cu(falloc(H, &F.d_Blo, (size_t)(F.brows * F.ldk)), "cudaMalloc B") ||
        !cu(falloc(H, &F.d_Ahi, (size_t)(arows * acols)), "cudaMalloc A") ||
        !cu(falloc(H, &F.d_Alo, (size_t)(arows * acols)), "cudaMalloc A"))
        return ANKH_ENOMEM;
    cudaMemset(F.d_Bhi, 0, sizeof(__half) * F.brows * F.ldk);
    cudaMemset(F.d_Blo, 0, sizeof(__half) * F.brows * F.ldk);
    {
        const int64_t tot = arows * acols;
        k_pre_m2l<<<(unsigned)((tot + 255) / 256), 256>>>(E, L, F.ldk, arows, g.box, xi, ec, F.d_Ahi, F.d_Alo);
        if (!cu(cudaGetLastError(), "M2L operator precompute")) return ANKH_ECUDA;
    }
    // interaction offsets per class (lexicographically positive half of Lambda)
    std::vector<int> tab, cbeg(8), ccnt(8);
    for (int cls = 0; cls < 8; ++cls) {
        const int p[3] = {cls >> 2, (cls >> 1) & 1, cls & 1};
        cbeg[cls] = (int)tab.size();
        for (int dx = -2 - p[0]; dx <= 3 - p[0]; ++dx)
            for (int dy = -2 - p[1]; dy <= 3 - p[1]; ++dy)
                for (int dz = -2 - p[2]; dz <= 3 - p[2]; ++dz) {
                    if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
                    const bool positive = dx > 0 || (dx == 0 && (dy > 0 || (dy == 0 && dz > 0)));
                    if (!positive) continue;
                    const int d[3] = {dx, dy, dz};
                    int q[3], D[3];
                    for (int a = 0; a < 3; ++a) {
                        q[a] = ((p[a] + d[a]) % 2 + 2) % 2;
                        D[a] = (p[a] + d[a] - q[a]) / 2;
                    }
                    const int sc = (q[0] << 2) | (q[1] << 1) | q[2];
                    tab.push_back(blk_of(dx, dy, dz) | (sc << 9) | ((D[0] + 1) << 12) | ((D[1] + 1) << 14) |
                                  ((D[2] + 1) << 16));
                }
        ccnt[cls] = (int)tab.size() - cbeg[cls];
    }
    F.ntab = (int)tab.size();
    if (!cu(falloc(H, &F.d_lev, (size_t)kFmmMaxLevels), "cudaMalloc level table")) return ANKH_ENOMEM;
    if (!cu(cudaMemcpy(F.d_lev, F.lev.lv, sizeof(F.lev.lv), cudaMemcpyHostToDevice), "upload level table"))
        return ANKH_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H.device) != cudaSuccess || sms <= 0) {
        err = "cudaDeviceGetAttribute (SM count) failed";
        return ANKH_ECUDA;
    }
    // work items: (level, class, tile, slice) with a range of the class's
    // offsets.  When there are few of them the offset ranges are split (the
    // energy of an item is linear in its offsets, so the pieces add) to give
    // about eight items per SM; then the items are dealt to the persistent
    // CTAs longest first, each to the least-loaded CTA (ties: lowest index),
    // and every CTA walks its own items in their original order.
    std::vector<int4> base;
    for (int e = E; e >= 1; --e) {
        const FmmLevel &lv = F.lev.lv[e];
        for (int t = 0; t < lv.tiles; ++t)
            for (int cls = 0; cls < 8; ++cls)
                for (int sl = 0; sl < F.slices; ++sl)
                    base.push_back(make_int4(e | (cls << 4) | (sl << 8), t, cbeg[cls], ccnt[cls]));
    }
    const int split = std::max(1, std::min(8, (8 * sms + (int)base.size() - 1) / (int)base.size()));
    std::vector<int4> items;
    for (const int4 &it : base)
        for (int c = 0; c < split; ++c) {
            const int lo = it.z + (int)((int64_t)it.w * c / split), hi = it.z + (int)((int64_t)it.w * (c + 1) / split);
            if (hi > lo) items.push_back(make_int4(it.x, it.y, lo, hi - lo));
        }
    F.nitems = (int)items.size();
    F.grid = std::min(F.nitems, sms);
    std::vector<int> order(items.size()), owner(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return items[a].w > items[b].w; });
    {
        // cost of an item: its offsets plus ~2 offsets' worth for finishing it
        std::vector<int64_t> load(F.grid, 0);
        for (int i : order) {
            int best = 0;
            for (int c = 1; c < F.grid; ++c)
                if (load[c] < load[best]) best = c;
            owner[i] = best;
            load[best] += (int64_t)items[i].w + 2;
        }
    }
    std::vector<int> cta_off(F.grid + 1, 0);
    for (size_t i = 0; i < items.size(); ++i) cta_off[owner[i] + 1]++;
    for (int c = 0; c < F.grid; ++c) cta_off[c + 1] += cta_off[c];
    std::vector<int4> dealt(items.size());
    {
        std::vector<int> fill(cta_off.begin(), cta_off.end() - 1);
        for (size_t i = 0; i < items.size(); ++i) dealt[fill[owner[i]]++] = items[i];
    }
    if (!cu(falloc(H, &F.d_tab, tab.size()), "cudaMalloc offsets") ||
        !cu(falloc(H, &F.d_items, dealt.size()), "cudaMalloc items") ||
        !cu(falloc(H, &F.d_ctaoff, cta_off.size()), "cudaMalloc item offsets"))
        return ANKH_ENOMEM;
    if (!cu(cudaMemcpy(F.d_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice), "upload offsets") ||
        !cu(cudaMemcpy(F.d_items, dealt.data(), dealt.size() * sizeof(int4), cudaMemcpyHostToDevice),
            "upload items") ||
        !cu(cudaMemcpy(F.d_ctaoff, cta_off.data(), cta_off.size() * sizeof(int), cudaMemcpyHostToDevice),
            "upload item offsets"))
        return ANKH_ECUDA;
    // M2M factors
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 8; ++k)
            for (int l = 0; l < 8; ++l)
                F.V[b][k][l] = (k < L && l < L) ? (float)lagrange(r, k, 0.5 * (2 * b - 1 + r[l])) : 0.f;
    // root operator
    {
        const std::vector<double> K = root_operator(L, g.box, xi, include_rec);
        if (!cu(falloc(H, &F.d_K, K.size()), "cudaMalloc K")) return ANKH_ENOMEM;
        if (!cu(cudaMemcpy(F.d_K, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice), "upload K"))
            return ANKH_ECUDA;
    }
    (void)P;
    // tensor maps and launch shape
    if (!encode_2d(&F.mAhi, F.d_Ahi, (uint64_t)acols, (uint64_t)arows, tcg::kKc, tcg::kRows, err) ||
        !encode_2d(&F.mAlo, F.d_Alo, (uint64_t)acols, (uint64_t)arows, tcg::kKc, tcg::kRows, err) ||
        !encode_2d(&F.mBhi, F.d_Bhi, (uint64_t)F.ldk, (uint64_t)F.brows, tcg::kKc, kBoxRows, err) ||
        !encode_2d(&F.mBlo, F.d_Blo, (uint64_t)F.ldk, (uint64_t)F.brows, tcg::kKc, kBoxRows, err))
        return ANKH_ECUDA;
    for (int e = 4; e <= E; ++e) {
        const FmmLevel &lv = F.lev.lv[e];
        const uint64_t nblk = (uint64_t)8 * lv.m * (lv.m + 2);
        const size_t off = (size_t)lv.rowbase * F.ldk;
        if (!encode_3d(&F.mB3hi[e - 4], F.d_Bhi + off, (uint64_t)F.ldk, (uint64_t)lv.rowstride, nblk,
                       (uint32_t)lv.S, (uint32_t)lv.R, err) ||
            !encode_3d(&F.mB3lo[e - 4], F.d_Blo + off, (uint64_t)F.ldk, (uint64_t)lv.rowstride, nblk,
                       (uint32_t)lv.S, (uint32_t)lv.R, err))
            return ANKH_ECUDA;
    }
    if (!cu(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m2l_smem_bytes()),
            "cudaFuncSetAttribute (shared memory)"))
        return ANKH_ECUDA;
    F.enabled = 1;
    return ANKH_OK;
}

int fmm_part_slots(const Handle &H)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H.device) != cudaSuccess || sms <= 0)
        sms = 1024;
    return sms;
}

static cudaError_t launch_m2m_chain(Handle &H, cudaStream_t s)
{
    FmmPlan &F = H.fmm;
    M2MTab V;
    std::memcpy(V.v, F.V, sizeof(V.v));
    for (int e = F.E - 1; e >= 0; --e) {
        const float *Mc = e + 1 == F.E ? H.d_M : F.d_Mlev[e + 1];
        const int ne = 1 << e;
        const unsigned nb = (unsigned)((int64_t)ne * ne * ne);
        ANKH_FMM_L_SWITCH(F.L, k_m2m<LL><<<nb, 128, 0, s>>>(Mc, F.d_Mlev[e], ne, H.g.ldm, V, H.d_mmax + e));
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

static cudaError_t launch_m2l(Handle &H, cudaStream_t s)
{
    FmmPlan &F = H.fmm;
    const int64_t nthr = F.brows * (F.ldk / 8);
    k_split_fmm<<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(F.lev, F.E, H.g.ldm, F.ldk, F.brows, H.d_mmax,
                                                             F.d_Bhi, F.d_Blo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    B3Maps b3;
    std::memcpy(b3.hi, F.mB3hi, sizeof(b3.hi));
    std::memcpy(b3.lo, F.mB3lo, sizeof(b3.lo));
    k_m2l_tc<<<F.grid, 576, m2l_smem_bytes(), s>>>(F.mAhi, F.mAlo, F.mBhi, F.mBlo, b3, F.d_lev, H.g.ldm, F.ldk,
                                                             F.d_items, F.d_ctaoff, F.d_tab, H.d_mmax, F.tmem_cols,
                                                             H.d_part + H.part_off[kPartCorr], H.d_flag);
    return cudaGetLastError();
}

// Alg. 3 on the stream: sort, self, P2M, M2M, M2L, root, near, reduce.
int run_fmm(Handle &H, const float *x, const float *q, const float *mu, const float *theta, cudaStream_t s)
{
    FmmPlan &F = H.fmm;
    auto chk = [](cudaError_t e, const char *what) -> int {
        if (e != cudaSuccess) {
            set_error(std::string(what) + ": " + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? (int)ANKH_ENOMEM : (int)ANKH_ECUDA;
        }
        return (int)ANKH_OK;
    };
    int rc;
    H.nrec = 0;
    mark_stage(H, -1, s);
    if ((rc = chk(launch_bin(H, x, s), "bin"))) return rc;
    if ((rc = chk(launch_scan(H, s), "scan"))) return rc;
    if ((rc = chk(launch_scatter_sort_gather(H, x, q, mu, theta, s), "sort"))) return rc;
    mark_stage(H, kStSort, s);
    if ((rc = chk(launch_self_dc(H, s), "self"))) return rc;
    mark_stage(H, kStSelf, s);
    if ((rc = chk(cudaMemsetAsync(H.d_mmax, 0, sizeof(unsigned) * (F.E + 1), s), "memset"))) return rc;
    if ((rc = chk(launch_p2m(H, s), "p2m"))) return rc;
    mark_stage(H, kStP2M, s);
    if ((rc = chk(launch_m2m_chain(H, s), "m2m"))) return rc;
    mark_stage(H, kStMerge, s);
    k_root<<<1, 256, 0, s>>>(F.d_Mlev[0], F.d_K, H.g.P, H.d_part + H.part_off[kPartGlob]);
    if ((rc = chk(cudaGetLastError(), "root"))) return rc;
    mark_stage(H, kStSpectral, s);
    if ((rc = chk(launch_m2l(H, s), "m2l"))) return rc;
    mark_stage(H, kStCorr, s);
    if ((rc = chk(launch_near(H, false, s), "near"))) return rc;
    mark_stage(H, kStNear, s);
    if ((rc = chk(launch_reduce(H, s), "reduce"))) return rc;
    mark_stage(H, kStReduce, s);
    return ANKH_OK;
}

}  // namespace ankh
