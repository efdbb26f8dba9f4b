// Adjacent-leaf correction on the 5th-generation tensor cores (tcgen05).
//
// Same contraction as k_corr.cu (see there for the definition):
//   Psi[ldm x N] = sum_{d=0..26} C_d[ldm x ldm] . B_d[ldm x N],
//   B_d[:, j] = M_{t_j + d},
// for tiles of R z-rows of the leaf grid, each padded to S >= n leaves (S a
// multiple of 8), the MMA width being N = R S rounded up to 16 (<= 128), and
// 128-row slices of the target nodes (ldm = 128 for L_u = 5; 224 for L_u = 6,
// two slices; rows beyond ldm are zero).
//
// Split precision "2xFP16": every FP32 operand x is scaled by a power of two
// (2^eC for C, fixed per box; 2^eM for M, from max |M| of the call, so that
// the largest scaled value is <= 2^14) and written as x_hi + x_lo with
// x_hi = fp16(x), x_lo = fp16(x - x_hi), both rounded to nearest: 11 + 11
// significant bits, ~2^-22 relative (an absolute floor of 2^-24 below the
// normal range of x_lo, i.e. ~1e-12 of the largest value).  C.M is
// accumulated in FP32 as C_hi.M_hi + C_hi.M_lo + C_lo.M_hi (kind::f16, twice
// the TF32 rate, half the bytes) and scaled back by 2^-(eC + eM) (exact).
//
// Data movement: A (= [C_0 | ... | C_26], hi and lo) and B (the leaf rows of
// the split modified charges, stored with a one-leaf halo along z so that
// the rows t + d of a z-row form one contiguous block) are fetched by TMA
// with the 128-byte swizzle (64 halves of K per row) into a 3-stage
// shared-memory ring; one thread issues tcgen05.mma (M = 128, K = 16) into
// FP32 accumulators in tensor memory; four epilogue warps read them back
// with tcgen05.ld, write the correction potential psi and form
// -1/2 sum M.psi in FP64.
//
// The tensor core rounds toward zero as it accumulates, so the large
// C_hi.M_hi products of one stage (four MMAs) go to one of two TMEM buffers
// and are drained after the stage into FP32 registers with round-to-nearest
// additions, while the next stage accumulates into the other buffer.  The
// small C_hi.M_lo + C_lo.M_hi corrections (2^-11 of the large ones) stay in a
// per-tile TMEM accumulator; their truncation bias is relative to their own
// small size and negligible.
//
// Every wait is bounded (clock64 budget); on timeout the kernel raises bit 2
// of the error flag, waits (bounded) for its own copies in flight, frees its
// tensor memory and returns.
#include "tcgen05.cuh"

#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <cmath>

namespace ankh {

int split_exponent(float maxabs)
{
    if (!(maxabs > 0.f) || !(maxabs <= 3.0e38f)) return 0;
    int ex;
    std::frexp(maxabs, &ex);
    return tcg::kMaxScaled - ex;
}

// Split of M for the tensor cores: rows of each z-row with a one-leaf halo
// (row j of z-row zr holds leaf z = n-1, 0, ..., n-1, 0 for j = 0 .. n+1;
// zeros in place of the wrapped rows for a non-periodic box),
// nodes padded to ldk with zeros, scaled by 2^eM and split into fp16 hi + lo.
// One thread per 8 nodes of a row.
__global__ void __launch_bounds__(256)
k_split_f16(Geo g, int ldk, int rowstride, const float *__restrict__ M, const unsigned *__restrict__ mmax,
            __half *__restrict__ Mhi, __half *__restrict__ Mlo)
{
    const int n = g.n, per_row = ldk / 8;
    const int64_t nrows = (int64_t)n * n * (n + 2);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrows * per_row) return;
    const int64_t r = t / per_row;
    const int node0 = (int)(t % per_row) * 8;
    const int j = (int)(r % (n + 2));
    const int64_t zr = r / (n + 2);
    const int cz = j == 0 ? n - 1 : (j == n + 1 ? 0 : j - 1);
    const float scale = ldexpf(1.f, split_exponent_dev(__uint_as_float(*mmax)));
    // the halo rows wrap around the z-row (periodic) or are zero (non-periodic)
    const bool halo_zero = g.nonperiodic && (j == 0 || j == n + 1);
    float v[8];
    if (node0 < g.ldm && !halo_zero) {
        const float4 *src = reinterpret_cast<const float4 *>(M + (zr * n + cz) * g.ldm + node0);
        const float4 a = src[0], b = src[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = 0.f;
    }
    __align__(16) __half hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float x = v[q] * scale;
        hi[q] = __float2half_rn(x);
        lo[q] = __float2half_rn(x - __half2float(hi[q]));
    }
    const int64_t o = (zr * rowstride + j) * ldk + node0;
    *reinterpret_cast<uint4 *>(Mhi + o) = *reinterpret_cast<const uint4 *>(hi);
    *reinterpret_cast<uint4 *>(Mlo + o) = *reinterpret_cast<const uint4 *>(lo);
}

// Persistent kernel: one CTA per SM walks the work items w = blockIdx.x,
// blockIdx.x + gridDim.x, ... (tile = w mod tiles, row slice = w / tiles);
// the TMA ring, the MMA stream and the drains run across item boundaries.
// TMEM (512 columns): two large-product buffers (drained after every stage)
// and two small-product accumulators, one per item parity.  When an item's
// last stage is drained, the epilogue warps fold their FP32 registers into
// that item's small accumulator (which then holds psi) and finish it -- the
// energy dot with M and the psi write, 8 columns per stage -- while the next
// item's MMAs run; the small accumulator is then released for the item after.
constexpr int kCorrEpiWarps = 16;                        // warp w: TMEM lanes 32 (w mod 4), columns 32 (w div 4)
constexpr int kCorrThreads = (kCorrEpiWarps + 2) * 32;   // + TMA producer + MMA issuer

template <bool FORCES>
__global__ void __launch_bounds__(kCorrThreads, 1)
k_corr_tc(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
          const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo, Geo g, int S,
          int R, int rowstride, int ldk, int eC, const unsigned *__restrict__ mmax, int ntiles, int nwork,
          int d0, int noff, uint32_t tmem_cols, const float *__restrict__ M, float *__restrict__ psi,
          double *__restrict__ part, int *__restrict__ errflag)
{
    using namespace tcg;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int N = R * S;                   // leaf columns of a tile
    const int Nm = (N + 15) & ~15;         // MMA width (<= kMaxN); rows N .. Nm-1 of B stay zero
    const int Nb = (Nm + 31) & ~31;        // TMEM column stride of the accumulator buffers
    const uint32_t bbytes = (uint32_t)Nm * kRowBytes;
    const uint32_t stage = 2 * kABytes + 2 * bbytes;
    const uint32_t txbytes = 2 * kABytes + 2 * (uint32_t)N * kRowBytes;   // what the copies of a stage deliver
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * stage);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;       // [kAccBufs] large buffer ready for draining
    uint64_t *acc_empty = acc_full + kAccBufs;  // [kAccBufs] large buffer drained (4 warp arrivals)
    uint64_t *small_free = acc_empty + kAccBufs;  // [2] small accumulator finished (4 warp arrivals)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(small_free + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *issued = abort_flag + 1;
    __shared__ double red[kCorrEpiWarps];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldm = g.ldm;
    const int kch = ldk / kKc;            // K chunks per offset d
    const int kIters = noff * kch;        // stages per work item
    const int nmine = blockIdx.x < nwork ? (nwork - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (Nm > N) {
        // B rows N .. Nm-1 of every stage: zero (no copy writes them), read by
        // the MMAs through the async proxy
        const int per = (Nm - N) * kRowBytes / 16;
        for (int i = threadIdx.x; i < kStages * 2 * per; i += blockDim.x) {
            const int st = i / (2 * per), hl = (i / per) % 2, o = i % per;
            *reinterpret_cast<uint4 *>(smem + (size_t)st * stage + 2 * kABytes + (size_t)hl * bbytes +
                                       (size_t)N * kRowBytes + (size_t)o * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kCorrEpiWarps);
        }
        for (int p = 0; p < 2; ++p) mbar_init(&small_free[p], kCorrEpiWarps);
        *abort_flag = 0;
        *issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int wprod = kCorrEpiWarps, wmma = kCorrEpiWarps + 1;
    if (warp == wmma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tcg::su32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n = g.n, nrow = n * n;

    if (warp == wprod && lane == 0) {
        // TMA producer.  A single thread issues every copy, so its per-stage
        // integer work sits on the critical path: the stages are walked as
        // nested loops (item, offset, K chunk) without divisions, the leaf
        // coordinates of the item's z-rows are computed once per item, and
        // neighbours wrap by compare.
        int gi = 0, s = 0;
        uint32_t ph = 0;
        bool stop = false;
        for (int j = 0; j < nmine && !stop; ++j) {
            const int w = (int)blockIdx.x + j * (int)gridDim.x;
            const int tile = w % ntiles, row0 = (w / ntiles) * kRows;
            int cxr[8], cyr[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                int zrow = tile * R + r;
                if (zrow >= nrow) zrow = nrow - 1;
                cxr[r] = zrow / n;
                cyr[r] = zrow - cxr[r] * n;
            }
            for (int jd = 0; jd < noff && !stop; ++jd) {
                // offset d = d0 + jd; its operator block is column block jd of A
                const int d = d0 + jd;
                const int dx = d / 9 - 1, dy = (d / 3) % 3 - 1, dz = d % 3 - 1;
                int brow[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    int ax = cxr[r] + dx, ay = cyr[r] + dy;
                    // a non-periodic box reads the all-zero z-row block n^2 beyond its faces
                    const bool outside = g.nonperiodic && (ax < 0 || ax >= n || ay < 0 || ay >= n);
                    ax += ax < 0 ? n : 0;
                    ax -= ax >= n ? n : 0;
                    ay += ay < 0 ? n : 0;
                    ay -= ay >= n ? n : 0;
                    brow[r] = (outside ? nrow : ax * n + ay) * rowstride + 1 + dz;
                }
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
                    mbar_expect_tx(&full[s], txbytes);
                    tma_2d(st, &tmAhi, &full[s], jd * ldk + kc * kKc, row0);
                    tma_2d(st + kABytes, &tmAlo, &full[s], jd * ldk + kc * kKc, row0);
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        if (r < R) {
                            tma_2d(st + 2 * kABytes + (size_t)r * S * kRowBytes, &tmBhi, &full[s], kc * kKc, brow[r]);
                            tma_2d(st + 2 * kABytes + bbytes + (size_t)r * S * kRowBytes, &tmBlo, &full[s], kc * kKc,
                                   brow[r]);
                        }
                    }
                    *issued = gi + 1;
                }
            }
        }
    } else if (warp == wmma && lane == 0) {
        // MMA issuer: large products of each stage into one of two TMEM buffers
        // (drained by the epilogue warps), small corrections into the item's
        // small accumulator
        const uint32_t idesc = idesc_f16(kRows, Nm);
        int consumed = 0, gi = 0, s = 0;
        uint32_t ph = 0;
        bool stop = false;
        for (int j = 0; j < nmine && !stop; ++j)
        for (int it = 0; it < kIters; ++it, ++gi, s = (s + 1 == kStages ? 0 : s + 1), ph ^= (s == 0 ? 1u : 0u)) {
            // (item j, stage it) walked as nested loops: no divisions per stage;
            // ring slot s = gi mod kStages, phase ph = (gi div kStages) mod 2
            const int b = gi % kAccBufs, u = gi / kAccBufs;
            const int par = j & 1;
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
            const uint32_t big = tmem + (uint32_t)(b * Nb);
            const uint32_t small = tmem + (uint32_t)((kAccBufs + par) * Nb);
            const uint32_t base = su32(smem + (size_t)s * stage);
            const uint32_t ahi = base, alo = base + kABytes, bhi = base + 2 * kABytes, blo = bhi + bbytes;
            // descriptors built once per stage; a K step of 16 halves (32 bytes
            // along the swizzled row) adds 2 to the encoded start address
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
        if (*abort_flag) {
            // release the epilogue and let every copy this CTA issued land
            for (int b = 0; b < kAccBufs; ++b) mma_commit(&acc_full[b]);
            const int nis = *issued;
            for (int g2 = consumed; g2 < nis; ++g2)
                mbar_wait(&full[g2 % kStages], (uint32_t)((g2 / kStages) & 1), kBudget);
        }
    }
    double e = 0.0;
    if (warp < kCorrEpiWarps) {
        // sixteen epilogue warps: warp w owns TMEM lanes 32 (w mod 4) and the 32
        // columns 32 (w div 4) .. (a group past N owns none but keeps the barriers)
        const int qd = warp & 3, grp = warp >> 2, col0 = grp * 32;
        const bool have = col0 < Nm;
        float acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0.f;
        bool ok = true;
        const uint32_t lanebase = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)col0;
        const float unscale = ldexpf(1.f, -(eC + split_exponent_dev(__uint_as_float(*mmax))));
        // the item whose small accumulator (= psi) is being finished, and the
        // next of this warp's columns to finish
        int pend = -1, pcol = 0;
        float pe0 = 0.f, pe1 = 0.f;   // FP32 partial dot of the pending item (two chains)
        auto finish_chunk = [&](int c0) {
            // columns col0 + c0 .. + 7 of item pend: psi from TMEM, M from global
            const int w = (int)blockIdx.x + pend * (int)gridDim.x;
            const int tile = w % ntiles, m = (w / ntiles) * kRows + qd * 32 + lane;
            float mv[8];
            int64_t ofs[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = col0 + c0 + q, slab = c / S, z = c % S, zrow = tile * R + slab;
                const bool valid = (m < ldm) && (c < N) && (z < n) && (zrow < nrow);
                ofs[q] = valid ? ((int64_t)zrow * n + z) * ldm + m : -1;
                mv[q] = valid ? __ldg(&M[ofs[q]]) : 0.f;
            }
            uint32_t v[8];
            tmem_ld8_nowait(lanebase + (uint32_t)((kAccBufs + (pend & 1)) * Nb + c0), v);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                // a padding column may hold anything: it takes no part
                const float pv = ofs[q] >= 0 ? __uint_as_float(v[q]) : 0.f;
                if (q & 1) pe1 = fmaf(mv[q], pv, pe1);
                else pe0 = fmaf(mv[q], pv, pe0);
                if (FORCES && ofs[q] >= 0) psi[ofs[q]] = pv;
            }
        };
        auto release_pending = [&]() {
            e += (double)pe0 + (double)pe1;
            pe0 = pe1 = 0.f;
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&small_free[pend & 1]);
            pend = -1;
        };
        const int ncols = have ? min(32, Nm - col0) : 0;   // a multiple of 8
        int gi = 0;
        for (int j = 0; j < nmine && ok; ++j)
        for (int it = 0; it < kIters; ++it, ++gi) {
            const int b = gi % kAccBufs, u = gi / kAccBufs;
            bool wok = mbar_wait(&acc_full[b], (uint32_t)(u & 1), 2 * kBudget);
            ok = __all_sync(0xffffffffu, wok && !*abort_flag);
            if (!ok) break;
            fence_after();
            if (have) {
                uint32_t v[32];
                tmem_ld32_nowait(lanebase + (uint32_t)(b * Nb), v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[q] += __uint_as_float(v[q]);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            // finish 8 columns of the previous item while this one streams
            if (pend >= 0) {
                if (pcol < ncols) finish_chunk(pcol);
                pcol += 8;
                if (pcol >= ncols) release_pending();
            }
            if (it == kIters - 1) {
                // item j complete (this arrival follows all of its MMAs): fold
                // the drained large products into its small accumulator
                while (pend >= 0) {
                    if (pcol < ncols) finish_chunk(pcol);
                    pcol += 8;
                    if (pcol >= ncols) release_pending();
                }
                if (have) {
                    const uint32_t ts = lanebase + (uint32_t)((kAccBufs + (j & 1)) * Nb);
                    uint32_t v[32];
                    tmem_ld32_nowait(ts, v);
                    tmem_wait_ld();
                    float o[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        o[q] = (acc[q] + __uint_as_float(v[q])) * unscale;
                        acc[q] = 0.f;
                    }
                    tmem_st32(ts, o);
                    tmem_wait_st();
                }
                pend = j;
                pcol = 0;
            }
        }
        if (ok) {
            while (pend >= 0) {
                if (pcol < ncols) finish_chunk(pcol);
                pcol += 8;
                if (pcol >= ncols) release_pending();
            }
        } else {
            *abort_flag = 1;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if (lane == 0) red[warp] = e;
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kCorrEpiWarps; ++w) t += red[w];
        part[blockIdx.x] = -0.5 * t;
        if (*abort_flag) atomicOr(errflag, 2);
    }
    if (warp == wmma) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// host side

// 2-D fp16 tensor map, rows of `inner` halves, boxes of 64 x box_outer (128-byte swizzle)
bool encode_2d(CUtensorMap *map, void *ptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
                      uint32_t box_outer, std::string &err)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            err = "cuTensorMapEncodeTiled not available";
            return false;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * sizeof(__half)};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ptr, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

// 3-D fp16 tensor map {inner, mid, outer} with boxes {64, box_mid, box_outer} (128-byte swizzle)
bool encode_3d(CUtensorMap *map, void *ptr, uint64_t inner, uint64_t mid, uint64_t outer, uint32_t box_mid,
               uint32_t box_outer, std::string &err)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            err = "cuTensorMapEncodeTiled not available";
            return false;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    cuuint64_t dims[3] = {inner, mid, outer};
    cuuint64_t strides[2] = {inner * sizeof(__half), inner * mid * sizeof(__half)};
    cuuint32_t box[3] = {(cuuint32_t)tcg::kKc, box_mid, box_outer};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, ptr, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled (3-D) failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

static size_t tc_smem_bytes(int N)
{
    const size_t stage = 2 * (size_t)tcg::kABytes + 2 * (size_t)N * tcg::kRowBytes;
    return (size_t)tcg::kStages * stage + 1024 + 256;
}

// Tile of R z-rows of S leaves (S >= n, a multiple of 8 so that every z-row
// block of B starts on a 1 KB swizzle atom), R <= 8, MMA width
// roundup16(R S) <= 128.
// R minimises the estimated time: waves of work items over the SMs times the
// cost of one item, whose stages move the A slice (as many bytes as 128 B
// rows) and the B rows -- so 128 + width.  Ties go to the larger R.
void tc_tile_shape(int n, int halves, int sms, int &S, int &R)
{
    S = ((n + 7) / 8) * 8;
    const int rmax = std::max(1, std::min(8, tcg::kMaxN / S));   // the producer tracks up to 8 z-rows
    int64_t best = -1;
    R = rmax;
    for (int r = rmax; r >= 1; --r) {
        const int64_t items = (int64_t)((n * n + r - 1) / r) * halves;
        const int64_t waves = (items + sms - 1) / sms;
        const int64_t width = ((int64_t)r * S + 15) / 16 * 16;
        const int64_t cost = waves * (128 + width);
        if (best < 0 || cost < best) {
            best = cost;
            R = r;
        }
    }
}

int tc_max_blocks(int n, int ldm, int sms)
{
    int S, R;
    const int halves = (ldm + tcg::kRows - 1) / tcg::kRows;
    tc_tile_shape(n, halves, sms, S, R);
    return ((n * n + R - 1) / R) * halves;
}

bool tc_prepare(Handle &H, std::string &err)
{
    H.tc.enabled = 0;
    const Geo &g = H.g;
    if (g.ldm % 32 != 0 || g.ldm > 512 || g.n > 128) return true;   // plain FP32 kernel is used
    int S, R;
    tc_tile_shape(g.n, (g.ldm + tcg::kRows - 1) / tcg::kRows, H.sm_count, S, R);
    H.tc.S = S;
    H.tc.R = R;
    H.tc.rowstride = S + 2;
    H.tc.N = (R * S + 15) / 16 * 16;   // MMA width
    const int nb = (H.tc.N + 31) / 32 * 32;
    H.tc.tmem_cols = 32;
    while ((int)H.tc.tmem_cols < (tcg::kAccBufs + 2) * nb) H.tc.tmem_cols <<= 1;   // large buffers + 2 small
    H.tc.tiles = (g.n * g.n + R - 1) / R;
    H.tc.halves = (g.ldm + tcg::kRows - 1) / tcg::kRows;
    if (H.tc.tiles * H.tc.halves > H.part_off[kPartCorr + 1] - H.part_off[kPartCorr]) {
        err = "tensor-core correction: more CTAs than energy partial slots";
        return false;
    }
    const uint64_t rows = ((uint64_t)g.n * g.n + (g.nonperiodic ? 1 : 0)) * H.tc.rowstride;
    const uint64_t arows = (uint64_t)H.tc.halves * tcg::kRows;
    const int ldk = H.tc.ldk;
    if (!encode_2d(&H.tc.mAhi, H.d_Chi, 27 * (uint64_t)ldk, arows, tcg::kKc, 128, err)) return false;
    if (!encode_2d(&H.tc.mAlo, H.d_Clo, 27 * (uint64_t)ldk, arows, tcg::kKc, 128, err)) return false;
    if (!encode_2d(&H.tc.mAhiE, H.d_ChiE, 14 * (uint64_t)ldk, arows, tcg::kKc, 128, err)) return false;
    if (!encode_2d(&H.tc.mAloE, H.d_CloE, 14 * (uint64_t)ldk, arows, tcg::kKc, 128, err)) return false;
    if (!encode_2d(&H.tc.mBhi, H.d_Mhi, ldk, rows, tcg::kKc, (uint32_t)S, err)) return false;
    if (!encode_2d(&H.tc.mBlo, H.d_Mlo, ldk, rows, tcg::kKc, (uint32_t)S, err)) return false;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H.device) != cudaSuccess || sms <= 0) {
        err = "cudaDeviceGetAttribute (SM count) failed";
        return false;
    }
    H.tc.grid = std::min(H.tc.tiles * H.tc.halves, sms);   // persistent: one CTA per SM
    // the attribute belongs to the kernel, not to the handle: set the largest
    // tile's need, so that handles of other tile widths keep launching
    const int smem = (int)tc_smem_bytes(tcg::kMaxN);
    if (cudaFuncSetAttribute(k_corr_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_corr_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        err = "cudaFuncSetAttribute (shared memory) failed";
        return false;
    }
    H.tc.enabled = 1;
    return true;
}

int corr_tc_blocks(const Handle &H) { return H.tc.grid; }

int tc_ldk(int ldm) { return ((ldm + tcg::kKc - 1) / tcg::kKc) * tcg::kKc; }

cudaError_t launch_split_f16(Handle &H, cudaStream_t s)
{
    const int64_t nthr = (int64_t)H.g.n * H.g.n * (H.g.n + 2) * (H.tc.ldk / 8);
    k_split_f16<<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(H.g, H.tc.ldk, H.tc.rowstride, H.d_M, H.d_mmax,
                                                               H.d_Mhi, H.d_Mlo);
    return cudaGetLastError();
}

cudaError_t launch_corr_tc(Handle &H, bool forces, cudaStream_t s)
{
    cudaError_t e = launch_split_f16(H, s);
    if (e != cudaSuccess) return e;
    const size_t smem = tc_smem_bytes(H.tc.N);
    double *part = H.d_part + H.part_off[kPartCorr];
    const int nwork = H.tc.tiles * H.tc.halves;
    // forces: all 27 offsets (psi at every leaf); energy alone: d = 0 and the 13
    // positive offsets against [C_0 | 2 C_d], since C_(-d) = C_d^T
    if (forces)
        k_corr_tc<true><<<H.tc.grid, kCorrThreads, smem, s>>>(H.tc.mAhi, H.tc.mAlo, H.tc.mBhi, H.tc.mBlo, H.g,
                                                               H.tc.S, H.tc.R, H.tc.rowstride, H.tc.ldk, H.tc.eC,
                                                               H.d_mmax, H.tc.tiles, nwork, 0, 27, H.tc.tmem_cols,
                                                               H.d_M, H.d_psi, part, H.d_flag);
    else
        k_corr_tc<false><<<H.tc.grid, kCorrThreads, smem, s>>>(H.tc.mAhiE, H.tc.mAloE, H.tc.mBhi, H.tc.mBlo, H.g,
                                                                H.tc.S, H.tc.R, H.tc.rowstride, H.tc.ldk, H.tc.eC,
                                                                H.d_mmax, H.tc.tiles, nwork, 13, 14, H.tc.tmem_cols,
                                                                H.d_M, H.d_psi, part, H.d_flag);
    return cudaGetLastError();
}

}  // namespace ankh
