// Adjacent-leaf correction on the 5th-generation tensor cores (tcgen05).
//
// Same contraction as k_corr.cu (see there for the definition):
//   Psi[ldm x N] = sum_{d=0..26} C_d[ldm x ldm] . B_d[ldm x N],
//   B_d[:, j] = M_{t_j + d},
// one CTA per 128-row slice of the target nodes (blockIdx.y; ldm = 128 for
// L_u = 5, 224 for L_u = 6, rows beyond ldm are zero),
// for a tile of N target leaves (R z-rows of the leaf grid, each padded to S
// columns).  Split precision "3xTF32": every FP32 operand x is written as
// x_hi + x_lo with x_hi = tf32(x) (round to nearest) and x_lo = tf32(x - x_hi);
// C.M is accumulated in FP32 as C_hi.M_hi + C_hi.M_lo + C_lo.M_hi, which
// keeps ~21 bits of every product.
//
// Data movement: A (= [C_0 | ... | C_26], hi and lo) and B (the leaf rows of
// the modified charges, hi and lo, stored with a one-leaf halo along z so
// that the rows t + d of a z-row form one contiguous block) are fetched by
// TMA with the 128-byte swizzle into a 3-stage shared-memory ring; one thread
// issues tcgen05.mma (kind::tf32, M = 128, K = 8) into an FP32 accumulator in
// tensor memory; four epilogue warps read it back with tcgen05.ld, write the
// correction potential psi and form -1/2 sum M.psi in FP64.
//
// The tensor core rounds toward zero as it accumulates; over the 27 x 48 MMA
// steps of a tile that bias reaches ~4e-5.  So the large C_hi.M_hi products
// of one stage (K = 32, four MMAs) go to one of three TMEM buffers and are
// drained after the stage into FP32 registers with round-to-nearest
// additions, while the next stage accumulates into the other buffer.  The
// small C_hi.M_lo + C_lo.M_hi corrections (2^-11 of the large ones) stay in a
// third TMEM accumulator for the whole tile; their truncation bias is
// relative to their own small size and negligible.
//
// Every wait is bounded (clock64 budget); on timeout the kernel raises bit 2
// of the error flag, waits (bounded) for its own copies in flight, frees its
// tensor memory and returns.
#include "ankh_internal.cuh"

#include <cudaTypedefs.h>

namespace ankh {

namespace tcg {

constexpr int kStages = 3;
constexpr int kAccBufs = 3;            // large-product accumulator buffers in TMEM
constexpr int kRows = 128;            // target-node rows per CTA (MMA M)
constexpr int kKc = 32;               // K floats per stage (128 bytes)
constexpr int kThreads = 192;         // warps 0-3 epilogue, 4 TMA producer, 5 MMA issuer
constexpr uint32_t kABytes = kRows * kKc * 4;
constexpr long long kBudget = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand, 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);      // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused here)
    d |= (uint64_t)(1024u >> 4) << 32;              // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                         // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                         // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtm, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tcg

template <bool FORCES>
__global__ void __launch_bounds__(tcg::kThreads, 1)
k_corr_tc(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
          const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo, Geo g, int S,
          int R, int rowstride, uint32_t tmem_cols, const float *__restrict__ M, float *__restrict__ psi,
          double *__restrict__ part, int *__restrict__ errflag)
{
    using namespace tcg;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int N = R * S;
    const uint32_t bbytes = (uint32_t)N * kKc * 4;
    const uint32_t stage = 2 * kABytes + 2 * bbytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * stage);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;     // [kAccBufs] accumulator buffer ready for draining
    uint64_t *acc_empty = acc_full + kAccBufs; // [kAccBufs] buffer drained (4 warp arrivals)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + kAccBufs);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *issued = abort_flag + 1;
    __shared__ double red[4];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldm = g.ldm;
    const int kch = ldm / kKc;            // K chunks per offset d
    const int kIters = 27 * kch;
    const int row0 = blockIdx.y * kRows;  // first target-node row of this CTA
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        *abort_flag = 0;
        *issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
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

    if (warp == 4 && lane == 0) {
        // TMA producer
        for (int it = 0; it < kIters; ++it) {
            const int s = it % kStages, k = it / kStages;
            if (it >= kStages && !mbar_wait(&empty[s], (uint32_t)((k - 1) & 1), kBudget)) {
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            const int d = it / kch, kc = it % kch;
            const int dx = d / 9 - 1, dy = (d / 3) % 3 - 1, dz = d % 3 - 1;
            unsigned char *st = smem + (size_t)s * stage;
            mbar_expect_tx(&full[s], stage);
            tma_2d(st, &tmAhi, &full[s], d * ldm + kc * kKc, row0);
            tma_2d(st + kABytes, &tmAlo, &full[s], d * ldm + kc * kKc, row0);
            for (int r = 0; r < R; ++r) {
                int zrow = blockIdx.x * R + r;
                if (zrow >= nrow) zrow = nrow - 1;
                const int cx = zrow / n, cy = zrow % n;
                const int ncx = (cx + dx + n) % n, ncy = (cy + dy + n) % n;
                const int brow = (ncx * n + ncy) * rowstride + 1 + dz;
                tma_2d(st + 2 * kABytes + (size_t)r * S * kKc * 4, &tmBhi, &full[s], kc * kKc, brow);
                tma_2d(st + 2 * kABytes + bbytes + (size_t)r * S * kKc * 4, &tmBlo, &full[s], kc * kKc, brow);
            }
            *issued = it + 1;
        }
    } else if (warp == 5 && lane == 0) {
        // MMA issuer: large products of each stage into one of two TMEM buffers
        // (drained by the epilogue warps), small corrections into a third one
        const uint32_t idesc = idesc_tf32(kRows, N);
        const uint32_t small = tmem + (uint32_t)(kAccBufs * N);
        int consumed = 0;
        for (int it = 0; it < kIters; ++it) {
            const int s = it % kStages, k = it / kStages, buf = it % kAccBufs;
            if (it >= kAccBufs &&
                !mbar_wait(&acc_empty[buf], (uint32_t)(((it / kAccBufs) - 1) & 1), kBudget)) {
                *abort_flag = 1;
                break;
            }
            if (!mbar_wait(&full[s], (uint32_t)(k & 1), kBudget)) {
                *abort_flag = 1;
                break;
            }
            consumed = it + 1;
            fence_after();
            const uint32_t big = tmem + (uint32_t)(buf * N);
            const uint32_t base = su32(smem + (size_t)s * stage);
            const uint32_t ahi = base, alo = base + kABytes, bhi = base + 2 * kABytes, blo = bhi + bbytes;
#pragma unroll
            for (int k8 = 0; k8 < kKc / 8; ++k8) {
                const uint32_t off = k8 * 32;
                mma_tf32(big, desc_sw128(ahi + off), desc_sw128(bhi + off), idesc, k8 > 0 ? 1u : 0u);
                mma_tf32(small, desc_sw128(ahi + off), desc_sw128(blo + off), idesc, (it > 0 || k8 > 0) ? 1u : 0u);
                mma_tf32(small, desc_sw128(alo + off), desc_sw128(bhi + off), idesc, 1u);
            }
            mma_commit(&empty[s]);
            mma_commit(&acc_full[buf]);
        }
        if (*abort_flag) {
            // release the epilogue and let every copy this CTA issued land
            for (int b = 0; b < kAccBufs; ++b) mma_commit(&acc_full[b]);
            const int nis = *issued;
            for (int it = consumed; it < nis; ++it)
                mbar_wait(&full[it % kStages], (uint32_t)((it / kStages) & 1), kBudget);
        }
    }
    double e = 0.0;
    if (warp < 4) {
        // drain every stage's large accumulator into FP32 registers (round to nearest)
        float acc[128];
#pragma unroll
        for (int j = 0; j < 128; ++j) acc[j] = 0.f;
        bool ok = true;
        const uint32_t lanebase = tmem + ((uint32_t)(warp * 32) << 16);
        for (int it = 0; it < kIters; ++it) {
            const int buf = it % kAccBufs;
            bool w = mbar_wait(&acc_full[buf], (uint32_t)((it / kAccBufs) & 1), 2 * kBudget);
            ok = __all_sync(0xffffffffu, w && !*abort_flag);
            if (!ok) break;
            fence_after();
            const uint32_t ta = lanebase + (uint32_t)(buf * N);
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
                if (c * 32 < N) {
                    uint32_t v[64];
                    tmem_ld32_nowait(ta + (uint32_t)(c * 32), v);
                    if ((c + 1) * 32 < N) tmem_ld32_nowait(ta + (uint32_t)((c + 1) * 32), v + 32);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[c * 32 + j] += __uint_as_float(v[j]);
                    if ((c + 1) * 32 < N) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[(c + 1) * 32 + j] += __uint_as_float(v[32 + j]);
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&acc_empty[buf]))
                                        : "memory");
        }
        if (ok) {
            // the small corrections, accumulated in TMEM over the whole tile (the
            // last acc_full arrival follows every MMA of the tile)
            const uint32_t ts = lanebase + (uint32_t)(kAccBufs * N);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c * 32 < N) {
                    uint32_t v[32];
                    tmem_ld32_nowait(ts + (uint32_t)(c * 32), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[c * 32 + j] += __uint_as_float(v[j]);
                }
            }
        }
        if (ok) {
            // energy dot and psi: M loads issued 16 at a time (independent), FP32
            // partial sums per thread (128 products), FP64 across threads
            const int m = row0 + warp * 32 + lane;
            const bool mrow = m < ldm;
            float e0 = 0.f, e1 = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < 128; c0 += 16) {
                if (c0 < N) {
                    float mv[16];
                    int64_t ofs[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = c0 + j;
                        const int slab = c / S, z = c % S;
                        const int zrow = blockIdx.x * R + slab;
                        const bool valid = mrow && (c < N) && (z < n) && (zrow < nrow);
                        ofs[j] = valid ? ((int64_t)zrow * n + z) * ldm + m : -1;
                        mv[j] = valid ? __ldg(&M[ofs[j]]) : 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (j & 1) e1 = fmaf(mv[j], acc[c0 + j], e1);
                        else e0 = fmaf(mv[j], acc[c0 + j], e0);
                        if (FORCES && ofs[j] >= 0) psi[ofs[j]] = acc[c0 + j];
                    }
                }
            }
            e = (double)e0 + (double)e1;
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
        part[blockIdx.y * gridDim.x + blockIdx.x] = -0.5 * (red[0] + red[1] + red[2] + red[3]);
        if (*abort_flag) atomicOr(errflag, 2);
    }
    if (warp == 5) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// host side

static bool encode_2d(CUtensorMap *map, void *ptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
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
    cuuint64_t strides[1] = {inner * sizeof(float)};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

static size_t tc_smem_bytes(int N)
{
    const size_t stage = 2 * (size_t)tcg::kABytes + 2 * (size_t)N * tcg::kKc * 4;
    return tcg::kStages * stage + 1024 + 256;
}

bool tc_prepare(Handle &H, std::string &err)
{
    H.tc.enabled = 0;
    const Geo &g = H.g;
    if (g.ldm % tcg::kKc != 0 || g.ldm > 512 || g.n > 128) return true;   // plain FP32 kernel is used
    const int S = ((g.n + 15) / 16) * 16;
    const int R = std::max(1, 128 / S);
    H.tc.S = S;
    H.tc.R = R;
    H.tc.rowstride = S + 2;
    H.tc.N = R * S;
    H.tc.tmem_cols = 32;
    while ((int)H.tc.tmem_cols < (tcg::kAccBufs + 1) * H.tc.N) H.tc.tmem_cols <<= 1;   // large buffers + small
    H.tc.tiles = (g.n * g.n + R - 1) / R;
    H.tc.halves = (g.ldm + tcg::kRows - 1) / tcg::kRows;
    const uint64_t rows = (uint64_t)g.n * g.n * H.tc.rowstride;
    const uint64_t arows = (uint64_t)H.tc.halves * tcg::kRows;
    if (!encode_2d(&H.tc.mAhi, H.d_Chi, 27 * (uint64_t)g.ldm, arows, tcg::kKc, 128, err)) return false;
    if (!encode_2d(&H.tc.mAlo, H.d_Clo, 27 * (uint64_t)g.ldm, arows, tcg::kKc, 128, err)) return false;
    if (!encode_2d(&H.tc.mBhi, H.d_Mhi, g.ldm, rows, tcg::kKc, (uint32_t)S, err)) return false;
    if (!encode_2d(&H.tc.mBlo, H.d_Mlo, g.ldm, rows, tcg::kKc, (uint32_t)S, err)) return false;
    const size_t smem = tc_smem_bytes(H.tc.N);
    if (cudaFuncSetAttribute(k_corr_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_corr_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        err = "cudaFuncSetAttribute (shared memory) failed";
        return false;
    }
    H.tc.enabled = 1;
    return true;
}

int corr_tc_blocks(const Handle &H) { return H.tc.tiles * H.tc.halves; }

cudaError_t launch_corr_tc(Handle &H, bool forces, cudaStream_t s)
{
    const size_t smem = tc_smem_bytes(H.tc.N);
    double *part = H.d_part + H.part_off[kPartCorr];
    const dim3 grid(H.tc.tiles, H.tc.halves);
    if (forces)
        k_corr_tc<true><<<grid, tcg::kThreads, smem, s>>>(H.tc.mAhi, H.tc.mAlo, H.tc.mBhi, H.tc.mBlo, H.g,
                                                                H.tc.S, H.tc.R, H.tc.rowstride, H.tc.tmem_cols,
                                                                H.d_M, H.d_psi, part, H.d_flag);
    else
        k_corr_tc<false><<<grid, tcg::kThreads, smem, s>>>(H.tc.mAhi, H.tc.mAlo, H.tc.mBhi, H.tc.mBlo, H.g,
                                                                 H.tc.S, H.tc.R, H.tc.rowstride, H.tc.tmem_cols,
                                                                 H.d_M, H.d_psi, part, H.d_flag);
    return cudaGetLastError();
}

}  // namespace ankh
