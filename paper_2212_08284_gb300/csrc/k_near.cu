// Near field of ANKH (Alg. 5 step 3; Sec. 3.2 N_real): every pair of atoms in
// the same or in adjacent leaves (26 neighbours, periodic, one image per
// offset), kernel H = erfc(xi r)/r, with the full multipole operator
//   e_ik = (q_i + mu_i.grad + Theta_i:grad grad) V_k(r),   r = x_i - x_k,
//   V_k(r) = (q_k - mu_k.grad + Theta_k:grad grad) H(r),
//   N_real = 1/2 sum_i sum_k e_ik.
//
// Source-field formulation: each target i accumulates, over all its near
// sources k, the potential V_k and its first two derivatives,
//   V, dV_a, G_ab = d_a d_b V,
// which depend on the source's multipoles only, and the quadrupole part of
// its force, F_c = sum_ab Theta_i,ab T_abc with T_abc = d_a d_b d_c V
// (contracted per pair, cheaper than accumulating the ten T_abc).  The rest
// of the target's multipoles enter once per atom at the end:
//   e_i = q_i V + mu_i.dV + Theta_i:G,       dE/dq_i = V, dE/dmu_i = dV,
//   dE/dTheta_i = G (stored-entry convention),
//   dE/dx_i = q_i dV + mu_i.G + F.
// With B_0 = H, B_l = -(1/r) dB_{l-1}/dr (upward recurrence
// B_l = [(2l-1) B_{l-1} + (2 xi^2)^l exp(-xi^2 r^2)/(xi sqrt(pi))]/r^2) and
// s = mu_k.r - tr Theta_k, u = r.Theta_k.r, Q = Theta_k r:
//   V    = q B0 + s B1 + u B2
//   A    = -(q B1 + s B2 + u B3),  A2 = q B2 + s B3 + u B4,  A3 = q B3 + s B4 + u B5
//   dV_a = mu_a B1 + 2 Q_a B2 + r_a A
//   G_ab = delta_ab A + r_a r_b A2 - (r_a P_b + r_b P_a) + 2 Theta_ab B2,   P = mu B2 + 2 Q B3
//   T_abc = sym3(delta_ab W_c) - r_a r_b r_c A3 + sym3(r_a r_b Z_c) - sym3(Y_ab r_c),
//           W = r A2 - mu B2 - 2 Q B3,  Z = mu B3 + 2 Q B4,  Y = 2 B3 Theta_k
// (sym3 sums the three distinct placements of the index pair), so with
// R = Theta_i r, u_i = r.R:
//   F = tr(Theta_i) W + 2 Theta_i W + u_i (Z - r A3) + r (2 R.Z - Theta_i:Y) - 2 Y R.
//
// Work layout: one warp per work item, an item being up to 32 targets of one
// leaf (the leaf-count scan lays the items out in leaf order, so a leaf with
// many atoms is spread over many warps).  The atoms of the 27 leaves around
// it are staged in shared memory (chunks of 64, coordinates shifted by the
// leaf offset); the warp's lanes are split into G = 32 / n_t groups, lane
// (i, g) accumulating target i over sources g, g + G, ...; the group partials
// are summed in a fixed order.  Every output is written by exactly one lane:
// no atomics, deterministic results.  Zero-distance pairs are counted per
// target; a count other than one (two atoms at one position, where the
// energy is infinite) sets bit 4 of the error flag.
#include "ankh_internal.cuh"

#include <algorithm>
#include <vector>

namespace ankh {


// How B0 = erfc(xi r)/r is evaluated (chosen per launch from xi * r_max, r_max
// the largest distance between atoms of adjacent leaves):
//   kErfcLib    erfcf (any xi r)
//   kSeriesLong 8 terms of the series (xi r_max <= 0.5; the next term is
//               below 2e-11 of B0)
//   kSeriesShort 4 terms (xi r_max <= 0.2; the next term is below 3e-9 of B0)
enum { kErfcLib = 0, kSeriesLong = 1, kSeriesShort = 2 };

// One warp per block: a block's energy partial waits for all its warps, and
// with several warps a warp that drew light items sat at that barrier holding
// its slot (four-warp blocks: 12 % of the warp slots parked there); a
// one-warp block frees its slot the moment its items are done.
constexpr int kNearWarps = 1;
constexpr int kNearChunk = 64;
// Items per warp: the launch covers the largest possible item count with
// max_items / (k kNearWarps) blocks, which the hardware hands to the SMs as
// earlier blocks retire.  A persistent grid (a fixed share of leaves per
// warp) left the SMs idle at the end, waiting for the warps that drew the
// heaviest leaves.  k = 4 where that still gives at least kNearMinWaves
// waves of resident blocks (fewer blocks, fewer energy partials), else 2 or
// 1, so that a box of some ten thousand atoms still fills every SM.
constexpr int kNearMaxItemsPerWarp = 4;
constexpr int kNearBlocksPerSM = 28;   // resident one-warp blocks (<= 73 registers per thread)
constexpr int kNearMinWaves = 8;

template <bool FORCES>
struct NAcc {
    static constexpr int K = FORCES ? 13 : 10;   // V, dV(3), G(6) [, F(3)]
};

struct TgtQ {
    float xx, xy, xz, yy, yz, zz;       // target quadrupole Theta_i
    float wxx, wxy, wxz, wyy, wyz, wzz; // 2 Theta_i + tr(Theta_i) 1
};

// A pair at zero distance (the target itself; two distinct atoms at one
// position are counted in nzero and reported by the caller) contributes 0:
// rinv and B0 are selected to 0, which zeroes every B_l.
template <bool FORCES, int MODE>
__device__ __forceinline__ void src_fields(float rx, float ry, float rz, const float4 s0, const float4 s1,
                                           const float4 s2, const float4 s3, const BCoef &bc, const TgtQ &T,
                                           float (&acc)[NAcc<FORCES>::K], int &nzero)
{
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    const bool zero = r2 == 0.f;
    nzero += zero ? 1 : 0;
    // rsqrtf (hardware approximation) refined by one Newton step: its error is
    // one-sided, and the pair sums of a water box cancel strongly enough to
    // turn it into a visible bias (2.5e-7 of E before, 3e-9 after)
    float y0 = rsqrtf(r2);
    y0 = y0 * fmaf(-0.5f * r2, y0 * y0, 1.5f);
    const float rinv = zero ? 0.f : y0;
    const float ri2 = rinv * rinv;
    const float y = bc.kap * r2;
    const float ex = exp2f(-y);
    float B0;
    if (MODE == kErfcLib) {
        B0 = erfcf(bc.xi * (r2 * rinv)) * rinv;   // 0 when rinv = 0
    } else {
        constexpr int NT = (MODE == kSeriesShort) ? 4 : 8;
        float p = bc.a[NT - 1];
#pragma unroll
        for (int k = NT - 2; k >= 0; --k) p = fmaf(p, y, bc.a[k]);
        B0 = zero ? 0.f : rinv - p;
    }
    const float B1 = fmaf(bc.c1, ex, B0) * ri2;
    const float B2 = fmaf(bc.c2, ex, 3.f * B1) * ri2;
    const float B3 = fmaf(bc.c3, ex, 5.f * B2) * ri2;
    const float B4 = fmaf(bc.c4, ex, 7.f * B3) * ri2;
    // source multipoles: s0 = (x, y, z, q), s1 = (mu, tr Theta), s2 = (xx, xy, xz, yy), s3 = (yz, zz, -, -)
    const float q = s0.w, mx = s1.x, my = s1.y, mz = s1.z;
    const float txx = s2.x, txy = s2.y, txz = s2.z, tyy = s2.w, tyz = s3.x, tzz = s3.y;
    const float Qx = fmaf(txz, rz, fmaf(txy, ry, txx * rx));
    const float Qy = fmaf(tyz, rz, fmaf(tyy, ry, txy * rx));
    const float Qz = fmaf(tzz, rz, fmaf(tyz, ry, txz * rx));
    const float s = fmaf(mz, rz, fmaf(my, ry, fmaf(mx, rx, -s1.w)));
    const float u = fmaf(rz, Qz, fmaf(ry, Qy, rx * Qx));
    const float nA = fmaf(u, B3, fmaf(s, B2, q * B1));      // -A
    const float A2 = fmaf(u, B4, fmaf(s, B3, q * B2));
    acc[0] = fmaf(u, B2, fmaf(s, B1, fmaf(q, B0, acc[0])));
    const float twoB2 = 2.f * B2;
    acc[1] = fmaf(-rx, nA, fmaf(twoB2, Qx, fmaf(mx, B1, acc[1])));
    acc[2] = fmaf(-ry, nA, fmaf(twoB2, Qy, fmaf(my, B1, acc[2])));
    acc[3] = fmaf(-rz, nA, fmaf(twoB2, Qz, fmaf(mz, B1, acc[3])));
    const float twoB3 = 2.f * B3;
    const float Px = fmaf(twoB3, Qx, mx * B2), Py = fmaf(twoB3, Qy, my * B2), Pz = fmaf(twoB3, Qz, mz * B2);
    const float Wx = fmaf(rx, A2, -Px), Wy = fmaf(ry, A2, -Py), Wz = fmaf(rz, A2, -Pz);
    // G_ab = delta_ab A + r_a W_b - r_b P_a + 2 B2 Theta_ab  (= delta A + r r A2 - r P - P r + 2 B2 Theta)
    acc[4] = fmaf(twoB2, txx, fmaf(-rx, Px, fmaf(rx, Wx, acc[4] - nA)));
    acc[5] = fmaf(twoB2, txy, fmaf(-ry, Px, fmaf(rx, Wy, acc[5])));
    acc[6] = fmaf(twoB2, txz, fmaf(-rz, Px, fmaf(rx, Wz, acc[6])));
    acc[7] = fmaf(twoB2, tyy, fmaf(-ry, Py, fmaf(ry, Wy, acc[7] - nA)));
    acc[8] = fmaf(twoB2, tyz, fmaf(-rz, Py, fmaf(ry, Wz, acc[8])));
    acc[9] = fmaf(twoB2, tzz, fmaf(-rz, Pz, fmaf(rz, Wz, acc[9] - nA)));
    if (FORCES) {
        const float B5 = fmaf(bc.c5, ex, 9.f * B4) * ri2;
        const float A3 = fmaf(u, B5, fmaf(s, B4, q * B3));
        const float twoB4 = 2.f * B4;
        const float Zx = fmaf(twoB4, Qx, mx * B3), Zy = fmaf(twoB4, Qy, my * B3), Zz = fmaf(twoB4, Qz, mz * B3);
        // R = Theta_i r, u_i = r.R, K R = Theta_k R, Theta_i : Theta_k
        const float Rx = fmaf(T.xz, rz, fmaf(T.xy, ry, T.xx * rx));
        const float Ry = fmaf(T.yz, rz, fmaf(T.yy, ry, T.xy * rx));
        const float Rz = fmaf(T.zz, rz, fmaf(T.yz, ry, T.xz * rx));
        const float ui = fmaf(rz, Rz, fmaf(ry, Ry, rx * Rx));
        const float KRx = fmaf(txz, Rz, fmaf(txy, Ry, txx * Rx));
        const float KRy = fmaf(tyz, Rz, fmaf(tyy, Ry, txy * Rx));
        const float KRz = fmaf(tzz, Rz, fmaf(tyz, Ry, txz * Rx));
        const float TK = fmaf(T.wyz, tyz, fmaf(T.wxz, txz, fmaf(T.wxy, txy,
                         fmaf(T.zz, tzz, fmaf(T.yy, tyy, T.xx * txx)))));
        const float RZ = fmaf(Rz, Zz, fmaf(Ry, Zy, Rx * Zx));
        const float sc = fmaf(2.f, RZ, -fmaf(ui, A3, twoB3 * TK));   // 2 R.Z - Theta_i:Y - u_i A3
        const float m4B3 = -2.f * twoB3;
        // F = (2 Theta_i + tr Theta_i) W + u_i Z + r sc - 4 B3 Theta_k R
        acc[10] = fmaf(m4B3, KRx, fmaf(rx, sc, fmaf(ui, Zx, fmaf(T.wxz, Wz, fmaf(T.wxy, Wy, fmaf(T.wxx, Wx, acc[10]))))));
        acc[11] = fmaf(m4B3, KRy, fmaf(ry, sc, fmaf(ui, Zy, fmaf(T.wyz, Wz, fmaf(T.wyy, Wy, fmaf(T.wxy, Wx, acc[11]))))));
        acc[12] = fmaf(m4B3, KRz, fmaf(rz, sc, fmaf(ui, Zz, fmaf(T.wzz, Wz, fmaf(T.wyz, Wy, fmaf(T.wxz, Wx, acc[12]))))));
    }
}

// What the near field of one box needs (the single-box launch passes it by
// value; the batched launch reads one per box from device memory).
struct NearBox {
    int n, nonperiodic;
    float hf, hf_lo;                 // leaf edge as FP32 hi + lo
    const int *start;
    const int2 *items;
    const int *nitems;
    const float4 *A0, *A1, *A2, *A3;
    float *gnear;
    int64_t Nslot;
    double *part;
    int *flag;
};

// Block lb of nblocks working on box a (the item loop strides over the box's
// blocks); the energy partial of the block goes to a.part[lb].
template <bool FORCES, int MODE>
__device__ __forceinline__ void near_block(const NearBox &a, const BCoef &bc, int lb, int nblocks)
{
    const int *__restrict__ start = a.start;
    const int2 *__restrict__ items = a.items;
    const float4 *__restrict__ A0 = a.A0;
    const float4 *__restrict__ A1 = a.A1;
    const float4 *__restrict__ A2 = a.A2;
    const float4 *__restrict__ A3 = a.A3;
    float *__restrict__ gnear = a.gnear;
    const int64_t Nslot = a.Nslot;
    int *__restrict__ flag = a.flag;
    const int nonperiodic = a.nonperiodic;
    constexpr int K = NAcc<FORCES>::K;
    __shared__ float4 sSrc[kNearWarps][kNearChunk][4];
    __shared__ int sBeg[kNearWarps][28], sPre[kNearWarps][32];
    __shared__ float sRed[kNearWarps][K][32];
    __shared__ int sZero[kNearWarps][32];
    __shared__ double sE[kNearWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = a.n;
    const float h = a.hf, hlo = a.hf_lo;
    double ew = 0.0;
    const int nit = *a.nitems;
    for (int it = lb * kNearWarps + warp; it < nit; it += nblocks * kNearWarps) {
        const int2 item = items[it];
        const int t = item.x, t0 = item.y;
        const int tb = start[t], nt_all = start[t + 1] - tb;
        const int cx = t / (n * n), cy = (t / n) % n, cz = t % n;
        // neighbour leaves: begin offsets and exclusive prefix of their counts
        int cnt = 0, beg = 0;
        if (lane < 27) {
            const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
            const int ax = cx + dx, ay = cy + dy, az = cz + dz;
            // non-periodic box: leaves beyond its faces do not exist
            const bool inside = !nonperiodic || (ax >= 0 && ax < n && ay >= 0 && ay < n && az >= 0 && az < n);
            if (inside) {
                const int nc = (((ax + n) % n) * n + (ay + n) % n) * n + (az + n) % n;
                beg = start[nc];
                cnt = start[nc + 1] - beg;
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int ns = __shfl_sync(0xffffffffu, incl, 26);
        if (lane < 27) {
            sBeg[warp][lane] = beg;
            sPre[warp][lane] = incl - cnt;
        }
        if (lane >= 27) sPre[warp][lane] = ns;
        __syncwarp();
        {
            const int nt = min(32, nt_all - t0);
            const int G = 32 / nt;
            const int il = lane % nt, grp = lane / nt;
            const bool active = grp < G;
            const int si = tb + t0 + il;
            const float4 ti = A0[si];
            TgtQ TQ;
            {
                const float4 t2 = A2[si], t3 = A3[si];
                TQ.xx = t2.x; TQ.xy = t2.y; TQ.xz = t2.z; TQ.yy = t2.w; TQ.yz = t3.x; TQ.zz = t3.y;
                const float tr = t2.x + t2.w + t3.y;
                TQ.wxx = fmaf(2.f, t2.x, tr); TQ.wyy = fmaf(2.f, t2.w, tr); TQ.wzz = fmaf(2.f, t3.y, tr);
                TQ.wxy = 2.f * t2.y; TQ.wxz = 2.f * t2.z; TQ.wyz = 2.f * t3.x;
            }
            float acc[K];
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = 0.f;
            int nzero = 0;
            for (int c0 = 0; c0 < ns; c0 += kNearChunk) {
                const int cs = min(kNearChunk, ns - c0);
                __syncwarp();
                for (int k = lane; k < cs; k += 32) {
                    const int f = c0 + k;
                    // leaf d with sPre[d] <= f < sPre[d+1]: five fixed halving steps
                    // over the prefixes, padded to 32 entries with ns (> f)
                    int d = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) d += sPre[warp][d + st] <= f ? st : 0;
                    const int slot = sBeg[warp][d] + (f - sPre[warp][d]);
                    float4 a0 = A0[slot];
                    const float4 a1 = A1[slot], a2 = A2[slot], a3 = A3[slot];
                    // shift into the target leaf's frame by d h with the FP64 leaf
                    // edge carried as hf + hf_lo (an FP32 h alone would bias every
                    // cross-leaf distance the same way)
                    const float sx = (float)(d / 9 - 1), sy = (float)((d / 3) % 3 - 1), sz = (float)(d % 3 - 1);
                    a0.x = fmaf(sx, h, a0.x) + sx * hlo;
                    a0.y = fmaf(sy, h, a0.y) + sy * hlo;
                    a0.z = fmaf(sz, h, a0.z) + sz * hlo;
                    sSrc[warp][k][0] = a0;
                    sSrc[warp][k][1] = make_float4(a1.x, a1.y, a1.z, a2.x + a2.w + a3.y);
                    sSrc[warp][k][2] = a2;
                    sSrc[warp][k][3] = a3;
                }
                __syncwarp();
                if (active) {
#pragma unroll 1
                    for (int k = grp; k < cs; k += G) {
                        const float4 s0 = sSrc[warp][k][0];
                        src_fields<FORCES, MODE>(ti.x - s0.x, ti.y - s0.y, ti.z - s0.z, s0, sSrc[warp][k][1],
                                                 sSrc[warp][k][2], sSrc[warp][k][3], bc, TQ, acc, nzero);
                    }
                }
            }
            // sum the group partials of each target in a fixed order
            __syncwarp();
#pragma unroll
            for (int k = 0; k < K; ++k) sRed[warp][k][lane] = active ? acc[k] : 0.f;
            sZero[warp][lane] = active ? nzero : 0;
            __syncwarp();
            if (lane < nt) {
                // exactly one zero-distance pair (the target itself) is expected
                int z = sZero[warp][lane];
                for (int gq = 1; gq < G; ++gq) z += sZero[warp][lane + gq * nt];
                if (z != 1) atomicOr(flag, 4);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    float v = sRed[warp][k][lane];
                    for (int gq = 1; gq < G; ++gq) v += sRed[warp][k][lane + gq * nt];
                    acc[k] = v;
                }
                const float4 a1 = A1[si], a2 = A2[si], a3 = A3[si];
                const float q = ti.w, mx = a1.x, my = a1.y, mz = a1.z;
                const float txx = a2.x, txy = a2.y, txz = a2.z, tyy = a2.w, tyz = a3.x, tzz = a3.y;
                // e_i = q V + mu.dV + Theta:G
                const float ei = q * acc[0] + mx * acc[1] + my * acc[2] + mz * acc[3] + txx * acc[4] +
                                 tyy * acc[7] + tzz * acc[9] + 2.f * (txy * acc[5] + txz * acc[6] + tyz * acc[8]);
                ew += 0.5 * (double)ei;
                if (FORCES) {
                    const int64_t S = Nslot;
                    // dE/dx = q dV + mu.G + F
                    const float Gm[3][3] = {{acc[4], acc[5], acc[6]}, {acc[5], acc[7], acc[8]}, {acc[6], acc[8], acc[9]}};
                    const float mu[3] = {mx, my, mz};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float f = q * acc[1 + c] + mu[0] * Gm[0][c] + mu[1] * Gm[1][c] + mu[2] * Gm[2][c]
                                      + acc[10 + c];
                        gnear[(int64_t)c * S + si] = f;
                    }
                    gnear[3 * S + si] = acc[0];
                    gnear[4 * S + si] = acc[1];
                    gnear[5 * S + si] = acc[2];
                    gnear[6 * S + si] = acc[3];
                    gnear[7 * S + si] = acc[4];
                    gnear[8 * S + si] = 2.f * acc[5];
                    gnear[9 * S + si] = 2.f * acc[6];
                    gnear[10 * S + si] = acc[7];
                    gnear[11 * S + si] = 2.f * acc[8];
                    gnear[12 * S + si] = acc[9];
                }
            }
        }
    }
    // fixed-order block reduction of the energy
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ew += __shfl_down_sync(0xffffffffu, ew, o);
    if (lane == 0) sE[warp] = ew;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < kNearWarps; ++w) u += sE[w];
        a.part[lb] = u;
    }
}

template <bool FORCES, int MODE>
__global__ void __launch_bounds__(kNearWarps * 32, kNearBlocksPerSM) k_near(const __grid_constant__ NearBox a, BCoef bc)
{
    near_block<FORCES, MODE>(a, bc, blockIdx.x, gridDim.x);
}

// All the boxes of a batch in one launch: box b owns blocks
// [block0[b], block0[b + 1]) (the boxes are laid out in order of decreasing
// cost, so the largest start first); every box keeps its own items, energy
// partials and gradients.  All boxes of one launch share xi (bc) and the
// B0 evaluation.
template <bool FORCES, int MODE>
__global__ void __launch_bounds__(kNearWarps * 32, kNearBlocksPerSM)
k_near_batch(const NearBox *__restrict__ boxes, const int *__restrict__ block0, int nbox, BCoef bc)
{
    __shared__ int sbox;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nbox;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (block0[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid;
        }
        sbox = lo;
    }
    __syncthreads();
    const int b = sbox;
    near_block<FORCES, MODE>(boxes[b], bc, (int)blockIdx.x - block0[b], block0[b + 1] - block0[b]);
}

int near_blocks(const Handle &H)
{
    const int64_t wave = (int64_t)kNearBlocksPerSM * H.sm_count;
    int k = kNearMaxItemsPerWarp;
    while (k > 1 && ((int64_t)H.max_items + kNearWarps * k - 1) / (kNearWarps * k) < kNearMinWaves * wave) k >>= 1;
    const int per_block = kNearWarps * k;
    return (H.max_items + per_block - 1) / per_block;
}

static BCoef near_coef(double xi)
{
    BCoef bc;
    const double log2e = 1.4426950408889634;
    bc.xi = (float)xi;
    bc.kap = (float)(xi * xi * log2e);
    // screening coefficients; all zero for the bare kernel (xi = 0, non-periodic):
    // B0 = 1/r and B_l = (2l - 1) B_{l-1} / r^2
    double cl[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double c = xi > 0.0 ? 1.0 / (xi * sqrt(M_PI)) : 0.0;
    for (int l = 1; l <= 5; ++l) {
        c *= 2.0 * xi * xi;
        cl[l] = c;
    }
    bc.c1 = (float)cl[1]; bc.c2 = (float)cl[2]; bc.c3 = (float)cl[3]; bc.c4 = (float)cl[4]; bc.c5 = (float)cl[5];
    // erf(z) = (2/sqrt(pi)) sum_k (-1)^k z^(2k+1) / (k! (2k+1))  (Maclaurin series), z = xi r,
    // so erf(xi r)/r = sum_k a_k y^k with y = xi^2 r^2 log2(e)
    double fact = 1.0, l2k = 1.0;
    for (int k = 0; k < 8; ++k) {
        if (k > 0) {
            fact *= k;
            l2k *= log2e;
        }
        bc.a[k] = (float)((k % 2 ? -1.0 : 1.0) * 2.0 * xi / sqrt(M_PI) / (fact * (2 * k + 1) * l2k));
    }
    return bc;
}

int near_mode(const Handle &H)
{
    const double zmax = H.g.xi * 2.0 * sqrt(3.0) * H.g.h;   // xi times the farthest pair of adjacent leaves
    return zmax <= 0.2 ? kSeriesShort : (zmax <= 0.5 ? kSeriesLong : kErfcLib);
}

static NearBox near_box(const Handle &H)
{
    NearBox a;
    a.n = H.g.n;
    a.nonperiodic = H.g.nonperiodic;
    a.hf = H.g.hf;
    a.hf_lo = H.g.hf_lo;
    a.start = H.d_start;
    a.items = H.d_items;
    a.nitems = H.d_nitems;
    a.A0 = H.d_A0;
    a.A1 = H.d_A1;
    a.A2 = H.d_A2;
    a.A3 = H.d_A3;
    a.gnear = H.d_gnear;
    a.Nslot = H.N;
    a.part = H.d_part + H.part_off[kPartNear];
    a.flag = H.d_flag;
    return a;
}

#define ANKH_NEAR_DISPATCH(forces, mode, LAUNCH)                         \
    do {                                                                 \
        if (forces) {                                                    \
            if (mode == kSeriesShort) LAUNCH(true, kSeriesShort);        \
            else if (mode == kSeriesLong) LAUNCH(true, kSeriesLong);     \
            else LAUNCH(true, kErfcLib);                                 \
        } else {                                                         \
            if (mode == kSeriesShort) LAUNCH(false, kSeriesShort);       \
            else if (mode == kSeriesLong) LAUNCH(false, kSeriesLong);    \
            else LAUNCH(false, kErfcLib);                                \
        }                                                                \
    } while (0)

cudaError_t launch_near(Handle &H, bool forces, cudaStream_t s)
{
    const BCoef bc = near_coef(H.g.xi);
    const NearBox a = near_box(H);
    const int mode = near_mode(H);
    const dim3 grid(near_blocks(H)), block(kNearWarps * 32);
#define ANKH_NEAR_ONE(F, M) k_near<F, M><<<grid, block, 0, s>>>(a, bc)
    ANKH_NEAR_DISPATCH(forces, mode, ANKH_NEAR_ONE);
#undef ANKH_NEAR_ONE
    return cudaGetLastError();
}

// The boxes of a batch that share xi and the B0 evaluation, in one launch.
// d_boxes / d_block0 are device arrays made by near_batch_tables.
cudaError_t launch_near_batch(const NearBatch &nb, bool forces, cudaStream_t s)
{
    if (nb.total_blocks == 0) return cudaSuccess;
    const dim3 grid(nb.total_blocks), block(kNearWarps * 32);
#define ANKH_NEAR_BATCH(F, M) k_near_batch<F, M><<<grid, block, 0, s>>>(nb.d_boxes, nb.d_block0, nb.nbox, nb.bc)
    ANKH_NEAR_DISPATCH(forces, nb.mode, ANKH_NEAR_BATCH);
#undef ANKH_NEAR_BATCH
    return cudaGetLastError();
}

// Device tables of one batched launch over the handles hs[0..nbox) (all with
// the same xi and B0 evaluation), in decreasing order of their atom counts.
bool near_batch_tables(Handle *const *hs, int nbox, NearBatch &nb, std::string &err)
{
    std::vector<int> order(nbox);
    for (int i = 0; i < nbox; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hs[x]->N > hs[y]->N; });
    std::vector<NearBox> boxes(nbox);
    std::vector<int> block0(nbox + 1, 0);
    for (int k = 0; k < nbox; ++k) {
        boxes[k] = near_box(*hs[order[k]]);
        block0[k + 1] = block0[k] + near_blocks(*hs[order[k]]);
    }
    nb.nbox = nbox;
    nb.total_blocks = block0[nbox];
    nb.mode = near_mode(*hs[0]);
    nb.bc = near_coef(hs[0]->g.xi);
    if (cudaMalloc(&nb.d_boxes, sizeof(NearBox) * nbox) != cudaSuccess ||
        cudaMalloc(&nb.d_block0, sizeof(int) * (nbox + 1)) != cudaSuccess ||
        cudaMemcpy(nb.d_boxes, boxes.data(), sizeof(NearBox) * nbox, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(nb.d_block0, block0.data(), sizeof(int) * (nbox + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "batched near-field tables";
        near_batch_free(nb);
        return false;
    }
    return true;
}

void near_batch_free(NearBatch &nb)
{
    if (nb.d_boxes) cudaFree(nb.d_boxes);
    if (nb.d_block0) cudaFree(nb.d_block0);
    nb.d_boxes = nullptr;
    nb.d_block0 = nullptr;
}

}  // namespace ankh
