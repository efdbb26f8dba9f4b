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
// Work layout: one warp per target leaf.  The atoms of the 27 leaves around
// it are staged in shared memory (chunks of 64, coordinates shifted by the
// leaf offset); the warp's lanes are split into G = 32 / n_t groups, lane
// (i, g) accumulating target i over sources g, g + G, ...; the group partials
// are summed in a fixed order.  Every output is written by exactly one lane:
// no atomics, deterministic results.
#include "ankh_internal.cuh"

namespace ankh {

struct BCoef {
    float xi, xi2;
    float c1, c2, c3, c4, c5;   // (2 xi^2)^l / (xi sqrt(pi))
    float e[8];                 // Maclaurin coefficients of erf(x)/x in x^2
    int series;                 // use the series (xi * r_max <= 0.5)
};

constexpr int kNearWarps = 4;
constexpr int kNearChunk = 64;

template <bool FORCES>
struct NAcc {
    static constexpr int K = FORCES ? 13 : 10;   // V, dV(3), G(6) [, F(3)]
};

struct TgtQ {
    float xx, xy, xz, yy, yz, zz, tr;            // target quadrupole
};

template <bool FORCES, bool SERIES>
__device__ __forceinline__ void src_fields(float rx, float ry, float rz, const float4 s0, const float4 s1,
                                           const float4 s2, const float4 s3, const BCoef &bc, const TgtQ &T,
                                           float (&acc)[NAcc<FORCES>::K])
{
    const float r2 = rx * rx + ry * ry + rz * rz;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float ri2 = rinv * rinv;
    const float ex = __expf(-bc.xi2 * r2);
    float B0;
    if (SERIES) {
        const float x = bc.xi * r, x2 = x * x;
        float p = bc.e[7];
#pragma unroll
        for (int k = 6; k >= 0; --k) p = fmaf(p, x2, bc.e[k]);
        B0 = fmaf(-x, p, 1.f) * rinv;
    } else {
        B0 = erfcf(bc.xi * r) * rinv;
    }
    const float B1 = fmaf(bc.c1, ex, B0) * ri2;
    const float B2 = fmaf(bc.c2, ex, 3.f * B1) * ri2;
    const float B3 = fmaf(bc.c3, ex, 5.f * B2) * ri2;
    const float B4 = fmaf(bc.c4, ex, 7.f * B3) * ri2;
    // source multipoles: s0 = (x, y, z, q), s1 = (mu, tr Theta), s2 = (xx, xy, xz, yy), s3 = (yz, zz, -, -)
    const float q = s0.w, mx = s1.x, my = s1.y, mz = s1.z;
    const float txx = s2.x, txy = s2.y, txz = s2.z, tyy = s2.w, tyz = s3.x, tzz = s3.y;
    const float Qx = txx * rx + txy * ry + txz * rz;
    const float Qy = txy * rx + tyy * ry + tyz * rz;
    const float Qz = txz * rx + tyz * ry + tzz * rz;
    const float s = mx * rx + my * ry + mz * rz - s1.w;
    const float u = rx * Qx + ry * Qy + rz * Qz;
    const float A = -(q * B1 + s * B2 + u * B3);
    const float A2 = q * B2 + s * B3 + u * B4;
    acc[0] += q * B0 + s * B1 + u * B2;
    const float twoB2 = 2.f * B2;
    acc[1] += mx * B1 + twoB2 * Qx + rx * A;
    acc[2] += my * B1 + twoB2 * Qy + ry * A;
    acc[3] += mz * B1 + twoB2 * Qz + rz * A;
    const float twoB3 = 2.f * B3;
    const float Px = mx * B2 + twoB3 * Qx, Py = my * B2 + twoB3 * Qy, Pz = mz * B2 + twoB3 * Qz;
    const float rxA2 = rx * A2, ryA2 = ry * A2, rzA2 = rz * A2;
    acc[4] += A + rx * rxA2 - 2.f * rx * Px + twoB2 * txx;
    acc[5] += rx * ryA2 - (rx * Py + ry * Px) + twoB2 * txy;
    acc[6] += rx * rzA2 - (rx * Pz + rz * Px) + twoB2 * txz;
    acc[7] += A + ry * ryA2 - 2.f * ry * Py + twoB2 * tyy;
    acc[8] += ry * rzA2 - (ry * Pz + rz * Py) + twoB2 * tyz;
    acc[9] += A + rz * rzA2 - 2.f * rz * Pz + twoB2 * tzz;
    if (FORCES) {
        const float B5 = fmaf(bc.c5, ex, 9.f * B4) * ri2;
        const float A3 = q * B3 + s * B4 + u * B5;
        const float twoB4 = 2.f * B4;
        const float Wx = rxA2 - Px, Wy = ryA2 - Py, Wz = rzA2 - Pz;   // r A2 - mu B2 - 2 Q B3
        const float Zx = mx * B3 + twoB4 * Qx, Zy = my * B3 + twoB4 * Qy, Zz = mz * B3 + twoB4 * Qz;
        // R = Theta_i r, u_i = r.R
        const float Rx = T.xx * rx + T.xy * ry + T.xz * rz;
        const float Ry = T.xy * rx + T.yy * ry + T.yz * rz;
        const float Rz = T.xz * rx + T.yz * ry + T.zz * rz;
        const float ui = rx * Rx + ry * Ry + rz * Rz;
        // Theta_i W, Theta_k R, Theta_i : Theta_k
        const float TWx = T.xx * Wx + T.xy * Wy + T.xz * Wz;
        const float TWy = T.xy * Wx + T.yy * Wy + T.yz * Wz;
        const float TWz = T.xz * Wx + T.yz * Wy + T.zz * Wz;
        const float KRx = txx * Rx + txy * Ry + txz * Rz;
        const float KRy = txy * Rx + tyy * Ry + tyz * Rz;
        const float KRz = txz * Rx + tyz * Ry + tzz * Rz;
        const float TK = T.xx * txx + T.yy * tyy + T.zz * tzz + 2.f * (T.xy * txy + T.xz * txz + T.yz * tyz);
        const float sc = 2.f * (Rx * Zx + Ry * Zy + Rz * Zz) - twoB3 * TK - ui * A3;
        const float fourB3 = 2.f * twoB3;
        acc[10] += T.tr * Wx + 2.f * TWx + ui * Zx + rx * sc - fourB3 * KRx;
        acc[11] += T.tr * Wy + 2.f * TWy + ui * Zy + ry * sc - fourB3 * KRy;
        acc[12] += T.tr * Wz + 2.f * TWz + ui * Zz + rz * sc - fourB3 * KRz;
    }
}

template <bool FORCES, bool SERIES>
__global__ void __launch_bounds__(kNearWarps * 32)
k_near(Geo g, const int *__restrict__ start, const float4 *__restrict__ A0, const float4 *__restrict__ A1,
       const float4 *__restrict__ A2, const float4 *__restrict__ A3, BCoef bc, float *__restrict__ gnear,
       int64_t Nslot, double *__restrict__ part)
{
    constexpr int K = NAcc<FORCES>::K;
    __shared__ float4 sSrc[kNearWarps][kNearChunk][4];
    __shared__ int sSlot[kNearWarps][kNearChunk];
    __shared__ int sBeg[kNearWarps][28], sPre[kNearWarps][28];
    __shared__ float sRed[kNearWarps][K][32];
    __shared__ double sE[kNearWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = g.n;
    const float h = g.hf;
    double ew = 0.0;
    for (int t = blockIdx.x * kNearWarps + warp; t < g.ncell; t += gridDim.x * kNearWarps) {
        const int tb = start[t], nt_all = start[t + 1] - tb;
        if (nt_all == 0) continue;
        const int cx = t / (n * n), cy = (t / n) % n, cz = t % n;
        // neighbour leaves: begin offsets and exclusive prefix of their counts
        int cnt = 0, beg = 0;
        if (lane < 27) {
            const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
            const int nc = (((cx + dx + n) % n) * n + (cy + dy + n) % n) * n + (cz + dz + n) % n;
            beg = start[nc];
            cnt = start[nc + 1] - beg;
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
        if (lane == 27) sPre[warp][27] = ns;
        __syncwarp();
        for (int t0 = 0; t0 < nt_all; t0 += 32) {
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
                TQ.tr = t2.x + t2.w + t3.y;
            }
            float acc[K];
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = 0.f;
            for (int c0 = 0; c0 < ns; c0 += kNearChunk) {
                const int cs = min(kNearChunk, ns - c0);
                __syncwarp();
                for (int k = lane; k < cs; k += 32) {
                    const int f = c0 + k;
                    // leaf d with sPre[d] <= f < sPre[d+1]
                    int lo = 0, hi = 27;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (sPre[warp][mid] <= f) lo = mid;
                        else hi = mid;
                    }
                    const int d = lo;
                    const int slot = sBeg[warp][d] + (f - sPre[warp][d]);
                    float4 a0 = A0[slot];
                    const float4 a1 = A1[slot], a2 = A2[slot], a3 = A3[slot];
                    a0.x += (d / 9 - 1) * h;
                    a0.y += ((d / 3) % 3 - 1) * h;
                    a0.z += (d % 3 - 1) * h;
                    sSrc[warp][k][0] = a0;
                    sSrc[warp][k][1] = make_float4(a1.x, a1.y, a1.z, a2.x + a2.w + a3.y);
                    sSrc[warp][k][2] = a2;
                    sSrc[warp][k][3] = a3;
                    sSlot[warp][k] = slot;
                }
                __syncwarp();
                if (active) {
#pragma unroll 2
                    for (int k = grp; k < cs; k += G) {
                        if (sSlot[warp][k] == si) continue;
                        const float4 s0 = sSrc[warp][k][0];
                        src_fields<FORCES, SERIES>(ti.x - s0.x, ti.y - s0.y, ti.z - s0.z, s0, sSrc[warp][k][1],
                                                   sSrc[warp][k][2], sSrc[warp][k][3], bc, TQ, acc);
                    }
                }
            }
            // sum the group partials of each target in a fixed order
            __syncwarp();
#pragma unroll
            for (int k = 0; k < K; ++k) sRed[warp][k][lane] = active ? acc[k] : 0.f;
            __syncwarp();
            if (lane < nt) {
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
        part[blockIdx.x] = u;
    }
}

int near_blocks(const Handle &H)
{
    (void)H;
    return 152 * 5;
}

cudaError_t launch_near(Handle &H, bool forces, cudaStream_t s)
{
    BCoef bc;
    const double xi = H.g.xi;
    bc.xi = (float)xi;
    bc.xi2 = (float)(xi * xi);
    double c = 1.0 / (xi * sqrt(M_PI));
    double cl[6];
    for (int l = 1; l <= 5; ++l) {
        c *= 2.0 * xi * xi;
        cl[l] = c;
    }
    bc.c1 = (float)cl[1]; bc.c2 = (float)cl[2]; bc.c3 = (float)cl[3]; bc.c4 = (float)cl[4]; bc.c5 = (float)cl[5];
    // erf(x) = (2/sqrt(pi)) sum_k (-1)^k x^(2k+1) / (k! (2k+1))  (Maclaurin series)
    double fact = 1.0;
    for (int k = 0; k < 8; ++k) {
        if (k > 0) fact *= k;
        bc.e[k] = (float)((k % 2 ? -1.0 : 1.0) * 2.0 / sqrt(M_PI) / (fact * (2 * k + 1)));
    }
    const double rmax = 2.0 * sqrt(3.0) * H.g.h;   // farthest pair of adjacent leaves
    bc.series = (xi * rmax <= 0.5) ? 1 : 0;
    double *part = H.d_part + H.part_off[kPartNear];
    const int nb = near_blocks(H);
    const int64_t S = H.N;
    if (forces) {
        if (bc.series)
            k_near<true, true><<<nb, kNearWarps * 32, 0, s>>>(H.g, H.d_start, H.d_A0, H.d_A1, H.d_A2, H.d_A3, bc,
                                                              H.d_gnear, S, part);
        else
            k_near<true, false><<<nb, kNearWarps * 32, 0, s>>>(H.g, H.d_start, H.d_A0, H.d_A1, H.d_A2, H.d_A3, bc,
                                                               H.d_gnear, S, part);
    } else {
        if (bc.series)
            k_near<false, true><<<nb, kNearWarps * 32, 0, s>>>(H.g, H.d_start, H.d_A0, H.d_A1, H.d_A2, H.d_A3, bc,
                                                               H.d_gnear, S, part);
        else
            k_near<false, false><<<nb, kNearWarps * 32, 0, s>>>(H.g, H.d_start, H.d_A0, H.d_A1, H.d_A2, H.d_A3,
                                                                bc, H.d_gnear, S, part);
    }
    return cudaGetLastError();
}

}  // namespace ankh
