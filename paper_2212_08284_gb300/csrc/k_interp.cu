// Interpolation kernels of ANKH-FFT.
//
//  * P2M (Alg. 2 fused with the Chebyshev -> equispaced re-interpolation of
//    Sec. 4.1): per atom and axis the Chebyshev polynomials T_0..T_{Lc-1}(x_hat)
//    by their recurrence, then u^(p) = W_p T with W_p = (2/h)^p E H D^p
//    (L_u x L_c, precomputed), and the ten tensor-product terms of Alg. 2
//    accumulated into the L_u^3 equispaced modified charges M_c of the leaf.
//  * Merge of the per-leaf nodes onto the periodic equispaced grid of n (L_u-1)
//    points per axis (nodes on leaf faces are shared, Fig. 4): the vector chi v
//    of Eq. fastotfft with the duplicated nodes summed.
//  * L2P: the adjoint of P2M -- from the node potentials of a leaf to
//    dE/dx, dE/dq, dE/dmu, dE/dTheta of each atom in it (Sec. 2.2: L2P is the
//    adjoint of P2M).
#include "ankh_internal.cuh"

namespace ankh {

// Basis values u^(p)_a(x_hat), p = 0..NP-1, a = 0..LU-1, for one coordinate.
// W is [4][LU][Lc] in global memory (already scaled by (2/h)^p).
template <int LU, int NP>
__device__ __forceinline__ void basis_1d(float xh, const float *__restrict__ W, int Lc,
                                         float (&u)[NP][LU])
{
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int a = 0; a < LU; ++a) u[p][a] = 0.f;
    float tm2 = 1.f, tm1 = xh;
    for (int k = 0; k < Lc; ++k) {
        float t;
        if (k == 0) t = 1.f;
        else if (k == 1) t = xh;
        else {
            t = 2.f * xh * tm1 - tm2;
            tm2 = tm1;
            tm1 = t;
        }
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int a = 0; a < LU; ++a) u[p][a] = fmaf(__ldg(&W[(p * LU + a) * Lc + k]), t, u[p][a]);
    }
}

// Same for L_c = L_u with W passed as a kernel parameter (read from the
// constant bank by the FMAs: no load instructions).
template <int LU>
struct WTab {
    float w[4 * LU * LU];   // [p][a][k]
};

template <int LU, int NP>
__device__ __forceinline__ void basis_1d_fixed(float xh, const WTab<LU> &W, float (&u)[NP][LU])
{
    float t[LU];
    t[0] = 1.f;
    if (LU > 1) t[1] = xh;
#pragma unroll
    for (int k = 2; k < LU; ++k) t[k] = 2.f * xh * t[k - 1] - t[k - 2];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int a = 0; a < LU; ++a) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < LU; ++k) v = fmaf(W.w[(p * LU + a) * LU + k], t[k], v);
            u[p][a] = v;
        }
}

template <int LU, bool FASTW, int NP>
__device__ __forceinline__ void basis_any(float xh, const float *__restrict__ W, int Lc, const WTab<LU> &Wc,
                                          float (&u)[NP][LU])
{
    if (FASTW) basis_1d_fixed<LU, NP>(xh, Wc, u);
    else basis_1d<LU, NP>(xh, W, Lc, u);
}

// One warp per leaf.  The ten terms of Alg. 2 factor by the x-derivative
// order: M[a,b,c] += sum_p ux^(p)[a] G_p[b,c] with G_0 = q uy0 uz0 + mu_y uy1 uz0
// + mu_z uy0 uz1 + Th_yy uy2 uz0 + 2 Th_yz uy1 uz1 + Th_zz uy0 uz2, G_1 = mu_x uy0 uz0
// + 2 Th_xy uy1 uz0 + 2 Th_xz uy0 uz1, G_2 = Th_xx uy0 uz0.  Each lane owns one
// (b, c) node column and all L_u values of a; per-atom data (basis values,
// multipoles) sit in shared memory and are read as broadcast float4s.
constexpr int kP2MWarps = 4;
constexpr int kP2MChunk = 16;

template <int LU>
struct P2MAtom {
    static constexpr int NX = (3 * LU + 3) / 4;       // float4s for ux^(0..2)[0..LU-1]
    float4 ux[NX];
    float4 mp[3];                                     // q mux muy muz | xx 2xy 2xz yy | 2yz zz - -
    float uy[3][LU];
    float uz[3][LU];
};

template <int LU, bool FASTW>
__global__ void __launch_bounds__(kP2MWarps * 32)
k_p2m(Geo g, const int *__restrict__ start, const float4 *__restrict__ A0,
      const float4 *__restrict__ A1, const float4 *__restrict__ A2, const float4 *__restrict__ A3,
      const float *__restrict__ W, const __grid_constant__ WTab<LU> Wc, float *__restrict__ M,
      unsigned *__restrict__ mmax)
{
    constexpr int P = LU * LU * LU;
    constexpr int NBC = LU * LU;
    constexpr int NPASS = (NBC + 31) / 32;
    __shared__ P2MAtom<LU> sA[kP2MWarps][kP2MChunk];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cell = blockIdx.x * kP2MWarps + warp;
    if (cell >= g.ncell) return;
    const int b = start[cell], e = start[cell + 1];
    float acc[NPASS][LU];
#pragma unroll
    for (int ps = 0; ps < NPASS; ++ps)
#pragma unroll
        for (int a = 0; a < LU; ++a) acc[ps][a] = 0.f;
    for (int c0 = b; c0 < e; c0 += kP2MChunk) {
        const int na = min(kP2MChunk, e - c0);
        __syncwarp();
        for (int it = lane; it < na * 3; it += 32) {
            const int at = it / 3, ax = it % 3;
            const float4 a0 = A0[c0 + at];
            const float l = ax == 0 ? a0.x : (ax == 1 ? a0.y : a0.z);
            float u[3][LU];
            basis_any<LU, FASTW, 3>(l * g.two_over_h, W, g.Lc, Wc, u);
            P2MAtom<LU> &rec = sA[warp][at];
            if (ax == 0) {
                float *ux = reinterpret_cast<float *>(rec.ux);
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int a = 0; a < LU; ++a) ux[p * LU + a] = u[p][a];
            } else {
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int a = 0; a < LU; ++a) (ax == 1 ? rec.uy : rec.uz)[p][a] = u[p][a];
            }
        }
        for (int at = lane; at < na; at += 32) {
            const float4 a0 = A0[c0 + at], a1 = A1[c0 + at], a2 = A2[c0 + at], a3 = A3[c0 + at];
            sA[warp][at].mp[0] = make_float4(a0.w, a1.x, a1.y, a1.z);
            sA[warp][at].mp[1] = make_float4(a2.x, 2.f * a2.y, 2.f * a2.z, a2.w);
            sA[warp][at].mp[2] = make_float4(2.f * a3.x, a3.y, 0.f, 0.f);
        }
        __syncwarp();
        for (int at = 0; at < na; ++at) {
            const P2MAtom<LU> &rec = sA[warp][at];
            const float4 m0 = rec.mp[0], m1 = rec.mp[1], m2 = rec.mp[2];
            float ux[P2MAtom<LU>::NX * 4];
#pragma unroll
            for (int k = 0; k < P2MAtom<LU>::NX; ++k) {
                const float4 v = rec.ux[k];
                ux[4 * k] = v.x; ux[4 * k + 1] = v.y; ux[4 * k + 2] = v.z; ux[4 * k + 3] = v.w;
            }
#pragma unroll
            for (int ps = 0; ps < NPASS; ++ps) {
                const int bc = lane + 32 * ps;
                if (bc < NBC) {
                    const int bb = bc / LU, cc = bc % LU;
                    const float uy0 = rec.uy[0][bb], uy1 = rec.uy[1][bb], uy2 = rec.uy[2][bb];
                    const float uz0 = rec.uz[0][cc], uz1 = rec.uz[1][cc], uz2 = rec.uz[2][cc];
                    const float y0z0 = uy0 * uz0;
                    const float G0 = m0.x * y0z0 + m0.z * uy1 * uz0 + m0.w * uy0 * uz1 + m1.w * uy2 * uz0
                                   + m2.x * uy1 * uz1 + m2.y * uy0 * uz2;
                    const float G1 = m0.y * y0z0 + m1.y * uy1 * uz0 + m1.z * uy0 * uz1;
                    const float G2 = m1.x * y0z0;
#pragma unroll
                    for (int a = 0; a < LU; ++a)
                        acc[ps][a] += ux[a] * G0 + ux[LU + a] * G1 + ux[2 * LU + a] * G2;
                }
            }
        }
    }
    float *Mrow = M + (int64_t)cell * g.ldm;
    // nodes a*LU^2 + bc: this lane's column; zero padding beyond P
    float amax = 0.f;
#pragma unroll
    for (int ps = 0; ps < NPASS; ++ps) {
        const int bc = lane + 32 * ps;
        if (bc < NBC) {
#pragma unroll
            for (int a = 0; a < LU; ++a) {
                Mrow[a * NBC + bc] = acc[ps][a];
                amax = fmaxf(amax, fabsf(acc[ps][a]));
            }
        }
    }
    for (int node = P + lane; node < g.ldm; node += 32) Mrow[node] = 0.f;
    if (mmax) {
        // max |M| for the scaling of the tensor-core operands (non-negative
        // floats order like their bit patterns)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if (lane == 0) atomicMax(mmax, __float_as_uint(amax));
    }
}

// Merged grid: rho[g] = sum of M over the (up to 8) leaf nodes at g.
// Periodic: nf = n (L_u - 1) points per axis, node 0 of leaf q is also node
// L_u - 1 of leaf q - 1 (mod n).  Non-periodic (NP): ng = n (L_u - 1) + 1
// nodes per axis written into the zero-padded FFT grid (stride nf), node 0
// of leaf q shared with leaf q - 1 only for q >= 1, and the last node
// (q = n) belongs to leaf n - 1 alone.
// Grid (ceil(ng / 128), ng, ng): x -> gz, y -> gy, z -> gx.
template <int LU, bool NP>
__global__ void __launch_bounds__(128) k_fine(Geo g, const float *__restrict__ M, float *__restrict__ rho)
{
    constexpr int Lm = LU - 1;
    const int gz = blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = g.nf, n = g.n, ldm = g.ldm;
    if (gz >= g.ng) return;
    const int gg[3] = {(int)blockIdx.z, (int)blockIdx.y, gz};
    // per axis: the (leaf, node) owners of the merged node -- the node itself
    // and, on a face, the last node of the previous leaf -- as offsets into M
    // (leaf strides n^2 ldm, n ldm, ldm; node strides LU^2, LU, 1)
    int64_t offx[2];
    int off[3][2];
    bool has[3][2];
    const int64_t cstride[3] = {(int64_t)n * n * ldm, (int64_t)n * ldm, (int64_t)ldm};
    const int nstride[3] = {LU * LU, LU, 1};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int q = gg[a] / Lm, r = gg[a] - q * Lm;
        const int qp = q == 0 ? n - 1 : q - 1;
        const int64_t o0 = q * cstride[a] + r * nstride[a], o1 = qp * cstride[a] + Lm * nstride[a];
        if (a == 0) {
            offx[0] = o0;
            offx[1] = o1;
        } else {
            off[a][0] = (int)o0;
            off[a][1] = (int)o1;
        }
        has[a][0] = true;
        has[a][1] = r == 0;
        if (NP) {
            if (r == 0 && q == 0) has[a][1] = false;             // first face: no previous leaf
            if (q == n) { has[a][0] = false; has[a][1] = true; } // last face: previous leaf only
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (has[0][i] && has[1][j] && has[2][k]) s += __ldg(&M[offx[i] + off[1][j] + off[2][k]]);
    rho[((int64_t)gg[0] * nf + gg[1]) * nf + gz] = s;
}

// L2P fused with the node potentials and the gradient assembly, one thread
// per sorted atom.  The node potentials of a leaf,
//   Pi_t[k] = phi[g(t,k)] / M - psi_t[k]
// (the merged-grid potential at the node minus the adjacent-leaf
// correction), are formed once per leaf: each warp stages them for the
// distinct leaves of its 32 atoms in shared memory (up to kL2PLeaves at a
// time, lane (a, b) writing the L_u nodes along z of its (x, y) node row).
// Each atom contracts them with its basis -- the adjoint of P2M --
//   V[p][q][r] = sum_abc Pi[a,b,c] ux^(p)[a] uy^(q)[b] uz^(r)[c],  p + q + r <= 3,
// z first, then y, then x; adds the near-field gradient, the self-term
// gradient and the k = 0 potential; forms torques and writes in the
// caller's atom order.
template <int LU>
struct L2PShape {
    static constexpr int CP = (LU + 3) & ~3;            // nodes along z, padded to float4s
    static constexpr int LEAF = LU * LU * CP;           // staged floats per leaf
    static constexpr int LEAVES = LU <= 6 ? 8 : 4;      // leaves staged per warp at a time
};

template <int LU, bool FASTW>
__global__ void __launch_bounds__(128, LU <= 5 ? 4 : 2)
k_l2p(Geo g, const int *__restrict__ scell, const int *__restrict__ perm, const float4 *__restrict__ A0,
      const float4 *__restrict__ A1, const float4 *__restrict__ A2, const float4 *__restrict__ A3,
      const float *__restrict__ W, const __grid_constant__ WTab<LU> Wc, const float *__restrict__ phi, float invM,
      const float *__restrict__ psi, const float *__restrict__ gnear, int64_t Nslot,
      const double *__restrict__ terms, float *__restrict__ dEdx, float *__restrict__ dEdq,
      float *__restrict__ dEdmu, float *__restrict__ dEdth, float *__restrict__ torque)
{
    constexpr int Lm = LU - 1, CP = L2PShape<LU>::CP, LEAF = L2PShape<LU>::LEAF, NL = L2PShape<LU>::LEAVES;
    __shared__ __align__(16) float sPi[4][NL][LEAF];
    __shared__ int sCell[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = s < Nslot;
    const int cell = active ? scell[s] : -1;
    // the warp's distinct leaves in order (slots are sorted by leaf)
    const int prev = __shfl_up_sync(0xffffffffu, cell, 1);
    const bool leader = active && (lane == 0 || cell != prev);
    const unsigned lead = __ballot_sync(0xffffffffu, leader);
    const int nl = __popc(lead);
    const int rank = __popc(lead & (0xffffffffu >> (31 - lane))) - 1;   // leaders at or below this lane, less one
    if (leader) sCell[warp][rank] = cell;
    const int n = g.n, nf = g.nf, ldm = g.ldm;
    float ux[4][LU], uy[4][LU], uz[4][LU];
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
        a0 = A0[s];
        basis_any<LU, FASTW, 4>(a0.x * g.two_over_h, W, g.Lc, Wc, ux);
        basis_any<LU, FASTW, 4>(a0.y * g.two_over_h, W, g.Lc, Wc, uy);
        basis_any<LU, FASTW, 4>(a0.z * g.two_over_h, W, g.Lc, Wc, uz);
    }
    float V[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) V[i][j][k] = 0.f;
    for (int j0 = 0; j0 < nl; j0 += NL) {
        const int nlc = min(NL, nl - j0);
        __syncwarp();
        for (int ab = lane; ab < LU * LU; ab += 32) {
            const int a = ab / LU, bb = ab - a * LU;
            for (int k = 0; k < nlc; ++k) {
                const int t = sCell[warp][j0 + k];
                const int cx = t / (n * n), cy = (t / n) - cx * n, cz = t - (t / n) * n;
                int gx = cx * Lm + a, gy = cy * Lm + bb;   // nf^3 <= 2^30: 32-bit offsets
                gx -= gx >= nf ? nf : 0;
                gy -= gy >= nf ? nf : 0;
                const float *__restrict__ prow = phi + (gx * nf + gy) * nf;
                const float *__restrict__ srow = psi + (int64_t)t * ldm + ab * LU;
                float *dst = &sPi[warp][k][ab * CP];
#pragma unroll
                for (int c = 0; c < LU; ++c) {
                    int gz = cz * Lm + c;
                    gz -= gz >= nf ? nf : 0;
                    dst[c] = fmaf(__ldg(&prow[gz]), invM, -__ldg(&srow[c]));
                }
            }
        }
        __syncwarp();
        if (active && rank >= j0 && rank < j0 + nlc) {
            const float *sp = &sPi[warp][rank - j0][0];
#pragma unroll
            for (int a = 0; a < LU; ++a) {
                float Wq[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) Wq[i][j] = 0.f;
#pragma unroll
                for (int bb = 0; bb < LU; ++bb) {
                    float pv[CP];
#pragma unroll
                    for (int c4 = 0; c4 < CP / 4; ++c4) {
                        const float4 v = *reinterpret_cast<const float4 *>(sp + (a * LU + bb) * CP + 4 * c4);
                        pv[4 * c4] = v.x;
                        pv[4 * c4 + 1] = v.y;
                        pv[4 * c4 + 2] = v.z;
                        pv[4 * c4 + 3] = v.w;
                    }
                    float Z[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        float z = 0.f;
#pragma unroll
                        for (int c = 0; c < LU; ++c) z = fmaf(pv[c], uz[r][c], z);
                        Z[r] = z;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int r = 0; r < 4 - q; ++r) Wq[q][r] = fmaf(Z[r], uy[q][bb], Wq[q][r]);
                }
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4 - p; ++q)
#pragma unroll
                        for (int r = 0; r < 4 - p - q; ++r) V[p][q][r] = fmaf(Wq[q][r], ux[p][a], V[p][q][r]);
            }
        }
    }
    if (!active) return;
    const float dcpot = (float)terms[6];
    const float xi = g.xi;
    {
        const float4 a1 = A1[s], a2 = A2[s], a3 = A3[s];
        const float q = a0.w, mx = a1.x, my = a1.y, mz = a1.z;
        const float xx = a2.x, xy = a2.y, xz = a2.z, yy = a2.w, yz = a3.x, zz = a3.y;
        const float txy2 = 2.f * xy, txz2 = 2.f * xz, tyz2 = 2.f * yz;
        float gv[13];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int ex = ax == 0, ey = ax == 1, ez = ax == 2;
            gv[ax] = q * V[ex][ey][ez] + mx * V[1 + ex][ey][ez] + my * V[ex][1 + ey][ez] + mz * V[ex][ey][1 + ez]
                   + xx * V[2 + ex][ey][ez] + txy2 * V[1 + ex][1 + ey][ez] + txz2 * V[1 + ex][ey][1 + ez]
                   + yy * V[ex][2 + ey][ez] + tyz2 * V[ex][1 + ey][1 + ez] + zz * V[ex][ey][2 + ez];
        }
        gv[3] = V[0][0][0];
        gv[4] = V[1][0][0];
        gv[5] = V[0][1][0];
        gv[6] = V[0][0][1];
        gv[7] = V[2][0][0];
        gv[8] = 2.f * V[1][1][0];
        gv[9] = 2.f * V[1][0][1];
        gv[10] = V[0][2][0];
        gv[11] = 2.f * V[0][1][1];
        gv[12] = V[0][0][2];
#pragma unroll
        for (int k = 0; k < 13; ++k) gv[k] += gnear[(int64_t)k * Nslot + s];
        // self-term gradient (Eq. ewald, general symmetric Theta) and k = 0 potential
        const float tr = xx + yy + zz;
        const float cc = xi * 0.56418958354775628f, x2 = xi * xi, x4 = x2 * x2;
        gv[3] += -cc * (2.f * q - (4.f * x2 / 3.f) * tr) + dcpot;
        gv[4] += -cc * (4.f * x2 / 3.f) * mx;
        gv[5] += -cc * (4.f * x2 / 3.f) * my;
        gv[6] += -cc * (4.f * x2 / 3.f) * mz;
        const float dg = -(4.f * x2 / 3.f) * q + (8.f * x4 / 5.f) * tr;
        const float k16 = 16.f * x4 / 5.f;
        gv[7] += -cc * (dg + k16 * xx);
        gv[8] += -cc * 2.f * k16 * xy;
        gv[9] += -cc * 2.f * k16 * xz;
        gv[10] += -cc * (dg + k16 * yy);
        gv[11] += -cc * 2.f * k16 * yz;
        gv[12] += -cc * (dg + k16 * zz);
        const int64_t ii = perm[s];
        if (dEdx) {
            dEdx[3 * ii] = gv[0];
            dEdx[3 * ii + 1] = gv[1];
            dEdx[3 * ii + 2] = gv[2];
        }
        if (dEdq) dEdq[ii] = gv[3];
        if (dEdmu) {
            dEdmu[3 * ii] = gv[4];
            dEdmu[3 * ii + 1] = gv[5];
            dEdmu[3 * ii + 2] = gv[6];
        }
        if (dEdth) {
#pragma unroll
            for (int k = 0; k < 6; ++k) dEdth[6 * ii + k] = gv[7 + k];
        }
        if (torque) {
            // tau = -(mu x g) - 2 axial(G Theta), G = dE/dTheta with each of the nine
            // entries independent (stored off-diagonal derivative / 2)
            const float gx = gv[4], gy = gv[5], gz = gv[6];
            const float G[3][3] = {{gv[7], 0.5f * gv[8], 0.5f * gv[9]},
                                   {0.5f * gv[8], gv[10], 0.5f * gv[11]},
                                   {0.5f * gv[9], 0.5f * gv[11], gv[12]}};
            const float T[3][3] = {{xx, xy, xz}, {xy, yy, yz}, {xz, yz, zz}};
            float X[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) X[a][c] = G[a][0] * T[0][c] + G[a][1] * T[1][c] + G[a][2] * T[2][c];
            torque[3 * ii] = -(my * gz - mz * gy) - 2.f * (X[2][1] - X[1][2]);
            torque[3 * ii + 1] = -(mz * gx - mx * gz) - 2.f * (X[0][2] - X[2][0]);
            torque[3 * ii + 2] = -(mx * gy - my * gx) - 2.f * (X[1][0] - X[0][1]);
        }
    }
}

#define ANKH_LU_SWITCH(LUV, ...)                                   \
    switch (LUV) {                                                 \
    case 2: { constexpr int LU = 2; __VA_ARGS__; } break;          \
    case 3: { constexpr int LU = 3; __VA_ARGS__; } break;          \
    case 4: { constexpr int LU = 4; __VA_ARGS__; } break;          \
    case 5: { constexpr int LU = 5; __VA_ARGS__; } break;          \
    case 6: { constexpr int LU = 6; __VA_ARGS__; } break;          \
    case 7: { constexpr int LU = 7; __VA_ARGS__; } break;          \
    case 8: { constexpr int LU = 8; __VA_ARGS__; } break;          \
    default: return cudaErrorInvalidValue;                         \
    }

template <int LU>
static WTab<LU> wtab(const Handle &H)
{
    WTab<LU> t;
    for (int k = 0; k < 4 * LU * LU; ++k) t.w[k] = H.h_Wf[k];
    return t;
}

cudaError_t launch_p2m(Handle &H, cudaStream_t s)
{
    // max |M| of the leaves: the fp16 split exponent of the tensor-core correction, or of the leaf level (ANKH-FMM)
    unsigned *mmax = H.fmm.enabled ? H.d_mmax + H.fmm.E : (H.tc.enabled ? H.d_mmax : nullptr);
    if (mmax) {
        const cudaError_t e = cudaMemsetAsync(mmax, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    const unsigned nb = (unsigned)((H.g.ncell + kP2MWarps - 1) / kP2MWarps);
    ANKH_LU_SWITCH(H.g.Lu,
        if (H.g.Lc == LU)
            k_p2m<LU, true><<<nb, kP2MWarps * 32, 0, s>>>(H.g, H.d_start, H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_W,
                                                          wtab<LU>(H), H.d_M, mmax);
        else
            k_p2m<LU, false><<<nb, kP2MWarps * 32, 0, s>>>(H.g, H.d_start, H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_W,
                                                           WTab<LU>{}, H.d_M, mmax));
    return cudaGetLastError();
}

cudaError_t launch_fine_gather(Handle &H, cudaStream_t s)
{
    const dim3 grid((unsigned)((H.g.ng + 127) / 128), (unsigned)H.g.ng, (unsigned)H.g.ng);
    if (H.g.nonperiodic) {
        ANKH_LU_SWITCH(H.g.Lu, k_fine<LU, true><<<grid, 128, 0, s>>>(H.g, H.d_M, H.d_rho));
    } else {
        ANKH_LU_SWITCH(H.g.Lu, k_fine<LU, false><<<grid, 128, 0, s>>>(H.g, H.d_M, H.d_rho));
    }
    return cudaGetLastError();
}

template <int LU>
static cudaError_t l2p_one(Handle &H, float *dEdx, float *dEdq, float *dEdmu, float *dEdtheta, float *torque,
                           cudaStream_t s)
{
    constexpr int P = LU * LU * LU;
    const float invM = (float)(1.0 / (double)H.g.M);
    (void)P;
    const unsigned nb = (unsigned)((H.N + 127) / 128);
    if (H.g.Lc == LU)
        k_l2p<LU, true><<<nb, 128, 0, s>>>(H.g, H.d_scell, H.d_perm, H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_W,
                                           wtab<LU>(H), H.d_phi, invM, H.d_psi, H.d_gnear, H.N, H.d_terms, dEdx,
                                           dEdq, dEdmu, dEdtheta, torque);
    else
        k_l2p<LU, false><<<nb, 128, 0, s>>>(H.g, H.d_scell, H.d_perm, H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_W,
                                            WTab<LU>{}, H.d_phi, invM, H.d_psi, H.d_gnear, H.N, H.d_terms, dEdx,
                                            dEdq, dEdmu, dEdtheta, torque);
    return cudaGetLastError();
}

cudaError_t launch_l2p(Handle &H, float *dEdx, float *dEdq, float *dEdmu, float *dEdtheta, float *torque,
                       cudaStream_t s)
{
    ANKH_LU_SWITCH(H.g.Lu, return l2p_one<LU>(H, dEdx, dEdq, dEdmu, dEdtheta, torque, s));
    return cudaSuccess;
}

}  // namespace ankh
