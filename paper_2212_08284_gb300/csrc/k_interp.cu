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

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int LU>
__global__ void __launch_bounds__(((LU * LU * LU + 31) / 32) * 32)
k_p2m(Geo g, const int *__restrict__ start, const float4 *__restrict__ A0,
      const float4 *__restrict__ A1, const float4 *__restrict__ A2, const float4 *__restrict__ A3,
      const float *__restrict__ W, float *__restrict__ M, float *__restrict__ Mhi, float *__restrict__ Mlo,
      int rowstride)
{
    constexpr int P = LU * LU * LU;
    constexpr int CH = 32;
    __shared__ float sU[CH][3][3][LU];
    __shared__ float sMp[CH][10];
    const int cell = blockIdx.x;
    const int b = start[cell], e = start[cell + 1];
    const int node = threadIdx.x;
    const int na_ = node / (LU * LU), nb_ = (node / LU) % LU, nc_ = node % LU;
    float acc = 0.f;
    for (int c0 = b; c0 < e; c0 += CH) {
        const int na = min(CH, e - c0);
        __syncthreads();
        for (int it = threadIdx.x; it < na * 3; it += blockDim.x) {
            const int at = it / 3, ax = it % 3;
            const float4 a0 = A0[c0 + at];
            const float l = ax == 0 ? a0.x : (ax == 1 ? a0.y : a0.z);
            float u[3][LU];
            basis_1d<LU, 3>(l * g.two_over_h, W, g.Lc, u);
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int a = 0; a < LU; ++a) sU[at][ax][p][a] = u[p][a];
        }
        for (int at = threadIdx.x; at < na; at += blockDim.x) {
            const float4 a0 = A0[c0 + at], a1 = A1[c0 + at], a2 = A2[c0 + at], a3 = A3[c0 + at];
            sMp[at][0] = a0.w;
            sMp[at][1] = a1.x; sMp[at][2] = a1.y; sMp[at][3] = a1.z;
            sMp[at][4] = a2.x; sMp[at][5] = 2.f * a2.y; sMp[at][6] = 2.f * a2.z;
            sMp[at][7] = a2.w; sMp[at][8] = 2.f * a3.x; sMp[at][9] = a3.y;
        }
        __syncthreads();
        if (node < P) {
            for (int at = 0; at < na; ++at) {
                const float ux0 = sU[at][0][0][na_], ux1 = sU[at][0][1][na_], ux2 = sU[at][0][2][na_];
                const float uy0 = sU[at][1][0][nb_], uy1 = sU[at][1][1][nb_], uy2 = sU[at][1][2][nb_];
                const float uz0 = sU[at][2][0][nc_], uz1 = sU[at][2][1][nc_], uz2 = sU[at][2][2][nc_];
                const float *m = sMp[at];
                // terms of Alg. 2 grouped by the x-derivative order
                float g0 = m[0] * uy0 * uz0 + m[2] * uy1 * uz0 + m[3] * uy0 * uz1
                         + m[7] * uy2 * uz0 + m[8] * uy1 * uz1 + m[9] * uy0 * uz2;
                float g1 = m[1] * uy0 * uz0 + m[5] * uy1 * uz0 + m[6] * uy0 * uz1;
                float g2 = m[4] * uy0 * uz0;
                acc += ux0 * g0 + ux1 * g1 + ux2 * g2;
            }
        }
    }
    if (node < g.ldm) {
        const float v = node < P ? acc : 0.f;
        M[(int64_t)cell * g.ldm + node] = v;
        if (Mhi) {
            // split for the tensor-core correction: rows of each z-row with a one-leaf halo
            const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
            const int n = g.n;
            const int cz = cell % n, zr = cell / n;
            const int64_t base = (int64_t)zr * rowstride;
            Mhi[(base + 1 + cz) * g.ldm + node] = hi;
            Mlo[(base + 1 + cz) * g.ldm + node] = lo;
            if (cz == n - 1) {
                Mhi[base * g.ldm + node] = hi;
                Mlo[base * g.ldm + node] = lo;
            }
            if (cz == 0) {
                Mhi[(base + n + 1) * g.ldm + node] = hi;
                Mlo[(base + n + 1) * g.ldm + node] = lo;
            }
        }
    }
}

// Merged periodic grid: rho[g] = sum of M over the (up to 8) leaf nodes at g.
__global__ void k_fine(Geo g, const float *__restrict__ M, float *__restrict__ rho)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.M) return;
    const int nf = g.nf, Lm = g.Lu - 1, n = g.n, Lu = g.Lu;
    const int gz = (int)(idx % nf), gy = (int)((idx / nf) % nf), gx = (int)(idx / ((int64_t)nf * nf));
    int oc[3][2], on[3][2], cnt[3];
    const int gg[3] = {gx, gy, gz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int q = gg[a] / Lm, r = gg[a] % Lm;
        oc[a][0] = q; on[a][0] = r; cnt[a] = 1;
        if (r == 0) {
            oc[a][1] = (q - 1 + n) % n;
            on[a][1] = Lm;
            cnt[a] = 2;
        }
    }
    float s = 0.f;
    for (int i = 0; i < cnt[0]; ++i)
        for (int j = 0; j < cnt[1]; ++j)
            for (int k = 0; k < cnt[2]; ++k) {
                const int cell = (oc[0][i] * n + oc[1][j]) * n + oc[2][k];
                const int node = (on[0][i] * Lu + on[1][j]) * Lu + on[2][k];
                s += M[(int64_t)cell * g.ldm + node];
            }
    rho[idx] = s;
}

// L2P: far-field gradient of each sorted atom from the node potentials of its leaf,
//   Pi_t[k] = phi[g(t,k)] / M - psi_t[k].
template <int LU>
__global__ void __launch_bounds__(128)
k_l2p(Geo g, int N, const int *__restrict__ scell, const float4 *__restrict__ A0,
      const float4 *__restrict__ A1, const float4 *__restrict__ A2, const float4 *__restrict__ A3,
      const float *__restrict__ W, const float *__restrict__ phi, float invM,
      const float *__restrict__ psi, float *__restrict__ gfar)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int cell = scell[s];
    const int n = g.n, nf = g.nf, Lm = LU - 1;
    const int cx = cell / (n * n), cy = (cell / n) % n, cz = cell % n;
    const float4 a0 = A0[s], a1 = A1[s], a2 = A2[s], a3 = A3[s];
    float ux[4][LU], uy[4][LU], uz[4][LU];
    basis_1d<LU, 4>(a0.x * g.two_over_h, W, g.Lc, ux);
    basis_1d<LU, 4>(a0.y * g.two_over_h, W, g.Lc, uy);
    basis_1d<LU, 4>(a0.z * g.two_over_h, W, g.Lc, uz);
    // V[px][py][pz] = sum_k Pi[k] ux^(px) uy^(py) uz^(pz), px + py + pz <= 3
    float V[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) V[i][j][k] = 0.f;
    const float *ps = psi + (int64_t)cell * g.ldm;
#pragma unroll 1
    for (int c = 0; c < LU; ++c) {
        const int gzz = (cz * Lm + c) % nf;
        float Y[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Y[i][j] = 0.f;
#pragma unroll
        for (int bb = 0; bb < LU; ++bb) {
            const int gyy = (cy * Lm + bb) % nf;
            float X[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < LU; ++a) {
                const int gxx = (cx * Lm + a) % nf;
                const float pi = __ldg(&phi[((int64_t)gxx * nf + gyy) * nf + gzz]) * invM
                               - __ldg(&ps[(a * LU + bb) * LU + c]);
#pragma unroll
                for (int p = 0; p < 4; ++p) X[p] = fmaf(pi, ux[p][a], X[p]);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4 - p; ++q) Y[p][q] = fmaf(X[p], uy[q][bb], Y[p][q]);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4 - p; ++q)
#pragma unroll
                for (int r = 0; r < 4 - p - q; ++r) V[p][q][r] = fmaf(Y[p][q], uz[r][c], V[p][q][r]);
    }
    const float q = a0.w, mx = a1.x, my = a1.y, mz = a1.z;
    const float txx = a2.x, txy = 2.f * a2.y, txz = 2.f * a2.z, tyy = a2.w, tyz = 2.f * a3.x, tzz = a3.y;
    float gx_[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int ex = ax == 0, ey = ax == 1, ez = ax == 2;
        gx_[ax] = q * V[ex][ey][ez] + mx * V[1 + ex][ey][ez] + my * V[ex][1 + ey][ez] + mz * V[ex][ey][1 + ez]
                + txx * V[2 + ex][ey][ez] + txy * V[1 + ex][1 + ey][ez] + txz * V[1 + ex][ey][1 + ez]
                + tyy * V[ex][2 + ey][ez] + tyz * V[ex][1 + ey][1 + ez] + tzz * V[ex][ey][2 + ez];
    }
    const int64_t S = N;
    gfar[0 * S + s] = gx_[0];
    gfar[1 * S + s] = gx_[1];
    gfar[2 * S + s] = gx_[2];
    gfar[3 * S + s] = V[0][0][0];
    gfar[4 * S + s] = V[1][0][0];
    gfar[5 * S + s] = V[0][1][0];
    gfar[6 * S + s] = V[0][0][1];
    gfar[7 * S + s] = V[2][0][0];
    gfar[8 * S + s] = 2.f * V[1][1][0];
    gfar[9 * S + s] = 2.f * V[1][0][1];
    gfar[10 * S + s] = V[0][2][0];
    gfar[11 * S + s] = 2.f * V[0][1][1];
    gfar[12 * S + s] = V[0][0][2];
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

cudaError_t launch_p2m(Handle &H, cudaStream_t s)
{
    ANKH_LU_SWITCH(H.g.Lu,
        k_p2m<LU><<<H.g.ncell, ((LU * LU * LU + 31) / 32) * 32, 0, s>>>(
            H.g, H.d_start, H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_W, H.d_M,
            H.tc.enabled ? H.d_Mhi : nullptr, H.tc.enabled ? H.d_Mlo : nullptr, H.tc.rowstride));
    return cudaGetLastError();
}

cudaError_t launch_fine_gather(Handle &H, cudaStream_t s)
{
    const int64_t nb = (H.g.M + 255) / 256;
    k_fine<<<(unsigned)nb, 256, 0, s>>>(H.g, H.d_M, H.d_rho);
    return cudaGetLastError();
}

cudaError_t launch_l2p(Handle &H, cudaStream_t s)
{
    const int N = (int)H.N;
    const float invM = (float)(1.0 / (double)H.g.M);
    ANKH_LU_SWITCH(H.g.Lu,
        k_l2p<LU><<<(N + 127) / 128, 128, 0, s>>>(H.g, N, H.d_scell, H.d_A0, H.d_A1, H.d_A2,
                                                   H.d_A3, H.d_W, H.d_phi, invM, H.d_psi, H.d_gfar));
    return cudaGetLastError();
}

}  // namespace ankh
