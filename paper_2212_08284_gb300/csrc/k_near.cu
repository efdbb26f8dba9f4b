// Near field of ANKH (Alg. 5 step 3; Sec. 3.2 N_real): every pair of atoms in
// the same or in adjacent leaves (26 neighbours, periodic, one image per
// offset), kernel H = erfc(xi r)/r, with the full multipole operator
//   e_ik = (q_i + mu_i.grad + Theta_i:grad grad)(q_k - mu_k.grad + Theta_k:grad grad) H(r),
//   r = x_i - x_k.
// N_real = 1/2 sum_i sum_k e_ik.  Each thread owns one target atom and visits
// all 27 leaves (both orders of every pair are evaluated), so every output is
// written by exactly one thread -- no atomics, deterministic results.
//
// The derivatives of the radial kernel are taken through the screened
// functions B_0 = H, B_l = -(1/r) dB_{l-1}/dr, computed upward:
//   B_l = [(2l-1) B_{l-1} + (2 xi^2)^l exp(-xi^2 r^2)/(xi sqrt(pi))] / r^2.
// In terms of s_i = mu_i.r, s_k = mu_k.r, t = tr Theta, u = r.Theta.r:
//   e = sum_{l=0..4} c_l B_l with
//   c0 = q_i q_k
//   c1 = q_i (s_k - t_k) - q_k (s_i + t_i) + mu_i.mu_k
//   c2 = q_i u_k + q_k u_i - (s_i + t_i)(s_k - t_k) + 2 mu_i.Theta_k r - 2 mu_k.Theta_i r
//        + 2 Theta_i:Theta_k
//   c3 = (s_k - t_k) u_i - (s_i + t_i) u_k - 4 (Theta_i r).(Theta_k r)
//   c4 = u_i u_k
// and grad e = sum_l (grad c_l) B_l - r sum_l c_l B_{l+1}; the potential,
// field and field gradient of the source at the target give dE/dq_i,
// dE/dmu_i and dE/dTheta_i.
#include "ankh_internal.cuh"

namespace ankh {

struct MPf {
    float q, dx, dy, dz, xx, xy, xz, yy, yz, zz, tr;
};

__device__ __forceinline__ MPf load_mp(const float4 a0, const float4 a1, const float4 a2, const float4 a3)
{
    MPf m;
    m.q = a0.w;
    m.dx = a1.x; m.dy = a1.y; m.dz = a1.z;
    m.xx = a2.x; m.xy = a2.y; m.xz = a2.z; m.yy = a2.w; m.yz = a3.x; m.zz = a3.y;
    m.tr = m.xx + m.yy + m.zz;
    return m;
}

struct BCoef {
    float xi, c1, c2, c3, c4, c5;  // c_l = (2 xi^2)^l / (xi sqrt(pi))
};

template <bool FORCES>
__device__ __forceinline__ void near_pair(float rx, float ry, float rz, const MPf &I, const MPf &K,
                                          const BCoef &bc, float &e, float (&gr)[3], float &V,
                                          float (&gV)[3], float (&ggV)[6])
{
    const float r2 = rx * rx + ry * ry + rz * rz;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float ri2 = rinv * rinv;
    const float ex = __expf(-bc.xi * bc.xi * r2);
    const float B0 = erfcf(bc.xi * r) * rinv;
    const float B1 = (B0 + bc.c1 * ex) * ri2;
    const float B2 = (3.f * B1 + bc.c2 * ex) * ri2;
    const float B3 = (5.f * B2 + bc.c3 * ex) * ri2;
    const float B4 = (7.f * B3 + bc.c4 * ex) * ri2;

    const float Qir0 = I.xx * rx + I.xy * ry + I.xz * rz;
    const float Qir1 = I.xy * rx + I.yy * ry + I.yz * rz;
    const float Qir2 = I.xz * rx + I.yz * ry + I.zz * rz;
    const float Qkr0 = K.xx * rx + K.xy * ry + K.xz * rz;
    const float Qkr1 = K.xy * rx + K.yy * ry + K.yz * rz;
    const float Qkr2 = K.xz * rx + K.yz * ry + K.zz * rz;
    const float si = I.dx * rx + I.dy * ry + I.dz * rz;
    const float sk = K.dx * rx + K.dy * ry + K.dz * rz;
    const float ui = rx * Qir0 + ry * Qir1 + rz * Qir2;
    const float uk = rx * Qkr0 + ry * Qkr1 + rz * Qkr2;
    const float didk = I.dx * K.dx + I.dy * K.dy + I.dz * K.dz;
    const float diQkr = I.dx * Qkr0 + I.dy * Qkr1 + I.dz * Qkr2;
    const float dkQir = K.dx * Qir0 + K.dy * Qir1 + K.dz * Qir2;
    const float QirQkr = Qir0 * Qkr0 + Qir1 * Qkr1 + Qir2 * Qkr2;
    const float QiQk = I.xx * K.xx + I.yy * K.yy + I.zz * K.zz
                     + 2.f * (I.xy * K.xy + I.xz * K.xz + I.yz * K.yz);
    const float ski = sk - K.tr, sit = si + I.tr;
    const float c0 = I.q * K.q;
    const float c1 = I.q * ski - K.q * sit + didk;
    const float c2 = I.q * uk + K.q * ui - sit * ski + 2.f * (diQkr - dkQir + QiQk);
    const float c3 = ski * ui - sit * uk - 4.f * QirQkr;
    const float c4 = ui * uk;
    e += c0 * B0 + c1 * B1 + c2 * B2 + c3 * B3 + c4 * B4;
    if (!FORCES) return;

    const float B5 = (9.f * B4 + bc.c5 * ex) * ri2;
    const float cb1 = c0 * B1 + c1 * B2 + c2 * B3 + c3 * B4 + c4 * B5;
    // Theta_k mu_i, Theta_i mu_k, Theta_i (Theta_k r), Theta_k (Theta_i r)
    const float Qkdi0 = K.xx * I.dx + K.xy * I.dy + K.xz * I.dz;
    const float Qkdi1 = K.xy * I.dx + K.yy * I.dy + K.yz * I.dz;
    const float Qkdi2 = K.xz * I.dx + K.yz * I.dy + K.zz * I.dz;
    const float Qidk0 = I.xx * K.dx + I.xy * K.dy + I.xz * K.dz;
    const float Qidk1 = I.xy * K.dx + I.yy * K.dy + I.yz * K.dz;
    const float Qidk2 = I.xz * K.dx + I.yz * K.dy + I.zz * K.dz;
    const float QQ0 = I.xx * Qkr0 + I.xy * Qkr1 + I.xz * Qkr2 + K.xx * Qir0 + K.xy * Qir1 + K.xz * Qir2;
    const float QQ1 = I.xy * Qkr0 + I.yy * Qkr1 + I.yz * Qkr2 + K.xy * Qir0 + K.yy * Qir1 + K.yz * Qir2;
    const float QQ2 = I.xz * Qkr0 + I.yz * Qkr1 + I.zz * Qkr2 + K.xz * Qir0 + K.yz * Qir1 + K.zz * Qir2;
    const float di[3] = {I.dx, I.dy, I.dz}, dk[3] = {K.dx, K.dy, K.dz};
    const float Qir[3] = {Qir0, Qir1, Qir2}, Qkr[3] = {Qkr0, Qkr1, Qkr2};
    const float Qkdi[3] = {Qkdi0, Qkdi1, Qkdi2}, Qidk[3] = {Qidk0, Qidk1, Qidk2}, QQ[3] = {QQ0, QQ1, QQ2};
    const float rr[3] = {rx, ry, rz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float g1 = I.q * dk[a] - K.q * di[a];
        const float g2 = 2.f * (I.q * Qkr[a] + K.q * Qir[a] + Qkdi[a] - Qidk[a]) - di[a] * ski - sit * dk[a];
        const float g3 = 2.f * (ski * Qir[a] - sit * Qkr[a]) + ui * dk[a] - uk * di[a] - 4.f * QQ[a];
        const float g4 = 2.f * (uk * Qir[a] + ui * Qkr[a]);
        gr[a] += g1 * B1 + g2 * B2 + g3 * B3 + g4 * B4 - rr[a] * cb1;
    }
    // potential, field and field gradient of the source at the target
    V += K.q * B0 + ski * B1 + uk * B2;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        gV[a] += B1 * (dk[a] - K.q * rr[a]) + B2 * (2.f * Qkr[a] - ski * rr[a]) - B3 * uk * rr[a];
    const float dA = -K.q * B1 - ski * B2 - uk * B3;
    const float rrA = K.q * B2 + ski * B3 + uk * B4;
    const float Kab[6] = {K.xx, K.xy, K.xz, K.yy, K.yz, K.zz};
    const int PA[6] = {0, 0, 0, 1, 1, 2}, PB[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const int a = PA[m], b = PB[m];
        float G = rr[a] * rr[b] * rrA - (dk[a] * rr[b] + rr[a] * dk[b]) * B2 + 2.f * Kab[m] * B2
                - 2.f * (rr[a] * Qkr[b] + Qkr[a] * rr[b]) * B3;
        if (a == b) G += dA;
        ggV[m] += (a == b) ? G : 2.f * G;
    }
}

template <bool FORCES>
__global__ void __launch_bounds__(128)
k_near(Geo g, int N, const int *__restrict__ start, const int *__restrict__ scell,
       const float4 *__restrict__ A0, const float4 *__restrict__ A1, const float4 *__restrict__ A2,
       const float4 *__restrict__ A3, BCoef bc, float *__restrict__ gnear, double *__restrict__ part)
{
    __shared__ double sh[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    float gr[3] = {0.f, 0.f, 0.f}, V = 0.f, gV[3] = {0.f, 0.f, 0.f};
    float ggV[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (s < N) {
        const float4 t0 = A0[s];
        const MPf I = load_mp(t0, A1[s], A2[s], A3[s]);
        const int cell = scell[s];
        const int n = g.n;
        const int cx = cell / (n * n), cy = (cell / n) % n, cz = cell % n;
        for (int dx = -1; dx <= 1; ++dx) {
            const int nx = (cx + dx + n) % n;
            for (int dy = -1; dy <= 1; ++dy) {
                const int ny = (cy + dy + n) % n;
                for (int dz = -1; dz <= 1; ++dz) {
                    const int nz = (cz + dz + n) % n;
                    const int nc = (nx * n + ny) * n + nz;
                    const float ox = dx * g.hf, oy = dy * g.hf, oz = dz * g.hf;
                    const bool same = (dx == 0 && dy == 0 && dz == 0);
                    const int jb = start[nc], je = start[nc + 1];
                    for (int j = jb; j < je; ++j) {
                        if (same && j == s) continue;
                        const float4 k0 = A0[j];
                        const MPf K = load_mp(k0, A1[j], A2[j], A3[j]);
                        const float rx = (t0.x - k0.x) - ox;
                        const float ry = (t0.y - k0.y) - oy;
                        const float rz = (t0.z - k0.z) - oz;
                        near_pair<FORCES>(rx, ry, rz, I, K, bc, e, gr, V, gV, ggV);
                    }
                }
            }
        }
        if (FORCES) {
            const int64_t S = N;
            gnear[0 * S + s] = gr[0];
            gnear[1 * S + s] = gr[1];
            gnear[2 * S + s] = gr[2];
            gnear[3 * S + s] = V;
            gnear[4 * S + s] = gV[0];
            gnear[5 * S + s] = gV[1];
            gnear[6 * S + s] = gV[2];
#pragma unroll
            for (int m = 0; m < 6; ++m) gnear[(7 + m) * S + s] = ggV[m];
        }
    }
    // per-target energy I_i . V_i; 1/2 for the double counting of ordered pairs
    double t = 0.5 * (double)e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += sh[w];
        part[blockIdx.x] = u;
    }
}

int near_blocks(const Handle &H) { return (int)((H.N + 127) / 128); }

cudaError_t launch_near(Handle &H, bool forces, cudaStream_t s)
{
    BCoef bc;
    const double xi = H.g.xi;
    bc.xi = (float)xi;
    double c = 1.0 / (xi * sqrt(M_PI));
    double cl[6];
    for (int l = 1; l <= 5; ++l) {
        c *= 2.0 * xi * xi;
        cl[l] = c;
    }
    bc.c1 = (float)cl[1]; bc.c2 = (float)cl[2]; bc.c3 = (float)cl[3]; bc.c4 = (float)cl[4]; bc.c5 = (float)cl[5];
    const int N = (int)H.N;
    double *part = H.d_part + H.part_off[kPartNear];
    if (forces)
        k_near<true><<<near_blocks(H), 128, 0, s>>>(H.g, N, H.d_start, H.d_scell, H.d_A0, H.d_A1, H.d_A2,
                                                    H.d_A3, bc, H.d_gnear, part);
    else
        k_near<false><<<near_blocks(H), 128, 0, s>>>(H.g, N, H.d_start, H.d_scell, H.d_A0, H.d_A1, H.d_A2,
                                                     H.d_A3, bc, H.d_gnear, part);
    return cudaGetLastError();
}

}  // namespace ankh
