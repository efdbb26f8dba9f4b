// k = 0 far-field term, gradient assembly and the FP64 energy reduction
// (Alg. 5 steps 4-5).  The self term of Eq. ewald (per atom in the gather
// kernel, k_sort.cu) is
// E_self = -(xi/sqrt(pi)) sum_i [q^2 + (2xi^2/3)|mu|^2 - (4xi^2/3) q tr(Theta)
//                                + (8xi^4/5) Theta:Theta + (4xi^4/5) tr(Theta)^2]
// (general symmetric Theta; for a traceless Theta this is the printed form).
// The k = 0 term of the far field is D_0 Q^2 / (2M) with Q = sum_i q_i exactly
// (partition of unity of the interpolation), evaluated in FP64; its
// potential D_0 Q / M is added to dE/dq.
#include "ankh_internal.cuh"

namespace ankh {

int self_blocks(const Handle &H) { return (int)((H.N + 255) / 256); }

// total charge and the k = 0 potential D0 Q / M -> terms[6], terms[7] (Q)
__global__ void __launch_bounds__(256) k_dc(const double *__restrict__ part_q, int nq, double D0, double invM,
                                            double *__restrict__ terms)
{
    __shared__ double sh[8];
    double Q = 0.0;
    for (int b = threadIdx.x; b < nq; b += 256) Q += part_q[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Q += __shfl_down_sync(0xffffffffu, Q, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = Q;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < 8; ++w) u += sh[w];
        terms[7] = u;
        terms[6] = D0 * u * invM;
    }
}

// Gradient assembly per sorted slot: far + near + self (+ k = 0 potential),
// torques, and the write to the caller's atom order.
__global__ void __launch_bounds__(256)
k_finalize(int N, const int *__restrict__ perm, const float4 *__restrict__ A0,
           const float4 *__restrict__ A1, const float4 *__restrict__ A2, const float4 *__restrict__ A3,
           const float *__restrict__ gfar, const float *__restrict__ gnear, const double *__restrict__ terms,
           float xi, float *__restrict__ dEdx, float *__restrict__ dEdq, float *__restrict__ dEdmu,
           float *__restrict__ dEdth, float *__restrict__ torque)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int64_t S = N;
    float gv[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) gv[k] = gfar[k * S + s] + gnear[k * S + s];
    const float4 a0 = A0[s], a1 = A1[s], a2 = A2[s], a3 = A3[s];
    const float q = a0.w;
    const float xx = a2.x, xy = a2.y, xz = a2.z, yy = a2.w, yz = a3.x, zz = a3.y;
    const float tr = xx + yy + zz;
    // self-term gradient
    const float c = xi * 0.56418958354775628f;  // xi / sqrt(pi)
    const float x2 = xi * xi, x4 = x2 * x2;
    gv[3] += -c * (2.f * q - (4.f * x2 / 3.f) * tr) + (float)terms[6];
    gv[4] += -c * (4.f * x2 / 3.f) * a1.x;
    gv[5] += -c * (4.f * x2 / 3.f) * a1.y;
    gv[6] += -c * (4.f * x2 / 3.f) * a1.z;
    const float dg = -(4.f * x2 / 3.f) * q + (8.f * x4 / 5.f) * tr;
    const float k16 = 16.f * x4 / 5.f;
    gv[7] += -c * (dg + k16 * xx);
    gv[8] += -c * 2.f * k16 * xy;
    gv[9] += -c * 2.f * k16 * xz;
    gv[10] += -c * (dg + k16 * yy);
    gv[11] += -c * 2.f * k16 * yz;
    gv[12] += -c * (dg + k16 * zz);

    const int i = perm[s];
    const int64_t ii = i;
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
            for (int b = 0; b < 3; ++b) X[a][b] = G[a][0] * T[0][b] + G[a][1] * T[1][b] + G[a][2] * T[2][b];
        const float mx = a1.x, my = a1.y, mz = a1.z;
        torque[3 * ii] = -(my * gz - mz * gy) - 2.f * (X[2][1] - X[1][2]);
        torque[3 * ii + 1] = -(mz * gx - mx * gz) - 2.f * (X[0][2] - X[2][0]);
        torque[3 * ii + 2] = -(mx * gy - my * gx) - 2.f * (X[1][0] - X[0][1]);
    }
}

// Fixed-order FP64 reduction of all energy partials.
// terms: [0] near [1] far (k != 0) [2] k = 0 [3] correction [4] self [5] total
//        [6] k = 0 potential [7] Q
__global__ void k_reduce(const double *__restrict__ part, const int *__restrict__ off_dev,
                         double invM2, double D0, const int *__restrict__ flag, double *__restrict__ terms,
                         int have_glob, int have_corr)
{
    __shared__ double sh[32];
    __shared__ double res[kPartCount];
    for (int slot = 0; slot < kPartCount; ++slot) {
        const int b = off_dev[slot], e = off_dev[slot + 1];
        double v = 0.0;
        for (int k = b + threadIdx.x; k < e; k += blockDim.x) v += part[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += sh[w];
            res[slot] = u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double Q = terms[7];
        const double near = res[kPartNear];
        const double glob = have_glob ? res[kPartGlob] * invM2 : 0.0;
        const double dc = have_glob ? D0 * Q * Q * invM2 : 0.0;
        const double corr = have_corr ? res[kPartCorr] : 0.0;
        const double self = res[kPartSelf];
        terms[0] = near;
        terms[1] = glob;
        terms[2] = dc;
        terms[3] = corr;
        terms[4] = self;
        terms[5] = near + glob + dc + corr + self;
        terms[8] = (double)(*flag);
        if (*flag) terms[5] = __longlong_as_double(0x7ff8000000000000LL);
    }
}

// the self term and Q partials are produced by the gather kernel (k_sort.cu)
cudaError_t launch_self_dc(Handle &H, cudaStream_t s)
{
    k_dc<<<1, 256, 0, s>>>(H.d_part + H.part_off[kPartQ], self_blocks(H), H.D0, 1.0 / (double)H.g.M,
                           H.d_terms);
    return cudaGetLastError();
}

cudaError_t launch_finalize(Handle &H, float *dEdx, float *dEdq, float *dEdmu, float *dEdtheta,
                            float *torque, cudaStream_t s)
{
    const int N = (int)H.N;
    k_finalize<<<(N + 255) / 256, 256, 0, s>>>(N, H.d_perm, H.d_A0, H.d_A1, H.d_A2, H.d_A3, H.d_gfar,
                                               H.d_gnear, H.d_terms, H.g.xi, dEdx, dEdq, dEdmu, dEdtheta,
                                               torque);
    return cudaGetLastError();
}

cudaError_t launch_reduce(Handle &H, cudaStream_t s)
{
    k_reduce<<<1, 256, 0, s>>>(H.d_part, H.d_partoff, 0.5 / (double)H.g.M, H.D0, H.d_flag, H.d_terms, 1, 1);
    return cudaGetLastError();
}

}  // namespace ankh
