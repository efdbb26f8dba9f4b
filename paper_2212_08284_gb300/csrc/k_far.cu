// Far field of ANKH-FFT on the merged periodic equispaced grid.
//
// The masked 6-D block-Toeplitz matrix A of Sec. 4.2 (blocks G~[t,s] zero for
// adjacent leaves, periodic images folded in, Sec. 4.3) is applied here as
//   F = 1/2 rho^T G rho  +  (adjacent-leaf correction, k_corr.cu)
// where rho is the grid charge with the duplicated face nodes summed and G is
// one circulant on the n (L_u - 1) grid (its transforms and the spectral
// product are in fft.cu):
//   G(z) = Phi(z) - [ |z|_inf < h ] H(z),  Phi(z) = sum_m H(z + L m),
// i.e. the interactions closer than one leaf width are taken out of the
// global kernel and every adjacent-leaf node pair at |z|_inf >= h is removed
// by the correction term.  The circulant is diagonalised by the DFT (Thm. 1,
// Cor. 1); its spectrum is real (Cor. 2), so only one forward transform is
// needed for the energy (Eq. realdiag):
//   F_glob = (1 / 2M) sum_k D_k |rho^_k|^2.
//
// Precomputation (FP64, once per box, the role of Alg. 4 and Sec. 4.3): Phi is
// evaluated in closed form by a second Ewald split with eta >> xi,
//   Phi(z) = sum_m erfc(eta |z+Lm|)/|z+Lm| + (4 pi / V) sum_{k!=0} c_k cos(k.z)
//          + (pi / V)(1/xi^2 - 1/eta^2),
//   c_k = (exp(-k^2/4eta^2) - [paper-literal] exp(-k^2/4xi^2)) / k^2;
// the real-space part (with the H subtraction) is transformed by a D2Z FFT and
// the band-limited reciprocal part is added directly in Fourier space (its
// DFT on the grid is M c_k, folded modulo the grid).  The constant pi/(V xi^2)
// multiplies Q^2 only and cancels the tin-foil neutralising term; both are
// dropped.
#include "ankh_internal.cuh"

#include <cmath>

namespace ankh {

// ----------------------------------------------------------------------------
// Precomputation kernels (FP64)

__global__ void k_pre_real(Geo g, double eta, double xi, double *__restrict__ T)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.M) return;
    const int nf = g.nf;
    const int j[3] = {(int)(idx / ((int64_t)nf * nf)), (int)((idx / nf) % nf), (int)(idx % nf)};
    int jm[3];
    int jmax = 0;
    for (int a = 0; a < 3; ++a) {
        jm[a] = j[a] > nf / 2 ? j[a] - nf : j[a];
        jmax = max(jmax, abs(jm[a]));
    }
    const double delta = g.box / nf;
    const double z[3] = {jm[0] * delta, jm[1] * delta, jm[2] * delta};
    const bool origin = (jm[0] == 0 && jm[1] == 0 && jm[2] == 0);
    double v = 0.0;
    for (int mx = -1; mx <= 1; ++mx)
        for (int my = -1; my <= 1; ++my)
            for (int mz = -1; mz <= 1; ++mz) {
                const double dx = z[0] + g.box * mx, dy = z[1] + g.box * my, dz = z[2] + g.box * mz;
                const double r = sqrt(dx * dx + dy * dy + dz * dz);
                if (origin && mx == 0 && my == 0 && mz == 0) {
                    // limit of (erfc(eta r) - erfc(xi r)) / r at r = 0
                    v += 2.0 / sqrt(M_PI) * (xi - eta);
                } else {
                    v += erfc(eta * r) / r;
                }
            }
    if (!origin && jmax <= g.Lu - 2) {
        const double r0 = sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
        v -= erfc(xi * r0) / r0;
    }
    T[idx] = v;
}

__global__ void k_pre_spec(Geo g, const cufftDoubleComplex *__restrict__ Tk, double eta, double xi,
                           int include_rec, int mmax, double kcut2, float *__restrict__ D,
                           double *__restrict__ D0)
{
    const int64_t total = (int64_t)g.nf * g.nf * g.nfh;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int nf = g.nf;
    const int kz = (int)(idx % g.nfh), ky = (int)((idx / g.nfh) % nf), kx = (int)(idx / ((int64_t)g.nfh * nf));
    const double V = g.box * g.box * g.box;
    const double tpl = 2.0 * M_PI / g.box;
    double sum = 0.0;
    const int P = mmax / nf + 2;
    for (int px = -P; px <= P; ++px) {
        const int mx = kx + px * nf;
        if (abs(mx) > mmax) continue;
        for (int py = -P; py <= P; ++py) {
            const int my = ky + py * nf;
            if (abs(my) > mmax) continue;
            for (int pz = -P; pz <= P; ++pz) {
                const int mz = kz + pz * nf;
                if (abs(mz) > mmax) continue;
                if (mx == 0 && my == 0 && mz == 0) continue;
                const double k2 = tpl * tpl * ((double)mx * mx + (double)my * my + (double)mz * mz);
                if (k2 > kcut2) continue;
                double c = exp(-k2 / (4.0 * eta * eta));
                if (!include_rec) c -= exp(-k2 / (4.0 * xi * xi));
                sum += c / k2;
            }
        }
    }
    const double Md = (double)g.M;
    double val = Tk[idx].x + Md * (4.0 * M_PI / V) * sum;
    if (idx == 0) {
        val += Md * (-M_PI / (V * eta * eta));
        *D0 = val;
        D[0] = 0.f;
    } else {
        D[idx] = (float)val;
    }
}

// Non-periodic kernel on the zero-padded grid (FP64): the linear
// convolution of the ng merged nodes per axis with
//   G(d) = H(d delta) = 1/(delta |d|)  if max_a |d_a| >= L_u - 1 (one leaf), else 0,
// displacements d in [-(ng-1), ng-1] per axis placed circularly (nf >= 2 ng - 1,
// so the wrap-around entries are never reached and stay 0).
__global__ void k_pre_np(Geo g, double *__restrict__ T)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.M) return;
    const int nf = g.nf, ng = g.ng, Lm = g.Lu - 1;
    const int j[3] = {(int)(idx / ((int64_t)nf * nf)), (int)((idx / nf) % nf), (int)(idx % nf)};
    int d[3];
    bool used = true;
    int dmax = 0;
    for (int a = 0; a < 3; ++a) {
        d[a] = j[a] < ng ? j[a] : (j[a] > nf - ng ? j[a] - nf : 0);
        if (j[a] >= ng && j[a] <= nf - ng) used = false;
        dmax = max(dmax, abs(d[a]));
    }
    double v = 0.0;
    if (used && dmax >= Lm) {
        const double delta = g.h / Lm;
        v = 1.0 / (delta * sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]));
    }
    T[idx] = v;
}

// D (FP32) from the D2Z transform of the non-periodic kernel; the k = 0 value
// is returned in FP64 and removed from D (its term D_0 Q^2 / 2M is added in FP64).
__global__ void k_pre_spec_np(Geo g, const cufftDoubleComplex *__restrict__ Tk, float *__restrict__ D,
                              double *__restrict__ D0)
{
    const int64_t total = (int64_t)g.nf * g.nf * g.nfh;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    if (idx == 0) {
        *D0 = Tk[0].x;
        D[0] = 0.f;
    } else {
        D[idx] = (float)Tk[idx].x;
    }
}

cudaError_t precompute_kernel_spectrum(Handle &H, double *D0_out, std::string &err)
{
    const Geo &g = H.g;
    const double eta = 14.0 / g.box;                 // erfc(eta L/2) = erfc(7) ~ 4e-23
    const double kcut = 12.8 * eta;                  // exp(-kcut^2 / 4 eta^2) ~ 1e-18
    const int mmax = (int)std::ceil(kcut * g.box / (2.0 * M_PI));
    double *dT = nullptr, *dD0 = nullptr;
    cufftDoubleComplex *dTk = nullptr;
    cufftHandle plan = 0;
    bool have_plan = false;
    cudaError_t ce = cudaSuccess;
    const int64_t nspec = (int64_t)g.nf * g.nf * g.nfh;
    auto fail = [&](const char *what) {
        err = std::string("precompute: ") + what;
        if (have_plan) cufftDestroy(plan);
        cudaFree(dT);
        cudaFree(dTk);
        cudaFree(dD0);
        return ce == cudaSuccess ? cudaErrorUnknown : ce;
    };
    if ((ce = cudaMalloc(&dT, sizeof(double) * g.M)) != cudaSuccess) return fail("cudaMalloc T");
    if ((ce = cudaMalloc(&dTk, sizeof(cufftDoubleComplex) * nspec)) != cudaSuccess) return fail("cudaMalloc Tk");
    if ((ce = cudaMalloc(&dD0, sizeof(double))) != cudaSuccess) return fail("cudaMalloc D0");
    if (g.nonperiodic) k_pre_np<<<(unsigned)((g.M + 255) / 256), 256>>>(g, dT);
    else k_pre_real<<<(unsigned)((g.M + 255) / 256), 256>>>(g, eta, (double)H.g.xi, dT);
    if ((ce = cudaGetLastError()) != cudaSuccess) return fail("kernel table");
    if (cufftPlan3d(&plan, g.nf, g.nf, g.nf, CUFFT_D2Z) != CUFFT_SUCCESS) return fail("cufftPlan3d D2Z");
    have_plan = true;
    if (cufftExecD2Z(plan, dT, dTk) != CUFFT_SUCCESS) return fail("cufftExecD2Z");
    if (g.nonperiodic)
        k_pre_spec_np<<<(unsigned)((nspec + 255) / 256), 256>>>(g, dTk, H.d_D, dD0);
    else
        k_pre_spec<<<(unsigned)((nspec + 255) / 256), 256>>>(g, dTk, eta, (double)H.g.xi,
                                                              (H.flags & ANKH_INCLUDE_REC) ? 1 : 0, mmax,
                                                              kcut * kcut, H.d_D, dD0);
    if ((ce = cudaGetLastError()) != cudaSuccess) return fail("k_pre_spec");
    if ((ce = cudaMemcpy(D0_out, dD0, sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail("copy D0");
    cufftDestroy(plan);
    cudaFree(dT);
    cudaFree(dTk);
    cudaFree(dD0);
    return cudaSuccess;
}

}  // namespace ankh
