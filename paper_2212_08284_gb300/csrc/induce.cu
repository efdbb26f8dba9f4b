// Induced dipoles of point-polarizable atoms by the ANKH field (the use named
// in Sec. 1 and 6 of the paper: repeated field evaluations in polarizable
// force fields).  Each atom i has an isotropic polarizability alpha_i and
//     mu_i = alpha_i (F_i^perm + F_i(mu)),   F_i = -dE/dmu_i,
// the field of all other atoms and all periodic images (the Ewald self term of
// the library removes the atom's own direct term).  The field of a dipole
// distribution is linear, F(mu) = T mu with T symmetric, so
//     A mu = F^perm,   A = diag(1/alpha) - T,
// solved by conjugate gradients with the Jacobi preconditioner diag(alpha).
// A v = v/alpha + dE/dmu(v), one library evaluation with charges and
// quadrupoles zero and dipoles v (the adjoint path).  Vectors are FP32 in the
// caller's atom order, dot products are reduced in FP64 (fixed order).
#include "ankh_internal.cuh"

#include <cmath>
#include <vector>

namespace ankh {

constexpr int kIndThreads = 256;

int induce_blocks(int64_t n3, int sm_count)
{
    return (int)std::min<int64_t>((n3 + kIndThreads - 1) / kIndThreads, (int64_t)sm_count * 8);
}

__device__ __forceinline__ double ind_block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kIndThreads / 32; ++w) t += sh[w];
    __syncthreads();
    return t;
}

// F = -dE/dmu of the permanent multipoles, x = alpha F (initial guess);
// a non-positive or non-finite alpha raises bit 16 of the flag
__global__ void __launch_bounds__(kIndThreads)
k_ind_init(int64_t n3, const float *__restrict__ alpha, const float *__restrict__ dEdmu, float *__restrict__ F,
           float *__restrict__ x, int *__restrict__ flag)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x) {
        const float a = alpha[k / 3];
        if (!(a > 0.f) || !isfinite(a)) atomicOr(flag, 16);
        const float f = -dEdmu[k];
        F[k] = f;
        x[k] = a * f;
    }
}

// r = F - (x/alpha + dEdmu(x)), z = alpha r, p = z; partials (r.z, r.r, F.F)
__global__ void __launch_bounds__(kIndThreads)
k_ind_resid(int64_t n3, const float *__restrict__ alpha, const float *__restrict__ F, const float *__restrict__ x,
            const float *__restrict__ dEdmu, float *__restrict__ r, float *__restrict__ z, float *__restrict__ p,
            double *__restrict__ part)
{
    __shared__ double sh[kIndThreads / 32];
    double rz = 0.0, rr = 0.0, ff = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x) {
        const float a = alpha[k / 3];
        const float rv = F[k] - (x[k] / a + dEdmu[k]);
        const float zv = a * rv;
        r[k] = rv;
        z[k] = zv;
        p[k] = zv;
        rz += (double)rv * zv;
        rr += (double)rv * rv;
        ff += (double)F[k] * F[k];
    }
    rz = ind_block_sum(rz, sh);
    rr = ind_block_sum(rr, sh);
    ff = ind_block_sum(ff, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = rz;
        part[3 * blockIdx.x + 1] = rr;
        part[3 * blockIdx.x + 2] = ff;
    }
}

// Ap = p/alpha + dEdmu(p); partial p.Ap
__global__ void __launch_bounds__(kIndThreads)
k_ind_ap(int64_t n3, const float *__restrict__ alpha, const float *__restrict__ p, const float *__restrict__ dEdmu,
         float *__restrict__ Ap, double *__restrict__ part)
{
    __shared__ double sh[kIndThreads / 32];
    double s = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x) {
        const float v = p[k] / alpha[k / 3] + dEdmu[k];
        Ap[k] = v;
        s += (double)p[k] * v;
    }
    s = ind_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// x += a p, r -= a Ap, z = alpha r; partials (r.z, r.r)
__global__ void __launch_bounds__(kIndThreads)
k_ind_update(int64_t n3, float a, const float *__restrict__ alpha, const float *__restrict__ p,
             const float *__restrict__ Ap, float *__restrict__ x, float *__restrict__ r, float *__restrict__ z,
             double *__restrict__ part)
{
    __shared__ double sh[kIndThreads / 32];
    double rz = 0.0, rr = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x) {
        x[k] = fmaf(a, p[k], x[k]);
        const float rv = fmaf(-a, Ap[k], r[k]);
        const float zv = alpha[k / 3] * rv;
        r[k] = rv;
        z[k] = zv;
        rz += (double)rv * zv;
        rr += (double)rv * rv;
    }
    rz = ind_block_sum(rz, sh);
    rr = ind_block_sum(rr, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = rz;
        part[2 * blockIdx.x + 1] = rr;
    }
}

// p = z + beta p
__global__ void __launch_bounds__(kIndThreads)
k_ind_dir(int64_t n3, float beta, const float *__restrict__ z, float *__restrict__ p)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
        p[k] = fmaf(beta, p[k], z[k]);
}

// partial u.v
__global__ void __launch_bounds__(kIndThreads)
k_ind_dot(int64_t n3, const float *__restrict__ u, const float *__restrict__ v, double *__restrict__ part)
{
    __shared__ double sh[kIndThreads / 32];
    double s = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
        s += (double)u[k] * v[k];
    s = ind_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// fixed-order host sum of k-interleaved block partials
static int fetch_sums(const double *d_part, int nb, int k, double *out, double *h_buf, cudaStream_t s)
{
    if (cudaMemcpyAsync(h_buf, d_part, sizeof(double) * nb * k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ANKH_ECUDA;
    for (int j = 0; j < k; ++j) out[j] = 0.0;
    for (int b = 0; b < nb; ++b)
        for (int j = 0; j < k; ++j) out[j] += h_buf[k * b + j];
    return ANKH_OK;
}

int induce_dipoles(Handle &H, const float *x, const float *q, const float *mu, const float *theta,
                   const float *alpha, double tol, int max_iter, float *mu_ind, double *E_pol, int *iterations,
                   cudaStream_t s, std::string &err)
{
    const int64_t N = H.N, n3 = 3 * N;
    const int nb = induce_blocks(n3, H.sm_count);
    if (!H.d_ind) {
        // workspace: F, r, z, p, Ap, dE/dmu (3N each), zero charges (N), partials
        if (cudaMalloc(&H.d_ind, sizeof(float) * (6 * n3 + N)) != cudaSuccess) {
            err = "cudaMalloc induced-dipole workspace";
            return ANKH_ENOMEM;
        }
        if (cudaMalloc(&H.d_ind_part, sizeof(double) * 3 * H.sm_count * 8) != cudaSuccess) {
            err = "cudaMalloc induced-dipole partials";
            return ANKH_ENOMEM;
        }
        H.device_bytes += (int64_t)sizeof(float) * (6 * n3 + N) + (int64_t)sizeof(double) * 3 * H.sm_count * 8;
        if (cudaMemset(H.d_ind + 6 * n3, 0, sizeof(float) * N) != cudaSuccess) {
            err = "cudaMemset zero charges";
            return ANKH_ECUDA;
        }
    }
    float *F = H.d_ind, *r = F + n3, *z = r + n3, *p = z + n3, *Ap = p + n3, *g = Ap + n3;
    const float *qzero = g + n3;
    double *part = H.d_ind_part;
    std::vector<double> hbuf((size_t)3 * nb);
    auto field_grad = [&](const float *xv, const float *qv, const float *mv, const float *tv) {
        // dE/dmu of (q, mu, theta) into g
        int rc = run_sequence(H, xv, qv, mv, tv, true, nullptr, nullptr, g, nullptr, nullptr, s);
        if (rc != ANKH_OK) return rc;
        rc = fetch_terms(H, nullptr, s);
        return rc;
    };
    // permanent field and the initial guess mu = alpha F
    int rc = field_grad(x, q, mu, theta);
    if (rc != ANKH_OK) return rc;
    k_ind_init<<<nb, kIndThreads, 0, s>>>(n3, alpha, g, F, mu_ind, H.d_flag);
    int flag = 0;
    if (cudaMemcpyAsync(&flag, H.d_flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        err = "induce: init";
        return ANKH_ECUDA;
    }
    if (flag & 16) {
        err = "induce: every polarizability must be finite and > 0";
        return ANKH_EINVAL;
    }
    // r = F - A x, z = alpha r, p = z
    if ((rc = field_grad(x, qzero, mu_ind, nullptr)) != ANKH_OK) return rc;
    k_ind_resid<<<nb, kIndThreads, 0, s>>>(n3, alpha, F, mu_ind, g, r, z, p, part);
    double sums[3];
    if (fetch_sums(part, nb, 3, sums, hbuf.data(), s) != ANKH_OK) {
        err = "induce: residual";
        return ANKH_ECUDA;
    }
    double rz = sums[0], rr = sums[1];
    const double bnorm = std::sqrt(sums[2]);
    int it = 0;
    bool conv = !(bnorm > 0.0) || std::sqrt(rr) <= tol * bnorm;
    while (!conv && it < max_iter) {
        if ((rc = field_grad(x, qzero, p, nullptr)) != ANKH_OK) return rc;
        k_ind_ap<<<nb, kIndThreads, 0, s>>>(n3, alpha, p, g, Ap, part);
        double pAp;
        if (fetch_sums(part, nb, 1, &pAp, hbuf.data(), s) != ANKH_OK) {
            err = "induce: p.Ap";
            return ANKH_ECUDA;
        }
        if (!(pAp > 0.0)) {
            err = "induce: the system is not positive definite (polarization catastrophe)";
            return ANKH_ENUMERIC;
        }
        const double a = rz / pAp;
        k_ind_update<<<nb, kIndThreads, 0, s>>>(n3, (float)a, alpha, p, Ap, mu_ind, r, z, part);
        if (fetch_sums(part, nb, 2, sums, hbuf.data(), s) != ANKH_OK) {
            err = "induce: update";
            return ANKH_ECUDA;
        }
        const double rz_new = sums[0];
        rr = sums[1];
        ++it;
        conv = std::sqrt(rr) <= tol * bnorm;
        if (!conv) {
            k_ind_dir<<<nb, kIndThreads, 0, s>>>(n3, (float)(rz_new / rz), z, p);
            rz = rz_new;
        }
    }
    // E_pol = -1/2 mu . F^perm
    k_ind_dot<<<nb, kIndThreads, 0, s>>>(n3, mu_ind, F, part);
    double d;
    if (fetch_sums(part, nb, 1, &d, hbuf.data(), s) != ANKH_OK) {
        err = "induce: energy";
        return ANKH_ECUDA;
    }
    if (E_pol) *E_pol = -0.5 * d;
    if (iterations) *iterations = it;
    if (!conv) {
        err = "induce: no convergence within max_iter";
        return ANKH_ENOTCONV;
    }
    return ANKH_OK;
}

}  // namespace ankh
