// Three-dimensional real FFT of the merged grid for the far field of
// ANKH-FFT (Thm. 1 and Cor. 1: the circulant kernel is diagonalised by the
// DFT; Cor. 2 and Eq. realdiag: its spectrum is real, so the energy is
// F_glob = (1/2M) sum_k D_k |rho^_k|^2 over the half spectrum of the real
// grid), with the spectral step fused into the transform along x:
//
//   pass Z   r2c along z: two real rows as one complex row, one complex FFT,
//            the two half spectra separated, X_k = (Z_k + conj Z_{L-k}) / 2,
//            Y_k = (Z_k - conj Z_{L-k}) / 2i, k = 0 .. L/2;
//   pass Y   complex FFT along y (forward);
//   pass X   complex FFT along x, then per point the energy term
//            w_kz D_k |rho^_k|^2 (w = 1 for kz = 0 and kz = L/2, else 2, the
//            Hermitian half) into FP64 block partials; with forces also
//            phi^ = D rho^ and the inverse FFT along x, written back in place;
//   pass Y'  inverse complex FFT along y;
//   pass Z'  c2r along z: two Hermitian half rows as one complex row
//            (Z_k = X_k + i Y_k, the imaginary parts of X_0 and X_{L/2} dropped
//            as for a real row), one inverse FFT, real and imaginary parts out.
// Transforms are unnormalised (forward e^{-2 pi i k n / L}, inverse e^{+...}).
// Spectrum layout [x][y][kz], kz fastest (L/2 + 1 values), the layout of the
// kernel spectrum D.
//
// Each 1-D transform is a mixed-radix Stockham FFT in shared memory (radices
// 2..8, the fewest stages): stage s with radix R and p = product of the
// earlier radices maps, for i in [0, L/R), k = i mod p,
//   u_r = a[i + r L/R] W^(r k L/(p R)),  U = DFT_R(u),  b[(i - k) R + k + r p] = U_r,
// and the result ends in natural order.  Twiddles W^e = e^{-2 pi i e/L} come
// from a table computed in FP64 on the host and rounded to FP32.  The lines
// of a block sit side by side in shared memory (point-major, line fastest),
// so consecutive threads touch consecutive words.
#include "ankh_internal.cuh"

#include <cmath>
#include <functional>
#include <vector>

namespace ankh {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// SIGN i z  (SIGN = -1 forward, +1 inverse)
template <int SIGN>
__device__ __forceinline__ float2 mul_si(float2 z)
{
    return SIGN > 0 ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

// Small DFTs U_q = sum_r u_r e^{SIGN 2 pi i r q / R}, in place.
template <int R, int SIGN>
struct Dft;

template <int SIGN>
struct Dft<2, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        const float2 a = u[0], b = u[1];
        u[0] = cadd(a, b);
        u[1] = csub(a, b);
    }
};

template <int SIGN>
struct Dft<3, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        const float2 t1 = cadd(u[1], u[2]), t2 = csub(u[1], u[2]);
        const float2 m = make_float2(fmaf(-0.5f, t1.x, u[0].x), fmaf(-0.5f, t1.y, u[0].y));
        const float2 s = mul_si<SIGN>(cscale(t2, 0.86602540378443865f));
        u[0] = cadd(u[0], t1);
        u[1] = cadd(m, s);
        u[2] = csub(m, s);
    }
};

template <int SIGN>
struct Dft<4, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        const float2 a = cadd(u[0], u[2]), b = csub(u[0], u[2]);
        const float2 c = cadd(u[1], u[3]), d = mul_si<SIGN>(csub(u[1], u[3]));
        u[0] = cadd(a, c);
        u[2] = csub(a, c);
        u[1] = cadd(b, d);
        u[3] = csub(b, d);
    }
};

template <int SIGN>
struct Dft<5, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        // cos and sin of 2 pi / 5 and 4 pi / 5
        const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;
        const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;
        const float2 t1 = cadd(u[1], u[4]), t2 = cadd(u[2], u[3]);
        const float2 t3 = csub(u[1], u[4]), t4 = csub(u[2], u[3]);
        const float2 a1 = make_float2(u[0].x + c1 * t1.x + c2 * t2.x, u[0].y + c1 * t1.y + c2 * t2.y);
        const float2 a2 = make_float2(u[0].x + c2 * t1.x + c1 * t2.x, u[0].y + c2 * t1.y + c1 * t2.y);
        const float2 b1 = mul_si<SIGN>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
        const float2 b2 = mul_si<SIGN>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
        u[0] = cadd(u[0], cadd(t1, t2));
        u[1] = cadd(a1, b1);
        u[4] = csub(a1, b1);
        u[2] = cadd(a2, b2);
        u[3] = csub(a2, b2);
    }
};

template <int SIGN>
struct Dft<6, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        // even and odd inputs, DFT_3 each, combined with e^{SIGN i pi q / 3}
        float2 e[3] = {u[0], u[2], u[4]}, o[3] = {u[1], u[3], u[5]};
        Dft<3, SIGN>::run(e);
        Dft<3, SIGN>::run(o);
        const float h = 0.86602540378443865f * (float)SIGN;
        const float2 o1 = cmul(o[1], make_float2(0.5f, h)), o2 = cmul(o[2], make_float2(-0.5f, h));
        u[0] = cadd(e[0], o[0]);
        u[3] = csub(e[0], o[0]);
        u[1] = cadd(e[1], o1);
        u[4] = csub(e[1], o1);
        u[2] = cadd(e[2], o2);
        u[5] = csub(e[2], o2);
    }
};

template <int SIGN>
struct Dft<7, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        // cos and sin of 2 pi m / 7, m = 1, 2, 3
        const float c[3] = {0.62348980185873353f, -0.22252093395631440f, -0.90096886790241913f};
        const float sn[3] = {0.78183148246802981f, 0.97492791218182361f, 0.43388373911755812f};
        float2 t[3], d[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            t[m] = cadd(u[1 + m], u[6 - m]);
            d[m] = csub(u[1 + m], u[6 - m]);
        }
        const float2 u0 = u[0];
        u[0] = cadd(u0, cadd(t[0], cadd(t[1], t[2])));
#pragma unroll
        for (int q = 1; q <= 3; ++q) {
            float2 a = u0, b = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int e = ((m + 1) * q) % 7;                  // angle index 1..6
                const int ei = e <= 3 ? e - 1 : 6 - e;             // cos/sin of 2 pi (ei+1) / 7
                const float cs = c[ei], ss = e <= 3 ? sn[ei] : -sn[ei];
                a = make_float2(fmaf(cs, t[m].x, a.x), fmaf(cs, t[m].y, a.y));
                b = make_float2(fmaf(ss, d[m].x, b.x), fmaf(ss, d[m].y, b.y));
            }
            const float2 bi = mul_si<SIGN>(b);
            u[q] = cadd(a, bi);
            u[7 - q] = csub(a, bi);
        }
    }
};

template <int SIGN>
struct Dft<8, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        float2 e[4] = {u[0], u[2], u[4], u[6]}, o[4] = {u[1], u[3], u[5], u[7]};
        Dft<4, SIGN>::run(e);
        Dft<4, SIGN>::run(o);
        const float r = 0.70710678118654752f, sg = (float)SIGN;
        const float2 o1 = cmul(o[1], make_float2(r, sg * r));
        const float2 o2 = mul_si<SIGN>(o[2]);
        const float2 o3 = cmul(o[3], make_float2(-r, sg * r));
        u[0] = cadd(e[0], o[0]);
        u[4] = csub(e[0], o[0]);
        u[1] = cadd(e[1], o1);
        u[5] = csub(e[1], o1);
        u[2] = cadd(e[2], o2);
        u[6] = csub(e[2], o2);
        u[3] = cadd(e[3], o3);
        u[7] = csub(e[3], o3);
    }
};

// One Stockham stage of radix R over the NL lines of a block (line stride
// ls in the point index).  tw: e^{-2 pi i e / L}, e = 0 .. L - 1.
template <int R, int SIGN>
__device__ __forceinline__ void fft_stage(const float2 *__restrict__ a, float2 *__restrict__ b, int L, int p, int NL,
                                          int ls, const float2 *__restrict__ tw)
{
    const int LR = L / R, tws = L / (p * R), nb = LR * NL;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int i = idx / NL, l = idx - i * NL;
        const int k = i % p;
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = a[(i + r * LR) * ls + l];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * k * tws];          // r k tws < L
                if (SIGN > 0) w.y = -w.y;
                u[r] = cmul(u[r], w);
            }
        }
        Dft<R, SIGN>::run(u);
        const int j = (i - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) b[(j + r * p) * ls + l] = u[r];
    }
}

// Transform the NL lines held in a (point-major, line stride ls); returns
// the buffer that holds the result (a or b).  Ends with a barrier.
template <int SIGN>
__device__ float2 *fft_lines(float2 *a, float2 *b, int NL, int ls, const FftPlan &pl, const float2 *tw)
{
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.radix[s], p = pl.p[s];
        switch (R) {
        case 2: fft_stage<2, SIGN>(a, b, pl.L, p, NL, ls, tw); break;
        case 3: fft_stage<3, SIGN>(a, b, pl.L, p, NL, ls, tw); break;
        case 4: fft_stage<4, SIGN>(a, b, pl.L, p, NL, ls, tw); break;
        case 5: fft_stage<5, SIGN>(a, b, pl.L, p, NL, ls, tw); break;
        case 6: fft_stage<6, SIGN>(a, b, pl.L, p, NL, ls, tw); break;
        case 7: fft_stage<7, SIGN>(a, b, pl.L, p, NL, ls, tw); break;
        default: fft_stage<8, SIGN>(a, b, pl.L, p, NL, ls, tw); break;
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    return a;
}

__device__ __forceinline__ void load_twiddles(float2 *stw, const float2 *__restrict__ tw, int L)
{
    for (int e = threadIdx.x; e < L; e += blockDim.x) stw[e] = tw[e];
}

// ---------------------------------------------------------------------------
// Pass Z: r2c along z.  Block: 2 * ZL consecutive rows (x, y) of L reals, as
// ZL complex lines; out: [rows][Lh] complex.
__global__ void __launch_bounds__(256) k_fft_z_r2c(FftPlan pl, int nrows, const float *__restrict__ in,
                                                   float2 *__restrict__ out, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int L = pl.L, Lh = pl.Lh, ZL = pl.zl, ls = ZL + 1;
    float2 *stw = sm, *a = sm + L, *b = a + L * ls;
    load_twiddles(stw, tw, L);
    const int row0 = blockIdx.x * 2 * ZL;
    for (int e = threadIdx.x; e < 2 * ZL * L; e += blockDim.x) {
        const int rr = e / L, n = e - rr * L;
        const int row = row0 + rr;
        const float v = row < nrows ? in[(int64_t)row * L + n] : 0.f;
        float *dst = reinterpret_cast<float *>(&a[n * ls + (rr >> 1)]);
        dst[rr & 1] = v;
    }
    __syncthreads();
    const float2 *z = fft_lines<-1>(a, b, ZL, ls, pl, stw);
    for (int e = threadIdx.x; e < 2 * ZL * Lh; e += blockDim.x) {
        const int rr = e / Lh, k = e - rr * Lh;
        const int row = row0 + rr;
        if (row >= nrows) continue;
        const int q = rr >> 1;
        const float2 zk = z[k * ls + q], zm = z[(k == 0 ? 0 : L - k) * ls + q];
        // X = (Z_k + conj Z_{L-k}) / 2,  Y = (Z_k - conj Z_{L-k}) / 2i
        const float2 v = (rr & 1) ? make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x))
                                  : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        out[(int64_t)row * Lh + k] = v;
    }
}

// Pass Z': c2r along z.  in: [rows][Lh] half spectra; out: [rows][L] reals.
__global__ void __launch_bounds__(256) k_fft_z_c2r(FftPlan pl, int nrows, const float2 *__restrict__ in,
                                                   float *__restrict__ out, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int L = pl.L, Lh = pl.Lh, ZL = pl.zl, ls = ZL + 1;
    float2 *stw = sm, *a = sm + L, *b = a + L * ls;
    load_twiddles(stw, tw, L);
    const int row0 = blockIdx.x * 2 * ZL;
    // Z_k = X_k + i Y_k over k = 0 .. L-1, X_{L-k} = conj X_k (Hermitian rows)
    for (int e = threadIdx.x; e < ZL * L; e += blockDim.x) {
        const int q = e / L, k = e - q * L;
        const int r0 = row0 + 2 * q, r1 = r0 + 1;
        const bool lowh = k < Lh;
        const int kk = lowh ? k : L - k;
        float2 X = r0 < nrows ? in[(int64_t)r0 * Lh + kk] : make_float2(0.f, 0.f);
        float2 Y = r1 < nrows ? in[(int64_t)r1 * Lh + kk] : make_float2(0.f, 0.f);
        if (kk == 0 || 2 * kk == L) {
            X.y = 0.f;
            Y.y = 0.f;
        }
        if (!lowh) {
            X.y = -X.y;
            Y.y = -Y.y;
        }
        a[k * ls + q] = make_float2(X.x - Y.y, X.y + Y.x);
    }
    __syncthreads();
    const float2 *z = fft_lines<1>(a, b, ZL, ls, pl, stw);
    for (int e = threadIdx.x; e < 2 * ZL * L; e += blockDim.x) {
        const int rr = e / L, n = e - rr * L;
        const int row = row0 + rr;
        if (row >= nrows) continue;
        const float2 v = z[n * ls + (rr >> 1)];
        out[(int64_t)row * L + n] = (rr & 1) ? v.y : v.x;
    }
}

// Pass Y / Y': complex FFT along y, in place.  Block (kz tile, x): the TK
// columns kz0 .. kz0 + TK - 1 of the plane x, all L values of y.
template <int SIGN>
__global__ void __launch_bounds__(256) k_fft_y(FftPlan pl, float2 *__restrict__ s, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int L = pl.L, Lh = pl.Lh, TK = pl.tk;
    float2 *stw = sm, *a = sm + L, *b = a + L * TK;
    load_twiddles(stw, tw, L);
    const int kz0 = blockIdx.x * TK, x = blockIdx.y;
    float2 *base = s + (int64_t)x * L * Lh + kz0;
    for (int e = threadIdx.x; e < L * TK; e += blockDim.x) {
        const int y = e / TK, l = e - y * TK;
        a[y * TK + l] = kz0 + l < Lh ? base[(int64_t)y * Lh + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2 *z = fft_lines<SIGN>(a, b, TK, TK, pl, stw);
    for (int e = threadIdx.x; e < L * TK; e += blockDim.x) {
        const int y = e / TK, l = e - y * TK;
        if (kz0 + l < Lh) base[(int64_t)y * Lh + l] = z[y * TK + l];
    }
}

// Pass X: forward FFT along x, the energy sum, and with forces the product
// with D and the inverse FFT along x, in place.  Block (kz tile, y).
// mode 0: energy only; 1: energy, D rho^ and the inverse along x written
// back (forces); 2: the forward transform written back (no energy; tests).
__global__ void __launch_bounds__(256) k_fft_x_spectral(FftPlan pl, float2 *__restrict__ s,
                                                        const float *__restrict__ D, const float2 *__restrict__ tw,
                                                        int mode, double *__restrict__ part)
{
    extern __shared__ float2 sm[];
    __shared__ double sred[8];
    const int L = pl.L, Lh = pl.Lh, TK = pl.tk;
    float2 *stw = sm, *a = sm + L, *b = a + L * TK;
    load_twiddles(stw, tw, L);
    const int kz0 = blockIdx.x * TK, y = blockIdx.y;
    const int64_t pstride = (int64_t)L * Lh;          // between x planes
    float2 *base = s + (int64_t)y * Lh + kz0;
    const float *Db = D + (int64_t)y * Lh + kz0;
    for (int e = threadIdx.x; e < L * TK; e += blockDim.x) {
        const int x = e / TK, l = e - x * TK;
        a[x * TK + l] = kz0 + l < Lh ? base[x * pstride + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 *z = fft_lines<-1>(a, b, TK, TK, pl, stw);
    if (mode == 2) {
        for (int e = threadIdx.x; e < L * TK; e += blockDim.x) {
            const int x = e / TK, l = e - x * TK;
            if (kz0 + l < Lh) base[x * pstride + l] = z[x * TK + l];
        }
        return;
    }
    const bool forces = mode == 1;
    float2 *o = z == a ? b : a;
    const bool even = (L & 1) == 0;
    double en = 0.0;
    for (int e = threadIdx.x; e < L * TK; e += blockDim.x) {
        const int x = e / TK, l = e - x * TK;
        const int kz = kz0 + l;
        if (kz >= Lh) continue;
        const float d = Db[x * pstride + l];
        float2 c = z[x * TK + l];
        const float w = (kz == 0 || (even && kz == Lh - 1)) ? 1.f : 2.f;
        en += (double)(w * d * (c.x * c.x + c.y * c.y));
        if (forces) z[x * TK + l] = cscale(c, d);
    }
    // fixed-order block sum of the energy partials
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) en += __shfl_down_sync(0xffffffffu, en, off);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = en;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sred[w];
        part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
    if (!forces) return;
    z = fft_lines<1>(z, o, TK, TK, pl, stw);
    for (int e = threadIdx.x; e < L * TK; e += blockDim.x) {
        const int x = e / TK, l = e - x * TK;
        if (kz0 + l < Lh) base[x * pstride + l] = z[x * TK + l];
    }
}

// ---------------------------------------------------------------------------
// Host side

bool fft_prepare(Handle &H, std::string &err)
{
    FftPlan &pl = H.fft;
    const int L = H.g.nf;
    pl.L = L;
    pl.Lh = L / 2 + 1;
    // fewest stages, larger radices first
    std::vector<int> best, cur;
    std::function<void(int)> rec = [&](int m) {
        if (m == 1) {
            if (best.empty() || cur.size() < best.size()) best = cur;
            return;
        }
        if (!best.empty() && cur.size() + 1 >= best.size()) return;
        for (int r : {8, 7, 6, 5, 4, 3, 2})
            if (m % r == 0) {
                cur.push_back(r);
                rec(m / r);
                cur.pop_back();
            }
    };
    rec(L);
    if (best.empty() || (int)best.size() > kFftMaxStages) {
        err = "FFT length " + std::to_string(L) + " has a prime factor above 7";
        return false;
    }
    pl.nst = (int)best.size();
    int p = 1;
    for (int s = 0; s < pl.nst; ++s) {
        pl.radix[s] = best[s];
        pl.p[s] = p;
        p *= best[s];
    }
    pl.tk = L <= 512 ? 16 : 8;
    pl.zl = L <= 512 ? 8 : 4;
    std::vector<float2> tw(L);
    for (int e = 0; e < L; ++e) {
        const double ang = -2.0 * M_PI * (double)e / (double)L;
        tw[e] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    if (cudaMalloc(&H.d_tw, sizeof(float2) * L) != cudaSuccess ||
        cudaMemcpy(H.d_tw, tw.data(), sizeof(float2) * L, cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "FFT twiddle table";
        return false;
    }
    H.device_bytes += (int64_t)sizeof(float2) * L;
    const int sz = (int)(sizeof(float2) * (L + 2 * L * (pl.zl + 1)));
    const int sy = (int)(sizeof(float2) * (L + 2 * L * pl.tk));
    if (cudaFuncSetAttribute(k_fft_z_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, sz) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_z_c2r, cudaFuncAttributeMaxDynamicSharedMemorySize, sz) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_x_spectral, cudaFuncAttributeMaxDynamicSharedMemorySize, sy) != cudaSuccess) {
        err = "cudaFuncSetAttribute (FFT shared memory)";
        return false;
    }
    return true;
}

int spectral_blocks(const Handle &H)
{
    const int L = H.g.nf, tk = L <= 512 ? 16 : 8;
    return ((L / 2 + 1 + tk - 1) / tk) * L;
}

static size_t smem_z(const FftPlan &pl) { return sizeof(float2) * (pl.L + 2 * pl.L * (pl.zl + 1)); }
static size_t smem_y(const FftPlan &pl) { return sizeof(float2) * (pl.L + 2 * pl.L * pl.tk); }

cudaError_t launch_fft_forward(Handle &H, cudaStream_t s)
{
    const FftPlan &pl = H.fft;
    const int nrows = pl.L * pl.L;
    float2 *spec = reinterpret_cast<float2 *>(H.d_rhohat);
    k_fft_z_r2c<<<(nrows + 2 * pl.zl - 1) / (2 * pl.zl), 256, smem_z(pl), s>>>(pl, nrows, H.d_rho, spec, H.d_tw);
    const dim3 g((pl.Lh + pl.tk - 1) / pl.tk, pl.L);
    k_fft_y<-1><<<g, 256, smem_y(pl), s>>>(pl, spec, H.d_tw);
    return cudaGetLastError();
}

cudaError_t launch_spectral(Handle &H, bool forces, cudaStream_t s)
{
    const FftPlan &pl = H.fft;
    const dim3 g((pl.Lh + pl.tk - 1) / pl.tk, pl.L);
    k_fft_x_spectral<<<g, 256, smem_y(pl), s>>>(pl, reinterpret_cast<float2 *>(H.d_rhohat), H.d_D, H.d_tw,
                                                forces ? 1 : 0, H.d_part + H.part_off[kPartGlob]);
    return cudaGetLastError();
}

static cudaError_t launch_forward_x_only(Handle &H, cudaStream_t s)
{
    const FftPlan &pl = H.fft;
    const dim3 g((pl.Lh + pl.tk - 1) / pl.tk, pl.L);
    k_fft_x_spectral<<<g, 256, smem_y(pl), s>>>(pl, reinterpret_cast<float2 *>(H.d_rhohat), H.d_D, H.d_tw, 2,
                                                H.d_part + H.part_off[kPartGlob]);
    return cudaGetLastError();
}

cudaError_t launch_fft_inverse(Handle &H, cudaStream_t s)
{
    const FftPlan &pl = H.fft;
    const int nrows = pl.L * pl.L;
    float2 *spec = reinterpret_cast<float2 *>(H.d_rhohat);
    const dim3 g((pl.Lh + pl.tk - 1) / pl.tk, pl.L);
    k_fft_y<1><<<g, 256, smem_y(pl), s>>>(pl, spec, H.d_tw);
    k_fft_z_c2r<<<(nrows + 2 * pl.zl - 1) / (2 * pl.zl), 256, smem_z(pl), s>>>(pl, nrows, spec, H.d_phi, H.d_tw);
    return cudaGetLastError();
}

}  // namespace ankh

using namespace ankh;


extern "C" int ankh_debug_fft(ankh_handle *hh, const float *rho, const float *D, int mode, double *E_glob,
                              void *out, void *cuda_stream)
{
    if (!hh || !rho || !out || (mode == 1 && !E_glob)) {
        set_error("ankh_debug_fft: handle, rho, out (and E_glob for mode 1) are required");
        return ANKH_EINVAL;
    }
    Handle &H = hh->h;
    if (H.fmm.enabled || !H.d_tw) {
        set_error("ankh_debug_fft: the handle has no merged-grid FFT (ANKH-FMM)");
        return ANKH_EINVAL;
    }
    if (mode != 0 && mode != 1) {
        set_error("ankh_debug_fft: mode must be 0 (forward) or 1 (far-field step)");
        return ANKH_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t nspec = (int64_t)H.g.nf * H.g.nf * H.g.nfh;
    float *D_keep = H.d_D, *D_tmp = nullptr;
    auto done = [&](cudaError_t e, const char *what) {
        H.d_D = D_keep;
        if (D_tmp) cudaFree(D_tmp);
        if (e != cudaSuccess) {
            set_error(std::string("ankh_debug_fft: ") + what + ": " + cudaGetErrorString(e));
            return ANKH_ECUDA;
        }
        return ANKH_OK;
    };
    cudaError_t e = cudaMemcpyAsync(H.d_rho, rho, sizeof(float) * H.g.M, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return done(e, "copy rho");
    if (D) {
        if ((e = cudaMalloc(&D_tmp, sizeof(float) * nspec)) != cudaSuccess) return done(e, "cudaMalloc D");
        if ((e = cudaMemcpyAsync(D_tmp, D, sizeof(float) * nspec, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return done(e, "copy D");
        H.d_D = D_tmp;
    }
    if ((e = launch_fft_forward(H, s)) != cudaSuccess) return done(e, "forward passes");
    if (mode == 0) {
        if ((e = launch_forward_x_only(H, s)) != cudaSuccess) return done(e, "forward along x");
        e = cudaMemcpyAsync(out, H.d_rhohat, sizeof(float2) * nspec, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return done(e, "copy spectrum");
    }
    if ((e = launch_spectral(H, true, s)) != cudaSuccess) return done(e, "spectral pass");
    if ((e = launch_fft_inverse(H, s)) != cudaSuccess) return done(e, "inverse passes");
    const int nb = spectral_blocks(H);
    std::vector<double> part(nb);
    e = cudaMemcpyAsync(part.data(), H.d_part + H.part_off[kPartGlob], sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, H.d_phi, sizeof(float) * H.g.M, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    double t = 0.0;
    for (double v : part) t += v;
    *E_glob = t / (2.0 * (double)H.g.M);
    return done(e, "copy results");
}
