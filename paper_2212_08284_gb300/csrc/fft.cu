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

#include <algorithm>
#include <cmath>
#include <functional>
#include <numeric>
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
struct Dft<9, SIGN> {
    static __device__ __forceinline__ void run(float2 *u)
    {
        // 9 = 3 x 3: X[k1 + 3 k2] = DFT_3 over b of w^(b k1) Y[b][k1],
        // Y[b][.] = DFT_3 over a of u[3a + b], w = e^{SIGN 2 pi i / 9}
        float2 y[3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float2 e[3] = {u[b], u[b + 3], u[b + 6]};
            Dft<3, SIGN>::run(e);
            y[b][0] = e[0];
            y[b][1] = e[1];
            y[b][2] = e[2];
        }
        const float sg = (float)SIGN;
        const float2 w1 = make_float2(0.76604444311897804f, sg * 0.64278760968653933f);    // 40 degrees
        const float2 w2 = make_float2(0.17364817766693035f, sg * 0.98480775301220806f);    // 80
        const float2 w4 = make_float2(-0.93969262078590838f, sg * 0.34202014332566873f);   // 160
        y[1][1] = cmul(y[1][1], w1);
        y[1][2] = cmul(y[1][2], w2);
        y[2][1] = cmul(y[2][1], w2);
        y[2][2] = cmul(y[2][2], w4);
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            float2 f[3] = {y[0][k1], y[1][k1], y[2][k1]};
            Dft<3, SIGN>::run(f);
            u[k1] = f[0];
            u[k1 + 3] = f[1];
            u[k1 + 6] = f[2];
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
// ls in the point index).  Butterfly f covers line f mod NL and index
// i = f / NL of the stage; k = i mod p with the division by p done as a
// multiplication by mag = ceil(2^20 / p) (exact for i, p < 1024, checked on
// the host).  The twiddles W^(r k L/(p R)), r = 1 .. R-1, are powers of the
// one read from the table.  tw: e^{-2 pi i e / L}, e = 0 .. L - 1.
template <int R, int SIGN, int NL>
__device__ __forceinline__ void fft_stage(const float2 *__restrict__ a, float2 *__restrict__ b, int L, int p,
                                          unsigned mag, int ls, const float2 *__restrict__ tw)
{
    constexpr int LG = NL == 16 ? 4 : (NL == 8 ? 3 : (NL == 4 ? 2 : 1));
    const int LR = L / R, tws = L / (p * R), nb = LR * NL;
    for (int f = threadIdx.x; f < nb; f += blockDim.x) {
        const int l = f & (NL - 1), i = f >> LG;
        const int g = (int)(((unsigned)i * mag) >> 20);
        const int k = i - g * p;
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = a[(i + r * LR) * ls + l];
        if (k != 0) {
            float2 w1 = tw[k * tws];
            if (SIGN > 0) w1.y = -w1.y;
            float2 w = w1;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                u[r] = cmul(u[r], w);
                if (r + 1 < R) w = cmul(w, w1);
            }
        }
        Dft<R, SIGN>::run(u);
        const int j = g * p * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) b[(j + r * p) * ls + l] = u[r];
    }
}

// Transform the NL lines held in a (point-major, line stride ls); returns
// the buffer that holds the result (a or b).  Ends with a barrier.
template <int SIGN, int NL>
__device__ float2 *fft_lines(float2 *a, float2 *b, int ls, const FftPlan &pl, const float2 *tw)
{
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.radix[s], p = pl.p[s];
        const unsigned mag = pl.mag[s];
        switch (R) {
        case 2: fft_stage<2, SIGN, NL>(a, b, pl.L, p, mag, ls, tw); break;
        case 3: fft_stage<3, SIGN, NL>(a, b, pl.L, p, mag, ls, tw); break;
        case 4: fft_stage<4, SIGN, NL>(a, b, pl.L, p, mag, ls, tw); break;
        case 5: fft_stage<5, SIGN, NL>(a, b, pl.L, p, mag, ls, tw); break;
        case 6: fft_stage<6, SIGN, NL>(a, b, pl.L, p, mag, ls, tw); break;
        case 7: fft_stage<7, SIGN, NL>(a, b, pl.L, p, mag, ls, tw); break;
        default: fft_stage<8, SIGN, NL>(a, b, pl.L, p, mag, ls, tw); break;
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    return a;
}

// q / d for the d of a plan: (q m) >> 32 with m = floor(2^32 / d) + 1
// (exact for the q, d of the plans, checked on the host)
__device__ __forceinline__ int udiv(int q, unsigned m) { return (int)__umulhi((unsigned)q, m); }

__device__ __forceinline__ void load_twiddles(float2 *stw, const float2 *__restrict__ tw, int L)
{
    for (int e = threadIdx.x; e < L; e += blockDim.x) stw[e] = tw[e];
}

// ---------------------------------------------------------------------------
// Pass Z: r2c along z.  Block: 2 ZL consecutive rows (x, y) of L reals, as
// ZL complex lines; out: [rows][Lh] complex.
template <int ZL>
__global__ void __launch_bounds__(512) k_fft_z_r2c(FftPlan pl, int nrows, const float *__restrict__ in,
                                                   float2 *__restrict__ out, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int L = pl.L, Lh = pl.Lh;
    constexpr int ls = ZL + 1;
    float2 *stw = sm, *a = sm + L, *b = a + L * ls;
    load_twiddles(stw, tw, L);
    const int row0 = blockIdx.x * 2 * ZL;
    const int tot = 2 * ZL * L;
    const float *src = in + (int64_t)row0 * L;              // the block's rows are contiguous
    const int64_t avail = ((int64_t)nrows - row0) * L;      // values left in the input
    float *af = reinterpret_cast<float *>(a);
    for (int f0 = threadIdx.x; f0 < tot; f0 += 8 * blockDim.x) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int f = f0 + u * blockDim.x;
            v[u] = (f < tot && f < avail) ? src[f] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int f = f0 + u * blockDim.x;
            if (f < tot) {
                const int rr = udiv(f, pl.magL), n = f - rr * L;
                af[2 * (n * ls + (rr >> 1)) + (rr & 1)] = v[u];
            }
        }
    }
    __syncthreads();
    const float2 *z = fft_lines<-1, ZL>(a, b, ls, pl, stw);
    const int toto = 2 * ZL * Lh;
    for (int f = threadIdx.x; f < toto; f += blockDim.x) {
        const int rr = udiv(f, pl.magLh), k = f - rr * Lh;
        const int row = row0 + rr;
        if (row >= nrows) continue;
        const int q = rr >> 1;
        const float2 zk = z[k * ls + q], zm = z[(k == 0 ? 0 : L - k) * ls + q];
        // X = (Z_k + conj Z_{L-k}) / 2,  Y = (Z_k - conj Z_{L-k}) / 2i
        const float2 v = (rr & 1) ? make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x))
                                  : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        out[(int64_t)row0 * Lh + f] = v;                    // rows of Lh values, contiguous
    }
}

// Pass Z': c2r along z.  in: [rows][Lh] half spectra; out: [rows][L] reals.
template <int ZL>
__global__ void __launch_bounds__(512) k_fft_z_c2r(FftPlan pl, int nrows, const float2 *__restrict__ in,
                                                   float *__restrict__ out, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int L = pl.L, Lh = pl.Lh;
    constexpr int ls = ZL + 1;
    float2 *stw = sm, *a = sm + L, *b = a + L * ls;
    load_twiddles(stw, tw, L);
    const int row0 = blockIdx.x * 2 * ZL;
    // Z_k = X_k + i Y_k over k = 0 .. L-1, X_{L-k} = conj X_k (Hermitian rows)
    const int tot = ZL * L;
    for (int f0 = threadIdx.x; f0 < tot; f0 += 4 * blockDim.x) {
        float2 X[4], Y[4];
        int kk4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int f = f0 + u * blockDim.x;
            const int q = udiv(f, pl.magL), k = f - q * L;
            const int r0 = row0 + 2 * q, r1 = r0 + 1;
            const int kk = k < Lh ? k : L - k;
            kk4[u] = kk;
            X[u] = (f < tot && r0 < nrows) ? in[(int64_t)r0 * Lh + kk] : make_float2(0.f, 0.f);
            Y[u] = (f < tot && r1 < nrows) ? in[(int64_t)r1 * Lh + kk] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int f = f0 + u * blockDim.x;
            if (f >= tot) continue;
            const int q = udiv(f, pl.magL), k = f - q * L;
            float2 x = X[u], y = Y[u];
            if (kk4[u] == 0 || 2 * kk4[u] == L) {
                x.y = 0.f;
                y.y = 0.f;
            }
            if (k >= Lh) {
                x.y = -x.y;
                y.y = -y.y;
            }
            a[k * ls + q] = make_float2(x.x - y.y, x.y + y.x);
        }
    }
    __syncthreads();
    const float2 *z = fft_lines<1, ZL>(a, b, ls, pl, stw);
    const float *zf = reinterpret_cast<const float *>(z);
    const int toto = 2 * ZL * L;
    for (int f = threadIdx.x; f < toto; f += blockDim.x) {
        const int rr = udiv(f, pl.magL), n = f - rr * L;
        if (row0 + rr >= nrows) continue;
        out[(int64_t)row0 * L + f] = zf[2 * (n * ls + (rr >> 1)) + (rr & 1)];
    }
}

// Load a tile of L points x TK lines (line l of point pos at
// base[pos * stride + l], lines beyond nvalid read as 0) into shared memory,
// point-major, with eight loads in flight per thread.
template <int TK>
__device__ __forceinline__ void tile_load(float2 *a, const float2 *__restrict__ base, int64_t stride, int L,
                                          bool full, int nvalid)
{
    constexpr int LG = TK == 16 ? 4 : 3;
    const int tot = L * TK;
    for (int f0 = threadIdx.x; f0 < tot; f0 += 8 * blockDim.x) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int f = f0 + u * blockDim.x;
            const int l = f & (TK - 1), pos = f >> LG;
            v[u] = (f < tot && (full || l < nvalid)) ? base[pos * stride + l] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int f = f0 + u * blockDim.x;
            if (f < tot) a[f] = v[u];
        }
    }
}

// Pass Y / Y': complex FFT along y, in place.  Block (kz tile, x): the TK
// columns kz0 .. kz0 + TK - 1 of the plane x, all L values of y.
template <int SIGN, int TK>
__global__ void __launch_bounds__(512) k_fft_y(FftPlan pl, float2 *__restrict__ s, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    constexpr int LG = TK == 16 ? 4 : 3;
    const int L = pl.L, Lh = pl.Lh;
    float2 *stw = sm, *a = sm + L, *b = a + L * TK;
    load_twiddles(stw, tw, L);
    const int kz0 = blockIdx.x * TK, x = blockIdx.y;
    float2 *base = s + (int64_t)x * L * Lh + kz0;
    const bool full = kz0 + TK <= Lh;
    tile_load<TK>(a, base, Lh, L, full, Lh - kz0);
    __syncthreads();
    const float2 *z = fft_lines<SIGN, TK>(a, b, TK, pl, stw);
    for (int f = threadIdx.x; f < L * TK; f += blockDim.x) {
        const int l = f & (TK - 1), y = f >> LG;
        if (full || kz0 + l < Lh) base[(int64_t)y * Lh + l] = z[f];
    }
}

// Pass X: forward FFT along x, the energy sum, and with forces the product
// with D and the inverse FFT along x, in place.  Block (kz tile, y).
// mode 0: energy only; 1: energy, D rho^ and the inverse along x written
// back (forces); 2: the forward transform written back (no energy; tests).
template <int TK>
__global__ void __launch_bounds__(512) k_fft_x_spectral(FftPlan pl, float2 *__restrict__ s,
                                                        const float *__restrict__ D, const float2 *__restrict__ tw,
                                                        int mode, double *__restrict__ part)
{
    extern __shared__ float2 sm[];
    __shared__ double sred[16];
    constexpr int LG = TK == 16 ? 4 : 3;
    const int L = pl.L, Lh = pl.Lh;
    float2 *stw = sm, *a = sm + L, *b = a + L * TK;
    load_twiddles(stw, tw, L);
    const int kz0 = blockIdx.x * TK, y = blockIdx.y;
    const int64_t pstride = (int64_t)L * Lh;          // between x planes
    float2 *base = s + (int64_t)y * Lh + kz0;
    const float *Db = D + (int64_t)y * Lh + kz0;
    const bool full = kz0 + TK <= Lh;
    float *sD = reinterpret_cast<float *>(b + L * TK);      // the D tile, loaded with the spectrum tile
    tile_load<TK>(a, base, pstride, L, full, Lh - kz0);
    if (mode != 2) {
        const int tot = L * TK;
        for (int f0 = threadIdx.x; f0 < tot; f0 += 8 * blockDim.x) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int f = f0 + u * blockDim.x;
                const int l = f & (TK - 1), x = f >> LG;
                v[u] = (f < tot && (full || kz0 + l < Lh)) ? Db[x * pstride + l] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int f = f0 + u * blockDim.x;
                if (f < tot) sD[f] = v[u];
            }
        }
    }
    __syncthreads();
    float2 *z = fft_lines<-1, TK>(a, b, TK, pl, stw);
    if (mode == 2) {
        for (int f = threadIdx.x; f < L * TK; f += blockDim.x) {
            const int l = f & (TK - 1), x = f >> LG;
            if (full || kz0 + l < Lh) base[x * pstride + l] = z[f];
        }
        return;
    }
    const bool forces = mode == 1;
    float2 *o = z == a ? b : a;
    const bool even = (L & 1) == 0;
    double en = 0.0;
    for (int f = threadIdx.x; f < L * TK; f += blockDim.x) {
        const int l = f & (TK - 1), x = f >> LG;
        const int kz = kz0 + l;
        if (kz >= Lh) continue;
        const float d = sD[f];
        const float2 c = z[f];
        const float w = (kz == 0 || (even && kz == Lh - 1)) ? 1.f : 2.f;
        en += (double)(w * d * (c.x * c.x + c.y * c.y));
        if (forces) z[f] = cscale(c, d);
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
    z = fft_lines<1, TK>(z, o, TK, pl, stw);
    for (int f = threadIdx.x; f < L * TK; f += blockDim.x) {
        const int l = f & (TK - 1), x = f >> LG;
        if (full || kz0 + l < Lh) base[x * pstride + l] = z[f];
    }
}

// ---------------------------------------------------------------------------
// Compile-time plans for the grid lengths of the library's default
// configurations and of boxes down to a few thousand atoms (the same
// Stockham stages, three of them, every index and trip count a constant).  The passes along y and x read their first stage's inputs from
// global memory and write their last stage's outputs there; the stages run
// in place in one shared tile (each thread reads all inputs of its
// butterflies, a barrier, then writes all outputs); the twiddles of a stage
// come from a per-stage table W^(r k L/(p R)), r = 1 .. R-1, k < p (1 for
// k = 0, so no branch).  Along x the forward transform's last stage keeps
// its outputs in registers for the spectral product, and the inverse runs
// the radices in reverse order, so that its first stage takes exactly those
// registers as inputs (forward stage 3, butterfly i, holds the points
// i + r L/R3, the inputs of inverse stage 1's butterfly i).
template <int L>
struct FftSpec;
template <>
struct FftSpec<216> {
    static constexpr int R1 = 6, R2 = 6, R3 = 6, NT = 288, MINB = 4;   // four blocks per SM: <= 56 registers
};
template <>
struct FftSpec<80> {
    static constexpr int R1 = 8, R2 = 5, R3 = 2, NT = 320;
};
template <>
struct FftSpec<72> {
    static constexpr int R1 = 8, R2 = 3, R3 = 3, NT = 192;
};
// the grids of smaller boxes (n = 6 .. 18 leaves per axis, L_u = 5 or 6)
template <>
struct FftSpec<24> {
    static constexpr int R1 = 4, R2 = 3, R3 = 2, NT = 96;
};
template <>
struct FftSpec<40> {
    static constexpr int R1 = 5, R2 = 4, R3 = 2, NT = 160;
};
template <>
struct FftSpec<45> {
    static constexpr int R1 = 5, R2 = 3, R3 = 3, NT = 128;
};
template <>
struct FftSpec<50> {
    static constexpr int R1 = 5, R2 = 5, R3 = 2, NT = 224;
};
template <>
struct FftSpec<60> {
    static constexpr int R1 = 5, R2 = 4, R3 = 3, NT = 160;
};
template <>
struct FftSpec<70> {
    static constexpr int R1 = 7, R2 = 5, R3 = 2, NT = 288;
};
template <>
struct FftSpec<75> {
    static constexpr int R1 = 5, R2 = 5, R3 = 3, NT = 224;
};
template <>
struct FftSpec<90> {
    static constexpr int R1 = 6, R2 = 5, R3 = 3, NT = 256;
};
// eight lines per block: also the test length of the radix-9 butterfly and
// of the narrow tile of the 432-point plan
template <>
struct FftSpec<54> {
    static constexpr int R1 = 9, R2 = 3, R3 = 2, NT = 128, TK = 8;
};
// the zero-padded grid of the non-periodic 1,008,000-atom box (n = 53):
// eight lines per block (27 KB of shared memory)
template <>
struct FftSpec<432> {
    static constexpr int R1 = 8, R2 = 6, R3 = 9, NT = 288, TK = 8;
};

// the lengths with a compile-time plan
#define ANKH_FFT_SPEC_LENGTHS(X) X(24) X(40) X(45) X(50) X(54) X(60) X(70) X(72) X(75) X(80) X(90) X(216) X(432)

constexpr int kSpecTK = 16;   // lines per block (kz columns, or complex z lines): default

// lines per block of a plan (kSpecTK unless the plan says)
template <class F, class = void>
struct SpecLines {
    static constexpr int v = kSpecTK;
};
template <class F>
struct SpecLines<F, decltype((void)F::TK)> {
    static constexpr int v = F::TK;
};

// resident blocks per SM the launch bounds ask for (1 unless the plan says)
template <class F, class = void>
struct SpecMinBlocks {
    static constexpr int v = 1;
};
template <class F>
struct SpecMinBlocks<F, decltype((void)F::MINB)> {
    static constexpr int v = F::MINB;
};

template <int L, int R, int NT, int TK = kSpecTK>
struct SpecStage {
    static constexpr int LR = L / R, NB = LR * TK, NBT = (NB + NT - 1) / NT;
};

// Butterfly f of a stage: line and index.  Line-fastest (the passes along y
// and x, whose lines are adjacent in memory) or index-fastest (the passes
// along z, whose points are).
template <int LR, int TK, bool IFAST>
__device__ __forceinline__ void spec_li(int f, int &l, int &i)
{
    if (IFAST) {
        l = f / LR;
        i = f - l * LR;
    } else {
        l = f % TK;
        i = f / TK;
    }
}

// Twiddle table of a stage (radix R, p earlier points): t[k (R-1) + r-1] =
// W^(r k L/(p R)) with W = e^{SIGN 2 pi i / L}, from the e^{-2 pi i e / L} table.
template <int L, int R, int P, int SIGN, int NT>
__device__ __forceinline__ void spec_twiddles(float2 *t, const float2 *__restrict__ tw)
{
    constexpr int TWS = L / (P * R);
    for (int e = threadIdx.x; e < P * (R - 1); e += NT) {
        const int k = e / (R - 1), r = e % (R - 1) + 1;
        float2 w = tw[(r * k * TWS) % L];
        if (SIGN > 0) w.y = -w.y;
        t[e] = w;
    }
}

// This thread's butterflies of a stage: m-th one is f = threadIdx.x + m NT,
// its line l and index i from spec_li; inputs at points i + r L/R.
template <int L, int R, int NT, int TK = kSpecTK, bool IFAST = false, class Src>
__device__ __forceinline__ void spec_gather(float2 (&u)[SpecStage<L, R, NT, TK>::NBT][R], Src src)
{
    using S = SpecStage<L, R, NT, TK>;
#pragma unroll
    for (int m = 0; m < S::NBT; ++m) {
        const int f = threadIdx.x + m * NT;
        if (S::NB % NT == 0 || f < S::NB) {
            int l, i;
            spec_li<S::LR, TK, IFAST>(f, l, i);
#pragma unroll
            for (int r = 0; r < R; ++r) u[m][r] = src(i + r * S::LR, l);
        }
    }
}

template <int L, int R, int P, int SIGN, int NT, int TK = kSpecTK, bool IFAST = false>
__device__ __forceinline__ void spec_butterflies(float2 (&u)[SpecStage<L, R, NT, TK>::NBT][R], const float2 *t)
{
    using S = SpecStage<L, R, NT, TK>;
#pragma unroll
    for (int m = 0; m < S::NBT; ++m) {
        const int f = threadIdx.x + m * NT;
        if (S::NB % NT == 0 || f < S::NB) {
            if (P > 1) {
                int l, i;
                spec_li<S::LR, TK, IFAST>(f, l, i);
                const int k = i % P;
#pragma unroll
                for (int r = 1; r < R; ++r) u[m][r] = cmul(u[m][r], t[k * (R - 1) + r - 1]);
            }
            Dft<R, SIGN>::run(u[m]);
        }
    }
}

// outputs of butterfly i at points (i / p) p R + i mod p + r p
template <int L, int R, int P, int NT, int TK = kSpecTK, bool IFAST = false, class Dst>
__device__ __forceinline__ void spec_scatter(const float2 (&u)[SpecStage<L, R, NT, TK>::NBT][R], Dst dst)
{
    using S = SpecStage<L, R, NT, TK>;
#pragma unroll
    for (int m = 0; m < S::NBT; ++m) {
        const int f = threadIdx.x + m * NT;
        if (S::NB % NT == 0 || f < S::NB) {
            int l, i;
            spec_li<S::LR, TK, IFAST>(f, l, i);
            const int j = (i / P) * P * R + i % P;
#pragma unroll
            for (int r = 0; r < R; ++r) dst(j + r * P, l, u[m][r]);
        }
    }
}

// Pass Y / Y' for a compile-time length: the TK columns kz0 .. kz0 + TK - 1
// of the plane x, all L values of y, in place in global memory.
template <int L, int SIGN>
__global__ void __launch_bounds__(FftSpec<L>::NT, SpecMinBlocks<FftSpec<L>>::v) k_fft_y_spec(int Lh, float2 *__restrict__ s,
                                                             const float2 *__restrict__ tw)
{
    using F = FftSpec<L>;
    constexpr int NT = F::NT, R1 = F::R1, R2 = F::R2, R3 = F::R3, TK = SpecLines<F>::v;
    __shared__ float2 a[L * TK];
    __shared__ float2 t2[R1 * (R2 - 1)], t3[R1 * R2 * (R3 - 1)];
    spec_twiddles<L, R2, R1, SIGN, NT>(t2, tw);
    spec_twiddles<L, R3, R1 * R2, SIGN, NT>(t3, tw);
    const int kz0 = blockIdx.x * TK, x = blockIdx.y;
    float2 *base = s + (int64_t)x * L * Lh + kz0;
    const int nvalid = min(TK, Lh - kz0);
    {
        float2 u[SpecStage<L, R1, NT, TK>::NBT][R1];
        spec_gather<L, R1, NT, TK>(u, [&](int pos, int l) {
            return l < nvalid ? base[(int64_t)pos * Lh + l] : make_float2(0.f, 0.f);
        });
        spec_butterflies<L, R1, 1, SIGN, NT, TK>(u, nullptr);
        spec_scatter<L, R1, 1, NT, TK>(u, [&](int pos, int l, float2 v) { a[pos * TK + l] = v; });
    }
    __syncthreads();
    {
        float2 u[SpecStage<L, R2, NT, TK>::NBT][R2];
        spec_gather<L, R2, NT, TK>(u, [&](int pos, int l) { return a[pos * TK + l]; });
        __syncthreads();
        spec_butterflies<L, R2, R1, SIGN, NT, TK>(u, t2);
        spec_scatter<L, R2, R1, NT, TK>(u, [&](int pos, int l, float2 v) { a[pos * TK + l] = v; });
    }
    __syncthreads();
    {
        float2 u[SpecStage<L, R3, NT, TK>::NBT][R3];
        spec_gather<L, R3, NT, TK>(u, [&](int pos, int l) { return a[pos * TK + l]; });
        spec_butterflies<L, R3, R1 * R2, SIGN, NT, TK>(u, t3);
        spec_scatter<L, R3, R1 * R2, NT, TK>(u, [&](int pos, int l, float2 v) {
            if (l < nvalid) base[(int64_t)pos * Lh + l] = v;
        });
    }
}

// Pass X for a compile-time length: forward FFT along x, the energy sum and
// with forces D rho^ and the inverse along x (modes as k_fft_x_spectral).
template <int L>
__global__ void __launch_bounds__(FftSpec<L>::NT, SpecMinBlocks<FftSpec<L>>::v) k_fft_x_spec(int Lh, float2 *__restrict__ s,
                                                             const float *__restrict__ D,
                                                             const float2 *__restrict__ tw, int mode,
                                                             double *__restrict__ part)
{
    using F = FftSpec<L>;
    constexpr int NT = F::NT, R1 = F::R1, R2 = F::R2, R3 = F::R3, TK = SpecLines<F>::v;
    __shared__ float2 a[L * TK];
    __shared__ float2 f2[R1 * (R2 - 1)], f3[R1 * R2 * (R3 - 1)];   // forward stages 2, 3
    __shared__ float2 i2[R3 * (R2 - 1)], i3[R3 * R2 * (R1 - 1)];   // inverse stages 2, 3 (radices R3, R2, R1)
    __shared__ double sred[NT / 32];
    spec_twiddles<L, R2, R1, -1, NT>(f2, tw);
    spec_twiddles<L, R3, R1 * R2, -1, NT>(f3, tw);
    spec_twiddles<L, R2, R3, 1, NT>(i2, tw);
    spec_twiddles<L, R1, R3 * R2, 1, NT>(i3, tw);
    const int kz0 = blockIdx.x * TK, y = blockIdx.y;
    const int64_t pstride = (int64_t)L * Lh;          // between x planes
    float2 *base = s + (int64_t)y * Lh + kz0;
    const float *Db = D + (int64_t)y * Lh + kz0;
    const int nvalid = min(TK, Lh - kz0);
    using S3 = SpecStage<L, R3, NT, TK>;
    // D at the frequencies this thread's forward stage-3 butterflies end
    // with, loaded first so that the loads overlap the forward stages
    float dv[S3::NBT][R3];
    if (mode != 2) {
#pragma unroll
        for (int m = 0; m < S3::NBT; ++m) {
            const int f = threadIdx.x + m * NT;
            const int l = f % TK, i = f / TK;
#pragma unroll
            for (int r = 0; r < R3; ++r)
                dv[m][r] = ((S3::NB % NT == 0 || f < S3::NB) && l < nvalid) ? Db[(i + r * S3::LR) * pstride + l]
                                                                             : 0.f;
        }
    }
    {
        float2 u[SpecStage<L, R1, NT, TK>::NBT][R1];
        spec_gather<L, R1, NT, TK>(u, [&](int pos, int l) {
            return l < nvalid ? base[pos * pstride + l] : make_float2(0.f, 0.f);
        });
        spec_butterflies<L, R1, 1, -1, NT, TK>(u, nullptr);
        spec_scatter<L, R1, 1, NT, TK>(u, [&](int pos, int l, float2 v) { a[pos * TK + l] = v; });
    }
    __syncthreads();
    {
        float2 u[SpecStage<L, R2, NT, TK>::NBT][R2];
        spec_gather<L, R2, NT, TK>(u, [&](int pos, int l) { return a[pos * TK + l]; });
        __syncthreads();
        spec_butterflies<L, R2, R1, -1, NT, TK>(u, f2);
        spec_scatter<L, R2, R1, NT, TK>(u, [&](int pos, int l, float2 v) { a[pos * TK + l] = v; });
    }
    __syncthreads();
    float2 u[S3::NBT][R3];
    spec_gather<L, R3, NT, TK>(u, [&](int pos, int l) { return a[pos * TK + l]; });
    spec_butterflies<L, R3, R1 * R2, -1, NT, TK>(u, f3);
    // forward stage 3, butterfly i (< L/R3 = R1 R2, so i / p = 0) holds the
    // frequencies kx = i + r L/R3
    if (mode == 2) {
        spec_scatter<L, R3, R1 * R2, NT, TK>(u, [&](int pos, int l, float2 v) {
            if (l < nvalid) base[pos * pstride + l] = v;
        });
        return;
    }
    const bool forces = mode == 1;
    const bool even = (L & 1) == 0;
    double en = 0.0;
#pragma unroll
    for (int m = 0; m < S3::NBT; ++m) {
        const int f = threadIdx.x + m * NT;
        if (S3::NB % NT == 0 || f < S3::NB) {
            const int l = f % TK, i = f / TK;
            const int kz = kz0 + l;
#pragma unroll
            for (int r = 0; r < R3; ++r) {
                const float2 c = u[m][r];
                const float d = dv[m][r];
                const float w = (kz == 0 || (even && kz == Lh - 1)) ? 1.f : 2.f;
                en += (double)(w * d * (c.x * c.x + c.y * c.y));
                u[m][r] = cscale(c, d);
            }
        }
    }
    // fixed-order block sum of the energy partials
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) en += __shfl_down_sync(0xffffffffu, en, off);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = en;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += sred[w];
        part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
    if (!forces) return;
    // inverse stage 1 (radix R3, no twiddles) on the registers
    spec_butterflies<L, R3, 1, 1, NT, TK>(u, nullptr);
    spec_scatter<L, R3, 1, NT, TK>(u, [&](int pos, int l, float2 v) { a[pos * TK + l] = v; });
    __syncthreads();
    {
        float2 v[SpecStage<L, R2, NT, TK>::NBT][R2];
        spec_gather<L, R2, NT, TK>(v, [&](int pos, int l) { return a[pos * TK + l]; });
        __syncthreads();
        spec_butterflies<L, R2, R3, 1, NT, TK>(v, i2);
        spec_scatter<L, R2, R3, NT, TK>(v, [&](int pos, int l, float2 w) { a[pos * TK + l] = w; });
    }
    __syncthreads();
    {
        float2 v[SpecStage<L, R1, NT, TK>::NBT][R1];
        spec_gather<L, R1, NT, TK>(v, [&](int pos, int l) { return a[pos * TK + l]; });
        spec_butterflies<L, R1, R3 * R2, 1, NT, TK>(v, i3);
        spec_scatter<L, R1, R3 * R2, NT, TK>(v, [&](int pos, int l, float2 w) {
            if (l < nvalid) base[pos * pstride + l] = w;
        });
    }
}

// Pass Z for a compile-time length: r2c along z.  Block: 2 TK consecutive
// rows (x, y) of L reals as TK complex lines (row 2q the real, row 2q + 1 the
// imaginary part of line q), lines held line-major in shared memory (points
// contiguous, as in global memory: the butterflies run index-fastest).
template <int L>
__global__ void __launch_bounds__(FftSpec<L>::NT, SpecMinBlocks<FftSpec<L>>::v) k_fft_z_r2c_spec(int nrows, const float *__restrict__ in,
                                                                 float2 *__restrict__ out,
                                                                 const float2 *__restrict__ tw)
{
    using F = FftSpec<L>;
    constexpr int NT = F::NT, R1 = F::R1, R2 = F::R2, R3 = F::R3, TK = SpecLines<F>::v, LP = L + 1, LH = L / 2 + 1;
    __shared__ float2 a[TK * LP];
    __shared__ float2 t2[R1 * (R2 - 1)], t3[R1 * R2 * (R3 - 1)];
    spec_twiddles<L, R2, R1, -1, NT>(t2, tw);
    spec_twiddles<L, R3, R1 * R2, -1, NT>(t3, tw);
    const int row0 = blockIdx.x * 2 * TK;
    {
        float2 u[SpecStage<L, R1, NT, TK>::NBT][R1];
        spec_gather<L, R1, NT, TK, true>(u, [&](int pos, int q) {
            const int r0 = row0 + 2 * q;
            const float re = r0 < nrows ? in[(int64_t)r0 * L + pos] : 0.f;
            const float im = r0 + 1 < nrows ? in[(int64_t)(r0 + 1) * L + pos] : 0.f;
            return make_float2(re, im);
        });
        spec_butterflies<L, R1, 1, -1, NT, TK, true>(u, nullptr);
        spec_scatter<L, R1, 1, NT, TK, true>(u, [&](int pos, int q, float2 v) { a[q * LP + pos] = v; });
    }
    __syncthreads();
    {
        float2 u[SpecStage<L, R2, NT, TK>::NBT][R2];
        spec_gather<L, R2, NT, TK, true>(u, [&](int pos, int q) { return a[q * LP + pos]; });
        __syncthreads();
        spec_butterflies<L, R2, R1, -1, NT, TK, true>(u, t2);
        spec_scatter<L, R2, R1, NT, TK, true>(u, [&](int pos, int q, float2 v) { a[q * LP + pos] = v; });
    }
    __syncthreads();
    {
        float2 u[SpecStage<L, R3, NT, TK>::NBT][R3];
        spec_gather<L, R3, NT, TK, true>(u, [&](int pos, int q) { return a[q * LP + pos]; });
        __syncthreads();
        spec_butterflies<L, R3, R1 * R2, -1, NT, TK, true>(u, t3);
        spec_scatter<L, R3, R1 * R2, NT, TK, true>(u, [&](int pos, int q, float2 v) { a[q * LP + pos] = v; });
    }
    __syncthreads();
    // X = (Z_k + conj Z_{L-k}) / 2,  Y = (Z_k - conj Z_{L-k}) / 2i,  k = 0 .. L/2
    for (int f = threadIdx.x; f < 2 * TK * LH; f += NT) {
        const int rr = f / LH, k = f - rr * LH;
        if (row0 + rr >= nrows) continue;
        const int q = rr >> 1;
        const float2 zk = a[q * LP + k], zm = a[q * LP + (k == 0 ? 0 : L - k)];
        const float2 v = (rr & 1) ? make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x))
                                  : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        out[(int64_t)row0 * LH + f] = v;                    // rows of L/2 + 1 values, contiguous
    }
}

// Pass Z' for a compile-time length: c2r along z.  Line q is Z_k = X_k + i Y_k
// of the Hermitian half rows 2q and 2q + 1 (X_{L-k} = conj X_k, the imaginary
// parts of X_0 and X_{L/2} dropped as for a real row); one inverse FFT; the
// real parts go to row 2q and the imaginary parts to row 2q + 1.
template <int L>
__global__ void __launch_bounds__(FftSpec<L>::NT, SpecMinBlocks<FftSpec<L>>::v) k_fft_z_c2r_spec(int nrows, const float2 *__restrict__ in,
                                                                 float *__restrict__ out,
                                                                 const float2 *__restrict__ tw)
{
    using F = FftSpec<L>;
    constexpr int NT = F::NT, R1 = F::R1, R2 = F::R2, R3 = F::R3, TK = SpecLines<F>::v, LP = L + 1, LH = L / 2 + 1;
    __shared__ float2 a[TK * LP];
    __shared__ float2 t2[R1 * (R2 - 1)], t3[R1 * R2 * (R3 - 1)];
    spec_twiddles<L, R2, R1, 1, NT>(t2, tw);
    spec_twiddles<L, R3, R1 * R2, 1, NT>(t3, tw);
    const int row0 = blockIdx.x * 2 * TK;
    {
        float2 u[SpecStage<L, R1, NT, TK>::NBT][R1];
        spec_gather<L, R1, NT, TK, true>(u, [&](int pos, int q) {
            const int r0 = row0 + 2 * q;
            const int kk = pos < LH ? pos : L - pos;
            float2 x = r0 < nrows ? in[(int64_t)r0 * LH + kk] : make_float2(0.f, 0.f);
            float2 y = r0 + 1 < nrows ? in[(int64_t)(r0 + 1) * LH + kk] : make_float2(0.f, 0.f);
            if (kk == 0 || 2 * kk == L) {
                x.y = 0.f;
                y.y = 0.f;
            }
            if (pos >= LH) {
                x.y = -x.y;
                y.y = -y.y;
            }
            return make_float2(x.x - y.y, x.y + y.x);
        });
        spec_butterflies<L, R1, 1, 1, NT, TK, true>(u, nullptr);
        spec_scatter<L, R1, 1, NT, TK, true>(u, [&](int pos, int q, float2 v) { a[q * LP + pos] = v; });
    }
    __syncthreads();
    {
        float2 u[SpecStage<L, R2, NT, TK>::NBT][R2];
        spec_gather<L, R2, NT, TK, true>(u, [&](int pos, int q) { return a[q * LP + pos]; });
        __syncthreads();
        spec_butterflies<L, R2, R1, 1, NT, TK, true>(u, t2);
        spec_scatter<L, R2, R1, NT, TK, true>(u, [&](int pos, int q, float2 v) { a[q * LP + pos] = v; });
    }
    __syncthreads();
    {
        float2 u[SpecStage<L, R3, NT, TK>::NBT][R3];
        spec_gather<L, R3, NT, TK, true>(u, [&](int pos, int q) { return a[q * LP + pos]; });
        spec_butterflies<L, R3, R1 * R2, 1, NT, TK, true>(u, t3);
        spec_scatter<L, R3, R1 * R2, NT, TK, true>(u, [&](int pos, int q, float2 v) {
            const int r0 = row0 + 2 * q;
            if (r0 < nrows) out[(int64_t)r0 * L + pos] = v.x;
            if (r0 + 1 < nrows) out[(int64_t)(r0 + 1) * L + pos] = v.y;
        });
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
    // division by p as (i mag) >> 20, checked for every index of the stage
    for (int st = 0; st < pl.nst; ++st) {
        const unsigned pp = (unsigned)pl.p[st];
        pl.mag[st] = (unsigned)(((1u << 20) + pp - 1) / pp);
        for (unsigned i = 0; i < (unsigned)L; ++i)
            if (((i * pl.mag[st]) >> 20) != i / pp) {
                err = "FFT index division check failed";
                return false;
            }
    }
    // threads per block: a multiple of 32 that divides the butterfly count of
    // every stage (every thread busy in every stage) when one of 128 .. 512
    // exists, else 256
    auto pick = [&](int NL) {
        int gg = 0;
        for (int st = 0; st < pl.nst; ++st) gg = std::gcd(gg, NL * (L / pl.radix[st]));
        for (int t = 512; t >= 128; t -= 32)
            if (gg % t == 0) return t;
        return 256;
    };
    pl.ty = pick(pl.tk);
    pl.tz = pick(pl.zl);
    // q / L and q / (L/2 + 1) as __umulhi(q, m), checked over the ranges used
    auto magic = [&](unsigned d, unsigned qmax, unsigned &m) {
        m = (unsigned)((1ull << 32) / d + 1);
        for (unsigned q = 0; q < qmax; ++q)
            if ((unsigned)(((unsigned long long)q * m) >> 32) != q / d) return false;
        return true;
    };
    if (!magic((unsigned)L, (unsigned)(2 * pl.zl * L), pl.magL) ||
        !magic((unsigned)pl.Lh, (unsigned)(2 * pl.zl * pl.Lh), pl.magLh)) {
        err = "FFT index division check failed";
        return false;
    }
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
    // the attribute belongs to the kernel, not to the handle: set the need of
    // the largest grid of each tile regime (L = 512 and 1024), so that handles
    // of other grid sizes keep launching
    auto need_z = [](int Lx) { return (int)(sizeof(float2) * (Lx + 2 * Lx * ((Lx <= 512 ? 8 : 4) + 1))); };
    auto need_y = [](int Lx) { return (int)(sizeof(float2) * (Lx + 2 * Lx * (Lx <= 512 ? 16 : 8))); };
    auto need_x = [&](int Lx) { return need_y(Lx) + (int)(sizeof(float) * Lx * (Lx <= 512 ? 16 : 8)); };
    const int sz = std::max(need_z(512), need_z(1024));
    const int sy = std::max(need_y(512), need_y(1024));
    const int sx = std::max(need_x(512), need_x(1024));
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(k_fft_z_r2c<8>, A, sz) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_z_r2c<4>, A, sz) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_z_c2r<8>, A, sz) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_z_c2r<4>, A, sz) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y<-1, 16>, A, sy) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y<-1, 8>, A, sy) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y<1, 16>, A, sy) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y<1, 8>, A, sy) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_x_spectral<16>, A, sx) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_x_spectral<8>, A, sx) != cudaSuccess) {
        err = "cudaFuncSetAttribute (FFT shared memory)";
        return false;
    }
    return true;
}

// lines per block of the pass along x: the compile-time plan's, else the run-time plan's
static int x_lines(int L)
{
    switch (L) {
#define ANKH_T(LV) case LV: return SpecLines<FftSpec<LV>>::v;
    ANKH_FFT_SPEC_LENGTHS(ANKH_T)
#undef ANKH_T
    default: return L <= 512 ? 16 : 8;
    }
}

int spectral_blocks(const Handle &H)
{
    const int L = H.g.nf, tk = x_lines(L);
    return ((L / 2 + 1 + tk - 1) / tk) * L;
}

static size_t smem_z(const FftPlan &pl) { return sizeof(float2) * (pl.L + 2 * pl.L * (pl.zl + 1)); }
static size_t smem_y(const FftPlan &pl) { return sizeof(float2) * (pl.L + 2 * pl.L * pl.tk); }
static size_t smem_x(const FftPlan &pl) { return smem_y(pl) + sizeof(float) * pl.L * pl.tk; }

template <int L>
static void launch_z_spec(int nrows, bool inverse, float *rho, float2 *spec, const float2 *tw, cudaStream_t s)
{
    constexpr int tk = SpecLines<FftSpec<L>>::v;
    const unsigned nb = (unsigned)((nrows + 2 * tk - 1) / (2 * tk));
    if (!inverse) k_fft_z_r2c_spec<L><<<nb, FftSpec<L>::NT, 0, s>>>(nrows, rho, spec, tw);
    else k_fft_z_c2r_spec<L><<<nb, FftSpec<L>::NT, 0, s>>>(nrows, spec, rho, tw);
}

static void launch_z(const FftPlan &pl, bool inverse, float *rho, float2 *spec, const float2 *tw, cudaStream_t s)
{
    const int nrows = pl.L * pl.L;
    switch (pl.L) {
#define ANKH_Z(LV) case LV: launch_z_spec<LV>(nrows, inverse, rho, spec, tw, s); return;
    ANKH_FFT_SPEC_LENGTHS(ANKH_Z)
#undef ANKH_Z
    default: break;
    }
    const unsigned nb = (unsigned)((nrows + 2 * pl.zl - 1) / (2 * pl.zl));
    if (!inverse) {
        if (pl.zl == 8) k_fft_z_r2c<8><<<nb, pl.tz, smem_z(pl), s>>>(pl, nrows, rho, spec, tw);
        else k_fft_z_r2c<4><<<nb, pl.tz, smem_z(pl), s>>>(pl, nrows, rho, spec, tw);
    } else {
        if (pl.zl == 8) k_fft_z_c2r<8><<<nb, pl.tz, smem_z(pl), s>>>(pl, nrows, spec, rho, tw);
        else k_fft_z_c2r<4><<<nb, pl.tz, smem_z(pl), s>>>(pl, nrows, spec, rho, tw);
    }
}

template <int SIGN>
static void launch_y(const FftPlan &pl, float2 *spec, const float2 *tw, cudaStream_t s)
{
    switch (pl.L) {
#define ANKH_Y(LV)                                                                                          \
    case LV: {                                                                                              \
        constexpr int tk = SpecLines<FftSpec<LV>>::v;                                                       \
        k_fft_y_spec<LV, SIGN><<<dim3((pl.Lh + tk - 1) / tk, pl.L), FftSpec<LV>::NT, 0, s>>>(pl.Lh, spec, tw); \
        return;                                                                                             \
    }
    ANKH_FFT_SPEC_LENGTHS(ANKH_Y)
#undef ANKH_Y
    default: break;
    }
    const dim3 g((pl.Lh + pl.tk - 1) / pl.tk, pl.L);
    if (pl.tk == 16) k_fft_y<SIGN, 16><<<g, pl.ty, smem_y(pl), s>>>(pl, spec, tw);
    else k_fft_y<SIGN, 8><<<g, pl.ty, smem_y(pl), s>>>(pl, spec, tw);
}

static void launch_x(const Handle &H, int mode, cudaStream_t s)
{
    const FftPlan &pl = H.fft;
    const dim3 g((pl.Lh + pl.tk - 1) / pl.tk, pl.L);
    float2 *spec = reinterpret_cast<float2 *>(H.d_rhohat);
    double *part = H.d_part + H.part_off[kPartGlob];
    switch (pl.L) {
#define ANKH_X(LV)                                                                                          \
    case LV: {                                                                                              \
        constexpr int tk = SpecLines<FftSpec<LV>>::v;                                                       \
        k_fft_x_spec<LV><<<dim3((pl.Lh + tk - 1) / tk, pl.L), FftSpec<LV>::NT, 0, s>>>(pl.Lh, spec, H.d_D,    \
                                                                                   H.d_tw, mode, part);    \
        return;                                                                                             \
    }
    ANKH_FFT_SPEC_LENGTHS(ANKH_X)
#undef ANKH_X
    default: break;
    }
    if (pl.tk == 16) k_fft_x_spectral<16><<<g, pl.ty, smem_x(pl), s>>>(pl, spec, H.d_D, H.d_tw, mode, part);
    else k_fft_x_spectral<8><<<g, pl.ty, smem_x(pl), s>>>(pl, spec, H.d_D, H.d_tw, mode, part);
}

cudaError_t launch_fft_forward(Handle &H, cudaStream_t s)
{
    float2 *spec = reinterpret_cast<float2 *>(H.d_rhohat);
    launch_z(H.fft, false, H.d_rho, spec, H.d_tw, s);
    launch_y<-1>(H.fft, spec, H.d_tw, s);
    return cudaGetLastError();
}

cudaError_t launch_spectral(Handle &H, bool forces, cudaStream_t s)
{
    launch_x(H, forces ? 1 : 0, s);
    return cudaGetLastError();
}

static cudaError_t launch_forward_x_only(Handle &H, cudaStream_t s)
{
    launch_x(H, 2, s);
    return cudaGetLastError();
}

cudaError_t launch_fft_inverse(Handle &H, cudaStream_t s)
{
    float2 *spec = reinterpret_cast<float2 *>(H.d_rhohat);
    launch_y<1>(H.fft, spec, H.d_tw, s);
    launch_z(H.fft, true, H.d_phi, spec, H.d_tw, s);
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
