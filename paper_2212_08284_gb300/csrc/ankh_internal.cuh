// Internal declarations of libankh (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <string>

#include "ankh.h"

namespace ankh {

constexpr int kMaxLu = 8;
constexpr int kMaxLc = 16;

// Device-side view of one handle's geometry and buffers, passed by value to kernels.
struct Geo {
    int n;            // leaves per axis
    int ncell;        // n^3
    int Lu, Lc;       // interpolation orders
    int P;            // Lu^3 nodes per leaf
    int ldm;          // padded leading dimension of per-leaf node arrays (multiple of 32)
    int nf;           // FFT grid points per axis: n (Lu - 1) (periodic) or the padded size
    int nfh;          // nf / 2 + 1
    int64_t M;        // nf^3
    int ng;           // merged equispaced nodes per axis: nf (periodic) or n (Lu - 1) + 1
    int nonperiodic;  // 1: no images, bare kernel, zero-padded linear convolution
    double box, rB, inv_box, h;
    float hf;         // leaf edge (float)
    float hf_lo;      // h - hf (float): hf + hf_lo carries the FP64 leaf edge
    float two_over_h; // chain-rule factor of x_hat = 2 (x - ctr) / h
    float xi;
    float Kf;         // n / L rounded to FP32 (the binning's FP32 screen)
};

// Near-field work items: a leaf's targets in chunks of at most this many
// (one warp each), laid out by the leaf-count scan.
constexpr int kNearItemTargets = 32;

// Stable LSD radix sort of the atoms by leaf id (k_sort.cu).
struct RadixPlan {
    int npass;              // 1 .. 3 digit passes, lowest digit first
    int bits[3], shift[3];  // digit width (<= 10 bits) and position of each pass
    int ntiles;             // tiles of 4096 consecutive elements
    int64_t hist_len;       // largest 2^bits * ntiles over the passes
    int bsum_len;           // block totals of the histogram scan
};
struct RadixBufs {
    int *vtmp[2];           // [N] values between passes (vtmp[1] only for three passes)
    int *hist, *goff;       // [hist_len] digit counts per tile, [hist_len + 1] their exclusive scan
    int *bsum;              // block totals of the scans
};
// wide_tiles: the most tiles for which one 12-bit pass replaces two (0: never)
RadixPlan radix_plan(int64_t N, int ncell, int wide_tiles = 0);
cudaError_t radix_prepare();   // shared-memory attribute of the wide scatter pass

// Hand-written 3-D real FFT of the merged grid (fft.cu): one mixed-radix
// Stockham plan for the L = nf points of every axis.
constexpr int kFftMaxStages = 12;
struct FftPlan {
    int L, Lh;                  // points per axis, L / 2 + 1
    int nst;                    // stages
    int radix[kFftMaxStages];   // radix of each stage (2 .. 8)
    int p[kFftMaxStages];       // product of the radices before each stage
    unsigned mag[kFftMaxStages];  // ceil(2^20 / p): i / p = (i mag) >> 20 for i < L
    unsigned magL, magLh;       // floor(2^32 / d) + 1 for d = L and L / 2 + 1
    int tk;                     // lines per block of the passes along y and x
    int zl;                     // complex lines (row pairs) per block of the passes along z
    int ty, tz;                 // threads per block of those passes
};

// Pipeline stages (for the optional per-stage timing)
enum Stage { kStSort = 0, kStSelf, kStP2M, kStMerge, kStFFTf, kStSpectral, kStCorr, kStNear, kStFFTi,
             kStL2P, kStUnused, kStReduce, kNumStages };

// Energy partial slots (FP64 per block, reduced in a fixed order).
enum PartSlot { kPartNear = 0, kPartGlob = 1, kPartCorr = 2, kPartSelf = 3, kPartQ = 4, kPartCount = 5 };
constexpr int kReduceBlocks = 32;   // blocks of the energy reduction (k_final.cu)

// Tensor-core correction (k_corr_tc.cu): tile geometry and TMA descriptors.
struct TcPlan {
    int enabled;
    int S, R, rowstride, N, tiles, halves;
    int grid;               // persistent CTAs (one per SM)
    int ldk;                // node stride of the fp16 operands (ldm rounded up to 64)
    int eC;                 // C_d scaled by 2^eC before the fp16 split
    uint32_t tmem_cols;
    CUtensorMap mAhi, mAlo, mBhi, mBlo;
    CUtensorMap mAhiE, mAloE;   // energy-only operator [C_0 | 2 C_d, d > 0] (14 blocks)
};

// ANKH-FMM (fmm.cu): perfect octree of depth E, L Chebyshev nodes per axis per cell.
constexpr int kFmmMaxLevels = 8;   // E <= 7

struct FmmLevel {
    const float *M;   // [(2m)^3][ldm] expansions of the level, natural cell order
    int m;            // parent cells per axis (2^(e-1)); the level has 2m cells per axis
    int S, R, tiles;  // z-row of m targets padded to S = max(16, m); R = 128 / S z-rows per tile; tiles per class
    int rowstride;    // S + 2 rows per z-row block of the split operand (one-cell z halo)
    int rowbase;      // first row of the level in the split operand
    int acol;         // first column of the level in the operator table
    int eC;           // C_e(d) scaled by 2^eC before the fp16 split
};

struct FmmLevels {
    FmmLevel lv[kFmmMaxLevels];   // lv[e], e = 1 .. E (lv[0] unused)
};

struct FmmPlan {
    int enabled;
    int E, L, ldk, kch, slices;
    int nitems, grid, ntab;
    int64_t brows;          // rows of the split operand (all levels)
    uint32_t tmem_cols;
    float *d_Mlev[kFmmMaxLevels];   // levels 0 .. E-1 (level E is Handle::d_M)
    __half *d_Bhi, *d_Blo;  // [brows][ldk] parity-major split expansions, one-cell y and z halos
    __half *d_Ahi, *d_Alo;  // [slices*128][E * 343 * ldk] split M2L operators C_e(d), d in [-3,3]^3
    int4 *d_items;          // work items (level | class << 4 | slice << 8, tile, first offset, offsets), per CTA
    int *d_ctaoff;          // [grid + 1] first item of each persistent CTA
    int *d_tab;             // interaction offsets per class (block | class' << 9 | (D + 1) << 12..16)
    double *d_K;            // [L^3][L^3] root operator of the images beyond the direct ones
    float V[2][8][8];       // M2M: V[b][k][l] = S_k((2b - 1 + r_l) / 2)
    FmmLevels lev;
    FmmLevel *d_lev;        // device copy of lev.lv
    CUtensorMap mAhi, mAlo, mBhi, mBlo;
    CUtensorMap mB3hi[4], mB3lo[4];   // 3-D maps of the levels with m >= 8 (slot e - 4)
};

struct Handle {
    Geo g;
    TcPlan tc;
    FmmPlan fmm;
    __half *d_Mhi, *d_Mlo;  // [n*n*rowstride][ldk] fp16 split of 2^eM M, z-halo rows (tensor-core path)
    __half *d_Chi, *d_Clo;  // [halves*128][27*ldk] fp16 split of 2^eC [C_0 | ... | C_26]
    __half *d_ChiE, *d_CloE;  // [halves*128][14*ldk] the same of [C_13 | 2 C_14 | ... | 2 C_26] (energy alone)
    unsigned *d_mmax;       // max |M| of the call (FP32 bits), sets eM (ANKH-FMM: one per level)
    float *d_ind;           // induced-dipole workspace (allocated on first use)
    double *d_ind_part;
    int64_t N;
    int max_order;
    unsigned flags;
    int device;
    int sm_count;           // multiprocessors of the device (grid sizing)
    double D0;              // k = 0 value of the far-field kernel spectrum (FP64)
    double precompute_ms;
    int tables_from_cache;  // 1: the per-box tables were read from a cache file
    int64_t device_bytes;

    // atoms (sorted by leaf)
    int *d_cellid, *d_count, *d_start, *d_perm, *d_scell, *d_flag, *d_bsum;
    int2 *d_items;          // near-field work items (leaf, first target), laid out by the leaf-count scan
    int *d_nitems;          // number of items of the call
    int max_items;          // ncell + ceil(N / kNearItemTargets): bound on the items of any input
    RadixPlan rs;           // leaf sort
    RadixBufs rsb;
    float4 *d_loc;          // [N] coordinates relative to the leaf centre (caller's order)
    float2 *d_ctr;          // [3n] leaf centres -r_B + (c + 1/2) h, c = -n .. 2n-1, as FP32 hi + lo
    float4 *d_A0, *d_A1, *d_A2, *d_A3;   // (lx, ly, lz, q) (mu, 0) (txx, txy, txz, tyy) (tyz, tzz, 0, 0)
    // interpolation
    float *d_W;             // [4][Lu][Lc] derivative matrices (2/h)^p E H D^p (E = I for ANKH-FMM)
    float h_Wf[4 * 8 * 8];  // host copy of W for L_c = L_u <= 8 (kernel-parameter basis tables)
    float *d_M;             // [ncell][ldm] modified charges at the leaf nodes (equispaced; Chebyshev for ANKH-FMM)
    float *d_rho;           // [nf^3] merged grid charges
    cufftComplex *d_rhohat; // [nf][nf][nfh]
    float *d_D;             // [nf][nf][nfh] real spectrum of the far-field kernel (k = 0 removed)
    float *d_phi;           // [nf^3] merged grid potential (unnormalised c2r output)
    float *d_C;             // [27][ldm][ldm] adjacent-leaf correction blocks (FP32)
    float *d_psi;           // [ncell][ldm] correction potential
    float *d_gnear;         // [13][Nslot] near-field gradient per sorted slot
    double *d_part;         // energy partials
    int part_off[kPartCount + 1];
    int *d_partoff;         // device copy of part_off
    double *d_rscr;         // [kReduceBlocks][kPartCount] per-block sums of the energy reduction
    unsigned *d_ticket;     // blocks of the energy reduction done (the last one resets it to 0)
    double *d_terms;        // [8] reduced energy terms
    double *h_terms;        // pinned host copy
    float *d_hostbuf;       // staging for the host-buffer entry point
    int64_t hostbuf_bytes;
    // host-buffer entry point: inputs copied on copy_stream (x first) while
    // the leaf sort runs; the gather waits for ev_inputs
    cudaStream_t copy_stream;
    cudaEvent_t ev_call, ev_x, ev_inputs;
    int have_copy_stream;
    cudaEvent_t gather_wait;  // set for one run_sequence call: event the gather waits for
    // ankh_energy / ankh_energy_forces: the evaluation as a CUDA graph per
    // variant (0 energy, 1 forces), captured on gcap and replayed while the
    // call's pointers and the timing switch stay the same
    cudaStream_t gcap;
    cudaGraphExec_t gexec[2];
    const void *gkey[2][10];
    int gvalid[2];
    double last_terms[6];
    FftPlan fft;
    float2 *d_tw;           // [L] FFT twiddles e^{-2 pi i e / L} (FP32 from FP64)
    // optional per-stage timing (events on the caller's stream)
    int timing;
    int have_events;
    int nrec;
    cudaEvent_t ev[kNumStages + 1];
    int ev_stage[kNumStages + 1];
};

int run_sequence(Handle &H, const float *x, const float *q, const float *mu, const float *theta, bool forces,
                 float *dEdx, float *dEdq, float *dEdmu, float *dEdtheta, float *torque, cudaStream_t s);

// error reporting (thread-local message)
void set_error(const std::string &msg);

// kernels launchers (each returns cudaGetLastError())
cudaError_t launch_bin(Handle &H, const float *x, cudaStream_t s);
cudaError_t launch_scan(Handle &H, cudaStream_t s);
int sort_launches(const Handle &H);   // kernels of the leaf sort stage
cudaError_t launch_scatter_sort_gather(Handle &H, const float *x, const float *q, const float *mu,
                                       const float *theta, cudaStream_t s);
cudaError_t launch_radix(int N, const int *cellid, const RadixPlan &rp, const RadixBufs &b, int *perm, int *inv,
                         cudaStream_t s);
cudaError_t launch_bin_sort_raw(int N, const float *x, const Geo &g, int *cellid, int *count, int *flag,
                                const RadixPlan &rp, const RadixBufs &b, int *start, int *perm, cudaStream_t s);
cudaError_t launch_p2m(Handle &H, cudaStream_t s);
cudaError_t launch_fine_gather(Handle &H, cudaStream_t s);
bool fft_prepare(Handle &H, std::string &err);
cudaError_t launch_fft_forward(Handle &H, cudaStream_t s);   // passes along z and y
cudaError_t launch_spectral(Handle &H, bool forces, cudaStream_t s);   // along x: energy [, D rho^, inverse along x]
cudaError_t launch_fft_inverse(Handle &H, cudaStream_t s);   // inverse passes along y and z
cudaError_t launch_corr(Handle &H, bool forces, cudaStream_t s);
cudaError_t launch_near(Handle &H, bool forces, cudaStream_t s);
cudaError_t launch_l2p(Handle &H, float *dEdx, float *dEdq, float *dEdmu, float *dEdtheta, float *torque,
                       cudaStream_t s);
cudaError_t launch_self_dc(Handle &H, cudaStream_t s);
int fetch_terms(Handle &H, double *E_host, cudaStream_t s);
int run_sequence(Handle &H, const float *x, const float *q, const float *mu, const float *theta, bool forces,
                 float *dEdx, float *dEdq, float *dEdmu, float *dEdtheta, float *torque, cudaStream_t s);
int induce_dipoles(Handle &H, const float *x, const float *q, const float *mu, const float *theta,
                   const float *alpha, double tol, int max_iter, float *mu_ind, double *E_pol, int *iterations,
                   cudaStream_t s, std::string &err);
cudaError_t launch_reduce(Handle &H, cudaStream_t s);

// precomputation on the device (FP64)
cudaError_t precompute_kernel_spectrum(Handle &H, double *D0_out, std::string &err);

bool tc_prepare(Handle &H, std::string &err);
bool encode_2d(CUtensorMap *map, void *ptr, uint64_t inner, uint64_t outer, uint32_t box_inner, uint32_t box_outer,
               std::string &err);   // 2-D fp16 tensor map, 128-byte swizzle
bool encode_3d(CUtensorMap *map, void *ptr, uint64_t inner, uint64_t mid, uint64_t outer, uint32_t box_mid,
               uint32_t box_outer, std::string &err);   // 3-D fp16 tensor map, boxes {64, box_mid, box_outer}
// ANKH-FMM (fmm.cu)
int fmm_prepare(Handle &H, double xi, bool include_rec, std::string &err);
void fmm_free(Handle &H);
int fmm_part_slots(const Handle &H);   // energy partial slots of the M2L launch
void mark_stage(Handle &H, int stage_done, cudaStream_t s);   // optional per-stage timing
int run_fmm(Handle &H, const float *x, const float *q, const float *mu, const float *theta, cudaStream_t s);
void tc_tile_shape(int n, int halves, int sms, int &S, int &R);
int tc_max_blocks(int n, int ldm, int sms);   // CTAs of the tensor-core correction (energy partial slots)
int tc_ldk(int ldm);                 // node stride of the fp16 split operands
int split_exponent(float maxabs);    // e with max |x| 2^e <= 2^14 (0 for 0 or non-finite)
int corr_tc_blocks(const Handle &H);
cudaError_t launch_corr_tc(Handle &H, bool forces, cudaStream_t s);

int near_blocks(const Handle &H);
int near_mode(const Handle &H);   // B0 evaluation of the near field (series lengths or erfcf), from xi h

// Screening coefficients of the near-field pair kernel (k_near.cu).
struct BCoef {
    float xi;
    float kap;                  // xi^2 log2(e):  y = kap r^2,  exp(-xi^2 r^2) = 2^-y
    float c1, c2, c3, c4, c5;   // (2 xi^2)^l / (xi sqrt(pi))
    float a[8];                 // erf(xi r)/r = sum_k a_k y^k (Maclaurin series of erf)
};

// One launch of the near field over several boxes (k_near.cu).
struct NearBox;
struct NearBatch {
    int nbox = 0, total_blocks = 0, mode = 0;
    BCoef bc;
    NearBox *d_boxes = nullptr;   // per box, in decreasing order of atom count
    int *d_block0 = nullptr;      // [nbox + 1] first block of each box
};
bool near_batch_tables(Handle *const *hs, int nbox, NearBatch &nb, std::string &err);
cudaError_t launch_near_batch(const NearBatch &nb, bool forces, cudaStream_t s);
void near_batch_free(NearBatch &nb);
int spectral_blocks(const Handle &H);
int corr_blocks(const Handle &H);
int self_blocks(const Handle &H);

}  // namespace ankh

// The opaque handle of the C ABI.
struct ankh_handle {
    ankh::Handle h;
};
