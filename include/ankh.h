/*
 * ankh.h -- C ABI of the GB300 implementation of ANKH: the periodic
 * point-multipole Coulomb energy of the paper's Eq. 1 (charges, dipoles,
 * quadrupoles on the lattice 2 r_B Z^3), evaluated by the interpolated-Ewald
 * split of Sec. 3-4 (ANKH-FFT, Alg. 5) and its exact gradient; the energy by
 * ANKH-FMM (Alg. 3, flag ANKH_FMM); the non-periodic energy of Sec. 5.2
 * (flag ANKH_NONPERIODIC); induced dipoles on the same field (ankh_induce).
 *
 * Units: positions in Angstrom, charges in e, dipoles in e*A, quadrupoles in
 * e*A^2, energies in e^2/A (no Coulomb constant, as in Eq. 1).
 *
 * Conventions shared by every entry point:
 *   - The box is cubic with edge L = 2 r_B, centred at the origin (Eq. 1 and
 *     Sec. 3.3).  Positions outside it are wrapped.
 *   - D_u = q_u + mu_u . grad + Theta_u : grad grad (Sec. 1); Theta is
 *     symmetric and passed as its six stored entries xx, xy, xz, yy, yz, zz.
 *   - dEdtheta is the derivative with respect to those six stored entries
 *     (a stored off-diagonal entry stands for both Theta_ab and Theta_ba).
 *   - Arrays are row-major, float32, in the caller's atom order.
 *   - Device pointers are caller-owned; the library never frees them and
 *     never keeps them after the call returns.
 *   - All device work is issued on the given CUDA stream (NULL = legacy
 *     default stream).  Calls on one handle must not overlap.
 *   - Return value: ANKH_OK or one of the error codes below; the message of
 *     the last error of the calling thread is returned by ankh_last_error().
 *     No C++ exception crosses the ABI.
 */
#ifndef ANKH_H
#define ANKH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ANKH_OK = 0,
    ANKH_EINVAL = 1,   /* invalid argument (sizes, orders, NULL pointer, box) */
    ANKH_ENOMEM = 2,   /* device or host allocation failed; nothing leaked */
    ANKH_ECUDA = 3,    /* a CUDA or cuFFT call failed */
    ANKH_ETIMEOUT = 4, /* a bounded device-side wait ran out */
    ANKH_ENUMERIC = 5, /* a non-finite input coordinate was seen, or two atoms
                          share one position (infinite energy) */
    ANKH_ENOTCONV = 6  /* an iterative solve (ankh_induce) did not converge */
};

/* flags */
#define ANKH_INCLUDE_REC 1u  /* add the smooth reciprocal part of the xi split
                                to the far-field kernel (approximates the full
                                Ewald energy; without it E_rec(xi) is neglected
                                as in Sec. 3.1) -- default on */
#define ANKH_MIXED 2u        /* adjacent-leaf correction on the tensor cores
                                (operands scaled by powers of two and split
                                into fp16 hi + lo, three products, FP32
                                accumulate: ~22 significant bits); otherwise
                                plain FP32 on the CUDA cores */
#define ANKH_NONPERIODIC 4u  /* no periodic images (Sec. 5.2, Eq. relerrnonperio):
                                bare kernel 1/r (xi and ANKH_INCLUDE_REC are
                                ignored), leaves tile the box [-L/2, L/2)^3
                                without wrapping, the far field is the linear
                                (zero-padded) convolution of the non-adjacent
                                leaves; every atom must lie inside the box,
                                else the energy calls return ANKH_EINVAL */
#define ANKH_FMM 8u          /* ANKH-FMM (Sec. 3, Alg. 3) in place of ANKH-FFT:
                                perfect octree with n_cells = 2^E leaves per
                                axis (2 <= E <= 7; 0 picks the leaf edge
                                nearest 4 A), L = Lu = Lc first-kind
                                Chebyshev nodes per axis in every cell (L <= 8),
                                M2M up the tree, mutual M2L on the tensor cores
                                (fp16 hi + lo split, FP32 accumulation),
                                images beyond the direct ones through the root
                                expansion.  Energy only: ankh_energy_forces,
                                the batch and ankh_induce return ANKH_EINVAL.
                                Periodic boxes only.  Stage timings: "merge"
                                holds M2M, "spectral" the root term, "corr"
                                the M2L; ankh_last_terms: [1] root term,
                                [2] 0, [3] M2L far field */

typedef struct {
    double xi;        /* Ewald screening [1/A]; Sec. 5 uses 0.01 */
    int n_cells;      /* leaves per axis n >= 3 (0 = from the accuracy table, see ankh_accuracy_rule) */
    int Lu;           /* equispaced interpolation order, 2..8 (0 = from the accuracy table) */
    int Lc;           /* Chebyshev interpolation order, 2..16 (0 = Lu) */
    int max_order;    /* 0 = charges, 1 = + dipoles, 2 = + quadrupoles */
    unsigned flags;   /* ANKH_* flags above */
} ankh_params;

typedef struct {
    int n_cells, Lu, Lc, nf;  /* leaves per axis, orders, fine grid points per axis = n (Lu-1) */
    int64_t n_atoms;
    double box, h, xi;
    double precompute_ms;     /* wall time of ankh_create's table set-up */
    int64_t device_bytes;     /* device memory held by the handle */
    int tables_from_cache;    /* 1: ankh_create_cached read the tables from its cache file */
} ankh_info;

typedef struct ankh_handle ankh_handle;

/* Fill *p with the defaults (xi = 0.01, n and Lu = Lc from the accuracy
 * table, quadrupoles, ANKH_INCLUDE_REC | ANKH_MIXED). */
void ankh_default_params(ankh_params *p);

/* Accuracy table of the defaults (the paper picks the interpolation order
 * for a target accuracy, Sec. 5.2-5.3; this table is calibrated, not
 * printed there).  For N atoms (max_order 0: charges only, else with
 * multipoles) and order Lu, *hmin and *hmax (may be NULL) receive the range
 * of leaf edges (A) over which the method's own error -- the FP64 ANKH-FFT
 * against FP64 Ewald, measured on synthetic water boxes of 24,000 / 96,000 /
 * 1,008,000 atoms with charges, dipoles and quadrupoles, and of 648 atoms
 * with charges only -- stayed within 5e-6 relative energy error and 3e-5
 * relative RMS force error at every measured leaf count, leaving the rest of
 * the 1e-5 / 1e-4 target for the FP32 arithmetic.  Orders 2..6 only (above 6
 * the FP32 far field loses that margin).  The box uses the class of its kind
 * with the largest atom count not above N.  Returns ANKH_OK, or ANKH_EINVAL
 * when Lu is not calibrated for that class or N is below the smallest class
 * of its kind (with multipoles: 24,000 atoms).  With n_cells = 0 and/or
 * Lu = 0, ankh_create takes the lowest calibrated order that has a leaf
 * count in its range, and the largest such leaf count whose grid the FFT
 * takes; a box below the smallest class uses that class's rules, and where
 * no rule applies (too small a box, ANKH-FMM) the defaults are L_u = 5 and
 * a leaf edge near 4 A: in both cases with no accuracy guarantee.  Host
 * only. */
int ankh_accuracy_rule(int64_t N, int max_order, int Lu, double *hmin, double *hmax);

/* Create a handle for a cubic box of edge box_edge (= 2 r_B) holding N atoms.
 * Runs the per-box precomputation (Alg. 4 / Sec. 4.3): the interpolation
 * matrices, the spectrum of the periodic far-field kernel on the merged
 * equispaced grid, and the adjacent-leaf correction blocks.  Allocates all
 * device scratch on the current device.  params may be NULL (defaults).
 * The merged grid of n (L_u - 1) points per axis (periodic) or its
 * zero-padded size (non-periodic, chosen by the library) is transformed by
 * the library's own FFT, which takes lengths with prime factors 2, 3, 5 and
 * 7 only, at most 1024.
 * Errors: ANKH_EINVAL (N < 1, box not finite and > 0, n < 3, orders out of
 * range, xi <= 0, a periodic grid n (L_u - 1) with a prime factor above 7
 * or above 1024 points), ANKH_ENOMEM, ANKH_ECUDA.  *out is NULL on error. */
int ankh_create(double box_edge, int64_t N, const ankh_params *params, ankh_handle **out);

/* Same as ankh_create, with the per-box tables that do not depend on the
 * atoms cached in the directory cache_dir (the paper's precomputation is its
 * slow step, done once per box: Sec. 4.3 and 5.6).  The tables are the
 * spectrum of the far-field kernel on the merged grid with its FP64 k = 0
 * value, and the adjacent-leaf correction blocks C_d; they depend on the box
 * edge, n, L_u, L_c, xi (as FP32), the grid size, ANKH_NONPERIODIC and
 * ANKH_INCLUDE_REC, which key the file (cache_dir/ankh_tables_<hash>.bin,
 * the key stored and compared in full).  A matching file is read instead of
 * computing the tables; otherwise they are computed and the file is written
 * (to a temporary name, then renamed).  Results are bit-identical to
 * ankh_create's.  ANKH-FMM handles compute their own tables (not cached).
 * Errors: as ankh_create; ANKH_EINVAL if cache_dir is NULL or empty or the
 * file cannot be written.  ankh_get_info reports tables_from_cache. */
int ankh_create_cached(double box_edge, int64_t N, const ankh_params *params, const char *cache_dir,
                       ankh_handle **out);

/* Energy of Eq. 1 by Alg. 5: near field over adjacent leaves (step 3), far
 * field by the diagonalised circulant (step 2), self term (step 4).
 * x: N x 3 device; q: N device; mu: N x 3 device or NULL; theta: N x 6 device
 * or NULL.  *E_host receives the energy after the stream work completes (the
 * call synchronises the stream).  Errors: ANKH_EINVAL, ANKH_ECUDA,
 * ANKH_ENUMERIC.
 * Execution (this call and ankh_energy_forces): the first call records the
 * evaluation's kernels into a CUDA graph on the handle's own stream and
 * launches it on cuda_stream; later calls with the same pointers (and the
 * same ankh_set_timing state) launch that graph again, which reads whatever
 * the buffers hold then; a different pointer records a new graph.  While
 * cuda_stream is itself being captured the kernels are launched directly. */
int ankh_energy(ankh_handle *h, const float *x, const float *q, const float *mu,
                const float *theta, double *E_host, void *cuda_stream);

/* Energy and its exact gradient (the adjoint of every step; forces are not in
 * the paper, which lists them as future work in Sec. 3.8 and 6).
 * Outputs (device, N x 3 / N / N x 3 / N x 6 / N x 3, each may be NULL):
 *   dEdx = dE/dx (minus the force), dEdq = potential, dEdmu = minus the field,
 *   dEdtheta (stored-entry convention), torque = -dE/d(rotation angle) of each
 *   atom's dipole and quadrupole about its own position.
 * E_host may be NULL (then the call does not synchronise). */
int ankh_energy_forces(ankh_handle *h, const float *x, const float *q, const float *mu,
                       const float *theta, double *E_host, float *dEdx, float *dEdq,
                       float *dEdmu, float *dEdtheta, float *torque, void *cuda_stream);

/* Same as ankh_energy_forces with HOST input and output arrays (pageable or
 * pinned): copies in, evaluates, copies out, synchronises. */
int ankh_energy_forces_host(ankh_handle *h, const float *x, const float *q, const float *mu,
                            const float *theta, double *E, float *dEdx, float *dEdq,
                            float *dEdmu, float *dEdtheta, float *torque, void *cuda_stream);

/* Induced dipoles of point-polarizable atoms (the polarizable force fields
 * named in Sec. 1 and 6 of the paper as a use of the repeated field
 * evaluations): every atom i carries an isotropic polarizability alpha_i
 * (A^3, > 0) and the induced dipole
 *     mu_ind_i = alpha_i (F_i^perm + F_i(mu_ind)),
 * where F_i = -dE/dmu_i is the field of all other atoms and all periodic
 * images (the periodic boundary of the handle; ANKH_NONPERIODIC: no images),
 * F^perm that of the permanent multipoles (q, mu, theta as for
 * ankh_energy).  Solved by conjugate gradients with the preconditioner
 * diag(alpha) on (diag(1/alpha) - T) mu_ind = F^perm, T mu = F(mu) being one
 * ANKH evaluation of the dipoles mu alone (the adjoint path); no damping of
 * the short-range dipole-dipole field (point polarizabilities: the system
 * must be positive definite).  Initial guess alpha F^perm; stops when
 * |residual| <= tol |F^perm| (2-norms) or after max_iter iterations.
 * x, q: N x 3 and N device; mu: N x 3 device or NULL; theta: N x 6 device or
 * NULL; alpha: N device; mu_ind: N x 3 device output (caller-allocated).
 * *E_pol (host, may be NULL) receives -1/2 sum mu_ind . F^perm; *iterations
 * (host, may be NULL) the number of CG iterations.  Synchronises the stream
 * once per iteration.  Errors: ANKH_EINVAL (NULL, tol <= 0, alpha <= 0),
 * ANKH_ENUMERIC (non-finite input, or the system is not positive definite),
 * ANKH_ENOTCONV (max_iter reached; mu_ind holds the last iterate),
 * ANKH_ENOMEM, ANKH_ECUDA. */
int ankh_induce(ankh_handle *h, const float *x, const float *q, const float *mu, const float *theta,
                const float *alpha, double tol, int max_iter, float *mu_ind, double *E_pol, int *iterations,
                void *cuda_stream);

/* Energy terms of the last completed call on h, in e^2/A:
 * [0] near field, [1] far field on the merged grid (k != 0), [2] its k = 0
 * term, [3] adjacent-leaf correction, [4] self term, [5] total. */
int ankh_last_terms(const ankh_handle *h, double terms[6]);

int ankh_get_info(const ankh_handle *h, ankh_info *info);

/* Kernels launched by one evaluation on h (forces != 0: ankh_energy_forces,
 * else ankh_energy) into *count: the count the library's launch sequence
 * issues, from its plan (digit passes of the leaf sort, the fp16 split of
 * the tensor-core correction, the levels of ANKH_FMM).  Errors: ANKH_EINVAL
 * (NULL, or forces on an ANKH_FMM handle). */
int ankh_launch_count(const ankh_handle *h, int forces, int *count);

/* Copy an internal device buffer of the last call into caller memory dst
 * (device pointer, at least *bytes long; with dst == NULL only *bytes is
 * set).  which: 0 = permutation (int32, sorted slot -> atom), 1 = leaf
 * start offsets (int32, n^3 + 1), 2 = equispaced modified charges M
 * (float32, n^3 x ldm), 3 = merged grid charges (float32, nf^3),
 * 4 = correction potential psi (float32, n^3 x ldm, forces calls only),
 * 5 = leaf id of each sorted slot (int32), 6 = far-field kernel spectrum D
 * (float32, nf x nf x (nf/2 + 1), k = 0 removed; set at creation).
 * ldm = ankh_ldm(h). */
int ankh_debug_copy(const ankh_handle *h, int which, void *dst, int64_t *bytes, void *cuda_stream);
int ankh_ldm(const ankh_handle *h);

/* Batched independent boxes (replicas of uneven size).  Each box has its own
 * handle (tables depend on the box edge); one call evaluates all boxes:
 * the per-box pipelines are recorded once into a CUDA graph with parallel
 * branches (small boxes run concurrently) and replayed while the caller's
 * pointers and stream stay the same (a change triggers a new capture).
 * Inputs/outputs are the per-box arrays concatenated in box order (box i
 * starts at atom offset sum_{j<i} n_atoms[j]); E_host receives nbox
 * energies; the call synchronises the stream.  The first call on a stream
 * must not itself be inside a stream capture. */
typedef struct ankh_batch ankh_batch;
int ankh_create_batch(int nbox, const double *box_edges, const int64_t *n_atoms, const ankh_params *params,
                      ankh_batch **out);
int ankh_energy_forces_batch(ankh_batch *b, const float *x, const float *q, const float *mu,
                             const float *theta, double *E_host, float *dEdx, float *dEdq, float *dEdmu,
                             float *dEdtheta, float *torque, void *cuda_stream);
/* Kernels launched by one ankh_energy_forces_batch call into *count: every
 * box's evaluation without its near field, plus one near-field launch over
 * all boxes per group sharing xi and the near-field kernel variant.
 * Errors: ANKH_EINVAL (NULL). */
int ankh_batch_launch_count(const ankh_batch *b, int *count);
/* Optional timing of the batched near field: with enable != 0 the next
 * batch call records CUDA events (inside its graph) before and after the
 * near-field launches, and ankh_batch_near_ms returns their interval in
 * milliseconds for the last such call (waiting for it).  Errors:
 * ANKH_EINVAL (NULL; for ankh_batch_near_ms, no timed call yet), ANKH_ECUDA. */
int ankh_batch_set_timing(ankh_batch *b, int enable);
int ankh_batch_near_ms(const ankh_batch *b, double *ms);
/* Borrow the handle of box i (owned by the batch; do not destroy it). */
int ankh_batch_box(const ankh_batch *b, int i, ankh_handle **h);
void ankh_destroy_batch(ankh_batch *b);

/* Optional per-stage timing with CUDA events recorded on the call's stream
 * (off by default).  Stages: 0 bin+sort, 1 self term, 2 P2M, 3 merge onto
 * the equispaced grid, 4 forward FFT, 5 spectral product, 6 adjacent-leaf
 * correction, 7 near field, 8 inverse FFT, 9 L2P fused with the gradient
 * assembly (far + near + self terms, torques, write in the caller's order),
 * 10 unused (always 0), 11 energy reduction.  ankh_stage_times waits for the last call's events
 * and returns each stage's duration in milliseconds (0 for stages that did
 * not run). */
#define ANKH_NUM_STAGES 12
int ankh_set_timing(ankh_handle *h, int enable);
int ankh_stage_times(const ankh_handle *h, double ms[ANKH_NUM_STAGES]);

/* Leaf binning and stable sort without any allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (an engine that plans all device memory at start-up and treats
 * a later allocation as an error, a host whose device allocator belongs to
 * another runtime and must not be bypassed).  Its output equals the output of the
 * sort stage of ankh_energy (the leaf of each atom by the correctly rounded
 * FP64 chain of that stage, without its FP32 screen, then the stable radix
 * sort by leaf), with its scratch in a static device array of the library
 * instead of allocated memory.
 *   x: N x 3 device positions; n_cells leaves per axis of a cubic box of edge
 *   box_edge; outputs (device, caller-owned): perm[N] = atom index of each
 *   sorted slot (ordered by leaf, then by atom index), leaf_start[n^3 + 1] =
 *   first slot of each leaf.  The cost per atom does not depend on how the
 *   atoms are spread over the leaves (all of them in one leaf included).
 *   Limits: N <= ANKH_NOALLOC_MAX_ATOMS, n_cells^3 <= ANKH_NOALLOC_MAX_LEAVES;
 *   larger sizes return ANKH_EINVAL with a message naming the limit.
 *   The static array (11 MiB) is held by every GPU that loads the library
 *   until the process exits.  Every call looks up the array's device address
 *   on the current device (cudaGetSymbolAddress); the first call on a device
 *   also loads the library's device code there, so make that first call
 *   before any stream capture.  All calls share the one array, which keeps
 *   the last call's contents: each call clears what must start at zero, but
 *   calls that overlap on the GPU (other streams, other threads) race.
 *   Non-finite coordinates are binned as 0 and not reported.  The call is
 *   asynchronous on cuda_stream. */
#define ANKH_NOALLOC_MAX_ATOMS 1048576
#define ANKH_NOALLOC_MAX_LEAVES 262144
int ankh_bin_sort_noalloc(const float *x, int64_t N, double box_edge, int n_cells, int32_t *perm,
                          int32_t *leaf_start, void *cuda_stream);

/* Measurement utility (not part of the method): the FP32 FMA throughput of
 * the current device in TFLOP/s (FMA = 2 flop), measured with CUDA events
 * over ten launches of independent FMA chains (8 blocks of 256 threads per
 * multiprocessor) on cuda_stream, after three warm-up launches; *ms (may be
 * NULL) receives the time of one launch.  It is the denominator of the near
 * field's roofline.  Synchronises the stream. */
int ankh_measure_fp32_peak(double *tflops, double *ms, void *cuda_stream);

/* Test access to the far-field transform step alone (no counterpart in the
 * paper's interface; the tests use it to check the hand-written FFT against a
 * library transform).  rho: nf^3 device floats (the merged grid, z fastest);
 * D: nf * nf * (nf/2 + 1) device floats in the spectrum layout [x][y][kz]
 * (NULL: the handle's kernel spectrum).  mode 0: out receives the forward
 * unnormalised 3-D real transform of rho, nf * nf * (nf/2 + 1) complex
 * (float2) values in the same layout.  mode 1: the far-field step of an
 * evaluation: *E_glob = (1/2M) sum over the full spectrum of D |rho^|^2
 * (M = nf^3), and out receives phi = the unnormalised inverse transform of
 * D rho^ (nf^3 floats).  Overwrites the handle's grid buffers; synchronises
 * the stream.  Errors: ANKH_EINVAL (NULL arguments, bad mode, ANKH-FMM
 * handle), ANKH_ECUDA. */
int ankh_debug_fft(ankh_handle *h, const float *rho, const float *D, int mode, double *E_glob, void *out,
                   void *cuda_stream);

/* Free everything the handle owns.  NULL is ignored. */
void ankh_destroy(ankh_handle *h);

/* Message of the last error on the calling thread ("" if none). */
const char *ankh_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int ankh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ANKH_H */
