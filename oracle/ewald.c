/*
 * oracle/ewald.c -- FP64 CPU reference ("oracle") for the periodic
 * point-multipole Coulomb energy of ANKH and for the erfc-screened pair sums
 * its near field uses.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline / reference legs may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * What it computes (units: e, Angstrom, energy in e^2/Angstrom; no Coulomb
 * constant, as in Eq. 1 of the paper):
 *
 *   E = 1/2 sum_t sum_i sum_j' D_i D_j 1/|x_i - x_j + t|            (Eq. 1)
 *   D_u = q_u + mu_u . grad + Theta_u : grad grad                    (Sec. 1)
 *
 * by classical Ewald summation with tin-foil boundary conditions (Sec. 3,
 * Eq. ewald, with the reciprocal-space constants restated in their standard
 * form; the ones printed in the paper are garbled):
 *
 *   E_real = 1/2 sum_t sum_i sum_j' P_ij erfc(a r)/r ,  r = x_i - x_j + t
 *   E_rec  = (2 pi / V) sum_{k != 0} exp(-k^2/4a^2)/k^2 |S(k)|^2
 *   S(k)   = sum_j (q_j + i mu_j.k - Theta_j : k k) exp(i k.x_j)
 *   E_self = -(a/sqrt(pi)) sum_i [ q^2 + (2a^2/3)|mu|^2 - (4a^2/3) q tr(Theta)
 *                                  + (8a^4/5) Theta:Theta + (4a^4/5) tr(Theta)^2 ]
 *   E_neut = -pi Q^2 / (2 V a^2),  Q = sum_i q_i
 *
 * The self term is -1/2 lim_{r->0} P_ii erf(a r)/r; for a traceless Theta it
 * is the one printed in Eq. ewald.  The pair operator is
 *   P_ij f = (q_i + mu_i.grad + Theta_i:grad grad)(q_j - mu_j.grad + Theta_j:grad grad) f(r)
 * (grad acts on r; the source's own derivative is -grad, Sec. 1).
 *
 * Multipole layout per atom (10 doubles): q, mu_x, mu_y, mu_z,
 *   Theta_xx, Theta_xy, Theta_xz, Theta_yy, Theta_yz, Theta_zz.
 * Gradient layout per atom (13 doubles): dE/dx (3), dE/dq, dE/dmu (3),
 *   dE/dTheta (6) -- the derivative with respect to the six STORED entries,
 *   where a stored off-diagonal entry stands for both Theta_ab and Theta_ba.
 *
 * Two independent evaluators of one pair term are provided:
 *   - or_pair_tensor: builds the Cartesian derivative tensors of the radial
 *     kernel up to rank 5 from the screened B-functions and contracts them
 *     entry by entry (slow, easy to audit);
 *   - or_pair_scalar: the same quantity expanded into scalar contractions
 *     e = sum_l c_l B_l (fast; used for the large systems).
 * The tests check one against the other on random pairs.
 */
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NMP 10
#define OR_NGR 13

int or_version(void) { return 3; }

/* ------------------------------------------------------------------------ */
/* Screened B-functions: B_0 = erfc(a r)/r,  B_l = -(1/r) dB_{l-1}/dr.
 * Upward recurrence B_l = [(2l-1) B_{l-1} + (2a^2)^l exp(-a^2 r^2)/(a sqrt(pi))]/r^2.
 * a == 0 gives the bare Coulomb kernel, B_l = (2l-1)!!/r^(2l+1).            */
void or_bfun(double r, double a, int lmax, double *B)
{
    double r2 = r * r;
    if (a == 0.0) {
        B[0] = 1.0 / r;
        for (int l = 1; l <= lmax; ++l) B[l] = (2 * l - 1) * B[l - 1] / r2;
        return;
    }
    double ex = exp(-a * a * r2);
    double pw = 1.0 / (a * sqrt(M_PI));
    B[0] = erfc(a * r) / r;
    for (int l = 1; l <= lmax; ++l) {
        pw *= 2.0 * a * a;
        B[l] = ((2 * l - 1) * B[l - 1] + pw * ex) / r2;
    }
}

/* ------------------------------------------------------------------------ */
/* Cartesian derivative tensors of a radial kernel f(r):
 *   d^n f / dr_{i1}..dr_{in} = sum over partial pairings of the n indices with
 *   p pairs:  (-1)^(n-p) B_{n-p} prod_{pairs} delta prod_{unpaired} r
 * (rank 1: -r B1; rank 2: -delta B1 + r r B2; rank 3: (delta r + 2 perms) B2
 * - r r r B3; ...).  For each rank n <= 5 and each index tuple we precompute
 * the list of monomials (p, ex, ey, ez, multiplicity).                        */
typedef struct { int p, e[3], mult; } or_term;
typedef struct { int nterm; or_term t[16]; } or_entry;
static or_entry g_tab[6][243];
static int g_tab_ready = 0;

static void enum_pairings(const int *idx, int n, int used, int p, int *ecount,
                          or_entry *ent)
{
    int first = -1;
    for (int i = 0; i < n; ++i) if (!(used & (1 << i))) { first = i; break; }
    if (first < 0) {
        /* record monomial */
        for (int k = 0; k < ent->nterm; ++k) {
            or_term *t = &ent->t[k];
            if (t->p == p && t->e[0] == ecount[0] && t->e[1] == ecount[1] && t->e[2] == ecount[2]) {
                t->mult++;
                return;
            }
        }
        or_term *t = &ent->t[ent->nterm++];
        t->p = p; t->e[0] = ecount[0]; t->e[1] = ecount[1]; t->e[2] = ecount[2]; t->mult = 1;
        return;
    }
    /* leave 'first' unpaired */
    ecount[idx[first]]++;
    enum_pairings(idx, n, used | (1 << first), p, ecount, ent);
    ecount[idx[first]]--;
    /* pair 'first' with a later equal index */
    for (int j = first + 1; j < n; ++j) {
        if (used & (1 << j)) continue;
        if (idx[j] != idx[first]) continue;
        enum_pairings(idx, n, used | (1 << first) | (1 << j), p + 1, ecount, ent);
    }
}

static void build_tab(void)
{
    if (g_tab_ready) return;
    for (int n = 0; n <= 5; ++n) {
        int cnt = 1;
        for (int k = 0; k < n; ++k) cnt *= 3;
        for (int flat = 0; flat < cnt; ++flat) {
            int idx[5], f = flat;
            for (int k = n - 1; k >= 0; --k) { idx[k] = f % 3; f /= 3; }
            or_entry *ent = &g_tab[n][flat];
            ent->nterm = 0;
            int ec[3] = {0, 0, 0};
            enum_pairings(idx, n, 0, 0, ec, ent);
        }
    }
    g_tab_ready = 1;
}

/* T_n at index tuple idx given r and B[0..5]. */
static double tensor_entry(int n, const int *idx, const double *rp[3], const double *B)
{
    int flat = 0;
    for (int k = 0; k < n; ++k) flat = flat * 3 + idx[k];
    const or_entry *ent = &g_tab[n][flat];
    double s = 0.0;
    for (int k = 0; k < ent->nterm; ++k) {
        const or_term *t = &ent->t[k];
        double mono = rp[0][t->e[0]] * rp[1][t->e[1]] * rp[2][t->e[2]];
        double sg = ((n - t->p) & 1) ? -1.0 : 1.0;
        s += sg * t->mult * B[n - t->p] * mono;
    }
    return s;
}

/* Expand a multipole vector into operator components (order, indices, weight).
 * Theta : grad grad uses all 9 entries (off-diagonals appear twice).           */
typedef struct { int order; int idx[2]; double w; int src; } or_comp;
static const int TH_ID[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};

static int expand_mp(const double *mp, or_comp *c)
{
    int n = 0;
    c[n].order = 0; c[n].w = mp[0]; c[n].src = 0; n++;
    for (int a = 0; a < 3; ++a) { c[n].order = 1; c[n].idx[0] = a; c[n].w = mp[1 + a]; c[n].src = 1 + a; n++; }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            c[n].order = 2; c[n].idx[0] = a; c[n].idx[1] = b;
            c[n].w = mp[TH_ID[a][b]]; c[n].src = TH_ID[a][b]; n++;
        }
    return n;
}

/* Pair term, explicit tensor contraction.
 * r = x_i - x_k (target i, source k), B[0..5] for |r|.
 * out[0]      = e = P_ik f
 * out[1..3]   = d e / d r            (= contribution to dE/dx_i)
 * out[4]      = d e / d q_i
 * out[5..7]   = d e / d mu_i
 * out[8..13]  = d e / d Theta_i      (stored-6 convention)                    */
void or_pair_tensor(const double *r, const double *B, const double *mi,
                    const double *mk, double *out)
{
    build_tab();
    double rpw[3][6];
    const double *rp[3];
    for (int a = 0; a < 3; ++a) {
        rpw[a][0] = 1.0;
        for (int e = 1; e < 6; ++e) rpw[a][e] = rpw[a][e - 1] * r[a];
        rp[a] = rpw[a];
    }
    or_comp ci[13], ck[13];
    int ni = expand_mp(mi, ci), nk = expand_mp(mk, ck);
    for (int k = 0; k < 14; ++k) out[k] = 0.0;
    for (int A = 0; A < ni; ++A) {
        for (int Bk = 0; Bk < nk; ++Bk) {
            int idx[6], n = 0;
            for (int k = 0; k < ci[A].order; ++k) idx[n++] = ci[A].idx[k];
            for (int k = 0; k < ck[Bk].order; ++k) idx[n++] = ck[Bk].idx[k];
            double sgn = (ck[Bk].order & 1) ? -1.0 : 1.0;   /* source acts with -grad */
            double T = tensor_entry(n, idx, rp, B);
            double wk = sgn * ck[Bk].w;
            /* energy */
            out[0] += ci[A].w * wk * T;
            /* derivative w.r.t. the target component (chain to stored entries) */
            int s = ci[A].src;
            double d = wk * T;
            if (s == 0) out[4] += d;
            else if (s <= 3) out[4 + s] += d;
            else out[4 + s] += d;   /* 8..13 : each of the 9 entries adds to its stored slot */
            /* position gradient: one more derivative */
            for (int e = 0; e < 3; ++e) {
                idx[n] = e;
                double T1 = tensor_entry(n + 1, idx, rp, B);
                out[1 + e] += ci[A].w * wk * T1;
            }
        }
    }
}

/* Pair term, closed-form scalar expansion (same outputs as or_pair_tensor).
 * With s_i = mu_i.r, s_k = mu_k.r, t_i = tr Theta_i, t_k = tr Theta_k,
 * u_i = r.Theta_i.r, u_k = r.Theta_k.r:
 *   c0 = q_i q_k
 *   c1 = q_i (s_k - t_k) - q_k (s_i + t_i) + mu_i.mu_k
 *   c2 = q_i u_k + q_k u_i - (s_i + t_i)(s_k - t_k) + 2 mu_i.Theta_k r
 *        - 2 mu_k.Theta_i r + 2 Theta_i:Theta_k
 *   c3 = (s_k - t_k) u_i - (s_i + t_i) u_k - 4 (Theta_i r).(Theta_k r)
 *   c4 = u_i u_k
 *   e  = sum_l c_l B_l,   grad e = sum_l (grad c_l) B_l - r sum_l c_l B_{l+1}  */
static inline void symv(const double *T, const double *v, double *o)
{
    o[0] = T[4] * v[0] + T[5] * v[1] + T[6] * v[2];
    o[1] = T[5] * v[0] + T[7] * v[1] + T[8] * v[2];
    o[2] = T[6] * v[0] + T[8] * v[1] + T[9] * v[2];
}

void or_pair_scalar(const double *r, const double *B, const double *mi,
                    const double *mk, double *out)
{
    const double qi = mi[0], qk = mk[0];
    const double *di = mi + 1, *dk = mk + 1;
    double Qir[3], Qkr[3];
    symv(mi, r, Qir);
    symv(mk, r, Qkr);
    double si = di[0] * r[0] + di[1] * r[1] + di[2] * r[2];
    double sk = dk[0] * r[0] + dk[1] * r[1] + dk[2] * r[2];
    double ti = mi[4] + mi[7] + mi[9];
    double tk = mk[4] + mk[7] + mk[9];
    double ui = r[0] * Qir[0] + r[1] * Qir[1] + r[2] * Qir[2];
    double uk = r[0] * Qkr[0] + r[1] * Qkr[1] + r[2] * Qkr[2];
    double didk = di[0] * dk[0] + di[1] * dk[1] + di[2] * dk[2];
    double diQkr = di[0] * Qkr[0] + di[1] * Qkr[1] + di[2] * Qkr[2];
    double dkQir = dk[0] * Qir[0] + dk[1] * Qir[1] + dk[2] * Qir[2];
    double QirQkr = Qir[0] * Qkr[0] + Qir[1] * Qkr[1] + Qir[2] * Qkr[2];
    double QiQk = mi[4] * mk[4] + mi[7] * mk[7] + mi[9] * mk[9]
                + 2.0 * (mi[5] * mk[5] + mi[6] * mk[6] + mi[8] * mk[8]);
    double ski = sk - tk, sit = si + ti;

    double c[5];
    c[0] = qi * qk;
    c[1] = qi * ski - qk * sit + didk;
    c[2] = qi * uk + qk * ui - sit * ski + 2.0 * diQkr - 2.0 * dkQir + 2.0 * QiQk;
    c[3] = ski * ui - sit * uk - 4.0 * QirQkr;
    c[4] = ui * uk;
    double e = 0.0, cb1 = 0.0;
    for (int l = 0; l < 5; ++l) { e += c[l] * B[l]; cb1 += c[l] * B[l + 1]; }
    out[0] = e;

    /* gradients of the c_l */
    double Qi_dk[3], Qk_di[3], Qi_Qkr[3], Qk_Qir[3];
    symv(mi, dk, Qi_dk);
    symv(mk, di, Qk_di);
    symv(mi, Qkr, Qi_Qkr);
    symv(mk, Qir, Qk_Qir);
    for (int a = 0; a < 3; ++a) {
        double g1 = qi * dk[a] - qk * di[a];
        double g2 = 2.0 * qi * Qkr[a] + 2.0 * qk * Qir[a] - di[a] * ski - sit * dk[a]
                  + 2.0 * Qk_di[a] - 2.0 * Qi_dk[a];
        double g3 = 2.0 * ski * Qir[a] + ui * dk[a] - 2.0 * sit * Qkr[a] - uk * di[a]
                  - 4.0 * (Qi_Qkr[a] + Qk_Qir[a]);
        double g4 = 2.0 * uk * Qir[a] + 2.0 * ui * Qkr[a];
        out[1 + a] = g1 * B[1] + g2 * B[2] + g3 * B[3] + g4 * B[4] - r[a] * cb1;
    }
    /* potential, field, field gradient of the source at the target */
    out[4] = qk * B[0] + ski * B[1] + uk * B[2];
    for (int a = 0; a < 3; ++a)
        out[5 + a] = B[1] * (dk[a] - qk * r[a]) + B[2] * (2.0 * Qkr[a] - ski * r[a]) - B[3] * uk * r[a];
    double dA = -qk * B[1] - ski * B[2] - uk * B[3];
    double rrA = qk * B[2] + ski * B[3] + uk * B[4];
    static const int PA[6] = {0, 0, 0, 1, 1, 2}, PB[6] = {0, 1, 2, 1, 2, 2};
    for (int m = 0; m < 6; ++m) {
        int a = PA[m], b = PB[m];
        double G = (a == b ? dA : 0.0) + r[a] * r[b] * rrA
                 - (dk[a] * r[b] + r[a] * dk[b]) * B[2]
                 + 2.0 * mk[TH_ID[a][b]] * B[2]
                 - 2.0 * (r[a] * Qkr[b] + Qkr[a] * r[b]) * B[3];
        out[8 + m] = (a == b) ? G : 2.0 * G;
    }
}

/* ------------------------------------------------------------------------ */
/* Sum over an explicit ordered pair list in CSR form (row = target atom).
 * For each target i and each listed (j, shift): r = x_i - x_j - shift.
 * E_out += sum of e over all listed ordered pairs (NOT halved).
 * grad (N x 13) += target-side derivatives.  a == 0: bare Coulomb.           */
int or_pair_csr(int64_t N, const double *x, const double *mp, const int64_t *rowptr,
                const int32_t *col, const double *shift, double a, int use_tensor,
                double *E_out, double *grad, int nthreads)
{
    double Etot = 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    double *Ei = (double *)calloc((size_t)N, sizeof(double));
    if (!Ei) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        double acc[14] = {0};
        double out[14], B[6], r[3];
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            for (int c = 0; c < 3; ++c) r[c] = x[3 * i + c] - x[3 * (int64_t)j + c] - shift[3 * p + c];
            double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            or_bfun(rr, a, 5, B);
            if (use_tensor) or_pair_tensor(r, B, mp + OR_NMP * i, mp + OR_NMP * (int64_t)j, out);
            else or_pair_scalar(r, B, mp + OR_NMP * i, mp + OR_NMP * (int64_t)j, out);
            for (int c = 0; c < 14; ++c) acc[c] += out[c];
        }
        Ei[i] = acc[0];
        if (grad)
            for (int c = 0; c < 13; ++c) grad[OR_NGR * i + c] += acc[1 + c];
    }
    /* Neumaier sum in index order: deterministic */
    double s = 0.0, comp = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double t = s + Ei[i];
        if (fabs(s) >= fabs(Ei[i])) comp += (s - t) + Ei[i];
        else comp += (Ei[i] - t) + s;
        s = t;
    }
    Etot = s + comp;
    free(Ei);
    *E_out += Etot;
    return 0;
}

/* ------------------------------------------------------------------------ */
static double neumaier(const double *v, int64_t n)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = s + v[i];
        if (fabs(s) >= fabs(v[i])) c += (s - t) + v[i];
        else c += (v[i] - t) + s;
        s = t;
    }
    return s + c;
}

static inline int64_t floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

/* Real-space Ewald sum (E_real) over all ordered pairs and images with
 * |r| < rcut, excluding i == j at zero shift.  Targets are restricted to the
 * list 'tgt' (ntgt entries) when tgt != NULL (used to time a bounded sample);
 * E_real then holds 1/2 sum over those targets' rows only.                   */
int or_ewald_real(int64_t N, const double *x, const double *mp, double box, double alpha,
                  double rcut, int use_tensor, const int64_t *tgt, int64_t ntgt,
                  double *E_real, double *grad, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    /* wrap positions into [0, box) */
    double *xw = (double *)malloc((size_t)N * 3 * sizeof(double));
    if (!xw) return -1;
    for (int64_t i = 0; i < 3 * N; ++i) {
        double s = x[i] / box;
        s -= floor(s);
        xw[i] = s * box;
        if (xw[i] >= box) xw[i] -= box;
    }
    int nb = (int)floor(box / (rcut / 3.0));
    if (nb < 1) nb = 1;
    if (nb > 256) nb = 256;
    double bsz = box / nb;
    int R = (int)ceil(rcut / bsz);
    int64_t nbin = (int64_t)nb * nb * nb;
    int64_t *bstart = (int64_t *)calloc((size_t)nbin + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    int64_t *bin_of = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    if (!bstart || !order || !bin_of) return -1;
    for (int64_t i = 0; i < N; ++i) {
        int b3[3];
        for (int c = 0; c < 3; ++c) {
            int b = (int)floor(xw[3 * i + c] / bsz);
            if (b >= nb) b = nb - 1;
            if (b < 0) b = 0;
            b3[c] = b;
        }
        bin_of[i] = ((int64_t)b3[0] * nb + b3[1]) * nb + b3[2];
        bstart[bin_of[i] + 1]++;
    }
    for (int64_t b = 0; b < nbin; ++b) bstart[b + 1] += bstart[b];
    {
        int64_t *fill = (int64_t *)malloc((size_t)nbin * sizeof(int64_t));
        memcpy(fill, bstart, (size_t)nbin * sizeof(int64_t));
        for (int64_t i = 0; i < N; ++i) order[fill[bin_of[i]]++] = i;
        free(fill);
    }
    int64_t nt = tgt ? ntgt : N;
    double *Ei = (double *)calloc((size_t)nt, sizeof(double));
    double rc2 = rcut * rcut;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t it = 0; it < nt; ++it) {
        int64_t i = tgt ? tgt[it] : it;
        int64_t bi = bin_of[i];
        int bx = (int)(bi / ((int64_t)nb * nb)), by = (int)((bi / nb) % nb), bz = (int)(bi % nb);
        double acc[14] = {0};
        double out[14], B[6], r[3];
        for (int ox = -R; ox <= R; ++ox) {
            double gx = (abs(ox) > 0 ? (abs(ox) - 1) * bsz : 0.0);
            for (int oy = -R; oy <= R; ++oy) {
                double gy = (abs(oy) > 0 ? (abs(oy) - 1) * bsz : 0.0);
                if (gx * gx + gy * gy > rc2) continue;
                for (int oz = -R; oz <= R; ++oz) {
                    double gz = (abs(oz) > 0 ? (abs(oz) - 1) * bsz : 0.0);
                    if (gx * gx + gy * gy + gz * gz > rc2) continue;
                    int64_t sx = bx + ox, sy = by + oy, sz = bz + oz;
                    int64_t wx = floordiv(sx, nb), wy = floordiv(sy, nb), wz = floordiv(sz, nb);
                    int64_t sb = ((sx - wx * nb) * nb + (sy - wy * nb)) * nb + (sz - wz * nb);
                    double shx = wx * box, shy = wy * box, shz = wz * box;
                    int self_img = (wx == 0 && wy == 0 && wz == 0);
                    for (int64_t p = bstart[sb]; p < bstart[sb + 1]; ++p) {
                        int64_t j = order[p];
                        if (self_img && j == i) continue;
                        r[0] = xw[3 * i] - xw[3 * j] - shx;
                        r[1] = xw[3 * i + 1] - xw[3 * j + 1] - shy;
                        r[2] = xw[3 * i + 2] - xw[3 * j + 2] - shz;
                        double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                        if (r2 >= rc2) continue;
                        or_bfun(sqrt(r2), alpha, 5, B);
                        if (use_tensor) or_pair_tensor(r, B, mp + OR_NMP * i, mp + OR_NMP * j, out);
                        else or_pair_scalar(r, B, mp + OR_NMP * i, mp + OR_NMP * j, out);
                        for (int c = 0; c < 14; ++c) acc[c] += out[c];
                    }
                }
            }
        }
        Ei[it] = 0.5 * acc[0];
        if (grad)
            for (int c = 0; c < 13; ++c) grad[OR_NGR * i + c] += acc[1 + c];
    }
    *E_real = neumaier(Ei, nt);
    free(Ei); free(xw); free(bstart); free(order); free(bin_of);
    return 0;
}

/* Reciprocal-space Ewald sum over k = 2 pi m / box, 0 < |k| <= kcut.
 * Half-space enumeration (weight 2).  'kstride' > 1 keeps only every
 * kstride-th k-vector (bounded timing sample; the result is then partial).   */
int or_ewald_rec(int64_t N, const double *x, const double *mp, double box, double alpha,
                 double kcut, int64_t kstride, double *E_rec, double *grad, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    if (kstride < 1) kstride = 1;
    const double V = box * box * box;
    const double tpl = 2.0 * M_PI / box;
    int mmax = (int)floor(kcut / tpl);
    /* enumerate half-space k vectors */
    int64_t cap = (int64_t)(2 * mmax + 1) * (2 * mmax + 1) * (mmax + 1) + 8;
    int *km = (int *)malloc((size_t)cap * 3 * sizeof(int));
    int64_t nk = 0, seen = 0;
    for (int mx = 0; mx <= mmax; ++mx)
        for (int my = -mmax; my <= mmax; ++my)
            for (int mz = -mmax; mz <= mmax; ++mz) {
                if (mx == 0 && (my < 0 || (my == 0 && mz <= 0))) continue;
                double k2 = tpl * tpl * ((double)mx * mx + (double)my * my + (double)mz * mz);
                if (k2 > kcut * kcut) continue;
                if ((seen++ % kstride) != 0) continue;
                km[3 * nk] = mx; km[3 * nk + 1] = my; km[3 * nk + 2] = mz; nk++;
            }
    double *Sre = (double *)calloc((size_t)nk, sizeof(double));
    double *Sim = (double *)calloc((size_t)nk, sizeof(double));
    double *gk = (double *)malloc((size_t)nk * sizeof(double));
    for (int64_t k = 0; k < nk; ++k) {
        double kx = tpl * km[3 * k], ky = tpl * km[3 * k + 1], kz = tpl * km[3 * k + 2];
        double k2 = kx * kx + ky * ky + kz * kz;
        gk[k] = exp(-k2 / (4.0 * alpha * alpha)) / k2;
    }
    int nm = 2 * mmax + 1;
    /* structure factors: atoms in chunks, per-thread accumulators */
#pragma omp parallel
    {
        double *sr = (double *)calloc((size_t)nk, sizeof(double));
        double *si = (double *)calloc((size_t)nk, sizeof(double));
        double *ex = (double *)malloc((size_t)3 * nm * 2 * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t j = 0; j < N; ++j) {
            for (int c = 0; c < 3; ++c) {
                for (int m = -mmax; m <= mmax; ++m) {
                    double ph = tpl * m * x[3 * j + c];
                    ex[(c * nm + (m + mmax)) * 2] = cos(ph);
                    ex[(c * nm + (m + mmax)) * 2 + 1] = sin(ph);
                }
            }
            const double *m0 = mp + OR_NMP * j;
            for (int64_t k = 0; k < nk; ++k) {
                int mx = km[3 * k], my = km[3 * k + 1], mz = km[3 * k + 2];
                const double *a = &ex[(0 * nm + mx + mmax) * 2];
                const double *b = &ex[(1 * nm + my + mmax) * 2];
                const double *cz = &ex[(2 * nm + mz + mmax) * 2];
                double abr = a[0] * b[0] - a[1] * b[1], abi = a[0] * b[1] + a[1] * b[0];
                double pr = abr * cz[0] - abi * cz[1], pi_ = abr * cz[1] + abi * cz[0];
                double kv[3] = {tpl * mx, tpl * my, tpl * mz};
                double Ar = m0[0] - (m0[4] * kv[0] * kv[0] + m0[7] * kv[1] * kv[1] + m0[9] * kv[2] * kv[2]
                           + 2.0 * (m0[5] * kv[0] * kv[1] + m0[6] * kv[0] * kv[2] + m0[8] * kv[1] * kv[2]));
                double Ai = m0[1] * kv[0] + m0[2] * kv[1] + m0[3] * kv[2];
                sr[k] += Ar * pr - Ai * pi_;
                si[k] += Ar * pi_ + Ai * pr;
            }
        }
#pragma omp critical
        {
            for (int64_t k = 0; k < nk; ++k) { Sre[k] += sr[k]; Sim[k] += si[k]; }
        }
        free(sr); free(si); free(ex);
    }
    double *ek = (double *)malloc((size_t)nk * sizeof(double));
    for (int64_t k = 0; k < nk; ++k) ek[k] = (4.0 * M_PI / V) * gk[k] * (Sre[k] * Sre[k] + Sim[k] * Sim[k]);
    *E_rec = neumaier(ek, nk);
    free(ek);
    if (grad) {
#pragma omp parallel
        {
            double *ex = (double *)malloc((size_t)3 * nm * 2 * sizeof(double));
#pragma omp for schedule(static)
            for (int64_t j = 0; j < N; ++j) {
                for (int c = 0; c < 3; ++c)
                    for (int m = -mmax; m <= mmax; ++m) {
                        double ph = tpl * m * x[3 * j + c];
                        ex[(c * nm + (m + mmax)) * 2] = cos(ph);
                        ex[(c * nm + (m + mmax)) * 2 + 1] = sin(ph);
                    }
                const double *m0 = mp + OR_NMP * j;
                double g[13] = {0};
                for (int64_t k = 0; k < nk; ++k) {
                    int mx = km[3 * k], my = km[3 * k + 1], mz = km[3 * k + 2];
                    const double *a = &ex[(0 * nm + mx + mmax) * 2];
                    const double *b = &ex[(1 * nm + my + mmax) * 2];
                    const double *cz = &ex[(2 * nm + mz + mmax) * 2];
                    double abr = a[0] * b[0] - a[1] * b[1], abi = a[0] * b[1] + a[1] * b[0];
                    double pr = abr * cz[0] - abi * cz[1], pi_ = abr * cz[1] + abi * cz[0];
                    /* f = conj(S) e^{ik.x_j} */
                    double fr = Sre[k] * pr + Sim[k] * pi_;
                    double fi = Sre[k] * pi_ - Sim[k] * pr;
                    double kv[3] = {tpl * mx, tpl * my, tpl * mz};
                    double w = (4.0 * M_PI / V) * gk[k] * 2.0;
                    double Ar = m0[0] - (m0[4] * kv[0] * kv[0] + m0[7] * kv[1] * kv[1] + m0[9] * kv[2] * kv[2]
                               + 2.0 * (m0[5] * kv[0] * kv[1] + m0[6] * kv[0] * kv[2] + m0[8] * kv[1] * kv[2]));
                    double Ai = m0[1] * kv[0] + m0[2] * kv[1] + m0[3] * kv[2];
                    double xr = -(Ar * fi + Ai * fr);
                    for (int c = 0; c < 3; ++c) g[c] += w * kv[c] * xr;
                    g[3] += w * fr;
                    for (int c = 0; c < 3; ++c) g[4 + c] += w * (-kv[c] * fi);
                    g[7] += -w * kv[0] * kv[0] * fr;
                    g[8] += -w * 2.0 * kv[0] * kv[1] * fr;
                    g[9] += -w * 2.0 * kv[0] * kv[2] * fr;
                    g[10] += -w * kv[1] * kv[1] * fr;
                    g[11] += -w * 2.0 * kv[1] * kv[2] * fr;
                    g[12] += -w * kv[2] * kv[2] * fr;
                }
                for (int c = 0; c < 13; ++c) grad[OR_NGR * j + c] += g[c];
            }
            free(ex);
        }
    }
    free(km); free(Sre); free(Sim); free(gk);
    return 0;
}

/* Self and neutralising terms (and their gradients). */
int or_ewald_self(int64_t N, const double *mp, double box, double alpha,
                  double *E_self, double *E_neut, double *grad)
{
    const double V = box * box * box;
    const double c = alpha / sqrt(M_PI), a2 = alpha * alpha, a4 = a2 * a2;
    double *es = (double *)malloc((size_t)N * sizeof(double));
    double Q = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        const double *m = mp + OR_NMP * i;
        double q = m[0];
        double mu2 = m[1] * m[1] + m[2] * m[2] + m[3] * m[3];
        double tr = m[4] + m[7] + m[9];
        double TT = m[4] * m[4] + m[7] * m[7] + m[9] * m[9] + 2.0 * (m[5] * m[5] + m[6] * m[6] + m[8] * m[8]);
        es[i] = -c * (q * q + (2.0 * a2 / 3.0) * mu2 - (4.0 * a2 / 3.0) * q * tr
                      + (8.0 * a4 / 5.0) * TT + (4.0 * a4 / 5.0) * tr * tr);
        Q += q;
        if (grad) {
            double *g = grad + OR_NGR * i;
            g[3] += -c * (2.0 * q - (4.0 * a2 / 3.0) * tr);
            for (int k = 0; k < 3; ++k) g[4 + k] += -c * (4.0 * a2 / 3.0) * m[1 + k];
            /* 9-entry derivative: -c[-(4a2/3) q delta + (16a4/5) Theta + (8a4/5) tr delta] */
            double dg = -(4.0 * a2 / 3.0) * q + (8.0 * a4 / 5.0) * tr;
            g[7] += -c * (dg + (16.0 * a4 / 5.0) * m[4]);
            g[8] += -c * 2.0 * (16.0 * a4 / 5.0) * m[5];
            g[9] += -c * 2.0 * (16.0 * a4 / 5.0) * m[6];
            g[10] += -c * (dg + (16.0 * a4 / 5.0) * m[7]);
            g[11] += -c * 2.0 * (16.0 * a4 / 5.0) * m[8];
            g[12] += -c * (dg + (16.0 * a4 / 5.0) * m[9]);
        }
    }
    *E_self = neumaier(es, N);
    free(es);
    /* neutralising background */
    double Qs = 0.0;
    for (int64_t i = 0; i < N; ++i) Qs += mp[OR_NMP * i];
    *E_neut = -M_PI * Qs * Qs / (2.0 * V * a2);
    if (grad)
        for (int64_t i = 0; i < N; ++i) grad[OR_NGR * i + 3] += -M_PI * Qs / (V * a2);
    (void)Q;
    return 0;
}
