/*
 * FP64 CPU oracle for RGDBEK — Randomized Greedy Double Block Extended
 * Kaczmarz (arXiv 2509.19267).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark call it; the library's product path never
 * does.  It shares no code, header, table or constant generator with the CUDA
 * library: both sides implement the same published definitions separately.
 *
 * Plain, single-threaded, double precision, no blocking or fusion.  Each
 * routine is either the plain definition of what it computes or the steps of
 * the paper's algorithm in the paper's order:
 *   - the problem Ax = b, A in R^{m x n}                       (Eq. 1)
 *   - the block update of z and x                              (Eq. 4)
 *   - column residual weights eps^z_j = (A_j^T z)^2/||A_j||^2 and row
 *     residual weights eps^x_i = (b_i - z_i - A^(i) x)^2/||A^(i)||^2, the
 *     probabilities P proportional to them                     (Section 2)
 *   - the outer loop with x_0 = 0, z_0 = b                     (Algorithm 1)
 *   - LSQR as the inner least-squares solver                   (Remark 3.1)
 *   - the relative square error RSE = ||Ax-b||^2/||b||^2       (Section 3.1)
 *   - the greedy threshold sets of GDBEK                       (Section 2)
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *   - "select eta*n columns using P": ceil(eta*len) independent draws with
 *     replacement from P; the block is the sorted set of distinct indices.
 *   - draws are made exact and order-independent: the weights are quantised
 *     to integers q_j = floor(2^K eps_j / eps_max), K = 62 - ceil(log2 len),
 *     and a draw picks the first j whose inclusive prefix sum of q exceeds
 *     floor(R * Q_total / 2^64), R a 64-bit Philox4x64-10 output word.
 *   - Philox key = (seed, system id), counter = (k, phase, t div 4, 0) with
 *     phase 0 for columns and 1 for rows; draw t uses word t mod 4.
 *   - the inner LSQR starts from 0 (so it returns the minimum-norm solution)
 *     and stops when ||B^T r|| <= tol ||B||_F ||r|| or ||r|| <= tol ||c||, or
 *     after inner_max steps.  In the column step it runs on A_U with its
 *     columns scaled to unit norm (the projection A_U A_U^+ z does not depend
 *     on which least-squares solution is used); in the row step, when |J| <= n,
 *     first on A^J with its rows scaled to unit norm, which has the same
 *     minimum-norm solution whenever the block system is consistent, and
 *     again unscaled when LSQR finds it inconsistent.
 *   - a block whose weights are all zero is empty and its update is skipped;
 *     when both blocks are empty x can no longer change and the solve ends.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of the 4x64 S-box with a Weyl key    */
/* schedule.  Multipliers and key increments are the published constants.   */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t key_in[2], const uint64_t ctr_in[4],
                       uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t k0 = key_in[0], k1 = key_in[1];
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Plain CSR products and norms (A given by row pointers, column indices and */
/* values; row i holds entries rp[i] .. rp[i+1]-1).                          */
/* ------------------------------------------------------------------------ */

/* y = A x */
void orc_spmv(int64_t m, const int64_t *rp, const int32_t *ci, const double *av,
              const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += av[e] * x[ci[e]];
        y[i] = s;
    }
}

/* g = A^T z, by its definition g_j = sum_i A_ij z_i (scattered row by row) */
void orc_spmv_t(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci,
                const double *av, const double *z, double *g)
{
    for (int64_t j = 0; j < n; ++j) g[j] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) g[ci[e]] += av[e] * z[i];
}

/* ||A^(i)||^2 for every row i */
void orc_row_norms2(int64_t m, const int64_t *rp, const double *av, double *rn2)
{
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += av[e] * av[e];
        rn2[i] = s;
    }
}

/* ||A_(j)||^2 for every column j */
void orc_col_norms2(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci,
                    const double *av, double *cn2)
{
    for (int64_t j = 0; j < n; ++j) cn2[j] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) cn2[ci[e]] += av[e] * av[e];
}

static double dot(int64_t len, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Residual weights (Section 2): eps_j = v_j^2 / norm2_j, 0 where the norm   */
/* is 0.  Returns max_j eps_j; sets *has_nan when a weight is not finite.    */
/* ------------------------------------------------------------------------ */
double orc_weights(int64_t len, const double *v, const double *norm2, double *eps,
                   int *has_nan)
{
    double emax = 0.0;
    *has_nan = 0;
    for (int64_t j = 0; j < len; ++j) {
        double e = norm2[j] > 0.0 ? (v[j] * v[j]) / norm2[j] : 0.0;
        eps[j] = e;
        if (!isfinite(e)) *has_nan = 1;
        else if (e > emax) emax = e;
    }
    return emax;
}

/* ------------------------------------------------------------------------ */
/* Block selection (Section 2, Algorithm 1): ceil(eta*len) draws with        */
/* replacement, each index j with probability eps_j / sum eps, kept as the  */
/* sorted set of distinct indices.  The probabilities are realised exactly  */
/* by integer quantisation (see the file header).  Returns the block size.  */
/* ------------------------------------------------------------------------ */
static int ceil_log2_i64(int64_t v)
{
    int c = 0;
    while (((int64_t)1 << c) < v) ++c;
    return c;
}

int64_t orc_num_draws(double eta, int64_t len)
{
    if (len <= 0) return 0;
    double s = ceil(eta * (double)len);
    if (s < 1.0) s = 1.0;
    return (int64_t)s;
}

int64_t orc_sample(int64_t len, const double *eps, double emax, int64_t s,
                   uint64_t seed, uint64_t sysid, uint64_t k, uint64_t phase,
                   int32_t *idx_out)
{
    if (len <= 0 || s <= 0 || !(emax > 0.0)) return 0;
    const int K = 62 - ceil_log2_i64(len);
    uint64_t *Q = (uint64_t *)malloc((size_t)len * sizeof(uint64_t));
    unsigned char *flag = (unsigned char *)calloc((size_t)len, 1);
    uint64_t acc = 0;
    for (int64_t j = 0; j < len; ++j) {
        double ratio = eps[j] / emax;
        uint64_t q = (uint64_t)floor(ldexp(ratio, K));
        acc += q;
        Q[j] = acc; /* inclusive prefix sum */
    }
    const uint64_t qtot = acc;
    const uint64_t key[2] = {seed, sysid};
    uint64_t block[4];
    for (int64_t t = 0; t < s; ++t) {
        if ((t & 3) == 0) {
            const uint64_t ctr[4] = {k, phase, (uint64_t)(t >> 2), 0};
            orc_philox4x64_10(key, ctr, block);
        }
        uint64_t R = block[t & 3];
        uint64_t target = (uint64_t)(((unsigned __int128)R * qtot) >> 64);
        /* first j with Q[j] > target */
        int64_t lo = 0, hi = len - 1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (Q[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        flag[lo] = 1;
    }
    int64_t cnt = 0;
    for (int64_t j = 0; j < len; ++j)
        if (flag[j]) idx_out[cnt++] = (int32_t)j;
    free(Q);
    free(flag);
    return cnt;
}

/* Greedy threshold set of GDBEK (Section 2): {j : eps_j >= eta * eps_max}. */
int64_t orc_select_greedy(int64_t len, const double *eps, double emax, double eta,
                          int32_t *idx_out)
{
    if (len <= 0 || !(emax > 0.0)) return 0;
    const double thr = eta * emax;
    int64_t cnt = 0;
    for (int64_t j = 0; j < len; ++j)
        if (eps[j] >= thr && eps[j] > 0.0) idx_out[cnt++] = (int32_t)j;
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* LSQR (Paige and Saunders, ACM TOMS 8(1), 1982) for min ||B y - c||, from  */
/* y = 0, with B an mb x nb CSR matrix.  This is the inner solver the paper  */
/* uses for the block pseudo-inverse products (Remark 3.1).  fro = ||B||_F.  */
/* Returns the number of steps taken; *fit (if not NULL) is set to 1 when   */
/* it stopped because the residual itself met the tolerance (||r|| <= tol   */
/* ||c||, or an exact fit), i.e. the block system was found consistent, and  */
/* to 2 when it ran out of steps.                                            */
/* ------------------------------------------------------------------------ */
int orc_lsqr_fit(int64_t mb, int64_t nb, const int64_t *rp, const int32_t *ci,
                 const double *av, const double *c, double tol, double fro, int maxit,
                 double *y, int *fit)
{
    if (fit) *fit = 0;
    double *u = (double *)malloc((size_t)(mb > 0 ? mb : 1) * sizeof(double));
    double *v = (double *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(double));
    double *w = (double *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(double));
    double *tmp_m = (double *)malloc((size_t)(mb > 0 ? mb : 1) * sizeof(double));
    double *tmp_n = (double *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(double));
    int steps = 0;
    for (int64_t j = 0; j < nb; ++j) y[j] = 0.0;

    /* beta_1 u_1 = c,  alpha_1 v_1 = B^T u_1 */
    for (int64_t i = 0; i < mb; ++i) u[i] = c[i];
    double beta = sqrt(dot(mb, u, u));
    const double beta1 = beta;
    double alpha = 0.0;
    if (beta > 0.0) {
        for (int64_t i = 0; i < mb; ++i) u[i] /= beta;
        orc_spmv_t(mb, nb, rp, ci, av, u, v);
        alpha = sqrt(dot(nb, v, v));
    }
    if (beta > 0.0 && alpha > 0.0) {
        for (int64_t j = 0; j < nb; ++j) {
            v[j] /= alpha;
            w[j] = v[j];
        }
        double phibar = beta, rhobar = alpha;
        for (int it = 1; it <= maxit; ++it) {
            steps = it;
            /* beta_{i+1} u_{i+1} = B v_i - alpha_i u_i */
            orc_spmv(mb, rp, ci, av, v, tmp_m);
            for (int64_t i = 0; i < mb; ++i) u[i] = tmp_m[i] - alpha * u[i];
            beta = sqrt(dot(mb, u, u));
            if (beta > 0.0) {
                for (int64_t i = 0; i < mb; ++i) u[i] /= beta;
                /* alpha_{i+1} v_{i+1} = B^T u_{i+1} - beta_{i+1} v_i */
                orc_spmv_t(mb, nb, rp, ci, av, u, tmp_n);
                for (int64_t j = 0; j < nb; ++j) v[j] = tmp_n[j] - beta * v[j];
                alpha = sqrt(dot(nb, v, v));
                if (alpha > 0.0)
                    for (int64_t j = 0; j < nb; ++j) v[j] /= alpha;
            } else {
                alpha = 0.0;
            }
            /* plane rotation */
            double rho = sqrt(rhobar * rhobar + beta * beta);
            double cs = rhobar / rho;
            double sn = beta / rho;
            double theta = sn * alpha;
            rhobar = -cs * alpha;
            double phi = cs * phibar;
            phibar = sn * phibar;
            /* y_i = y_{i-1} + (phi_i / rho_i) w_i;  w_{i+1} = v_{i+1} - (theta/rho) w_i */
            for (int64_t j = 0; j < nb; ++j) {
                y[j] += (phi / rho) * w[j];
                w[j] = v[j] - (theta / rho) * w[j];
            }
            /* ||r_i|| = phibar_{i+1},  ||B^T r_i|| = phibar_{i+1} alpha_{i+1} |c_i| */
            double rnorm = phibar;
            double arnorm = phibar * alpha * fabs(cs);
            if (arnorm <= tol * fro * rnorm || rnorm <= tol * beta1 || alpha == 0.0 ||
                beta == 0.0) {
                if (fit) *fit = (rnorm <= tol * beta1 || beta == 0.0) ? 1 : 0;
                break;
            }
            if (it == maxit && fit) *fit = 2;
        }
    }
    free(u); free(v); free(w); free(tmp_m); free(tmp_n);
    return steps;
}

int orc_lsqr(int64_t mb, int64_t nb, const int64_t *rp, const int32_t *ci,
             const double *av, const double *c, double tol, double fro, int maxit,
             double *y)
{
    return orc_lsqr_fit(mb, nb, rp, ci, av, c, tol, fro, maxit, y, NULL);
}

/* ------------------------------------------------------------------------ */
/* Sub-matrices of A as CSR: A_U (all m rows, the columns in U, renumbered   */
/* 0..|U|-1) and A^J (the rows in J, all n columns).                         */
/* ------------------------------------------------------------------------ */
static void extract_columns(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci,
                            const double *av, int64_t nu, const int32_t *U,
                            int64_t *srp, int32_t *sci, double *sav)
{
    int32_t *pos = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    for (int64_t j = 0; j < n; ++j) pos[j] = -1;
    for (int64_t p = 0; p < nu; ++p) pos[U[p]] = (int32_t)p;
    int64_t cnt = 0;
    srp[0] = 0;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (pos[ci[e]] >= 0) {
                sci[cnt] = pos[ci[e]];
                sav[cnt] = av[e];
                ++cnt;
            }
        }
        srp[i + 1] = cnt;
    }
    free(pos);
}

static void extract_rows(const int64_t *rp, const int32_t *ci, const double *av,
                         int64_t nj, const int32_t *J, int64_t *srp, int32_t *sci,
                         double *sav)
{
    int64_t cnt = 0;
    srp[0] = 0;
    for (int64_t p = 0; p < nj; ++p) {
        int64_t i = J[p];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            sci[cnt] = ci[e];
            sav[cnt] = av[e];
            ++cnt;
        }
        srp[p + 1] = cnt;
    }
}

/* ------------------------------------------------------------------------ */
/* Options, statistics and the optional per-iteration trace.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    double eta_col, eta_row;  /* block fractions (eta of Algorithm 1)        */
    int selection;            /* 0 randomized (Algorithm 1), 1 greedy (GDBEK) */
    double inner_tol;         /* LSQR tolerance                              */
    int inner_max;            /* LSQR step cap                               */
    int stop_rule;            /* 0,2 normal eq.; 1 rel. residual; 3 RSE      */
    double tol;
    int64_t max_iter;
    uint64_t seed, sysid;
    int warm;                 /* 1: x holds x_0 on entry (else x_0 = 0)       */
    double inner_adapt;       /* > 0: inner tolerance of iteration k is
                                 max(inner_tol, min(0.1, inner_adapt * r_k)),
                                 r_k the stopping rule's measure of x_k       */
    int64_t k0;               /* number of the first iteration (0 for a fresh solve);
                                 max_iter caps the iteration number, not the count */
    double *z_state;          /* NULL: z_0 = b.  Otherwise z at iteration k0 on
                                 entry (a resumed solve; x holds x_k0 with warm = 1)
                                 and z at the last iteration on return, so that a
                                 solve cut into pieces draws and computes exactly
                                 what one uninterrupted solve does (the draws depend
                                 on (seed, k) only)                             */
} OrcOpts;

typedef struct {
    int64_t iters, inner_u, inner_j;
    double rel_res, normal_res, rse;
    int status; /* 0 converged, 1 iteration cap reached, -2 NaN met */
} OrcStats;

typedef struct {
    int64_t cap_iters;  /* iteration records the buffers can hold                */
    int64_t *counts;    /* [cap_iters][4] = |U_k|, |J_k|, LSQR steps (U), (J)     */
    int64_t list_cap;   /* capacity of lists                                     */
    int32_t *lists;     /* U_0, J_0, U_1, J_1, ... concatenated                  */
    int64_t list_len;   /* out: entries written                                  */
    int64_t n_iters;    /* out: records written                                  */
    double *zs;         /* optional [cap_iters + 1][m]: z_k at the start of iteration k */
    double *xs;         /* optional [cap_iters + 1][n]: x_k                      */
    /* optional lockstep input: take U_k and J_k from here instead of sampling */
    const int64_t *lock_counts; /* [lock_iters][2] = |U_k|, |J_k|            */
    const int32_t *lock_lists;
    int64_t lock_iters;
} OrcTrace;

static int stop_test(int rule, double tol, double rel, double nrm)
{
    switch (rule) {
    case 1: return rel <= tol;
    case 3: return rel * rel <= tol;
    default: return nrm <= tol;
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1.  x (length n) receives the result.                          */
/* ------------------------------------------------------------------------ */
int orc_solve(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci,
              const double *av, const double *b, const OrcOpts *o, double *x,
              OrcStats *st, OrcTrace *tr)
{
    const int64_t nnz = rp[m];
    double *rn2 = malloc((size_t)m * sizeof(double));
    double *cn2 = malloc((size_t)n * sizeof(double));
    double *z = malloc((size_t)m * sizeof(double));
    double *t = malloc((size_t)m * sizeof(double));
    double *r = malloc((size_t)m * sizeof(double));
    double *Ax = malloc((size_t)m * sizeof(double));
    double *g = malloc((size_t)n * sizeof(double));
    double *h = malloc((size_t)n * sizeof(double));
    double *epsz = malloc((size_t)n * sizeof(double));
    double *epsx = malloc((size_t)m * sizeof(double));
    double *y = malloc((size_t)n * sizeof(double));
    double *d = malloc((size_t)n * sizeof(double));
    double *rJ = malloc((size_t)m * sizeof(double));
    int32_t *U = malloc((size_t)n * sizeof(int32_t));
    int32_t *J = malloc((size_t)m * sizeof(int32_t));
    int64_t *srp = malloc((size_t)(m + 1) * sizeof(int64_t));
    int32_t *sci = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    double *sav = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    double *bsc = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    double *dcol = malloc((size_t)n * sizeof(double));

    orc_row_norms2(m, rp, av, rn2);
    orc_col_norms2(m, n, rp, ci, av, cn2);

    /* x_0 = 0 (or the given x_0), z_0 = b (or the given z of a resumed solve) */
    if (!o->warm)
        for (int64_t j = 0; j < n; ++j) x[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) z[i] = o->z_state ? o->z_state[i] : b[i];
    const double bnorm = sqrt(dot(m, b, b));
    orc_spmv_t(m, n, rp, ci, av, b, h);
    const double atbnorm = sqrt(dot(n, h, h));

    int64_t list_len = 0, n_rec = 0;
    int status = 1;
    int64_t k = 0;
    double rel = 0.0, nrm = 0.0;
    st->inner_u = 0;
    st->inner_j = 0;
    if (!isfinite(bnorm) || !isfinite(atbnorm)) {
        /* a non-finite entry in b (or an overflowing norm) is reported, not solved */
        st->iters = 0;
        st->rel_res = st->normal_res = st->rse = NAN;
        st->status = -2;
        if (tr) { tr->list_len = 0; tr->n_iters = 0; }
        free(rn2); free(cn2); free(z); free(t); free(r); free(Ax); free(g); free(h);
        free(epsz); free(epsx); free(y); free(d); free(rJ); free(U); free(J);
        free(srp); free(sci); free(sav); free(bsc); free(dcol);
        return -2;
    }
    for (k = o->k0;; ++k) {
        /* stopping test on x_k: t = b - A x_k */
        orc_spmv(m, rp, ci, av, x, Ax);
        for (int64_t i = 0; i < m; ++i) t[i] = b[i] - Ax[i];
        orc_spmv_t(m, n, rp, ci, av, t, h);
        rel = bnorm > 0.0 ? sqrt(dot(m, t, t)) / bnorm : 0.0;
        nrm = atbnorm > 0.0 ? sqrt(dot(n, h, h)) / atbnorm : 0.0;
        if (tr && tr->zs && k <= tr->cap_iters) memcpy(tr->zs + k * m, z, (size_t)m * sizeof(double));
        if (tr && tr->xs && k <= tr->cap_iters) memcpy(tr->xs + k * n, x, (size_t)n * sizeof(double));
        if (stop_test(o->stop_rule, o->tol, rel, nrm)) {
            status = 0;
            break;
        }
        if (k >= o->max_iter) {
            status = 1;
            break;
        }
        const int lock = tr && tr->lock_counts && k < tr->lock_iters;
        /* inner tolerance of this iteration: fixed, or tied to how far x_k is
           from the stopping rule (looser block solves while far away) */
        double itol = o->inner_tol;
        if (o->inner_adapt > 0.0) {
            const double rk = o->stop_rule == 1 ? rel : (o->stop_rule == 3 ? rel * rel : nrm);
            double a = o->inner_adapt * rk;
            if (a > 0.1) a = 0.1;
            if (a > itol) itol = a;
        }

        /* column step: eps^z_j = (A_j^T z_k)^2 / ||A_j||^2, sample U_k,
           z_{k+1} = z_k - A_U A_U^+ z_k */
        orc_spmv_t(m, n, rp, ci, av, z, g);
        int nan = 0;
        double emax = orc_weights(n, g, cn2, epsz, &nan);
        if (nan) {
            status = -2;
            break;
        }
        int64_t nu;
        if (lock) {
            nu = tr->lock_counts[2 * k];
            memcpy(U, tr->lock_lists + list_len, (size_t)nu * sizeof(int32_t));
        } else if (o->selection == 1) {
            nu = orc_select_greedy(n, epsz, emax, o->eta_col, U);
        } else {
            nu = orc_sample(n, epsz, emax, orc_num_draws(o->eta_col, n), o->seed, o->sysid,
                            (uint64_t)k, 0, U);
        }
        int steps_u = 0;
        if (nu > 0) {
            /* The least-squares problem min ||A_U y - z_k|| is solved by LSQR
               on B = A_U D with D = diag(1 / ||A_j||) (unit columns), then
               y = D y^.  Every least-squares solution gives the same A_U y,
               the projection of z_k onto range(A_U), so the scaling changes
               only the path of the inner solver, not z_{k+1}.  A selected
               column has a positive weight, hence a positive norm. */
            extract_columns(m, n, rp, ci, av, nu, U, srp, sci, sav);
            for (int64_t p = 0; p < nu; ++p) dcol[p] = 1.0 / sqrt(cn2[U[p]]);
            for (int64_t e = 0; e < srp[m]; ++e) bsc[e] = sav[e] * dcol[sci[e]];
            steps_u = orc_lsqr(m, nu, srp, sci, bsc, z, itol, sqrt((double)nu),
                               o->inner_max, y);
            for (int64_t p = 0; p < nu; ++p) y[p] *= dcol[p];
            orc_spmv(m, srp, sci, sav, y, Ax); /* A_U y */
            for (int64_t i = 0; i < m; ++i) z[i] -= Ax[i];
        }

        /* row step: r = b - z_{k+1} - A x_k, eps^x_i = r_i^2/||A^(i)||^2,
           sample J_k, x_{k+1} = x_k + (A^J)^+ r_J */
        orc_spmv(m, rp, ci, av, x, Ax);
        for (int64_t i = 0; i < m; ++i) r[i] = b[i] - z[i] - Ax[i];
        emax = orc_weights(m, r, rn2, epsx, &nan);
        if (nan) {
            status = -2;
            break;
        }
        int64_t nj;
        if (lock) {
            nj = tr->lock_counts[2 * k + 1];
            memcpy(J, tr->lock_lists + list_len + nu, (size_t)nj * sizeof(int32_t));
        } else if (o->selection == 1) {
            nj = orc_select_greedy(m, epsx, emax, o->eta_row, J);
        } else {
            nj = orc_sample(m, epsx, emax, orc_num_draws(o->eta_row, m), o->seed, o->sysid,
                            (uint64_t)k, 1, J);
        }
        int steps_j = 0;
        if (nj > 0) {
            /* (A^J)^+ r_J by LSQR.  When |J| <= n the block is first solved
               with its rows scaled to unit norm, D (A^J) d = D r_J with
               D = diag(1/||A^(i)||): if that system is consistent it has the
               same solutions as A^J d = r_J, so LSQR from 0 returns the same
               minimum-norm d.  Only when LSQR finds it inconsistent (it stops
               on the normal-equation test, not on the residual) is the block
               solved again unscaled, as (A^J)^+ r_J requires.  In exact
               arithmetic r lies in range(A) (b - z_{k+1} is a sum of
               projections onto it), so this happens at rounding level only.
               A selected row has a positive weight, hence a positive norm. */
            extract_rows(rp, ci, av, nj, J, srp, sci, sav);
            double fro2 = 0.0;
            for (int64_t p = 0; p < nj; ++p) {
                fro2 += rn2[J[p]];
                rJ[p] = r[J[p]];
            }
            int fit = 0;
            if (nj <= n) {
                for (int64_t p = 0; p < nj; ++p) {
                    const double dr = 1.0 / sqrt(rn2[J[p]]);
                    for (int64_t e = srp[p]; e < srp[p + 1]; ++e) bsc[e] = sav[e] * dr;
                    rJ[p] *= dr;
                }
                steps_j = orc_lsqr_fit(nj, n, srp, sci, bsc, rJ, itol,
                                       sqrt((double)nj), o->inner_max, d, &fit);
                if (fit == 0)
                    for (int64_t p = 0; p < nj; ++p) rJ[p] = r[J[p]];
            }
            if (nj > n || fit == 0)
                steps_j += orc_lsqr(nj, n, srp, sci, sav, rJ, itol, sqrt(fro2),
                                    o->inner_max, d);
            for (int64_t j = 0; j < n; ++j) x[j] += d[j];
        }
        st->inner_u += steps_u;
        st->inner_j += steps_j;

        if (tr) {
            if (k < tr->cap_iters) {
                tr->counts[4 * k + 0] = nu;
                tr->counts[4 * k + 1] = nj;
                tr->counts[4 * k + 2] = steps_u;
                tr->counts[4 * k + 3] = steps_j;
                n_rec = k + 1;
            }
            if (!lock && tr->lists && list_len + nu + nj <= tr->list_cap) {
                memcpy(tr->lists + list_len, U, (size_t)nu * sizeof(int32_t));
                memcpy(tr->lists + list_len + nu, J, (size_t)nj * sizeof(int32_t));
            }
        }
        list_len += nu + nj;

        if (nu == 0 && nj == 0) {
            /* both blocks empty: x_{k+1} = x_k and nothing can change any more */
            status = 0;
            break;
        }
    }
    if (tr) {
        tr->list_len = list_len;
        tr->n_iters = n_rec;
    }
    if (o->z_state)
        for (int64_t i = 0; i < m; ++i) o->z_state[i] = z[i];
    st->iters = k;
    st->rel_res = rel;
    st->normal_res = nrm;
    st->rse = rel * rel;
    st->status = status;

    free(rn2); free(cn2); free(z); free(t); free(r); free(Ax); free(g); free(h);
    free(epsz); free(epsx); free(y); free(d); free(rJ); free(U); free(J);
    free(srp); free(sci); free(sav); free(bsc); free(dcol);
    return status;
}
