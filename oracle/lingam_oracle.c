/*
 * lingam_oracle.c -- plain FP64 CPU oracle for DirectLiNGAM causal ordering.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference arm may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path, and the CUDA path
 * never calls it.
 *
 * What it computes (AcceleratedLiNGAM, arXiv 2403.03772):
 *   - Algorithm 1 ("search_causal_order"): for every ordered pair (i, j) of the
 *     remaining variables U, standardise x_i and x_j, form both least-squares
 *     residuals r_i^j = _residual(xi_std, xj_std) and r_j^i, evaluate
 *     _diff_mutual_info, accumulate min(0, .)^2 into k and return U[argmax(-k)].
 *   - Sec. 2.2 (DirectLiNGAM outer loop): append the chosen variable to the
 *     order and regress it out of every other remaining variable by least
 *     squares, then repeat on the residuals.
 *
 * Readings where the paper is silent (Algorithm 1 names _residual and
 * _diff_mutual_info but does not define them):
 *   - _residual(a, b) = a - (cov(a,b)/var(b)) * b with cov and var both
 *     normalised by 1/n, so the residual is exactly orthogonal to b.
 *   - _diff_mutual_info(xi, xj, ri_j, rj_i) =
 *         (H(xj) + H(ri_j)) - (H(xi) + H(rj_i)),
 *     the pairwise likelihood-ratio measure of Hyvarinen & Smith (2013), cited
 *     in Sec. 1; a positive value supports x_i -> x_j.
 *   - H(v) is the maximum-entropy approximation (Hyvarinen 1998) applied to v
 *     standardised by its own mean and standard deviation (ddof 0):
 *         H(v) = (1 + ln 2pi)/2 - K1 (E[log cosh u] - GAMMA)^2
 *                               - K2 (E[u exp(-u^2/2)])^2,
 *     K1 = 79.047, K2 = 7.4129, GAMMA = 0.37457 (constants of that literature,
 *     not of this paper).  log cosh u = |u| + log1p(exp(-2|u|)) - ln 2.
 *   - k_list is indexed by position in U; ties in argmax go to the first
 *     position, i.e. the smallest original index because U stays ascending.
 *   - Means and sums use pairwise (recursive halving) summation in FP64.
 *
 * Two modes of the per-step search, bitwise identical by construction:
 *   literal  -- Algorithm 1 exactly as written: every ordered pair recomputes
 *               both standardisations, both residuals and all four entropies.
 *   memoised -- computes each value that the literal mode would compute more
 *               than once only once: the standardised columns and their
 *               entropies per step, and for the unordered pair {a,b} the two
 *               residual entropies; I(b,a) is then Q - P where I(a,b) = P - Q,
 *               which is exactly the literal (H(xa)+H(rb_a)) - (H(xb)+H(ra_b)).
 *               The per-row accumulation of k runs over j in the same order.
 *
 * Build: cc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math), so
 * that no multiply-add is fused and x86-64 and aarch64 round alike.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_NONFINITE 2
#define ORACLE_ERR_DEGENERATE 3
#define ORACLE_ERR_NOMEM 5

static const double K1 = 79.047;
static const double K2 = 7.4129;
static const double GAMMA = 0.37457;
static const double LN2 = 0.69314718055994530942;
static const double TWO_PI = 6.28318530717958647692;

/* relative thresholds below which a variance counts as zero */
static const double DEGENERATE_REL = 1e-12;

/* ---------------------------------------------------------------- sums -- */

/* pairwise sum of v[0..n) */
static double psum(const double *v, int64_t n)
{
    if (n <= 8) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += v[i];
        return s;
    }
    int64_t h = n / 2;
    return psum(v, h) + psum(v + h, n - h);
}

double oracle_mean(const double *v, int64_t n) { return psum(v, n) / (double)n; }

/* population variance (ddof 0): mean((v - mean v)^2); tmp holds n doubles */
static double var_pop(const double *v, int64_t n, double *tmp)
{
    double mu = oracle_mean(v, n);
    for (int64_t s = 0; s < n; ++s) {
        double c = v[s] - mu;
        tmp[s] = c * c;
    }
    return psum(tmp, n) / (double)n;
}

/* population covariance (1/n) sum (a - mean a)(b - mean b) */
static double cov_pop(const double *a, const double *b, int64_t n, double *tmp)
{
    double ma = oracle_mean(a, n), mb = oracle_mean(b, n);
    for (int64_t s = 0; s < n; ++s) tmp[s] = (a[s] - ma) * (b[s] - mb);
    return psum(tmp, n) / (double)n;
}

/* ------------------------------------------------- Algorithm 1 helpers -- */

/* xi_std = (xi - mean(xi)) / std(xi), ddof 0 (Algorithm 1, standardisation). */
int oracle_standardize(const double *x, int64_t n, double *out, double *tmp)
{
    double mu = oracle_mean(x, n);
    double var = var_pop(x, n, tmp);
    if (!(var > 0.0) || !isfinite(var)) return ORACLE_ERR_DEGENERATE;
    double sd = sqrt(var);
    for (int64_t s = 0; s < n; ++s) out[s] = (x[s] - mu) / sd;
    return ORACLE_OK;
}

/* _residual(a, b) = a - (cov(a, b) / var(b)) * b  (least squares of a on b). */
int oracle_residual(const double *a, const double *b, int64_t n, double *out, double *tmp)
{
    double v = var_pop(b, n, tmp);
    if (!(v > 0.0)) return ORACLE_ERR_DEGENERATE;
    double c = cov_pop(a, b, n, tmp);
    double coef = c / v;
    for (int64_t s = 0; s < n; ++s) out[s] = a[s] - coef * b[s];
    return ORACLE_OK;
}

static double logcosh(double u)
{
    double a = fabs(u);
    return a + log1p(exp(-2.0 * a)) - LN2;
}

/* Moments of v standardised by its own mean and std (ddof 0):
 * m1 = E[log cosh u], m2 = E[u exp(-u^2/2)].  *var_out = var(v). */
int oracle_moments(const double *v, int64_t n, double *m1, double *m2, double *var_out,
                   double *tmp)
{
    double mu = oracle_mean(v, n);
    double var = var_pop(v, n, tmp);
    if (var_out) *var_out = var;
    if (!(var > 0.0) || !isfinite(var)) return ORACLE_ERR_DEGENERATE;
    double sd = sqrt(var);
    for (int64_t s = 0; s < n; ++s) tmp[s] = logcosh((v[s] - mu) / sd);
    *m1 = psum(tmp, n) / (double)n;
    for (int64_t s = 0; s < n; ++s) {
        double u = (v[s] - mu) / sd;
        tmp[s] = u * exp(-0.5 * u * u);
    }
    *m2 = psum(tmp, n) / (double)n;
    return ORACLE_OK;
}

/* Maximum-entropy approximation H(v) of a standardised copy of v. */
double oracle_entropy_from_moments(double m1, double m2)
{
    double a = m1 - GAMMA;
    return (1.0 + log(TWO_PI)) / 2.0 - K1 * a * a - K2 * m2 * m2;
}

int oracle_entropy(const double *v, int64_t n, double *H, double *tmp)
{
    double m1, m2;
    int st = oracle_moments(v, n, &m1, &m2, NULL, tmp);
    if (st) return st;
    *H = oracle_entropy_from_moments(m1, m2);
    return ORACLE_OK;
}

/* Entropy of a residual; a residual variance at or below DEGENERATE_REL of
 * its (unit-variance) inputs means |rho| = 1 within rounding. */
static int residual_entropy(const double *r, int64_t n, double *H, double *tmp)
{
    double m1, m2, var;
    int st = oracle_moments(r, n, &m1, &m2, &var, tmp);
    if (st) return st;
    if (var <= DEGENERATE_REL) return ORACLE_ERR_DEGENERATE;
    *H = oracle_entropy_from_moments(m1, m2);
    return ORACLE_OK;
}

/* _diff_mutual_info(xi_std, xj_std, ri_j, rj_i) =
 *     (H(xj_std) + H(ri_j)) - (H(xi_std) + H(rj_i)). */
int oracle_diff_mutual_info(const double *xi_std, const double *xj_std, const double *ri_j,
                            const double *rj_i, int64_t n, double *out, double *tmp)
{
    double hxi, hxj, hri, hrj;
    int st;
    if ((st = oracle_entropy(xj_std, n, &hxj, tmp))) return st;
    if ((st = residual_entropy(ri_j, n, &hri, tmp))) return st;
    if ((st = oracle_entropy(xi_std, n, &hxi, tmp))) return st;
    if ((st = residual_entropy(rj_i, n, &hrj, tmp))) return st;
    *out = (hxj + hri) - (hxi + hrj);
    return ORACLE_OK;
}

/* first maximum */
int oracle_argmax_first(const double *v, int64_t p)
{
    int best = 0;
    for (int64_t a = 1; a < p; ++a)
        if (v[a] > v[best]) best = (int)a;
    return best;
}

/* ------------------------------------------------ one ordering step ------ */

/*
 * One call of Algorithm 1 on the current residual data.
 *   R      column-major FP64 data: variable i is R[i*ldr .. i*ldr+n).
 *   U      p original indices (ascending), ref_var[i] = variance of the
 *          original variable i (degeneracy reference), may be NULL.
 *   k_list out [p]: k_list[a] = -sum_{b != a} min(0, I(U[a], U[b]))^2.
 *   I_out  optional [p*p] row-major I(U[a], U[b]) (diagonal 0).
 *   Hz_out optional [p]  H(xi_std) per position.
 *   m_pos  out: argmax position.
 */
int oracle_search_step(const double *R, int64_t n, int64_t ldr, const int32_t *U, int64_t p,
                       const double *ref_var, int literal, int nthreads, double *k_list,
                       double *I_out, double *Hz_out, int *m_pos)
{
    if (n < 2 || p < 1 || ldr < n || !U || !k_list) return ORACLE_ERR_ARG;
    if (nthreads < 1) nthreads = 1;
    int status = ORACLE_OK;

    /* column degeneracy against the original variance */
    for (int64_t a = 0; a < p; ++a) {
        double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
        if (!tmp) return ORACLE_ERR_NOMEM;
        double v = var_pop(R + (int64_t)U[a] * ldr, n, tmp);
        free(tmp);
        double ref = ref_var ? ref_var[U[a]] : 1.0;
        if (!isfinite(v)) return ORACLE_ERR_NONFINITE;
        if (!(v > DEGENERATE_REL * ref)) return ORACLE_ERR_DEGENERATE;
    }
    if (p == 1) {
        k_list[0] = -0.0;
        if (I_out) I_out[0] = 0.0;
        if (m_pos) *m_pos = 0;
        if (Hz_out) {
            double *xs = (double *)malloc(sizeof(double) * (size_t)n * 2);
            if (!xs) return ORACLE_ERR_NOMEM;
            int st = oracle_standardize(R + (int64_t)U[0] * ldr, n, xs, xs + n);
            if (!st) st = oracle_entropy(xs, n, &Hz_out[0], xs + n);
            free(xs);
            if (st) return st;
        }
        return ORACLE_OK;
    }

    double *I = (double *)calloc((size_t)(p * p), sizeof(double));
    if (!I) return ORACLE_ERR_NOMEM;

    if (literal) {
        /* Algorithm 1 as written: every ordered pair from scratch. */
#pragma omp parallel num_threads(nthreads)
        {
            double *buf = (double *)malloc(sizeof(double) * (size_t)n * 5);
            int local = buf ? ORACLE_OK : ORACLE_ERR_NOMEM;
#pragma omp for schedule(dynamic, 1)
            for (int64_t a = 0; a < p; ++a) {
                if (local) continue;
                for (int64_t b = 0; b < p; ++b) {
                    if (a == b || local) continue;
                    double *xi_std = buf, *xj_std = buf + n, *ri_j = buf + 2 * n,
                           *rj_i = buf + 3 * n, *tmp = buf + 4 * n;
                    const double *xi = R + (int64_t)U[a] * ldr, *xj = R + (int64_t)U[b] * ldr;
                    double mi;
                    if ((local = oracle_standardize(xi, n, xi_std, tmp))) break;
                    if ((local = oracle_standardize(xj, n, xj_std, tmp))) break;
                    if ((local = oracle_residual(xi_std, xj_std, n, ri_j, tmp))) break;
                    if ((local = oracle_residual(xj_std, xi_std, n, rj_i, tmp))) break;
                    if ((local = oracle_diff_mutual_info(xi_std, xj_std, ri_j, rj_i, n, &mi, tmp)))
                        break;
                    I[a * p + b] = mi;
                }
            }
            free(buf);
#pragma omp critical
            if (local && !status) status = local;
        }
        if (Hz_out && !status) {
            double *xs = (double *)malloc(sizeof(double) * (size_t)n * 2);
            if (!xs) status = ORACLE_ERR_NOMEM;
            for (int64_t a = 0; a < p && !status; ++a) {
                status = oracle_standardize(R + (int64_t)U[a] * ldr, n, xs, xs + n);
                if (!status) status = oracle_entropy(xs, n, &Hz_out[a], xs + n);
            }
            free(xs);
        }
    } else {
        /* Memoised: standardised columns and their entropies once per step. */
        double *Z = (double *)malloc(sizeof(double) * (size_t)(n * p));
        double *Hz = (double *)malloc(sizeof(double) * (size_t)p);
        if (!Z || !Hz) {
            free(Z); free(Hz); free(I);
            return ORACLE_ERR_NOMEM;
        }
#pragma omp parallel num_threads(nthreads)
        {
            double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
            int local = tmp ? ORACLE_OK : ORACLE_ERR_NOMEM;
#pragma omp for schedule(dynamic, 1)
            for (int64_t a = 0; a < p; ++a) {
                if (local) continue;
                local = oracle_standardize(R + (int64_t)U[a] * ldr, n, Z + a * n, tmp);
                if (!local) local = oracle_entropy(Z + a * n, n, &Hz[a], tmp);
            }
            free(tmp);
#pragma omp critical
            if (local && !status) status = local;
        }
        if (!status) {
            int64_t npairs = p * (p - 1) / 2;
#pragma omp parallel num_threads(nthreads)
            {
                double *buf = (double *)malloc(sizeof(double) * (size_t)n * 3);
                int local = buf ? ORACLE_OK : ORACLE_ERR_NOMEM;
#pragma omp for schedule(dynamic, 16)
                for (int64_t q = 0; q < npairs; ++q) {
                    if (local) continue;
                    /* unordered pair index q -> (a, b), a < b */
                    int64_t a = 0, rem = q;
                    while (rem >= p - 1 - a) { rem -= p - 1 - a; ++a; }
                    int64_t b = a + 1 + rem;
                    double *ra_b = buf, *rb_a = buf + n, *tmp = buf + 2 * n;
                    double hra, hrb;
                    /* Algorithm 1 for i = U[a], j = U[b]: ri_j, rj_i */
                    if ((local = oracle_residual(Z + a * n, Z + b * n, n, ra_b, tmp))) continue;
                    if ((local = oracle_residual(Z + b * n, Z + a * n, n, rb_a, tmp))) continue;
                    if ((local = residual_entropy(ra_b, n, &hra, tmp))) continue;
                    if ((local = residual_entropy(rb_a, n, &hrb, tmp))) continue;
                    double P = Hz[b] + hra;   /* H(xj_std) + H(ri_j) for (a,b) */
                    double Q = Hz[a] + hrb;   /* H(xi_std) + H(rj_i) for (a,b) */
                    I[a * p + b] = P - Q;
                    I[b * p + a] = Q - P;
                }
                free(buf);
#pragma omp critical
                if (local && !status) status = local;
            }
        }
        if (Hz_out && !status) memcpy(Hz_out, Hz, sizeof(double) * (size_t)p);
        free(Z);
        free(Hz);
    }

    if (!status) {
        for (int64_t a = 0; a < p; ++a) {
            double k = 0.0;
            for (int64_t b = 0; b < p; ++b) {
                if (a == b) continue;
                double v = fmin(0.0, I[a * p + b]);
                k += v * v;
            }
            k_list[a] = -k;
        }
        if (I_out) memcpy(I_out, I, sizeof(double) * (size_t)(p * p));
        if (m_pos) *m_pos = oracle_argmax_first(k_list, p);
    }
    free(I);
    return status;
}

/*
 * Algorithm 1's k_list restricted to the positions rows[0..nrows): for each
 * such i, the literal inner loop over every j in U.  Same helper calls in the
 * same order as the literal mode of oracle_search_step, so each value equals
 * the corresponding k_list entry bitwise.  Used to check sampled rows of a
 * step that is too large to score in full on the CPU.
 */
int oracle_row_scores(const double *R, int64_t n, int64_t ldr, const int32_t *U, int64_t p,
                      const int32_t *rows, int64_t nrows, int nthreads, double *k_out)
{
    if (n < 2 || p < 2 || ldr < n || !U || !rows || !k_out) return ORACLE_ERR_ARG;
    if (nthreads < 1) nthreads = 1;
    int status = ORACLE_OK;
#pragma omp parallel num_threads(nthreads)
    {
        double *buf = (double *)malloc(sizeof(double) * (size_t)n * 5);
        int local = buf ? ORACLE_OK : ORACLE_ERR_NOMEM;
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            if (local) continue;
            const int64_t a = rows[r];
            if (a < 0 || a >= p) { local = ORACLE_ERR_ARG; continue; }
            double k = 0.0;
            for (int64_t b = 0; b < p; ++b) {
                if (a == b || local) continue;
                double *xi_std = buf, *xj_std = buf + n, *ri_j = buf + 2 * n,
                       *rj_i = buf + 3 * n, *tmp = buf + 4 * n;
                const double *xi = R + (int64_t)U[a] * ldr, *xj = R + (int64_t)U[b] * ldr;
                double mi;
                if ((local = oracle_standardize(xi, n, xi_std, tmp))) break;
                if ((local = oracle_standardize(xj, n, xj_std, tmp))) break;
                if ((local = oracle_residual(xi_std, xj_std, n, ri_j, tmp))) break;
                if ((local = oracle_residual(xj_std, xi_std, n, rj_i, tmp))) break;
                if ((local = oracle_diff_mutual_info(xi_std, xj_std, ri_j, rj_i, n, &mi, tmp)))
                    break;
                double v = fmin(0.0, mi);
                k += v * v;
            }
            k_out[r] = -k;
        }
        free(buf);
#pragma omp critical
        if (local && !status) status = local;
    }
    return status;
}

/* ------------------------------------------------ DirectLiNGAM order ----- */

/*
 * Causal order of X (row-major FP64 [n][d], the paper's [m, dim] layout).
 *   order  out [d] original indices, first = most exogenous.
 *   scores optional out [d*d]: row t holds k_list of step t scattered to the
 *          original indices (NaN for variables already removed); the last row
 *          holds 0 for the single remaining variable.
 *   max_steps  if > 0, stop after that many search steps (order entries past
 *          them are -1); used to time a bounded sample of a run.
 */
/*
 * Prior knowledge of ancestry (not in the paper; the DirectLiNGAM literature
 * lets a user state known causal relations, and this is the reading used
 * here).  prior[i * d + j] = 1: x_j is known to be an ancestor of x_i (a
 * directed path j -> i); 0: x_j is known not to be an ancestor of x_i; -1:
 * unknown; the diagonal is ignored.  At each step, among the remaining
 * variables U:
 *   - i may be chosen only if no other remaining j is a known ancestor of it;
 *   - if some remaining i has every other remaining j known not to be an
 *     ancestor (known exogenous among U), the choice is restricted to those.
 * The scores k_list are computed as without prior knowledge; the argmax
 * (ties to the first position) runs over the allowed positions only.  No
 * allowed position (contradictory knowledge) is ORACLE_ERR_ARG.
 */
static int prior_allowed(const int8_t *prior, int64_t d, const int32_t *U, int64_t p,
                         unsigned char *allow)
{
    int any_exo = 0, any = 0;
    for (int64_t a = 0; a < p; ++a) {
        int anc = 0, exo = 1;
        for (int64_t b = 0; b < p; ++b) {
            if (b == a) continue;
            const int8_t v = prior[(int64_t)U[a] * d + U[b]];
            anc |= v == 1;
            exo &= v == 0;
        }
        allow[a] = (unsigned char)((anc ? 0 : 1) | (exo && !anc ? 2 : 0));
        any_exo |= (allow[a] & 2) != 0;
    }
    for (int64_t a = 0; a < p; ++a) {
        allow[a] = any_exo ? (allow[a] & 2) != 0 : (allow[a] & 1) != 0;
        any |= allow[a];
    }
    return any ? ORACLE_OK : ORACLE_ERR_ARG;
}

int oracle_causal_order_prior(const double *X, int64_t n, int64_t d, int literal, int nthreads,
                              const int8_t *prior, int32_t *order, double *scores,
                              int64_t max_steps);

int oracle_causal_order(const double *X, int64_t n, int64_t d, int literal, int nthreads,
                        int32_t *order, double *scores, int64_t max_steps)
{
    return oracle_causal_order_prior(X, n, d, literal, nthreads, NULL, order, scores, max_steps);
}

int oracle_causal_order_prior(const double *X, int64_t n, int64_t d, int literal, int nthreads,
                              const int8_t *prior, int32_t *order, double *scores,
                              int64_t max_steps)
{
    if (!X || !order || n < 2 || d < 1) return ORACLE_ERR_ARG;
    for (int64_t k = 0; k < n * d; ++k)
        if (!isfinite(X[k])) return ORACLE_ERR_NONFINITE;

    double *R = (double *)malloc(sizeof(double) * (size_t)(n * d));
    int32_t *U = (int32_t *)malloc(sizeof(int32_t) * (size_t)d);
    double *kl = (double *)malloc(sizeof(double) * (size_t)d);
    double *ref = (double *)malloc(sizeof(double) * (size_t)d);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n * 2);
    unsigned char *allow = (unsigned char *)malloc((size_t)d);
    if (!R || !U || !kl || !ref || !tmp || !allow) {
        free(R); free(U); free(kl); free(ref); free(tmp); free(allow);
        return ORACLE_ERR_NOMEM;
    }
    for (int64_t i = 0; i < d; ++i) {
        for (int64_t s = 0; s < n; ++s) R[i * n + s] = X[s * d + i];
        U[i] = (int32_t)i;
        ref[i] = var_pop(R + i * n, n, tmp);
        order[i] = -1;
    }
    if (scores)
        for (int64_t k = 0; k < d * d; ++k) scores[k] = NAN;

    int status = ORACLE_OK;
    int64_t p = d, t = 0;
    while (p > 1 && status == ORACLE_OK) {
        if (max_steps > 0 && t >= max_steps) break;
        int mpos = 0;
        status = oracle_search_step(R, n, n, U, p, ref, literal, nthreads, kl, NULL, NULL, &mpos);
        if (status) break;
        if (prior) {
            status = prior_allowed(prior, d, U, p, allow);
            if (status) break;
            mpos = -1;
            for (int64_t a = 0; a < p; ++a)
                if (allow[a] && (mpos < 0 || kl[a] > kl[mpos])) mpos = (int)a;
        }
        if (scores)
            for (int64_t a = 0; a < p; ++a) scores[t * d + U[a]] = kl[a];
        int32_t m = U[mpos];
        order[t] = m;
        /* Sec. 2.2: regress the chosen variable out of the others. */
        double *rm = R + (int64_t)m * n;
        for (int64_t a = 0; a < p && !status; ++a) {
            if (a == mpos) continue;
            double *ri = R + (int64_t)U[a] * n;
            status = oracle_residual(ri, rm, n, tmp, tmp + n);
            if (!status) memcpy(ri, tmp, sizeof(double) * (size_t)n);
        }
        for (int64_t a = mpos; a + 1 < p; ++a) U[a] = U[a + 1];
        --p;
        ++t;
    }
    if (status == ORACLE_OK && p == 1) {
        order[t] = U[0];
        if (scores) scores[t * d + U[0]] = 0.0;
    }
    free(R); free(U); free(kl); free(ref); free(tmp); free(allow);
    return status;
}

/*
 * Sec. 2.2's regress-out step applied along a given order: R is column-major
 * [d][n] (variable i at R + i n), U[0..p) the remaining variables ascending.
 * For k = t0 .. t1-1 the variable order[k] is regressed out of every other
 * remaining variable with the same _residual helper and in the same sequence
 * as oracle_causal_order, then removed from U.  On return *p is the number of
 * remaining variables.  With `order` the oracle's own order, R and U then
 * equal its internal state at step t1 bitwise, so sampled scores of a late
 * step can be checked one row at a time.
 */
int oracle_regress_along(double *R, int64_t n, int64_t d, int32_t *U, int64_t *p,
                         const int32_t *order, int64_t t0, int64_t t1)
{
    if (!R || !U || !p || !order || n < 2 || *p < 1 || *p > d || t0 < 0 || t1 < t0)
        return ORACLE_ERR_ARG;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n * 2);
    if (!tmp) return ORACLE_ERR_NOMEM;
    int status = ORACLE_OK;
    for (int64_t k = t0; k < t1 && status == ORACLE_OK; ++k) {
        int64_t mpos = -1;
        for (int64_t a = 0; a < *p; ++a)
            if (U[a] == order[k]) mpos = a;
        if (mpos < 0) {
            status = ORACLE_ERR_ARG;
            break;
        }
        const double *rm = R + (int64_t)order[k] * n;
        for (int64_t a = 0; a < *p && !status; ++a) {
            if (a == mpos) continue;
            double *ri = R + (int64_t)U[a] * n;
            status = oracle_residual(ri, rm, n, tmp, tmp + n);
            if (!status) memcpy(ri, tmp, sizeof(double) * (size_t)n);
        }
        for (int64_t a = mpos; a + 1 < *p; ++a) U[a] = U[a + 1];
        --*p;
    }
    free(tmp);
    return status;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
