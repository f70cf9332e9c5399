/*
 * CPU oracle for the conditional draw of beta (test infrastructure only).
 *
 * This file is the plain, slow FP64 statement of what the CUDA path computes.
 * It exists so that the tests, the smoke check and the CPU-baseline leg of
 * the benchmark have an independent answer to compare with; the library
 * itself never calls it.  It shares no code, header or constant with the
 * CUDA sources.
 *
 * Paper: Nishimura & Suchard, "Prior-preconditioned conjugate gradient
 * method for accelerated Gibbs sampling in 'large n & large p' Bayesian
 * sparse regression".
 *
 *   target (Eq. 1.2):  beta | omega, lambda, tau ~ N(Phi^-1 X^T Omega z, Phi^-1),
 *                      Phi = X^T Omega X + tau^-2 Lambda^-2
 *   Prop. 2.1 / Eq. 2.3:  b = X^T Omega z + X^T Omega^1/2 eta + tau^-1 Lambda^-1 delta
 *   Eq. 2.4:              solve Phi beta = b
 *   Sec. 2.4:             preconditioner M = tau^-2 Lambda^-2, used only through
 *                         v -> M^-1 v = tau^2 lambda^2 (.) v
 *   Algorithm S1 (Sec. S2): the CG recursion, applied to the preconditioned
 *                         system in the standard PCG form
 *   Eq. S2 (Sec. S4.2):   stop when p^-1/2 || tau lambda (.) r ||_2 <= tol
 *
 * X is binary and is held as indices only: CSR (row_ptr int64[n+1],
 * col_idx int32[nnz]) and CSC (col_ptr int64[p+1], row_idx int32[nnz]).
 *
 * Readings of the paper taken here (each is also listed with the design
 * notes):
 *  - Algorithm S1 writes r = Phi beta - b but then updates beta += a s,
 *    r -= a v, which is only consistent with r = b - Phi beta; that sign is
 *    used.  The stop norm does not depend on the sign.
 *  - Preconditioned CG is written in the usual form with z = M^-1 r, which is
 *    CG on the system of Eq. 2.6 mapped back to beta (Sec. 2.4).
 *  - The iteration count k is the number of products v = Phi s (= number of
 *    beta updates); the stop test is evaluated before the first product.
 *  - Stop rules: RMS  sqrt(rho/p) <= tol  (Eq. S2, rho = ||tau lambda r||^2),
 *                RELATIVE sqrt(rho/rho_0) <= tol  (same norm, relative to b).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_STOP_RMS 0
#define ORACLE_STOP_RELATIVE 1

#define ORACLE_OK 0
#define ORACLE_MAXITER 1
#define ORACLE_BREAKDOWN 2
#define ORACLE_NONFINITE 3

/* out = X v, out_i = sum over the nonzeros of row i of v_j (CSR walk). */
void oracle_x_mul(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                  const double *v, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            acc += v[col_idx[k]];
        out[i] = acc;
    }
}

/* out = X^T w, out_j = sum over the nonzeros of column j of w_i (CSC walk). */
void oracle_xt_mul(int64_t p, const int64_t *col_ptr, const int32_t *row_idx,
                   const double *w, double *out)
{
    for (int64_t j = 0; j < p; ++j) {
        double acc = 0.0;
        for (int64_t k = col_ptr[j]; k < col_ptr[j + 1]; ++k)
            acc += w[row_idx[k]];
        out[j] = acc;
    }
}

/* Prior precision diagonal tau^-2 lambda_j^-2 (Eq. 1.2). */
static double prior_prec(double tau, double lam) { return 1.0 / (tau * tau * lam * lam); }

/* Preconditioner inverse M^-1 = tau^2 lambda_j^2 (Sec. 2.4). */
static double prior_var(double tau, double lam) { return tau * tau * lam * lam; }

/*
 * out = Phi v = X^T (Omega (X v)) + tau^-2 Lambda^-2 v, never forming Phi
 * (Sec. 1: the products v -> X v and w -> X^T w and elementwise work).
 * work: n doubles.
 */
void oracle_phi_mul(int64_t n, int64_t p,
                    const int64_t *row_ptr, const int32_t *col_idx,
                    const int64_t *col_ptr, const int32_t *row_idx,
                    const double *omega, const double *lam, double tau,
                    const double *v, double *out, double *work)
{
    oracle_x_mul(n, row_ptr, col_idx, v, work);
    for (int64_t i = 0; i < n; ++i)
        work[i] = omega[i] * work[i];
    oracle_xt_mul(p, col_ptr, row_idx, work, out);
    for (int64_t j = 0; j < p; ++j)
        out[j] = out[j] + prior_prec(tau, lam[j]) * v[j];
}

/*
 * Right-hand side of Prop. 2.1, Eq. 2.3, term by term:
 *   b = X^T (Omega z) + X^T (Omega^1/2 eta) + tau^-1 Lambda^-1 delta.
 * work: n + p doubles.
 */
void oracle_build_b(int64_t n, int64_t p,
                    const int64_t *col_ptr, const int32_t *row_idx,
                    const double *omega, const double *z, const double *lam, double tau,
                    const double *eta, const double *delta, double *b, double *work)
{
    double *w = work;          /* n */
    double *t = work + n;      /* p */
    /* first term: X^T Omega z */
    for (int64_t i = 0; i < n; ++i)
        w[i] = omega[i] * z[i];
    oracle_xt_mul(p, col_ptr, row_idx, w, b);
    /* second term: X^T Omega^1/2 eta */
    for (int64_t i = 0; i < n; ++i)
        w[i] = sqrt(omega[i]) * eta[i];
    oracle_xt_mul(p, col_ptr, row_idx, w, t);
    for (int64_t j = 0; j < p; ++j)
        b[j] = b[j] + t[j];
    /* third term: tau^-1 Lambda^-1 delta */
    for (int64_t j = 0; j < p; ++j)
        b[j] = b[j] + delta[j] / (tau * lam[j]);
}

/*
 * Compensated summation (Neumaier 1974, the Kahan-Babuska scheme): the
 * running sum `s` and, in `c`, the rounding error of every addition, which is
 * added back at the end.  Used by the ORACLE_SUM_COMPENSATED mode, whose
 * sums are the same sums as the plain ones, accumulated more accurately.
 */
typedef struct { double s, c; } comp_sum;

static void comp_add(comp_sum *a, double x)
{
    const double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double comp_value(const comp_sum *a) { return a->s + a->c; }

/* X v with each row sum accumulated by compensated summation. */
void oracle_x_mul_comp(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       const double *v, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        comp_sum acc = {0.0, 0.0};
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            comp_add(&acc, v[col_idx[k]]);
        out[i] = comp_value(&acc);
    }
}

/* X^T w with each column sum accumulated by compensated summation. */
void oracle_xt_mul_comp(int64_t p, const int64_t *col_ptr, const int32_t *row_idx,
                        const double *w, double *out)
{
    for (int64_t j = 0; j < p; ++j) {
        comp_sum acc = {0.0, 0.0};
        for (int64_t k = col_ptr[j]; k < col_ptr[j + 1]; ++k)
            comp_add(&acc, w[row_idx[k]]);
        out[j] = comp_value(&acc);
    }
}

/* a . b: the rounded products a_j b_j summed by compensated summation. */
double oracle_dot_comp(int64_t p, const double *a, const double *b)
{
    comp_sum acc = {0.0, 0.0};
    for (int64_t j = 0; j < p; ++j)
        comp_add(&acc, a[j] * b[j]);
    return comp_value(&acc);
}

static double dot(int64_t p, const double *a, const double *b)
{
    double acc = 0.0;
    for (int64_t j = 0; j < p; ++j)
        acc += a[j] * b[j];
    return acc;
}

#define ORACLE_SUM_PLAIN 0        /* every sum accumulated left to right, as written above */
#define ORACLE_SUM_COMPENSATED 1  /* products' and dot products' sums compensated */
#define ORACLE_SUM_FLOAT32 2      /* products' sums accumulated left to right in float32,
                                     dot products compensated in float64 */

static double dot_mode(int sum_mode, int64_t p, const double *a, const double *b)
{
    return sum_mode == ORACLE_SUM_PLAIN ? dot(p, a, b) : oracle_dot_comp(p, a, b);
}

/* X v with each row sum accumulated left to right in float32. */
void oracle_x_mul_f32(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                      const double *v, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        float acc = 0.0f;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            acc = acc + (float)v[col_idx[k]];
        out[i] = (double)acc;
    }
}

/* X^T w with each column sum accumulated left to right in float32. */
void oracle_xt_mul_f32(int64_t p, const int64_t *col_ptr, const int32_t *row_idx,
                       const double *w, double *out)
{
    for (int64_t j = 0; j < p; ++j) {
        float acc = 0.0f;
        for (int64_t k = col_ptr[j]; k < col_ptr[j + 1]; ++k)
            acc = acc + (float)w[row_idx[k]];
        out[j] = (double)acc;
    }
}

/* Storage formats of the products' operands (ORACLE_VEC_*): float64 as is,
 * a pair of float32 (hi = float32(x), lo = float32(x - hi), value hi + lo,
 * about 48 significant bits), or one float32. */
#define ORACLE_VEC_F64 0
#define ORACLE_VEC_F32X2 1
#define ORACLE_VEC_F32 2

static double stored(int vec, double x)
{
    if (vec == ORACLE_VEC_F32X2) {
        const float hi = (float)x;
        const float lo = (float)(x - (double)hi);
        return (double)hi + (double)lo;
    }
    if (vec == ORACLE_VEC_F32)
        return (double)(float)x;
    return x;
}

/*
 * Phi v as oracle_phi_mul, with the products' sums in the given mode and
 * their operands and results held in the given storage format:
 *   u = stored(stored(omega) * stored(X stored(v)));  out = stored(X^T u) + d v
 * (the diagonal term and the output in float64).  work: n doubles.
 */
static void phi_mul_mode(int sum_mode, int vec, int64_t n, int64_t p,
                         const int64_t *row_ptr, const int32_t *col_idx,
                         const int64_t *col_ptr, const int32_t *row_idx,
                         const double *omega, const double *lam, double tau,
                         const double *v, double *out, double *work)
{
    if (sum_mode != ORACLE_SUM_COMPENSATED && vec == ORACLE_VEC_F64) {
        oracle_phi_mul(n, p, row_ptr, col_idx, col_ptr, row_idx, omega, lam, tau, v, out, work);
        return;
    }
    const double *vs = v;
    double *vr = NULL;
    if (vec != ORACLE_VEC_F64) {
        vr = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
        for (int64_t j = 0; j < p; ++j)
            vr[j] = stored(vec, v[j]);
        vs = vr;
    }
    if (sum_mode == ORACLE_SUM_COMPENSATED)
        oracle_x_mul_comp(n, row_ptr, col_idx, vs, work);
    else if (sum_mode == ORACLE_SUM_FLOAT32)
        oracle_x_mul_f32(n, row_ptr, col_idx, vs, work);
    else
        oracle_x_mul(n, row_ptr, col_idx, vs, work);
    for (int64_t i = 0; i < n; ++i)
        work[i] = stored(vec, stored(vec, work[i]) * stored(vec, omega[i]));
    if (sum_mode == ORACLE_SUM_COMPENSATED)
        oracle_xt_mul_comp(p, col_ptr, row_idx, work, out);
    else if (sum_mode == ORACLE_SUM_FLOAT32)
        oracle_xt_mul_f32(p, col_ptr, row_idx, work, out);
    else
        oracle_xt_mul(p, col_ptr, row_idx, work, out);
    for (int64_t j = 0; j < p; ++j)
        out[j] = stored(vec, out[j]) + v[j] * prior_prec(tau, lam[j]);
    free(vr);
}

/*
 * Diagonal of Phi, the Jacobi preconditioner M = diag(Phi_11 .. Phi_pp)
 * (Sec. 2.4): for binary X, Phi_jj = sum over the rows i of column j of
 * omega_i, plus tau^-2 lambda_j^-2.
 */
void oracle_phi_diag(int64_t p, const int64_t *col_ptr, const int32_t *row_idx,
                     const double *omega, const double *lam, double tau, double *out)
{
    oracle_xt_mul(p, col_ptr, row_idx, omega, out);
    for (int64_t j = 0; j < p; ++j)
        out[j] = out[j] + prior_prec(tau, lam[j]);
}

static int stop_met(int rule, double rho, double rho0, int64_t p, double tol)
{
    if (rule == ORACLE_STOP_RELATIVE)
        return rho0 > 0.0 ? sqrt(rho / rho0) <= tol : 1;
    return sqrt(rho / (double)p) <= tol;
}

static double resid_of(int rule, double rho, double rho0, int64_t p)
{
    if (rule == ORACLE_STOP_RELATIVE)
        return rho0 > 0.0 ? sqrt(rho / rho0) : 0.0;
    return sqrt(rho / (double)p);
}

/* ||tau lambda (.) r||^2 = r . (tau^2 lambda^2 r), the squared norm of the
 * prior-preconditioned residual that Eq. S2 tests. */
static double stop_norm2(int sum_mode, int64_t p, const double *r, const double *lam, double tau,
                         double *tmp)
{
    for (int64_t j = 0; j < p; ++j)
        tmp[j] = prior_var(tau, lam[j]) * r[j];
    return dot_mode(sum_mode, p, r, tmp);
}

/*
 * Preconditioned CG on Phi beta = b (Algorithm S1 in PCG form), general
 * form:
 *   minv   NULL: the prior preconditioner, M^-1 = tau^2 Lambda^2 (Sec. 2.4);
 *          else the diagonal M^-1 to use (the Jacobi preconditioner of
 *          Sec. 2.4 passes 1 / diag(Phi)).
 *   beta0  NULL: beta_0 = 0 (Sec. 2.7); else the initial vector (Sec. S4.1),
 *          with r_0 = b - Phi beta_0.
 *   sum_mode  ORACLE_SUM_PLAIN or ORACLE_SUM_COMPENSATED for every sum of
 *          the products and dot products; ORACLE_SUM_FLOAT32 accumulates the
 *          products' sums in float32 (left to right) and the dot products
 *          compensated.
 *   vec    ORACLE_VEC_F64, or the storage format (ORACLE_VEC_F32X2,
 *          ORACLE_VEC_F32) in which the products' operands and results are
 *          held (phi_mul_mode); every other quantity stays float64.
 * The stop rule always tests the prior-preconditioned residual of Eq. S2,
 * rho_s = ||tau lambda (.) r||^2: sqrt(rho_s / p) <= tol (RMS), or
 * sqrt(rho_s / rho_b) <= tol (RELATIVE, rho_b = ||tau lambda (.) b||^2, the
 * value at beta = 0, so a warm start does not move the target).  With the
 * prior preconditioner rho_s is the CG's own rho = r.z.
 *
 *   r = b - Phi beta0; z = M^-1 r; s = z; rho = r.z
 *   repeat: v = Phi s; alpha = rho / (s.v)
 *           beta += alpha s; r -= alpha v; z = M^-1 r; rho' = r.z; k += 1
 *           stop on rho_s (Eq. S2) or k == max_iter
 *           s = z + (rho'/rho) s; rho = rho'
 *
 * fixed_iters > 0 runs exactly that many iterations without testing the
 * stop rule (for same-k comparisons); fixed_iters == 0 uses tol/max_iter.
 * rho_hist (optional, max(max_iter, fixed_iters) + 1 doubles) receives rho_s
 * before the first product and after each product.
 * Returns ORACLE_OK, ORACLE_MAXITER, ORACLE_BREAKDOWN (s.v <= 0 or rho <= 0)
 * or ORACLE_NONFINITE (a NaN or infinite CG scalar).
 */
int oracle_pcg_ex(int64_t n, int64_t p,
                  const int64_t *row_ptr, const int32_t *col_idx,
                  const int64_t *col_ptr, const int32_t *row_idx,
                  const double *omega, const double *lam, double tau,
                  const double *b, const double *minv, const double *beta0,
                  double tol, int stop_rule, int max_iter, int fixed_iters, int sum_mode,
                  int vec, double *beta, int *iters, double *resid, double *rho_hist)
{
    const size_t np = (size_t)(p > 0 ? p : 1);
    double *r = (double *)malloc(sizeof(double) * np);
    double *z = (double *)malloc(sizeof(double) * np);
    double *s = (double *)malloc(sizeof(double) * np);
    double *v = (double *)malloc(sizeof(double) * np);
    double *tmp = (double *)malloc(sizeof(double) * np);
    double *work = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int status = ORACLE_OK;
    int k = 0;

    if (beta0) {
        phi_mul_mode(sum_mode, ORACLE_VEC_F64, n, p, row_ptr, col_idx, col_ptr, row_idx, omega,
                     lam, tau, beta0, v, work);
        for (int64_t j = 0; j < p; ++j) {
            beta[j] = beta0[j];
            r[j] = b[j] - v[j];            /* r_0 = b - Phi beta_0 */
        }
    } else {
        for (int64_t j = 0; j < p; ++j) {
            beta[j] = 0.0;
            r[j] = b[j];                   /* r_0 = b - Phi beta_0 = b */
        }
    }
    for (int64_t j = 0; j < p; ++j) {
        z[j] = minv ? minv[j] * r[j] : prior_var(tau, lam[j]) * r[j];
        s[j] = z[j];
    }
    double rho = dot_mode(sum_mode, p, r, z);
    /* the stop quantity: rho itself under the prior preconditioner */
    double rho_s = (minv == NULL) ? rho : stop_norm2(sum_mode, p, r, lam, tau, tmp);
    const double rho_b = (beta0 == NULL) ? rho_s : stop_norm2(sum_mode, p, b, lam, tau, tmp);
    if (rho_hist) rho_hist[0] = rho_s;

    if (!isfinite(rho) || !isfinite(rho_s)) {
        status = ORACLE_NONFINITE;
    } else if (fixed_iters > 0 || !stop_met(stop_rule, rho_s, rho_b, p, tol)) {
        int limit = fixed_iters > 0 ? fixed_iters : max_iter;
        if (limit <= 0) status = ORACLE_MAXITER;
        while (k < limit) {
            phi_mul_mode(sum_mode, vec, n, p, row_ptr, col_idx, col_ptr, row_idx, omega, lam, tau,
                         s, v, work);
            double sigma = dot_mode(sum_mode, p, s, v);
            if (!isfinite(sigma)) { status = ORACLE_NONFINITE; break; }
            if (sigma <= 0.0 || rho <= 0.0) { status = ORACLE_BREAKDOWN; break; }
            double alpha = rho / sigma;
            for (int64_t j = 0; j < p; ++j) {
                beta[j] = beta[j] + alpha * s[j];
                r[j] = r[j] - alpha * v[j];
                z[j] = minv ? minv[j] * r[j] : prior_var(tau, lam[j]) * r[j];
            }
            double rho_new = dot_mode(sum_mode, p, r, z);
            rho_s = (minv == NULL) ? rho_new : stop_norm2(sum_mode, p, r, lam, tau, tmp);
            k += 1;
            if (rho_hist) rho_hist[k] = rho_s;
            if (!isfinite(rho_new) || !isfinite(rho_s)) { status = ORACLE_NONFINITE; break; }
            if (fixed_iters == 0) {
                if (stop_met(stop_rule, rho_s, rho_b, p, tol)) break;
                if (k == max_iter) { status = ORACLE_MAXITER; break; }
            }
            double gamma = rho_new / rho;
            for (int64_t j = 0; j < p; ++j)
                s[j] = z[j] + gamma * s[j];
            rho = rho_new;
        }
    }
    *iters = k;
    *resid = resid_of(stop_rule, rho_s, rho_b, p);
    free(r); free(z); free(s); free(v); free(tmp); free(work);
    return status;
}

/*
 * Prior-preconditioned CG from beta_0 = 0 with plain sums: oracle_pcg_ex
 * with minv = NULL, beta0 = NULL and ORACLE_SUM_PLAIN.
 */
int oracle_pcg(int64_t n, int64_t p,
               const int64_t *row_ptr, const int32_t *col_idx,
               const int64_t *col_ptr, const int32_t *row_idx,
               const double *omega, const double *lam, double tau,
               const double *b, double tol, int stop_rule, int max_iter, int fixed_iters,
               double *beta, int *iters, double *resid, double *rho_hist)
{
    return oracle_pcg_ex(n, p, row_ptr, col_idx, col_ptr, row_idx, omega, lam, tau, b, NULL, NULL,
                         tol, stop_rule, max_iter, fixed_iters, ORACLE_SUM_PLAIN, ORACLE_VEC_F64,
                         beta, iters, resid, rho_hist);
}

/* X v and X^T w with the sums of a summation mode (plain or compensated). */
static void x_mode(int sum_mode, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                   const double *v, double *out)
{
    if (sum_mode == ORACLE_SUM_COMPENSATED) oracle_x_mul_comp(n, row_ptr, col_idx, v, out);
    else oracle_x_mul(n, row_ptr, col_idx, v, out);
}

static void xt_mode(int sum_mode, int64_t p, const int64_t *col_ptr, const int32_t *row_idx,
                    const double *w, double *out)
{
    if (sum_mode == ORACLE_SUM_COMPENSATED) oracle_xt_mul_comp(p, col_ptr, row_idx, w, out);
    else oracle_xt_mul(p, col_ptr, row_idx, w, out);
}

/*
 * LSQR (Paige and Saunders 1982) on the least-squares form of Eq. 2.4 (Sec.
 * S7.1, Eq. S6): Phi = Xt^T Xt with Xt = [Omega^1/2 X; tau^-1 Lambda^-1] and
 * Phi beta = Xt^T bt for bt = [Omega^1/2 z + eta; delta], so beta minimises
 * ||Xt beta - bt||.  LSQR runs on A = Xt D with D = diag(tau lambda) (the
 * prior preconditioner applied on the right, Sec. 2.4), A = [Omega^1/2 X D; I],
 * for x = D^-1 beta:
 *
 *   beta_1 u_1 = bt;  alpha_1 v_1 = A^T u_1;  w = v_1;  x = 0;
 *   phibar = beta_1;  rhobar = alpha_1
 *   repeat (k = 1, 2, ...):
 *     beta_{k+1} u_{k+1} = A v_k - alpha_k u_k
 *     alpha_{k+1} v_{k+1} = A^T u_{k+1} - beta_{k+1} v_k
 *     rho = sqrt(rhobar^2 + beta_{k+1}^2); c = rhobar / rho; s = beta_{k+1} / rho
 *     theta = s alpha_{k+1}; rhobar = -c alpha_{k+1}; phi = c phibar; phibar = s phibar
 *     x += (phi / rho) w;  w = v_{k+1} - (theta / rho) w
 *     stop on ||A^T r_k|| = phibar alpha_{k+1} |c|
 *
 * A^T (bt - A x) = D (b - Phi beta) = tau lambda (.) r, the prior-
 * preconditioned residual of Eq. S2, so the stop rules are those of PCG:
 * sqrt(||A^T r||^2 / p) <= tol (RMS) or ||A^T r|| / ||A^T bt|| <= tol
 * (RELATIVE; ||A^T bt|| = alpha_1 beta_1 = ||tau lambda (.) b||).  The
 * iteration count is the number of x updates (one product with A and one
 * with A^T each).  beta = D x on return.  Returns ORACLE_OK, ORACLE_MAXITER
 * or ORACLE_NONFINITE (ORACLE_BREAKDOWN when alpha_1 or beta_1 is not
 * positive while the stop rule is unmet).  sum_mode: ORACLE_SUM_PLAIN or
 * ORACLE_SUM_COMPENSATED for the products' sums and the norms.
 */
int oracle_lsqr(int64_t n, int64_t p,
                const int64_t *row_ptr, const int32_t *col_idx,
                const int64_t *col_ptr, const int32_t *row_idx,
                const double *omega, const double *z, const double *lam, double tau,
                const double *eta, const double *delta, double tol, int stop_rule, int max_iter,
                int sum_mode, double *beta, int *iters, double *resid)
{
    const size_t nn = (size_t)(n > 0 ? n : 1), np = (size_t)(p > 0 ? p : 1);
    double *u = (double *)malloc(sizeof(double) * (nn + np));   /* [top n; bottom p] */
    double *v = (double *)malloc(sizeof(double) * np);
    double *w = (double *)malloc(sizeof(double) * np);
    double *x = (double *)malloc(sizeof(double) * np);
    double *t = (double *)malloc(sizeof(double) * np);
    double *tn = (double *)malloc(sizeof(double) * nn);
    double *dsc = (double *)malloc(sizeof(double) * np);          /* D = tau lambda */
    int status = ORACLE_OK, k = 0;
    for (int64_t j = 0; j < p; ++j)
        dsc[j] = tau * lam[j];
    /* u = bt / ||bt|| */
    for (int64_t i = 0; i < n; ++i)
        u[i] = sqrt(omega[i]) * z[i] + eta[i];
    for (int64_t j = 0; j < p; ++j)
        u[n + j] = delta[j];
    double bet = sqrt(dot_mode(sum_mode, n + p, u, u));
    if (bet > 0.0)
        for (int64_t i = 0; i < n + p; ++i) u[i] = u[i] / bet;
    /* v = A^T u / ||A^T u||,  A^T u = D X^T (Omega^1/2 u_top) + u_bot */
    for (int64_t i = 0; i < n; ++i)
        tn[i] = sqrt(omega[i]) * u[i];
    xt_mode(sum_mode, p, col_ptr, row_idx, tn, t);
    for (int64_t j = 0; j < p; ++j)
        v[j] = dsc[j] * t[j] + u[n + j];
    double alf = sqrt(dot_mode(sum_mode, p, v, v));
    if (alf > 0.0)
        for (int64_t j = 0; j < p; ++j) v[j] = v[j] / alf;
    for (int64_t j = 0; j < p; ++j) {
        w[j] = v[j];
        x[j] = 0.0;
    }
    double phibar = bet, rhobar = alf;
    const double ref = alf * bet;                 /* ||A^T bt|| = ||tau lambda (.) b|| */
    double arnorm = ref;
    double q = stop_rule == ORACLE_STOP_RELATIVE ? (ref > 0.0 ? arnorm / ref : 0.0)
                                                 : sqrt(arnorm * arnorm / (double)p);
    if (!isfinite(q) || !isfinite(alf) || !isfinite(bet)) {
        status = ORACLE_NONFINITE;
    } else if (q > tol) {
        if (!(alf > 0.0) || !(bet > 0.0)) status = ORACLE_BREAKDOWN;
        else if (max_iter <= 0) status = ORACLE_MAXITER;
        while (status == ORACLE_OK) {
            /* u = A v - alpha u,  A v = [Omega^1/2 X (D v); v] */
            for (int64_t j = 0; j < p; ++j)
                t[j] = dsc[j] * v[j];
            x_mode(sum_mode, n, row_ptr, col_idx, t, tn);
            for (int64_t i = 0; i < n; ++i)
                u[i] = sqrt(omega[i]) * tn[i] - alf * u[i];
            for (int64_t j = 0; j < p; ++j)
                u[n + j] = v[j] - alf * u[n + j];
            bet = sqrt(dot_mode(sum_mode, n + p, u, u));
            if (bet > 0.0)
                for (int64_t i = 0; i < n + p; ++i) u[i] = u[i] / bet;
            /* v = A^T u - beta v */
            for (int64_t i = 0; i < n; ++i)
                tn[i] = sqrt(omega[i]) * u[i];
            xt_mode(sum_mode, p, col_ptr, row_idx, tn, t);
            for (int64_t j = 0; j < p; ++j)
                v[j] = dsc[j] * t[j] + u[n + j] - bet * v[j];
            alf = sqrt(dot_mode(sum_mode, p, v, v));
            if (alf > 0.0)
                for (int64_t j = 0; j < p; ++j) v[j] = v[j] / alf;
            /* plane rotation */
            const double rho = sqrt(rhobar * rhobar + bet * bet);
            const double c = rhobar / rho, sn = bet / rho;
            const double theta = sn * alf;
            rhobar = -c * alf;
            const double phi = c * phibar;
            phibar = sn * phibar;
            for (int64_t j = 0; j < p; ++j) {
                x[j] = x[j] + (phi / rho) * w[j];
                w[j] = v[j] - (theta / rho) * w[j];
            }
            k += 1;
            arnorm = phibar * alf * fabs(c);
            q = stop_rule == ORACLE_STOP_RELATIVE ? arnorm / ref : sqrt(arnorm * arnorm / (double)p);
            if (!isfinite(q) || !isfinite(rho)) { status = ORACLE_NONFINITE; break; }
            if (q <= tol) break;
            if (k == max_iter) { status = ORACLE_MAXITER; break; }
        }
    }
    for (int64_t j = 0; j < p; ++j)
        beta[j] = dsc[j] * x[j];
    *iters = k;
    *resid = q;
    free(u); free(v); free(w); free(x); free(t); free(tn); free(dsc);
    return status;
}

/*
 * Dense Phi = X^T Omega X + tau^-2 Lambda^-2 (p x p, row-major), the matrix
 * the direct sampler forms (Sec. 1; Sec. S7.2).  For binary X,
 * (X^T Omega X)_{jk} = sum over rows i holding both j and k of omega_i.
 */
void oracle_dense_phi(int64_t n, int64_t p, const int64_t *row_ptr, const int32_t *col_idx,
                      const double *omega, const double *lam, double tau, double *phi)
{
    memset(phi, 0, sizeof(double) * (size_t)(p * p));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t a = row_ptr[i]; a < row_ptr[i + 1]; ++a)
            for (int64_t c = row_ptr[i]; c < row_ptr[i + 1]; ++c)
                phi[(int64_t)col_idx[a] * p + col_idx[c]] += omega[i];
    for (int64_t j = 0; j < p; ++j)
        phi[j * p + j] += prior_prec(tau, lam[j]);
}

/*
 * In-place Cholesky A = L L^T of a p x p row-major SPD matrix (lower
 * triangle receives L, the strict upper triangle is zeroed).
 * Returns 0, or -1 - j when the pivot of column j is not positive.
 */
int oracle_cholesky(int64_t p, double *a)
{
    for (int64_t j = 0; j < p; ++j) {
        double d = a[j * p + j];
        for (int64_t k = 0; k < j; ++k)
            d -= a[j * p + k] * a[j * p + k];
        if (!(d > 0.0)) return (int)(-1 - j);
        double ljj = sqrt(d);
        a[j * p + j] = ljj;
        for (int64_t i = j + 1; i < p; ++i) {
            double e = a[i * p + j];
            for (int64_t k = 0; k < j; ++k)
                e -= a[i * p + k] * a[j * p + k];
            a[i * p + j] = e / ljj;
        }
        for (int64_t i = 0; i < j; ++i)
            a[i * p + j] = 0.0;
    }
    return 0;
}

/* Solve L L^T x = b with L from oracle_cholesky (forward, then backward). */
void oracle_chol_solve(int64_t p, const double *l, const double *b, double *x)
{
    for (int64_t i = 0; i < p; ++i) {
        double e = b[i];
        for (int64_t k = 0; k < i; ++k)
            e -= l[i * p + k] * x[k];
        x[i] = e / l[i * p + i];
    }
    for (int64_t i = p - 1; i >= 0; --i) {
        double e = x[i];
        for (int64_t k = i + 1; k < p; ++k)
            e -= l[k * p + i] * x[k];
        x[i] = e / l[i * p + i];
    }
}

/* ===========================================================================
 * The rest of the Gibbs cycle of Sec. S1 (row f3): tau | beta, lambda;
 * lambda | beta, tau; omega | beta ~ PolyaGamma(1, x_i^T beta); then the beta
 * draw above.  Horseshoe prior: half-Cauchy local scales lambda_j and global
 * scale tau (Sec. S1 names it beside the bridge), updated through the
 * auxiliary variables of Makalic and Schmidt (2016): with nu_j, xi,
 *   lambda_j^2 | nu_j ~ InvGamma(1/2, 1/nu_j),  nu_j ~ InvGamma(1/2, 1)
 * (so lambda_j ~ C+(0, 1)), and likewise tau^2 with xi, the conditionals are
 *   xi | tau          ~ InvGamma(1, 1 + 1/tau^2)
 *   tau^2 | beta, lambda, xi ~ InvGamma((p + 1)/2, 1/xi + sum_j beta_j^2 / (2 lambda_j^2))
 *   nu_j | lambda_j   ~ InvGamma(1, 1 + 1/lambda_j^2)
 *   lambda_j^2 | beta_j, tau, nu_j ~ InvGamma(1, 1/nu_j + beta_j^2 / (2 tau^2)).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw 2011), a
 * counter-based generator, keyed by a 64-bit seed; each quantity reads its own
 * counter (index, stream, step, draw), so every element's numbers are fixed
 * whatever order the elements are computed in.
 * =========================================================================== */

#define ORACLE_STREAM_XI 1u
#define ORACLE_STREAM_TAU 2u
#define ORACLE_STREAM_NU 3u
#define ORACLE_STREAM_LAMBDA 4u
#define ORACLE_STREAM_OMEGA 5u
#define ORACLE_STREAM_ETA 6u
#define ORACLE_STREAM_DELTA 7u

/* One Philox4x32-10 block: ten rounds of the Philox S-box on the 4-word
 * counter, the key bumped by the Weyl constants between rounds. */
void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A stream of uniforms for one (index, stream, step): each block gives two
 * doubles in (0, 1), ((w0 >> 5) 2^26 + (w1 >> 6) + 1/2) / 2^53 and the same
 * from (w2, w3); the fourth counter word counts blocks. */
typedef struct {
    uint32_t key[2], ctr[3], draw;
    double buf[2];
    int have;
} orng;

static void orng_init(orng *g, uint64_t seed, uint32_t index, uint32_t stream, uint32_t step)
{
    g->key[0] = (uint32_t)seed;
    g->key[1] = (uint32_t)(seed >> 32);
    g->ctr[0] = index;
    g->ctr[1] = stream;
    g->ctr[2] = step;
    g->draw = 0;
    g->have = 0;
}

static double orng_u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) / 9007199254740992.0;
}

static double orng_uniform(orng *g)
{
    if (g->have == 0) {
        const uint32_t c[4] = {g->ctr[0], g->ctr[1], g->ctr[2], g->draw};
        uint32_t w[4];
        oracle_philox(c, g->key, w);
        g->draw += 1;
        g->buf[0] = orng_u53(w[0], w[1]);
        g->buf[1] = orng_u53(w[2], w[3]);
        g->have = 2;
    }
    g->have -= 1;
    return g->buf[1 - g->have];
}

/* Exponential(1) by inversion; standard normal by Box and Muller (the cosine
 * branch only: two uniforms per normal). */
static double orng_exp(orng *g) { return -log(orng_uniform(g)); }

static double orng_normal(orng *g)
{
    const double u1 = orng_uniform(g), u2 = orng_uniform(g);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Gamma(a, 1), a >= 1 (Marsaglia and Tsang 2000): d = a - 1/3, c = 1/sqrt(9d);
 * repeat x ~ N(0,1), v = (1 + c x)^3 until v > 0 and log U < x^2/2 + d - d v + d log v. */
static double orng_gamma(orng *g, double a)
{
    const double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (int attempt = 0; attempt < 100000; ++attempt) {
        const double x = orng_normal(g);
        double v = 1.0 + c * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        const double u = orng_uniform(g);
        if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
    }
    return NAN;
}

/* Standard normal CDF. */
static double ophi(double x) { return 0.5 * erfc(-x / 1.4142135623730951); }

/* n-th coefficient of the alternating series of the J*(1, 0) density
 * (Devroye's piecewise form, split at t). */
static double pg_coef(int n, double x, double t)
{
    const double h = n + 0.5;
    if (x > t) return 3.141592653589793 * h * exp(-h * h * 9.869604401089358 * x / 2.0);
    return 3.141592653589793 * h * pow(2.0 / (3.141592653589793 * x), 1.5) * exp(-2.0 * h * h / x);
}

/* The J*(1, 0) density by its alternating series, sum_{n < terms} (-1)^n a_n(x),
 * with the coefficients of the form chosen by t (x <= t: the small-x form,
 * x > t: the large-x form).  Both forms represent the same density. */
double oracle_pg_series(double x, double t, int terms)
{
    double s = 0.0;
    for (int n = 0; n < terms; ++n)
        s += (n & 1) ? -pg_coef(n, x, t) : pg_coef(n, x, t);
    return s;
}

/* Inverse Gaussian IG(mu, 1) truncated to (0, t) (Polson, Scott and Windle 2013). */
static double pg_trunc_ig(orng *g, double z, double t)
{
    const double mu = z > 0.0 ? 1.0 / z : INFINITY;
    if (mu > t) {
        for (int attempt = 0; attempt < 100000; ++attempt) {
            double e1, e2;
            do {
                e1 = orng_exp(g);
                e2 = orng_exp(g);
            } while (e1 * e1 > 2.0 * e2 / t);
            const double x = t / ((1.0 + t * e1) * (1.0 + t * e1));
            const double alpha = exp(-0.5 * z * z * x);
            if (orng_uniform(g) <= alpha) return x;
        }
        return NAN;
    }
    for (int attempt = 0; attempt < 100000; ++attempt) {
        const double y0 = orng_normal(g);
        const double y = y0 * y0;
        double x = mu + 0.5 * mu * mu * y - 0.5 * mu * sqrt(4.0 * mu * y + (mu * y) * (mu * y));
        if (orng_uniform(g) > mu / (mu + x)) x = mu * mu / x;
        if (x <= t) return x;
    }
    return NAN;
}

/*
 * One draw of PolyaGamma(1, c) (Polson, Scott and Windle 2013): X ~ J*(1, z),
 * z = |c|/2, by Devroye's alternating-series method with the proposal mixing
 * a truncated exponential on (t, inf) and a truncated inverse Gaussian on
 * (0, t), t = 0.64; omega = X / 4.
 */
double oracle_pg1_draw(double c, orng *g)
{
    const double t = 0.64, z = 0.5 * fabs(c);
    const double K = 9.869604401089358 / 8.0 + 0.5 * z * z;
    const double p = 3.141592653589793 / (2.0 * K) * exp(-K * t);
    double q;
    if (z > 0.0) {
        const double mu = 1.0 / z, rt = sqrt(1.0 / t);
        q = 2.0 * exp(-z) * (ophi(rt * (t / mu - 1.0)) + exp(2.0 / mu) * ophi(-rt * (t / mu + 1.0)));
    } else {
        q = 4.0 * ophi(-sqrt(1.0 / t));
    }
    const double r = p / (p + q);
    /* a proposal is accepted with probability above 0.99 and the series decides
     * within a few terms: the caps only end a sampler that is broken (NaN) */
    for (int attempt = 0; attempt < 100000; ++attempt) {
        double x;
        if (orng_uniform(g) < r) x = t + orng_exp(g) / K;
        else x = pg_trunc_ig(g, z, t);
        double s = pg_coef(0, x, t);
        const double y = orng_uniform(g) * s;
        for (int n = 1; n < 1000; ++n) {
            if (n & 1) {
                s -= pg_coef(n, x, t);
                if (y <= s) return 0.25 * x;
            } else {
                s += pg_coef(n, x, t);
                if (y > s) break;
            }
        }
    }
    return NAN;
}

/* out[k] = PolyaGamma(1, c[k]) with index k's numbers of (seed, stream, step). */
void oracle_pg1(int64_t m, const double *c, uint64_t seed, uint32_t stream, uint32_t step, double *out)
{
    for (int64_t k = 0; k < m; ++k) {
        orng g;
        orng_init(&g, seed, (uint32_t)k, stream, step);
        out[k] = oracle_pg1_draw(c[k], &g);
    }
}

/* Uniforms, exponentials, normals and Gamma(a) draws of one counter (pins). */
void oracle_rng_draws(int kind, int64_t m, uint64_t seed, uint32_t index, uint32_t stream,
                      uint32_t step, double a, double *out)
{
    orng g;
    orng_init(&g, seed, index, stream, step);
    for (int64_t k = 0; k < m; ++k)
        out[k] = kind == 0 ? orng_uniform(&g) : kind == 1 ? orng_exp(&g)
               : kind == 2 ? orng_normal(&g) : orng_gamma(&g, a);
}

/*
 * The scale updates of one Gibbs cycle (steps 1-2 of Sec. S1):
 *   xi ~ IG(1, 1 + 1/tau^2), tau^2 ~ IG((p+1)/2, 1/xi + sum_j beta_j^2/(2 lambda_j^2)),
 *   nu_j ~ IG(1, 1 + 1/lambda_j^2), lambda_j^2 ~ IG(1, 1/nu_j + beta_j^2/(2 tau^2)),
 * with IG(a, b) = b / Gamma(a, 1) (Gamma(1, 1) = Exponential(1)).  tau, xi:
 * in/out scalars; lambda, nu: in/out p-vectors.
 */
void oracle_gibbs_scales(int64_t p, const double *beta, double *lam, double *nu, double *tau,
                         double *xi, uint64_t seed, uint32_t step)
{
    orng g;
    orng_init(&g, seed, 0u, ORACLE_STREAM_XI, step);
    *xi = (1.0 + 1.0 / ((*tau) * (*tau))) / orng_exp(&g);
    double ssq = 0.0;
    for (int64_t j = 0; j < p; ++j)
        ssq += beta[j] * beta[j] / (2.0 * lam[j] * lam[j]);
    orng_init(&g, seed, 0u, ORACLE_STREAM_TAU, step);
    *tau = sqrt((1.0 / *xi + ssq) / orng_gamma(&g, 0.5 * (double)(p + 1)));
    for (int64_t j = 0; j < p; ++j) {
        orng_init(&g, seed, (uint32_t)j, ORACLE_STREAM_NU, step);
        nu[j] = (1.0 + 1.0 / (lam[j] * lam[j])) / orng_exp(&g);
        orng_init(&g, seed, (uint32_t)j, ORACLE_STREAM_LAMBDA, step);
        lam[j] = sqrt((1.0 / nu[j] + beta[j] * beta[j] / (2.0 * (*tau) * (*tau))) / orng_exp(&g));
    }
}

/*
 * Step 3 of Sec. S1 and the Gaussian vectors of Prop. 2.1 for step 4:
 *   psi = X beta; omega_i ~ PolyaGamma(1, psi_i); z_i = (y_i - 1/2) / omega_i (Eq. 1.1);
 *   eta ~ N(0, I_n), delta ~ N(0, I_p).
 */
void oracle_gibbs_omega(int64_t n, int64_t p, const int64_t *row_ptr, const int32_t *col_idx,
                        const double *y, const double *beta, uint64_t seed, uint32_t step,
                        double *omega, double *z, double *eta, double *delta)
{
    double *psi = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    oracle_x_mul(n, row_ptr, col_idx, beta, psi);
    oracle_pg1(n, psi, seed, ORACLE_STREAM_OMEGA, step, omega);
    for (int64_t i = 0; i < n; ++i) {
        z[i] = (y[i] - 0.5) / omega[i];
        orng g;
        orng_init(&g, seed, (uint32_t)i, ORACLE_STREAM_ETA, step);
        eta[i] = orng_normal(&g);
    }
    for (int64_t j = 0; j < p; ++j) {
        orng g;
        orng_init(&g, seed, (uint32_t)j, ORACLE_STREAM_DELTA, step);
        delta[j] = orng_normal(&g);
    }
    free(psi);
}
