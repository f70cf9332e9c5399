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

static double dot(int64_t p, const double *a, const double *b)
{
    double acc = 0.0;
    for (int64_t j = 0; j < p; ++j)
        acc += a[j] * b[j];
    return acc;
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

/*
 * Prior-preconditioned CG on Phi beta = b from beta_0 = 0 (Sec. 2.7,
 * Algorithm S1 in PCG form).
 *
 *   beta = 0; r = b; z = m r; s = z; rho = r.z        (m = tau^2 lambda^2)
 *   repeat: v = Phi s; alpha = rho / (s.v)
 *           beta += alpha s; r -= alpha v; z = m r; rho' = r.z; k += 1
 *           stop on rho' (Eq. S2) or k == max_iter
 *           s = z + (rho'/rho) s; rho = rho'
 *
 * fixed_iters > 0 runs exactly that many iterations without testing the
 * stop rule (for same-k comparisons); fixed_iters == 0 uses tol/max_iter.
 * rho_hist (optional, max(max_iter, fixed_iters) + 1 doubles) receives rho
 * before the first product and after each product.
 * Returns ORACLE_OK, ORACLE_MAXITER, ORACLE_BREAKDOWN or ORACLE_NONFINITE.
 */
int oracle_pcg(int64_t n, int64_t p,
               const int64_t *row_ptr, const int32_t *col_idx,
               const int64_t *col_ptr, const int32_t *row_idx,
               const double *omega, const double *lam, double tau,
               const double *b, double tol, int stop_rule, int max_iter, int fixed_iters,
               double *beta, int *iters, double *resid, double *rho_hist)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
    double *s = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
    double *v = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
    double *work = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int status = ORACLE_OK;
    int k = 0;

    for (int64_t j = 0; j < p; ++j) {
        beta[j] = 0.0;
        r[j] = b[j];                       /* r_0 = b - Phi beta_0 = b */
        z[j] = prior_var(tau, lam[j]) * r[j];
        s[j] = z[j];
    }
    double rho = dot(p, r, z);
    const double rho0 = rho;
    double rho_new = rho;
    if (rho_hist) rho_hist[0] = rho;

    if (!isfinite(rho)) {
        status = ORACLE_NONFINITE;
    } else if (fixed_iters > 0 || !stop_met(stop_rule, rho, rho0, p, tol)) {
        int limit = fixed_iters > 0 ? fixed_iters : max_iter;
        if (limit <= 0) status = ORACLE_MAXITER;
        while (k < limit) {
            oracle_phi_mul(n, p, row_ptr, col_idx, col_ptr, row_idx, omega, lam, tau, s, v, work);
            double sigma = dot(p, s, v);
            if (!isfinite(sigma)) { status = ORACLE_NONFINITE; break; }
            if (sigma <= 0.0 || rho <= 0.0) { status = ORACLE_BREAKDOWN; break; }
            double alpha = rho / sigma;
            for (int64_t j = 0; j < p; ++j) {
                beta[j] = beta[j] + alpha * s[j];
                r[j] = r[j] - alpha * v[j];
                z[j] = prior_var(tau, lam[j]) * r[j];
            }
            rho_new = dot(p, r, z);
            k += 1;
            if (rho_hist) rho_hist[k] = rho_new;
            if (!isfinite(rho_new)) { status = ORACLE_NONFINITE; break; }
            if (fixed_iters == 0) {
                if (stop_met(stop_rule, rho_new, rho0, p, tol)) break;
                if (k == max_iter) { status = ORACLE_MAXITER; break; }
            }
            double gamma = rho_new / rho;
            for (int64_t j = 0; j < p; ++j)
                s[j] = z[j] + gamma * s[j];
            rho = rho_new;
        }
    }
    *iters = k;
    *resid = resid_of(stop_rule, rho_new, rho0, p);
    free(r); free(z); free(s); free(v); free(work);
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
