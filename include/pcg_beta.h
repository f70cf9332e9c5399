/*
 * pcg_beta.h -- C ABI of the GB300 library for the conditional draw of the
 * regression coefficients in the CG-accelerated Gibbs sampler of Nishimura &
 * Suchard, "Prior-preconditioned conjugate gradient method for accelerated
 * Gibbs sampling in 'large n & large p' Bayesian sparse regression".
 *
 * The draw (Eq. 1.2 and Prop. 2.1):
 *     beta ~ N(Phi^-1 X^T Omega z, Phi^-1),  Phi = X^T Omega X + tau^-2 Lambda^-2,
 * computed as
 *     b    = X^T Omega z + X^T Omega^1/2 eta + tau^-1 Lambda^-1 delta   (Eq. 2.3)
 *     solve Phi beta = b                                              (Eq. 2.4)
 * by conjugate gradient preconditioned with the prior precision
 * M = tau^-2 Lambda^-2 (Sec. 2.4), from beta_0 = 0 (Sec. 2.7), with the
 * recursion of Algorithm S1 (Sec. S2) in its preconditioned form and the
 * stop rule of Eq. S2 (Sec. S4.2).  Phi is never formed: each iteration
 * applies u = Omega (X s) and v = X^T u + tau^-2 Lambda^-2 s (Sec. 1).
 *
 * Conventions for every entry point:
 *  - X is binary (every stored entry is 1) and is passed as indices only,
 *    in both layouts: CSR (row_ptr int64[n+1], col_idx int32[nnz], columns
 *    strictly increasing within a row) and CSC (col_ptr int64[p+1],
 *    row_idx int32[nnz], rows strictly increasing within a column).  Both
 *    must describe the same X; pcg_check_design verifies that.
 *  - Every array pointer is a DEVICE pointer to memory owned by the caller
 *    (the library never frees it and keeps no reference after the call
 *    returns), except where a parameter is marked "host".
 *  - Vectors are contiguous float64 unless stated.  Batched inputs are
 *    chain-major: chain r's omega is omega[r*n .. r*n+n-1], and so on.
 *  - Work is queued on the stream given to pcg_ctx_create (a cudaStream_t
 *    passed as void*; NULL means the legacy default stream).  Each entry
 *    point returns after its host outputs are written, which is the only
 *    synchronisation it performs.
 *  - Every entry point returns a pcg_status and never aborts the process.
 *    On PCG_MAXITER the output holds the last iterate.  pcg_last_error gives
 *    a one-line description of the most recent non-OK status of a context.
 *  - Preconditions: omega_i > 0, lambda_j > 0, tau > 0 (PCG_BADARG is
 *    returned for non-positive tau; non-finite results give
 *    PCG_NONFINITE; a non-positive curvature s.Phi s gives PCG_BREAKDOWN).
 */
#ifndef PCG_BETA_H
#define PCG_BETA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcg_ctx pcg_ctx;

typedef enum pcg_status {
    PCG_OK = 0,         /* converged under the stop rule */
    PCG_MAXITER = 1,    /* max_iter reached first; output is the last iterate */
    PCG_BREAKDOWN = 2,  /* s.Phi s <= 0 or rho <= 0 (Phi not SPD in floating point) */
    PCG_NONFINITE = 3,  /* NaN or Inf in a CG scalar */
    PCG_BADARG = 4,     /* invalid sizes, pointers, options or design */
    PCG_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    PCG_CUDA = 6        /* a CUDA runtime call failed */
} pcg_status;

/* Arithmetic of the products u = Omega X s and v = X^T u. */
enum {
    PCG_PREC_FP64 = 0,          /* gathers and sums in float64 */
    PCG_PREC_FP32_REFINED = 1,  /* float32 gathers and sums; CG scalars, beta and r in
                                   float64; r = b - Phi beta recomputed in float64
                                   every reliable_k iterations and before stopping */
    PCG_PREC_FP32 = 2,          /* float32 products, float64 scalars, no recomputation */
    PCG_PREC_DF32 = 3,          /* double-float products: each gathered value held as a pair
                                   of float32 (hi + lo) and summed with error-free float32
                                   TwoSum, about 48 significant bits at float32 arithmetic
                                   cost; CG scalars, beta and r in float64 */
    PCG_PREC_FX64 = 4           /* fixed-point products: the vectors are float32 pairs as in
                                   PCG_PREC_DF32; each tile of the gathered vector is scaled,
                                   per right-hand side, by a power of two and rounded to
                                   64-bit integers (grid: 2^(hb-60) of the tile's largest
                                   value, where a segment sums fewer than 2^hb values, so no
                                   sum can overflow; about 2^-51 at n = 5e5, p = 5e4), summed
                                   exactly in integer arithmetic, and each sum converted back
                                   to a float32 pair (the tiled products only; elsewhere as
                                   PCG_PREC_DF32) */
};

/* Stop rules.  With rho = r.(M^-1 r) = ||tau lambda (.) r||^2 (Sec. S4.2):
 *   PCG_STOP_PAPER_RMS  stop when sqrt(rho / p) <= tol          (Eq. S2)
 *   PCG_STOP_RELATIVE   stop when sqrt(rho / rho_0) <= tol      (rho_0 at beta_0 = 0)
 * (with the Jacobi preconditioner or a warm start, rho is still ||tau lambda (.) r||^2
 * and rho_0 = ||tau lambda (.) b||^2). */
enum { PCG_STOP_PAPER_RMS = 0, PCG_STOP_RELATIVE = 1 };

/* Preconditioners of the single-RHS CG (Sec. 2.4): the prior precision
 * M = tau^-2 Lambda^-2 (the paper's choice), or the Jacobi preconditioner
 * M = diag(Phi_11 .. Phi_pp), diag(Phi)_j = sum_{i: X_ij = 1} omega_i + tau^-2
 * lambda_j^-2 for binary X (the alternative Sec. 2.4 names and Sec. 3 compares).
 * Whatever the preconditioner, the stop rule tests the prior-preconditioned
 * residual of Eq. S2, ||tau lambda (.) r||, so both stop at the same accuracy. */
enum { PCG_PRECOND_PRIOR = 0, PCG_PRECOND_JACOBI = 1 };

/* Adjoint modes: gradient with b as an input, or with b built inside from (z, eta, delta). */
enum { PCG_ADJ_SOLVE = 0, PCG_ADJ_DRAW = 1 };

typedef struct pcg_csr {
    int64_t n, p, nnz;
    const int64_t *row_ptr;   /* device, n+1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
    const int32_t *col_idx;   /* device, nnz entries in [0, p) */
} pcg_csr;

typedef struct pcg_csc {
    int64_t n, p, nnz;
    const int64_t *col_ptr;   /* device, p+1 entries, col_ptr[0] = 0, col_ptr[p] = nnz */
    const int32_t *row_idx;   /* device, nnz entries in [0, n) */
} pcg_csc;

typedef struct pcg_options {
    int precision;              /* PCG_PREC_*, default PCG_PREC_DF32 */
    int reliable_k;             /* refined mode: also recompute r every k iterations (0: only
                                   before stopping); default 50 */
    int stop_rule;              /* PCG_STOP_*, default PCG_STOP_PAPER_RMS */
    int use_graph;              /* 1 (default): the whole draw is one CUDA-graph launch whose
                                   iteration loop is a device-side while node; 0: plain launches
                                   with a host check every 8 iterations */
    const char *autotune_cache; /* host path of a text file caching tuned launch shapes, or NULL */
    int profile;                /* 1: time every kernel with CUDA events on the context stream
                                   (forces plain launches); read with pcg_profile_entry */
    double idle_limit_s;        /* uneven batch: a CTA that finds no work gives up, and the
                                   call returns PCG_TIMEOUT, once no tile of any problem has
                                   completed for this many seconds; default 2.0, accepted
                                   range [1e-6, 3600] (PCG_BADARG at pcg_ctx_create otherwise) */
    int preconditioner;         /* PCG_PRECOND_*, default PCG_PRECOND_PRIOR; pcg_draw_beta and
                                   pcg_solve (and the adjoint's solve) only: the batched and
                                   uneven entry points return PCG_BADARG for JACOBI */
    int warm_start;             /* 1: pcg_draw_beta and pcg_solve start CG from the initial
                                   vector beta_0 that the output buffer holds on entry (Sec.
                                   S4.1; r_0 = b - Phi beta_0, one float64 product), instead
                                   of beta_0 = 0; the RELATIVE rule still measures against
                                   ||tau lambda (.) b|| so the target does not move.  Default 0;
                                   the batched, uneven and adjoint entry points return
                                   PCG_BADARG when it is set */
} pcg_options;

/* Fills *opt with the defaults listed above. */
pcg_status pcg_options_default(pcg_options *opt);

/* Creates a context bound to the current CUDA device and to `stream`.  The
 * context owns its workspace (grown on demand, freed by pcg_ctx_destroy), its
 * cached graphs and its cached product plans: the tiled products' plan (tile
 * offsets, work split, bank order) depends on X alone, so it is built on the
 * first call for a design and reused while the design's pointers, sizes and
 * index contents are unchanged (each call hashes the four index arrays on the
 * device; a different design in the same buffers rebuilds the plan).  A context
 * must not be used by two host threads at once. */
pcg_status pcg_ctx_create(pcg_ctx **ctx, const pcg_options *opt, void *stream);
void pcg_ctx_destroy(pcg_ctx *ctx);
const char *pcg_last_error(const pcg_ctx *ctx);

/*
 * Unshrunk coefficients (Sec. S4.3): coefficients 0 .. q1-1 (an intercept,
 * predictors of interest) take independent Gaussian priors N(0, sigma_j^2)
 * instead of the shrinkage prior, so that
 *     Phi = X^T Omega X + diag(sigma_0^-2 .. sigma_{q1-1}^-2, tau^-2 lambda_q1^-2 ..),
 * the prior term of Eq. 2.3 is sigma_j^-1 delta_j for them, and the CG
 * preconditioner is M = diag(gamma^-2, tau^-2 Lambda^-2) with the scales
 * gamma_j of Sec. S4.3 (c times an estimate of the posterior standard
 * deviation of beta_j, c >= 1); the stop rule's norm ||M^-1/2 r|| uses that M.
 * prior_prec: device, q1 entries sigma_j^-2 >= 0 (0: the flat prior of an
 * uninformative coefficient); precond_scale: device, q1 entries gamma_j > 0.
 * Both are copied into the context (the caller keeps ownership) and apply to
 * the later pcg_draw_beta, pcg_solve, pcg_draw_beta_batched (every chain),
 * pcg_build_rhs and pcg_phi_mul calls on this context, where lambda[j] is
 * then not read for j < q1; q1 = 0 switches them off.  PCG_BADARG for q1 < 0,
 * NULL vectors, a negative or non-finite precision or a non-positive or
 * non-finite gamma (the setting is then cleared), for a later call whose X has
 * fewer than q1 columns, and for pcg_draw_beta_uneven and pcg_adjoint while
 * set (their tau and lambda derivatives assume the shrinkage prior throughout).
 */
pcg_status pcg_set_unshrunk(pcg_ctx *ctx, int q1, const double *prior_prec, const double *precond_scale);

/* Checks on the device that csr and csc are valid, agree in n, p and nnz and
 * hold the same set of (i, j) entries; never dereferences a stored index.
 * Returns PCG_OK or PCG_BADARG. */
pcg_status pcg_check_design(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc);

/*
 * Right-hand side of Prop. 2.1, Eq. 2.3, in float64:
 *   b_j = sum_{i : X_ij = 1} (omega_i z_i + sqrt(omega_i) eta_i) + delta_j / (tau lambda_j).
 * omega, z, eta: n; lambda, delta: p; b (out): p.
 */
pcg_status pcg_build_rhs(pcg_ctx *ctx, const pcg_csc *X_csc, const double *omega, const double *z,
                         const double *lambda, double tau, const double *eta,
                         const double *delta, double *b);

/*
 * Matrix-free product of Sec. 1:  out = X^T (Omega (X v)) + tau^-2 Lambda^-2 v,
 * with the products in the context's precision (float32 sums in the FP32
 * modes, float64 otherwise) and the diagonal term in float64.
 * v, out: p (float64); omega: n; lambda: p.
 */
pcg_status pcg_phi_mul(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc,
                       const double *omega, const double *lambda, double tau,
                       const double *v, double *out);

/*
 * One conditional draw: b by Eq. 2.3, then prior-preconditioned CG on Eq. 2.4.
 * beta (out, p) receives the draw; *iters (host) the number of CG iterations
 * (products Phi s); *resid (host) the final value of the stop quantity
 * (sqrt(rho/p) or sqrt(rho/rho_0)).  max_iter >= 0; tol >= 0.
 */
pcg_status pcg_draw_beta(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc,
                         const double *omega, const double *z, const double *lambda, double tau,
                         const double *eta, const double *delta, double tol, int max_iter,
                         double *beta, int *iters, double *resid);

/*
 * The same draw by LSQR (Paige and Saunders 1982) on the least-squares form
 * of Sec. S7.1 (Eq. S6): beta minimises ||Xt beta - bt|| with Xt = [Omega^1/2 X;
 * tau^-1 Lambda^-1] and bt = [Omega^1/2 z + eta; delta], whose normal equations
 * are Phi beta = b of Eq. 2.3-2.4.  LSQR is run on Xt diag(tau lambda) (the
 * prior preconditioner applied on the right), so its estimate of ||A^T r||
 * equals ||tau lambda (.) (b - Phi beta)|| and it stops under the context's
 * stop rule exactly as pcg_draw_beta does.  In exact arithmetic its iterates
 * are those of the prior-preconditioned CG.  Arithmetic: float64 products and
 * scalars whatever the context's precision.  Arguments and outputs as
 * pcg_draw_beta; PCG_BADARG while unshrunk coefficients, the Jacobi
 * preconditioner or warm starts are set on the context.
 */
pcg_status pcg_draw_beta_lsqr(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc,
                              const double *omega, const double *z, const double *lambda, double tau,
                              const double *eta, const double *delta, double tol, int max_iter,
                              double *beta, int *iters, double *resid);

/*
 * One cycle of the Gibbs sampler of Sec. S1 for sparse logistic regression with
 * Polya-Gamma augmentation and the horseshoe prior (half-Cauchy local scales
 * lambda_j and global scale tau, Sec. S1), in the order the paper gives:
 *   1. tau | beta, lambda   2. lambda | beta, tau   3. omega_i | beta ~ PolyaGamma(1, x_i^T beta)
 *   4. beta | omega, tau, lambda, y by pcg_draw_beta with z_i = (y_i - 1/2) / omega_i (Eq. 1.1)
 *      and fresh eta ~ N(0, I_n), delta ~ N(0, I_p).
 * Steps 1-2 use the auxiliary variables of Makalic and Schmidt (2016): xi ~
 * IG(1, 1 + 1/tau^2), tau^2 ~ IG((p+1)/2, 1/xi + sum beta_j^2 / (2 lambda_j^2)),
 * nu_j ~ IG(1, 1 + 1/lambda_j^2), lambda_j^2 ~ IG(1, 1/nu_j + beta_j^2 / (2 tau^2)).
 * Random numbers: Philox4x32-10 keyed by `seed`, one counter per (element,
 * quantity, step): the cycle is a deterministic function of (state, seed, step).
 * y: device, n values in {0, 1}.  In/out state: omega (device, n; out only),
 * lambda, nu, beta (device, p), *tau and *xi (host).  beta holds beta* on entry
 * (the previous draw, also beta_0 under warm_start) and the new draw on return.
 * The draw uses the context's precision, stop rule and preconditioner; tol,
 * max_iter, iters and resid as pcg_draw_beta.  PCG_BADARG while unshrunk
 * coefficients are set; PCG_NONFINITE if an update leaves tau or xi
 * non-finite.
 */
pcg_status pcg_gibbs_step(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc, const double *y,
                          uint64_t seed, uint32_t step, double *omega, double *lambda, double *nu,
                          double *tau, double *xi, double *beta, double tol, int max_iter, int *iters,
                          double *resid);

/*
 * CG solve of Phi x = rhs (Eq. 2.4) for a given right-hand side (no Eq. 2.3
 * step); same outputs as pcg_draw_beta.  Used by the adjoint, whose second
 * solve Phi g = c shares Phi and the preconditioner.
 */
pcg_status pcg_solve(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc,
                     const double *omega, const double *lambda, double tau, const double *rhs,
                     double tol, int max_iter, double *x, int *iters, double *resid);

/*
 * nrhs draws sharing X in one launch: each chain r has its own omega, z,
 * lambda, tau, eta and delta (chain-major, see above; tau: device, nrhs) and
 * runs its own CG scalars and stop test; the products are one sparse-times-
 * dense-block pass per iteration over the RHS block.  beta (out): nrhs*p,
 * chain-major.  iters, resid, status (host, nrhs each) receive each chain's
 * result; the return value is the worst status.  1 <= nrhs <= 32.
 * Precisions PCG_PREC_DF32, PCG_PREC_FX64, PCG_PREC_FP32_REFINED and
 * PCG_PREC_FP32 (PCG_PREC_FP64 returns PCG_BADARG).  PCG_PREC_DF32 and
 * PCG_PREC_FX64 exist only as tiled products: for a design beyond the tiled
 * plan's 32-bit positions (pcg_tiled_plan_applies false with nonzeros;
 * about 4e9 of them) they return PCG_BADARG, and the float32 modes run
 * untiled.
 */
pcg_status pcg_draw_beta_batched(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc,
                                 int nrhs, const double *omega, const double *z,
                                 const double *lambda, const double *tau, const double *eta,
                                 const double *delta, double tol, int max_iter, double *beta,
                                 int *iters, double *resid, int *status);

/* One independent problem of an uneven batch (all pointers device). */
typedef struct pcg_problem {
    pcg_csr X_csr;
    pcg_csc X_csc;
    const double *omega, *z, *lambda, *eta, *delta;
    double tau;
    double *beta;   /* out, p */
} pcg_problem;

/*
 * Independent problems of uneven n and p, solved together by one persistent
 * kernel launched from a CUDA graph: CTAs take (problem, tile) work items
 * from a device queue; each problem advances its own CG with per-problem
 * barriers whose waits are bounded (PCG_TIMEOUT if one gives up).
 * probs: host array of nprob descriptors.  iters, resid, status: host, nprob.
 * Its products are float64 (PCG_PREC_FP64), double-float (PCG_PREC_DF32, and
 * PCG_PREC_FX64, which runs as double-float here: float pairs gathered from L2
 * and summed with TwoSum), or float32 (PCG_PREC_FP32, and PCG_PREC_FP32_REFINED
 * with the float64 recomputation of r).
 */
pcg_status pcg_draw_beta_uneven(pcg_ctx *ctx, int nprob, const pcg_problem *probs, double tol,
                                int max_iter, int *iters, double *resid, int *status);

/*
 * Adjoint of the draw for a loss L with dL/dbeta = grad_beta (p):
 * one more prior-preconditioned CG solve Phi g = grad_beta, then
 *   g_b        = g                                     (p)
 *   g_omega    = -(X g) (.) (X beta)   [+ (X g) (.) (z + eta / (2 sqrt omega)) in DRAW mode]  (n)
 *   g_loglambda = 2 d (.) g (.) beta    [- g (.) delta / (tau lambda) in DRAW mode]           (p)
 *   *g_logtau (host) = sum_j g_loglambda_j
 * with d = tau^-2 lambda^-2.  beta is the draw whose gradient is wanted
 * (output of pcg_draw_beta).  In SOLVE mode z, eta, delta may be NULL.
 * iters/resid (host) describe the adjoint solve.  Not in the paper: implicit
 * differentiation of beta = Phi^-1 b with dPhi = X^T dOmega X + d(diag d).
 */
pcg_status pcg_adjoint(pcg_ctx *ctx, const pcg_csr *X_csr, const pcg_csc *X_csc,
                       const double *omega, const double *z, const double *lambda, double tau,
                       const double *eta, const double *delta, const double *beta,
                       const double *grad_beta, int mode, double tol, int max_iter,
                       double *g_b, double *g_omega, double *g_loglambda, double *g_logtau,
                       int *iters, double *resid);

/*
 * Whether the shared-memory tiled products serve a design of this shape:
 * returns 1 and the tile counts (host outputs, may be NULL) if they do, 0 if
 * the calls fall back to the untiled products (empty X, or a shape whose
 * padded 16-bit index stream or segment count exceeds the plan's 32-bit
 * positions and int counts).  rhs_group: right-hand sides staged together
 * (1 for the single-RHS path; 1, 2 or 4 in the batched path); precision:
 * PCG_PREC_*.  Host arithmetic only (no context, no GPU).  The paper's
 * products are plain sparse-BLAS calls (Sec. S7.2); this is the layout of
 * Sec. 1's two products on GB300.
 */
int pcg_tiled_plan_applies(int64_t n, int64_t p, int64_t nnz, int precision, int rhs_group,
                           int *col_tiles, int *row_strips);

/*
 * Measurement hooks (not in the paper; the paper times each linear-algebra
 * operation separately in Sec. S7.2).  With opt.profile = 1 every kernel
 * launch is bracketed by CUDA events on the context stream and accumulated
 * per kernel name.  pcg_profile_count gives the number of distinct kernels
 * seen; pcg_profile_entry(i) their name (valid until the next reset),
 * total milliseconds and launch count; pcg_profile_reset clears them.
 * pcg_last_kernel_launches gives the number of kernels the last entry point
 * launched (every node of the CUDA graph that ran counts once per run).
 */
int pcg_profile_count(const pcg_ctx *ctx);
pcg_status pcg_profile_entry(const pcg_ctx *ctx, int i, const char **name, double *total_ms,
                             int64_t *launches);
void pcg_profile_reset(pcg_ctx *ctx);
int64_t pcg_last_kernel_launches(const pcg_ctx *ctx);

/*
 * Allocation-free variant of pcg_phi_mul, for callers that cannot allocate
 * device memory: code running while a stream is captured into a CUDA graph,
 * host runtimes whose allocator owns the whole device, and loops where an
 * allocation could synchronise the device.  The paper has no counterpart.
 *
 * Computes out = X^T (Omega (X v)) + tau^-2 Lambda^-2 v in float64 (as
 * pcg_phi_mul does in PCG_PREC_FP64 mode) without a context: the caller
 * passes all inputs and outputs (device pointers, as everywhere) and the
 * stream (a cudaStream_t as void*, NULL for the legacy default stream).  The
 * call only queues the two kernels on `stream` and returns; `out` is ready
 * when the stream reaches that point.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * The intermediate u = Omega (X v) (n float64) lives in one file-scope device
 * array of PCG_NOALLOC_MAX_N doubles (8 MiB) that every GPU loading the
 * library holds until the process exits.  Sizes: n <= PCG_NOALLOC_MAX_N, else
 * PCG_BADARG is returned before any GPU work.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, once per
 * device); make that first call outside any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents (each call
 * writes every entry it reads, so nothing needs clearing): calls that overlap
 * on the GPU, e.g. on two streams at once, race on it.  Returns PCG_OK,
 * PCG_BADARG (NULL pointer, size mismatch, n too large, tau <= 0) or PCG_CUDA.
 */
#define PCG_NOALLOC_MAX_N 1048576
pcg_status pcg_phi_mul_noalloc(const pcg_csr *X_csr, const pcg_csc *X_csc, const double *omega,
                               const double *lambda, double tau, const double *v, double *out,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PCG_BETA_H */
