// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (see include/pcg_beta.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/pcg_beta.h"

namespace pcg {

constexpr int kMaxBatch = 32;          // largest RHS block of the batched path
constexpr int kMaxReduceBlocks = 4096; // capacity of the grid-reduction partial buffers

// Precisions whose vectors (s, omega) and product partials are float pairs:
// double-float sums, or fixed-point sums of each tile (PCG_PREC_FX64).
inline bool prec_pairs(int precision) { return precision == PCG_PREC_DF32 || precision == PCG_PREC_FX64; }

// Per-chain CG state kept in device memory.  Written only by the single
// "last block" of a grid reduction, read by every later kernel.
struct CgScalars {
    double rho;       // r . (M^-1 r) of the current residual
    double rho0;      // rho at beta_0 = 0
    double rho_prev;  // rho before the latest beta update
    double sigma;     // s . Phi s
    double alpha;     // rho / sigma
    double gamma;     // rho_new / rho_prev
    double resid;     // stop quantity of the current residual
    int iter;         // completed CG iterations (products Phi s)
    int status;       // kRunning, then a pcg_status
    int need_ru;      // recompute r = b - Phi beta before the next direction
    int pending;      // recursion met the stop rule; waiting for the recomputed r
    int done;         // nonzero once the chain has finished
    int ru_trips;     // iterations that ran the float64 recomputation of r
};
constexpr int kRunning = -1;

// Launch-time description of one single-RHS draw, copied to the device
// before each launch so that cached graphs need no parameter updates.
struct DrawDesc {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *omega;
    const double *z;
    const double *lambda;
    const double *eta;
    const double *delta;
    const double *rhs;     // solve mode: given right-hand side (else NULL)
    double *beta;          // output
    int64_t n, p, nnz;
    double tau, tol;
    int max_iter, stop_rule, refined, reliable_k;
    int df;                // double-float products: keep s (and omega) as float pairs too
    // unshrunk coefficients 0 .. q1-1 (Sec. S4.3): prior precision ud[j] = sigma_j^-2
    // (0: flat prior) and preconditioner variance um[j] = gamma_j^2 (device, q1 each)
    int q1;
    const double *ud, *um;
    // preconditioner M^-1 (device, p): the Jacobi 1 / diag(Phi), or NULL for the
    // prior preconditioner (the stop rule's weights either way)
    const double *mj;
    int warm;              // beta holds beta_0 on entry (Sec. S4.1)
};

// Device workspace of the single-RHS path (sizes grow on demand).
struct SingleWs {
    double *b, *r, *s64, *v64;    // p each
    float *s32;                   // p
    float2 *sdf;                  // p (s as double-float pairs, DF32 mode)
    void *u;                      // n doubles (aliased as n floats in FP32 modes)
    float *om32;                  // n
    double *om64;                 // n (float64 omega for the tiled float64 products)
    float2 *omdf;                 // n (omega as double-float pairs, DF32 mode)
    double *mj;                   // p (Jacobi preconditioner 1 / diag(Phi))
    double *partials;             // kMaxReduceBlocks * 4
    unsigned int *counters;       // 16
    CgScalars *sc;                // 1
    DrawDesc *desc;               // 1
};

struct LaunchShape {
    int csr_tpr = 32;     // threads per CSR row
    int csc_tpc = 32;     // threads per CSC column
    int blocks = 0;       // grid of the streaming kernels (0: SMs * blocks_per_sm)
    int threads = 256;
};

struct GraphKey {
    int64_t n, p;
    int precision, mode;  // mode: 0 draw, 1 solve
    bool operator<(const GraphKey &o) const {
        if (n != o.n) return n < o.n;
        if (p != o.p) return p < o.p;
        if (precision != o.precision) return precision < o.precision;
        return mode < o.mode;
    }
};

}  // namespace pcg

struct pcg_ctx {
    pcg_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    std::string last_error;

    // single-RHS workspace
    pcg::SingleWs ws{};
    int64_t cap_n = -1, cap_p = -1;
    pcg::DrawDesc *h_desc = nullptr;     // pinned host staging
    pcg::CgScalars *h_sc = nullptr;      // pinned host result
    std::map<pcg::GraphKey, cudaGraphExec_t> graphs;
    pcg::LaunchShape shape;

    // generic growable device buffers used by the batched / uneven / adjoint paths
    std::map<std::string, std::pair<void *, size_t>> bufs;
    std::map<std::string, std::pair<void *, size_t>> hbufs;   // pinned host
    std::map<std::string, cudaGraphExec_t> named_graphs;
    std::map<std::string, std::vector<int>> tuned;            // autotune results

    // measurement: per-kernel event timing (opt.profile) and launch counting
    struct ProfRec {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<double, int64_t>> prof;
    std::vector<std::string> prof_names;
    int64_t last_launches = 0;
    // shared-memory tiled products (on unless PCG_BETA_TILED=0 in the environment)
    bool tiled_enabled = true;
    // bank-aware entry order in the tiled plan (on unless PCG_BETA_BANK_PERMUTE=0)
    bool bank_permute = true;
    // tiled plans kept across calls (tiled.cu), per plan tag: the plan and the
    // key and design-content hash it was built for (PCG_BETA_PLAN_CACHE=0: off)
    std::map<std::string, std::vector<unsigned char>> plan_cache;
    bool plan_cache_enabled = true;
    // unshrunk coefficients set by pcg_set_unshrunk (context-owned device copies)
    int unshrunk_q1 = 0;
    double *unshrunk_d = nullptr, *unshrunk_m = nullptr;
};

namespace pcg {

// error helpers (capi.cu)
pcg_status set_error(pcg_ctx *ctx, pcg_status st, const std::string &msg);
pcg_status cuda_error(pcg_ctx *ctx, cudaError_t e, const char *what);
void *grow(pcg_ctx *ctx, const std::string &name, size_t bytes, cudaError_t *err);
void *grow_host(pcg_ctx *ctx, const std::string &name, size_t bytes, cudaError_t *err);
int grid_for(pcg_ctx *ctx, int threads, int per_sm);

#define PCG_CUDA_TRY(ctx, call)                                   \
    do {                                                          \
        cudaError_t e__ = (call);                                 \
        if (e__ != cudaSuccess) return ::pcg::cuda_error((ctx), e__, #call); \
    } while (0)

// per-kernel timing (capi.cu): bracket a launch with events when profiling
int prof_begin(pcg_ctx *ctx, const char *name);
void prof_end(pcg_ctx *ctx, int slot);
void prof_collect(pcg_ctx *ctx);   // after the stream has been synchronised

struct ProfScope {
    pcg_ctx *ctx;
    int slot;
    ProfScope(pcg_ctx *c, const char *name) : ctx(c), slot(c->opt.profile ? prof_begin(c, name) : -1) {}
    ~ProfScope() {
        if (slot >= 0) prof_end(ctx, slot);
    }
};
#define PCG_PROF(ctx, name, ...)                  \
    do {                                          \
        ::pcg::ProfScope ps__((ctx), (name));     \
        __VA_ARGS__;                              \
        ++(ctx)->last_launches;                   \
    } while (0)

// single-RHS path (single.cu)
pcg_status ensure_single_ws(pcg_ctx *ctx, int64_t n, int64_t p);
pcg_status run_single(pcg_ctx *ctx, const DrawDesc &d, int precision, int mode, int *iters,
                      double *resid);
pcg_status launch_build_rhs(pcg_ctx *ctx, const pcg_csc *X, const double *omega, const double *z,
                            const double *lambda, double tau, const double *eta,
                            const double *delta, double *b);
pcg_status launch_phi_mul(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                          const double *lambda, double tau, const double *v, double *out);
pcg_status launch_check_design(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc);

// batched path (batched.cu)
pcg_status run_batched(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, int nrhs,
                       const double *omega, const double *z, const double *lambda,
                       const double *tau, const double *eta, const double *delta, double tol,
                       int max_iter, double *beta, int *iters, double *resid, int *status);

// LSQR on the least-squares form (lsqr.cu)
pcg_status run_lsqr(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                    const double *z, const double *lambda, double tau, const double *eta,
                    const double *delta, double tol, int max_iter, double *beta, int *iters,
                    double *resid);

// the rest of the Gibbs cycle (gibbs.cu): tau, lambda, omega and the Gaussian
// vectors of Prop. 2.1 into context workspace (z, eta, delta)
pcg_status run_gibbs_updates(pcg_ctx *ctx, const pcg_csr *Xr, const double *y, uint64_t seed, uint32_t step,
                             double *omega, double *lambda, double *nu, double *tau, double *xi,
                             const double *beta, const double **z_out, const double **eta_out,
                             const double **delta_out);

// uneven batch (uneven.cu)
pcg_status run_uneven(pcg_ctx *ctx, int nprob, const pcg_problem *probs, double tol, int max_iter,
                      int *iters, double *resid, int *status);

// adjoint elementwise + products (adjoint.cu)
pcg_status launch_adjoint_terms(pcg_ctx *ctx, const pcg_csr *Xr, const double *omega,
                                const double *z, const double *lambda, double tau,
                                const double *eta, const double *delta, const double *beta,
                                const double *g, int mode, double *g_omega, double *g_loglambda,
                                double *g_logtau);

}  // namespace pcg
