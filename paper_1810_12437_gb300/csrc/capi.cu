// C ABI of the library (include/pcg_beta.h): context lifecycle, argument
// checks, the on-device design checker, and the entry points, which forward
// to the single-RHS, batched, uneven-batch and adjoint paths.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "device_common.cuh"
#include "internal.h"
#include "tiled.h"

namespace pcg {

pcg_status set_error(pcg_ctx *ctx, pcg_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

pcg_status cuda_error(pcg_ctx *ctx, cudaError_t e, const char *what) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error in %s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    cudaGetLastError();   // clear a sticky launch error so the context stays usable
    return set_error(ctx, PCG_CUDA, buf);
}

void *grow(pcg_ctx *ctx, const std::string &name, size_t bytes, cudaError_t *err) {
    *err = cudaSuccess;
    auto &slot = ctx->bufs[name];
    if (slot.second >= bytes && slot.first) return slot.first;
    cudaStreamSynchronize(ctx->stream);
    if (slot.first) cudaFree(slot.first);
    slot = {nullptr, 0};
    const size_t sz = std::max<size_t>(bytes, 256);
    void *p = nullptr;
    *err = cudaMalloc(&p, sz);
    if (*err != cudaSuccess) return nullptr;
    slot = {p, sz};
    return p;
}

void *grow_host(pcg_ctx *ctx, const std::string &name, size_t bytes, cudaError_t *err) {
    *err = cudaSuccess;
    auto &slot = ctx->hbufs[name];
    if (slot.second >= bytes && slot.first) return slot.first;
    cudaStreamSynchronize(ctx->stream);
    if (slot.first) cudaFreeHost(slot.first);
    slot = {nullptr, 0};
    const size_t sz = std::max<size_t>(bytes, 256);
    void *p = nullptr;
    *err = cudaMallocHost(&p, sz);
    if (*err != cudaSuccess) return nullptr;
    slot = {p, sz};
    return p;
}

int grid_for(pcg_ctx *ctx, int threads, int per_sm) {
    (void)threads;
    return std::min(ctx->num_sms * per_sm, kMaxReduceBlocks);
}

// ---------------------------------------------------------------------------
// design checker: pointer arrays valid, indices in range and strictly
// increasing per segment, and CSR and CSC holding the same entry set (by two
// order-independent 64-bit hash sums).  Stored indices are only compared,
// never used as addresses.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ void entry_hash(uint64_t i, uint64_t j, uint64_t &h1, uint64_t &h2) {
    const uint64_t a = mix64(i * 0x9e3779b97f4a7c15ull + j);
    h1 += a;
    h2 += mix64(a ^ 0x2545f4914f6cdd1dull);
}

// acc[0] = error flag, acc[1], acc[2] = hash sums, acc[3] = entries seen.
// seg_is_row: the segment index is the row (CSR) rather than the column (CSC).
__global__ void k_check(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                        int64_t nseg, int64_t nnz, int64_t limit, int seg_is_row,
                        unsigned long long *acc) {
    uint64_t h1 = 0, h2 = 0, cnt = 0;
    int bad = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = ptr[s], b = ptr[s + 1];
        if (s == 0 && a != 0) bad = 1;
        if (s == nseg - 1 && b != nnz) bad = 1;
        if (a < 0 || b < a || b > nnz) {
            bad = 1;
            continue;
        }
        int64_t prev = -1;
        for (int64_t k = a; k < b; ++k) {
            const int64_t v = idx[k];
            if (v < 0 || v >= limit || v <= prev) bad = 1;
            prev = v;
            if (seg_is_row) entry_hash((uint64_t)s, (uint64_t)v, h1, h2);
            else entry_hash((uint64_t)v, (uint64_t)s, h1, h2);
            ++cnt;
        }
    }
    if (bad) atomicOr((unsigned long long *)&acc[0], 1ull);
    atomicAdd(&acc[1], (unsigned long long)h1);
    atomicAdd(&acc[2], (unsigned long long)h2);
    atomicAdd(&acc[3], (unsigned long long)cnt);
}

pcg_status launch_check_design(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc) {
    cudaError_t e;
    unsigned long long *acc = (unsigned long long *)grow(ctx, "check", 8 * sizeof(unsigned long long), &e);
    if (!acc) return cuda_error(ctx, e, "allocating the check buffer");
    unsigned long long *h = (unsigned long long *)grow_host(ctx, "check_h", 8 * sizeof(unsigned long long), &e);
    if (!h) return cuda_error(ctx, e, "allocating the host check buffer");
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, 8 * sizeof(unsigned long long), ctx->stream));
    const int grid = grid_for(ctx, 256, 4);
    if (Xr->n > 0)
        PCG_PROF(ctx, "check_design", k_check<<<grid, 256, 0, ctx->stream>>>(Xr->row_ptr, Xr->col_idx, Xr->n, Xr->nnz, Xr->p, 1, acc));
    if (Xc->p > 0)
        PCG_PROF(ctx, "check_design", k_check<<<grid, 256, 0, ctx->stream>>>(Xc->col_ptr, Xc->row_idx, Xc->p, Xc->nnz, Xc->n, 0, acc + 4));
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(h, acc, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    if (h[0] || h[4]) return set_error(ctx, PCG_BADARG, "design: invalid pointers or indices (out of range, unsorted or repeated)");
    if ((uint64_t)h[3] != (uint64_t)Xr->nnz || (uint64_t)h[7] != (uint64_t)Xc->nnz)
        return set_error(ctx, PCG_BADARG, "design: entry count differs from nnz");
    if (h[1] != h[5] || h[2] != h[6])
        return set_error(ctx, PCG_BADARG, "design: CSR and CSC hold different entries");
    return PCG_OK;
}

static pcg_status check_shapes(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc) {
    if (!Xr || !Xc) return set_error(ctx, PCG_BADARG, "NULL design");
    if (Xr->n < 0 || Xr->p < 0 || Xr->nnz < 0) return set_error(ctx, PCG_BADARG, "negative size");
    if (Xr->n != Xc->n || Xr->p != Xc->p || Xr->nnz != Xc->nnz)
        return set_error(ctx, PCG_BADARG, "CSR and CSC sizes differ");
    if (Xr->n >= (int64_t)INT32_MAX || Xr->p >= (int64_t)INT32_MAX)
        return set_error(ctx, PCG_BADARG, "n and p must fit int32 indices");
    if ((Xr->n > 0 && !Xr->row_ptr) || (Xr->p > 0 && !Xc->col_ptr))
        return set_error(ctx, PCG_BADARG, "NULL pointer array");
    if (Xr->nnz > 0 && (!Xr->col_idx || !Xc->row_idx))
        return set_error(ctx, PCG_BADARG, "NULL index array");
    return PCG_OK;
}

static bool bad_scalar(double x) { return !(x > 0.0) || !isfinite(x); }

// ---------------------------------------------------------------------------
// per-kernel timing
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(pcg_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int prof_begin(pcg_ctx *ctx, const char *name) {
    pcg_ctx::ProfRec r{name, take_event(ctx), take_event(ctx)};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, ctx->stream);
    ctx->prof_pending.push_back(r);
    return (int)ctx->prof_pending.size() - 1;
}

void prof_end(pcg_ctx *ctx, int slot) {
    if (slot >= 0 && slot < (int)ctx->prof_pending.size())
        cudaEventRecord(ctx->prof_pending[slot].b, ctx->stream);
}

void prof_collect(pcg_ctx *ctx) {
    for (auto &r : ctx->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto &acc = ctx->prof[r.name];
            acc.first += ms;
            acc.second += 1;
        } else {
            cudaGetLastError();
        }
        ctx->event_pool.push_back(r.a);
        ctx->event_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
}

}  // namespace pcg

using namespace pcg;

// um[j] = gamma_j^2 and ud[j] = prior precision; *bad = 1 if some prior
// precision is negative or not finite, or some gamma is not positive and finite
__global__ void k_unshrunk(const double *__restrict__ prec, const double *__restrict__ gamma, int q1,
                           double *__restrict__ ud, double *__restrict__ um, int *__restrict__ bad) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q1; j += gridDim.x * blockDim.x) {
        const double a = prec[j], g = gamma[j];
        if (!(a >= 0.0) || !isfinite(a) || !(g > 0.0) || !isfinite(g)) *bad = 1;
        ud[j] = a;
        um[j] = g * g;
    }
}

extern "C" {

int pcg_tiled_plan_applies(int64_t n, int64_t p, int64_t nnz, int precision, int rhs_group,
                           int *col_tiles, int *row_strips) {
    if (precision < 0 || precision > PCG_PREC_FX64 || rhs_group <= 0) return 0;
    const int vsize = pcg::tiled_vtype(precision) == pcg::kVtF32 ? 4 : 8;
    int Wc = 0, Tc = 0, Wr = 0, Tr = 0;
    if (!pcg::tiled_geometry(n, p, nnz, rhs_group, vsize, &Wc, &Tc, &Wr, &Tr)) return 0;
    if (col_tiles) *col_tiles = Tc;
    if (row_strips) *row_strips = Tr;
    return 1;
}

pcg_status pcg_options_default(pcg_options *opt) {
    if (!opt) return PCG_BADARG;
    opt->precision = PCG_PREC_DF32;
    opt->reliable_k = 50;
    opt->stop_rule = PCG_STOP_PAPER_RMS;
    opt->use_graph = 1;
    opt->autotune_cache = nullptr;
    opt->profile = 0;
    opt->idle_limit_s = 2.0;
    opt->preconditioner = PCG_PRECOND_PRIOR;
    opt->warm_start = 0;
    return PCG_OK;
}

pcg_status pcg_ctx_create(pcg_ctx **out, const pcg_options *opt, void *stream) {
    if (!out) return PCG_BADARG;
    *out = nullptr;
    pcg_ctx *ctx = new pcg_ctx();
    if (opt) ctx->opt = *opt;
    else pcg_options_default(&ctx->opt);
    if (ctx->opt.precision < 0 || ctx->opt.precision > PCG_PREC_FX64 || ctx->opt.stop_rule < 0 ||
        ctx->opt.stop_rule > 1 || ctx->opt.reliable_k < 0 ||
        !(ctx->opt.idle_limit_s >= 1e-6 && ctx->opt.idle_limit_s <= 3600.0) ||
        (ctx->opt.preconditioner != PCG_PRECOND_PRIOR && ctx->opt.preconditioner != PCG_PRECOND_JACOBI) ||
        (ctx->opt.warm_start != 0 && ctx->opt.warm_start != 1)) {
        delete ctx;
        return PCG_BADARG;
    }
    ctx->stream = (cudaStream_t)stream;
    const char *tiled = getenv("PCG_BETA_TILED");
    ctx->tiled_enabled = !(tiled && tiled[0] == '0');
    const char *perm = getenv("PCG_BETA_BANK_PERMUTE");
    ctx->bank_permute = !(perm && perm[0] == '0');
    const char *pcache = getenv("PCG_BETA_PLAN_CACHE");
    ctx->plan_cache_enabled = !(pcache && pcache[0] == '0');
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return PCG_CUDA;
    }
    *out = ctx;
    return PCG_OK;
}

void pcg_ctx_destroy(pcg_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &g : ctx->named_graphs) cudaGraphExecDestroy(g.second);
    if (ctx->ws.b) cudaFree(ctx->ws.b);
    if (ctx->ws.u) cudaFree(ctx->ws.u);
    for (auto &b : ctx->bufs)
        if (b.second.first) cudaFree(b.second.first);
    for (auto &b : ctx->hbufs)
        if (b.second.first) cudaFreeHost(b.second.first);
    for (auto &r : ctx->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
    if (ctx->h_sc) cudaFreeHost(ctx->h_sc);
    delete ctx;
}

const char *pcg_last_error(const pcg_ctx *ctx) {
    return ctx ? ctx->last_error.c_str() : "NULL context";
}

pcg_status pcg_set_unshrunk(pcg_ctx *ctx, int q1, const double *prior_prec, const double *precond_scale) {
    if (!ctx) return PCG_BADARG;
    if (q1 < 0) return set_error(ctx, PCG_BADARG, "negative count of unshrunk coefficients");
    if (q1 == 0) {
        ctx->unshrunk_q1 = 0;
        return PCG_OK;
    }
    if (!prior_prec || !precond_scale) return set_error(ctx, PCG_BADARG, "NULL vector");
    cudaError_t e;
    double *ud = (double *)grow(ctx, "unshrunk_d", sizeof(double) * (size_t)q1, &e);
    if (!ud) return cuda_error(ctx, e, "allocating the unshrunk coefficients");
    double *um = (double *)grow(ctx, "unshrunk_m", sizeof(double) * (size_t)q1, &e);
    if (!um) return cuda_error(ctx, e, "allocating the unshrunk coefficients");
    int *dbad = (int *)grow(ctx, "unshrunk_bad", sizeof(int), &e);
    if (!dbad) return cuda_error(ctx, e, "allocating the unshrunk coefficients");
    int *hbad = (int *)grow_host(ctx, "unshrunk_bad", sizeof(int), &e);
    if (!hbad) return cuda_error(ctx, e, "allocating the unshrunk coefficients");
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(dbad, 0, sizeof(int), ctx->stream));
    k_unshrunk<<<std::min(1024, (q1 + 255) / 256), 256, 0, ctx->stream>>>(prior_prec, precond_scale, q1, ud, um,
                                                                         dbad);
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (*hbad) {
        ctx->unshrunk_q1 = 0;
        return set_error(ctx, PCG_BADARG, "prior precisions must be >= 0 and gammas > 0, all finite");
    }
    ctx->unshrunk_q1 = q1;
    ctx->unshrunk_d = ud;
    ctx->unshrunk_m = um;
    return PCG_OK;
}

pcg_status pcg_check_design(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc) {
    if (!ctx) return PCG_BADARG;
    ctx->last_launches = 0;
    pcg_status st = check_shapes(ctx, Xr, Xc);
    if (st != PCG_OK) return st;
    return launch_check_design(ctx, Xr, Xc);
}

pcg_status pcg_build_rhs(pcg_ctx *ctx, const pcg_csc *X, const double *omega, const double *z,
                         const double *lambda, double tau, const double *eta,
                         const double *delta, double *b) {
    if (!ctx || !X) return PCG_BADARG;
    ctx->last_launches = 0;
    if (X->n < 0 || X->p < 0 || X->nnz < 0) return set_error(ctx, PCG_BADARG, "negative size");
    if (bad_scalar(tau)) return set_error(ctx, PCG_BADARG, "tau must be positive and finite");
    if (X->p == 0) return PCG_OK;
    if ((X->n > 0 && (!omega || !z || !eta)) || !lambda || !delta || !b || !X->col_ptr)
        return set_error(ctx, PCG_BADARG, "NULL vector");
    return launch_build_rhs(ctx, X, omega, z, lambda, tau, eta, delta, b);
}

pcg_status pcg_phi_mul(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                       const double *lambda, double tau, const double *v, double *out) {
    if (!ctx) return PCG_BADARG;
    ctx->last_launches = 0;
    pcg_status st = check_shapes(ctx, Xr, Xc);
    if (st != PCG_OK) return st;
    if (bad_scalar(tau)) return set_error(ctx, PCG_BADARG, "tau must be positive and finite");
    if (Xr->p == 0) return PCG_OK;
    if ((Xr->n > 0 && !omega) || !lambda || !v || !out) return set_error(ctx, PCG_BADARG, "NULL vector");
    return launch_phi_mul(ctx, Xr, Xc, omega, lambda, tau, v, out);
}

static pcg_status draw_or_solve(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc,
                                const double *omega, const double *z, const double *lambda,
                                double tau, const double *eta, const double *delta,
                                const double *rhs, double tol, int max_iter, double *beta,
                                int *iters, double *resid) {
    if (!ctx) return PCG_BADARG;
    ctx->last_launches = 0;
    if (!iters || !resid) return set_error(ctx, PCG_BADARG, "NULL host output");
    *iters = 0;
    *resid = 0.0;
    pcg_status st = check_shapes(ctx, Xr, Xc);
    if (st != PCG_OK) return st;
    if (bad_scalar(tau)) return set_error(ctx, PCG_BADARG, "tau must be positive and finite");
    if (!(tol >= 0.0) || max_iter < 0) return set_error(ctx, PCG_BADARG, "tol >= 0 and max_iter >= 0 required");
    if (Xr->p == 0) return PCG_OK;
    if ((Xr->n > 0 && !omega) || !lambda || !beta) return set_error(ctx, PCG_BADARG, "NULL vector");
    if (!rhs && (!delta || (Xr->n > 0 && (!z || !eta))))
        return set_error(ctx, PCG_BADARG, "NULL vector");
    DrawDesc d{};
    d.row_ptr = Xr->row_ptr;
    d.col_idx = Xr->col_idx;
    d.col_ptr = Xc->col_ptr;
    d.row_idx = Xc->row_idx;
    d.omega = omega;
    d.z = z;
    d.lambda = lambda;
    d.eta = eta;
    d.delta = delta;
    d.rhs = rhs;
    d.beta = beta;
    d.n = Xr->n;
    d.p = Xr->p;
    d.nnz = Xr->nnz;
    d.tau = tau;
    d.tol = tol;
    d.max_iter = max_iter;
    d.stop_rule = ctx->opt.stop_rule;
    d.warm = ctx->opt.warm_start;
    return run_single(ctx, d, ctx->opt.precision, rhs ? 1 : 0, iters, resid);
}

pcg_status pcg_draw_beta(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                         const double *z, const double *lambda, double tau, const double *eta,
                         const double *delta, double tol, int max_iter, double *beta, int *iters,
                         double *resid) {
    return draw_or_solve(ctx, Xr, Xc, omega, z, lambda, tau, eta, delta, nullptr, tol, max_iter,
                         beta, iters, resid);
}

pcg_status pcg_draw_beta_lsqr(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                              const double *z, const double *lambda, double tau, const double *eta,
                              const double *delta, double tol, int max_iter, double *beta, int *iters,
                              double *resid) {
    if (!ctx) return PCG_BADARG;
    ctx->last_launches = 0;
    if (!iters || !resid) return set_error(ctx, PCG_BADARG, "NULL host output");
    *iters = 0;
    *resid = 0.0;
    pcg_status st = check_shapes(ctx, Xr, Xc);
    if (st != PCG_OK) return st;
    if (bad_scalar(tau)) return set_error(ctx, PCG_BADARG, "tau must be positive and finite");
    if (!(tol >= 0.0) || max_iter < 0) return set_error(ctx, PCG_BADARG, "tol >= 0 and max_iter >= 0 required");
    if (ctx->unshrunk_q1 > 0 || ctx->opt.preconditioner != PCG_PRECOND_PRIOR || ctx->opt.warm_start)
        return set_error(ctx, PCG_BADARG, "LSQR runs the shrinkage model's prior preconditioner from 0");
    if (Xr->p == 0) return PCG_OK;
    if ((Xr->n > 0 && (!omega || !z || !eta)) || !lambda || !delta || !beta)
        return set_error(ctx, PCG_BADARG, "NULL vector");
    return run_lsqr(ctx, Xr, Xc, omega, z, lambda, tau, eta, delta, tol, max_iter, beta, iters, resid);
}

pcg_status pcg_gibbs_step(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *y, uint64_t seed,
                          uint32_t step, double *omega, double *lambda, double *nu, double *tau, double *xi,
                          double *beta, double tol, int max_iter, int *iters, double *resid) {
    if (!ctx) return PCG_BADARG;
    ctx->last_launches = 0;
    if (!iters || !resid || !tau || !xi) return set_error(ctx, PCG_BADARG, "NULL host argument");
    *iters = 0;
    *resid = 0.0;
    pcg_status st = check_shapes(ctx, Xr, Xc);
    if (st != PCG_OK) return st;
    if (bad_scalar(*tau) || bad_scalar(*xi)) return set_error(ctx, PCG_BADARG, "tau and xi must be positive and finite");
    if (!(tol >= 0.0) || max_iter < 0) return set_error(ctx, PCG_BADARG, "tol >= 0 and max_iter >= 0 required");
    if (ctx->unshrunk_q1 > 0)
        return set_error(ctx, PCG_BADARG, "the Gibbs step puts every coefficient under the horseshoe prior");
    if (Xr->p == 0) return PCG_OK;
    if ((Xr->n > 0 && (!y || !omega)) || !lambda || !nu || !beta) return set_error(ctx, PCG_BADARG, "NULL vector");
    const double *z = nullptr, *eta = nullptr, *delta = nullptr;
    st = run_gibbs_updates(ctx, Xr, y, seed, step, omega, lambda, nu, tau, xi, beta, &z, &eta, &delta);
    if (st != PCG_OK) return st;
    const int64_t upd = ctx->last_launches;
    st = pcg_draw_beta(ctx, Xr, Xc, omega, z, lambda, *tau, eta, delta, tol, max_iter, beta, iters, resid);
    ctx->last_launches += upd;
    return st;
}

pcg_status pcg_solve(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                     const double *lambda, double tau, const double *rhs, double tol, int max_iter,
                     double *x, int *iters, double *resid) {
    if (!rhs && ctx) return set_error(ctx, PCG_BADARG, "NULL right-hand side");
    return draw_or_solve(ctx, Xr, Xc, omega, nullptr, lambda, tau, nullptr, nullptr, rhs, tol,
                         max_iter, x, iters, resid);
}

pcg_status pcg_draw_beta_batched(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, int nrhs,
                                 const double *omega, const double *z, const double *lambda,
                                 const double *tau, const double *eta, const double *delta,
                                 double tol, int max_iter, double *beta, int *iters, double *resid,
                                 int *status) {
    if (!ctx) return PCG_BADARG;
    ctx->last_launches = 0;
    pcg_status st = check_shapes(ctx, Xr, Xc);
    if (st != PCG_OK) return st;
    if (nrhs < 1 || nrhs > kMaxBatch) return set_error(ctx, PCG_BADARG, "nrhs must be in [1, 32]");
    if (ctx->opt.preconditioner != PCG_PRECOND_PRIOR || ctx->opt.warm_start)
        return set_error(ctx, PCG_BADARG, "the batched path runs the prior preconditioner from beta_0 = 0");
    if (!iters || !resid || !status) return set_error(ctx, PCG_BADARG, "NULL host output");
    if (!(tol >= 0.0) || max_iter < 0) return set_error(ctx, PCG_BADARG, "tol >= 0 and max_iter >= 0 required");
    for (int r = 0; r < nrhs; ++r) {
        iters[r] = 0;
        resid[r] = 0.0;
        status[r] = PCG_OK;
    }
    if (Xr->p == 0) return PCG_OK;
    if ((Xr->n > 0 && (!omega || !z || !eta)) || !lambda || !tau || !delta || !beta)
        return set_error(ctx, PCG_BADARG, "NULL vector");
    return run_batched(ctx, Xr, Xc, nrhs, omega, z, lambda, tau, eta, delta, tol, max_iter, beta,
                       iters, resid, status);
}

pcg_status pcg_draw_beta_uneven(pcg_ctx *ctx, int nprob, const pcg_problem *probs, double tol,
                                int max_iter, int *iters, double *resid, int *status) {
    if (!ctx) return PCG_BADARG;
    ctx->last_launches = 0;
    if (nprob < 0 || (nprob > 0 && (!probs || !iters || !resid || !status)))
        return set_error(ctx, PCG_BADARG, "bad problem list");
    if (!(tol >= 0.0) || max_iter < 0) return set_error(ctx, PCG_BADARG, "tol >= 0 and max_iter >= 0 required");
    if (ctx->unshrunk_q1 > 0)
        return set_error(ctx, PCG_BADARG, "the uneven batch takes no unshrunk coefficients (pcg_set_unshrunk)");
    if (ctx->opt.preconditioner != PCG_PRECOND_PRIOR || ctx->opt.warm_start)
        return set_error(ctx, PCG_BADARG, "the uneven batch runs the prior preconditioner from beta_0 = 0");
    for (int q = 0; q < nprob; ++q) {
        pcg_status st = check_shapes(ctx, &probs[q].X_csr, &probs[q].X_csc);
        if (st != PCG_OK) return st;
        if (bad_scalar(probs[q].tau)) return set_error(ctx, PCG_BADARG, "tau must be positive and finite");
        if (probs[q].X_csr.p > 0 &&
            ((probs[q].X_csr.n > 0 && (!probs[q].omega || !probs[q].z || !probs[q].eta)) ||
             !probs[q].lambda || !probs[q].delta || !probs[q].beta))
            return set_error(ctx, PCG_BADARG, "NULL vector in a problem");
    }
    if (nprob == 0) return PCG_OK;
    return run_uneven(ctx, nprob, probs, tol, max_iter, iters, resid, status);
}

pcg_status pcg_adjoint(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                       const double *z, const double *lambda, double tau, const double *eta,
                       const double *delta, const double *beta, const double *grad_beta, int mode,
                       double tol, int max_iter, double *g_b, double *g_omega, double *g_loglambda,
                       double *g_logtau, int *iters, double *resid) {
    if (!ctx) return PCG_BADARG;
    if (mode != PCG_ADJ_SOLVE && mode != PCG_ADJ_DRAW) return set_error(ctx, PCG_BADARG, "bad adjoint mode");
    if (ctx->unshrunk_q1 > 0)
        return set_error(ctx, PCG_BADARG, "the adjoint takes no unshrunk coefficients (pcg_set_unshrunk)");
    if (ctx->opt.warm_start)
        return set_error(ctx, PCG_BADARG, "the adjoint's solve starts from 0 (warm_start must be off)");
    if (!g_logtau || !iters || !resid) return set_error(ctx, PCG_BADARG, "NULL host output");
    *g_logtau = 0.0;
    pcg_status st = check_shapes(ctx, Xr, Xc);
    if (st != PCG_OK) return st;
    if (Xr->p == 0) return PCG_OK;
    if (!beta || !grad_beta || !g_b || !g_loglambda || (Xr->n > 0 && (!g_omega || !omega)))
        return set_error(ctx, PCG_BADARG, "NULL vector");
    if (mode == PCG_ADJ_DRAW && (!delta || (Xr->n > 0 && (!z || !eta))))
        return set_error(ctx, PCG_BADARG, "DRAW mode needs z, eta and delta");
    // the second prior-preconditioned CG solve: Phi g = grad_beta
    ctx->last_launches = 0;
    st = draw_or_solve(ctx, Xr, Xc, omega, nullptr, lambda, tau, nullptr, nullptr, grad_beta, tol,
                       max_iter, g_b, iters, resid);
    // a solve stopped by max_iter still yields the gradient of its last iterate
    if (st != PCG_OK && st != PCG_MAXITER) return st;
    const pcg_status solve_st = st;
    const int64_t solve_launches = ctx->last_launches;
    st = launch_adjoint_terms(ctx, Xr, omega, z, lambda, tau, eta, delta, beta, g_b, mode,
                                g_omega, g_loglambda, g_logtau);
    ctx->last_launches += solve_launches;
    return st != PCG_OK ? st : solve_st;
}

int pcg_profile_count(const pcg_ctx *ctx) { return ctx ? (int)ctx->prof.size() : 0; }

pcg_status pcg_profile_entry(const pcg_ctx *ctx, int i, const char **name, double *total_ms,
                             int64_t *launches) {
    if (!ctx || i < 0 || i >= (int)ctx->prof.size() || !name || !total_ms || !launches)
        return PCG_BADARG;
    auto it = ctx->prof.begin();
    std::advance(it, i);
    *name = it->first.c_str();
    *total_ms = it->second.first;
    *launches = it->second.second;
    return PCG_OK;
}

void pcg_profile_reset(pcg_ctx *ctx) {
    if (ctx) ctx->prof.clear();
}

int64_t pcg_last_kernel_launches(const pcg_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

}  // extern "C"
