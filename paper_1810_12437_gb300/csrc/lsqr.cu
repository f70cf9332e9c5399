// LSQR (Paige and Saunders 1982) on the least-squares form of the draw
// (Sec. S7.1, Eq. S6): Phi = Xt^T Xt with Xt = [Omega^1/2 X; tau^-1 Lambda^-1],
// so beta minimises ||Xt beta - bt|| for bt = [Omega^1/2 z + eta; delta], the
// same b of Eq. 2.3 (Xt^T bt = b).  LSQR runs on A = Xt D, D = diag(tau lambda)
// (the prior preconditioner of Sec. 2.4 applied on the right), which makes
// A = [Omega^1/2 X D; I] and A^T (bt - A x) = tau lambda (.) (b - Phi beta):
// LSQR's own estimate of ||A^T r|| is the prior-preconditioned residual of
// Eq. S2, so it stops under the same rule as the CG path.  Float64 throughout.
//
// The Golub-Kahan vectors are kept unnormalised (u~ = beta u, v~ = alpha v)
// and the scales carried as scalars, so one iteration is two fused kernels:
//   k_l_rows  rows i:  u~top_i <- sqrt(omega_i) (X y)_i / alpha - (alpha/beta) u~top_i,
//                      q~_i = sqrt(omega_i) u~top_i  (the vector the CSC pass gathers);
//             cols j:  u~bot_j <- v~_j / alpha - (alpha/beta) u~bot_j, plus the x and w
//                      updates left pending by the previous iteration's rotation;
//             beta_{k+1} = ||u~||                    (y = tau lambda (.) v~)
//   k_l_cols  cols j:  v~_j <- (tau lambda_j (X^T q~)_j + u~bot_j) / beta - beta v~_j / alpha,
//                      y_j = tau lambda_j v~_j;  alpha_{k+1} = ||v~||; the last block
//                      applies the plane rotation and the stop test.
// A final kernel applies the last pending x update and writes beta = D x.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>

#include "device_common.cuh"
#include "internal.h"

namespace pcg {

struct LsqrDesc {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *omega, *z, *lambda, *eta, *delta;
    double *beta;
    int64_t n, p;
    double tau, tol;
    int max_iter, stop_rule;
};

struct LsqrScalars {
    double alpha, beta;        // current Golub-Kahan scales
    double rhobar, phibar;     // rotation state
    double phi_rho;            // phi_k / rho_k: pending x += phi_rho w
    double theta_rho;          // theta_{k+1} / rho_k: pending w = v - theta_rho w
    double ref;                // ||A^T bt|| = alpha_1 beta_1 = ||tau lambda (.) b||
    double resid;              // stop quantity
    int iter, status, done, pending;   // pending: an x update waits (k >= 1)
};

struct LsqrWs {
    double *ut, *qt, *sqw;     // n: u~ top, sqrt(omega) (.) u~ top, sqrt(omega)
    double *ub, *vt, *y, *w, *x;   // p
    double *partials;          // kMaxReduceBlocks
    unsigned *counters;        // 4
    LsqrScalars *sc;
    LsqrDesc *desc;
};

__device__ __forceinline__ double lsqr_stop(const LsqrDesc *d, double arnorm, double ref) {
    if (d->stop_rule == PCG_STOP_RELATIVE) return ref > 0.0 ? arnorm / ref : 0.0;
    return d->p > 0 ? sqrt(arnorm * arnorm / (double)d->p) : 0.0;
}

// Start: u~ = bt = [sqrt(omega) z + eta; delta], beta_1 = ||bt||.
__global__ void __launch_bounds__(256) k_l_start(const LsqrDesc *__restrict__ d, LsqrWs ws) {
    __shared__ double red[32];
    __shared__ double sums[1];
    const int64_t n = d->n, p = d->p;
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n + p;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n) {
            const double so = sqrt(d->omega[t]);
            const double u = so * d->z[t] + d->eta[t];
            ws.sqw[t] = so;
            ws.ut[t] = u;
            ws.qt[t] = so * u;
            acc += u * u;
        } else {
            const int64_t j = t - n;
            const double u = d->delta[j];
            ws.ub[j] = u;
            ws.x[j] = 0.0;
            acc += u * u;
        }
    }
    const double tot = block_sum(acc, red);
    if (grid_reduce<1>(&tot, ws.partials, ws.counters + 0, sums, red) && threadIdx.x == 0) {
        LsqrScalars *sc = ws.sc;
        sc->beta = sqrt(sums[0]);
        sc->alpha = 0.0;
        sc->iter = 0;
        sc->pending = 0;
        sc->done = 0;
        sc->status = kRunning;
    }
}

// Iteration k, rows and the p-part (see the file comment).  first: the
// first pass after the start, where w = v_1 and no x update is pending.
template <int G>
__global__ void __launch_bounds__(256) k_l_rows(const LsqrDesc *__restrict__ d, LsqrWs ws) {
    __shared__ double red[32];
    __shared__ double sums[1];
    const LsqrScalars *sc = ws.sc;
    if (*(volatile const int *)&sc->done) return;
    const int64_t n = d->n, p = d->p;
    const double alpha = sc->alpha, ab = sc->alpha / sc->beta, ia = 1.0 / sc->alpha;
    const bool pend = sc->pending != 0;
    const double phi_rho = sc->phi_rho, theta_rho = sc->theta_rho;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    double acc2 = 0.0;
    for (int64_t base = warp * gpw; base < n; base += nwarps * gpw) {
        const int64_t i = base + sub;
        double xy = 0.0;
        if (i < n) xy = segment_partial<G, double>(d->col_idx, d->row_ptr[i], d->row_ptr[i + 1], ws.y, lane);
        xy = group_sum<G>(xy);
        if (i < n && lane == 0) {
            const double so = ws.sqw[i];
            const double u = so * xy * ia - ab * ws.ut[i];
            ws.ut[i] = u;
            ws.qt[i] = so * u;
            acc2 += u * u;
        }
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double v = ws.vt[j] * ia;
        const double u = v - ab * ws.ub[j];
        ws.ub[j] = u;
        acc2 += u * u;
        if (pend) {
            const double w = ws.w[j];
            ws.x[j] += phi_rho * w;
            ws.w[j] = v - theta_rho * w;
        } else {
            ws.w[j] = v;
        }
    }
    (void)alpha;
    const double tot = block_sum(acc2, red);
    if (grid_reduce<1>(&tot, ws.partials, ws.counters + 1, sums, red) && threadIdx.x == 0)
        ws.sc->beta = sqrt(sums[0]);
}

// Iteration k, columns: v~ = A^T u - beta v, alpha_{k+1}, rotation, stop test.
// first: the start's A^T u_1 (no - beta v term), which sets alpha_1 and the
// rotation's initial state.
template <int G>
__global__ void __launch_bounds__(256) k_l_cols(const LsqrDesc *__restrict__ d, LsqrWs ws, int first,
                                                cudaGraphConditionalHandle h_while, int use_cond) {
    __shared__ double red[32];
    __shared__ double sums[1];
    LsqrScalars *sc = ws.sc;
    if (*(volatile const int *)&sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_while, 0u);
        return;
    }
    const int64_t p = d->p;
    const double beta = sc->beta, ib = sc->beta > 0.0 ? 1.0 / sc->beta : 0.0;
    const double ba = first ? 0.0 : sc->beta / sc->alpha;
    const double tau = d->tau;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    double acc2 = 0.0;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        double z = 0.0;
        if (j < p) z = segment_partial<G, double>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], ws.qt, lane);
        z = group_sum<G>(z);
        if (j < p && lane == 0) {
            const double dj = tau * d->lambda[j];
            const double v = (dj * z + ws.ub[j]) * ib - ba * ws.vt[j];
            ws.vt[j] = v;
            ws.y[j] = dj * v;
            acc2 += v * v;
        }
    }
    (void)beta;
    const double tot = block_sum(acc2, red);
    if (grid_reduce<1>(&tot, ws.partials, ws.counters + 2, sums, red) && threadIdx.x == 0) {
        const double alpha = sqrt(sums[0]);
        const double bet = sc->beta;
        if (first) {
            sc->alpha = alpha;
            sc->rhobar = alpha;
            sc->phibar = bet;
            sc->ref = alpha * bet;
            sc->resid = lsqr_stop(d, sc->ref, sc->ref);
            if (!isfinite(sc->resid) || !isfinite(alpha) || !isfinite(bet)) {
                sc->status = PCG_NONFINITE;
                sc->done = 1;
            } else if (sc->resid <= d->tol) {
                sc->status = PCG_OK;
                sc->done = 1;
            } else if (!(alpha > 0.0) || !(bet > 0.0)) {
                sc->status = PCG_BREAKDOWN;
                sc->done = 1;
            } else if (d->max_iter <= 0) {
                sc->status = PCG_MAXITER;
                sc->done = 1;
            }
        } else {
            const double rho = sqrt(sc->rhobar * sc->rhobar + bet * bet);
            const double c = sc->rhobar / rho, s = bet / rho;
            const double theta = s * alpha;
            sc->rhobar = -c * alpha;
            const double phi = c * sc->phibar;
            sc->phibar = s * sc->phibar;
            sc->phi_rho = phi / rho;
            sc->theta_rho = theta / rho;
            sc->alpha = alpha;
            sc->pending = 1;
            sc->iter += 1;
            sc->resid = lsqr_stop(d, sc->phibar * alpha * fabs(c), sc->ref);
            if (!isfinite(sc->resid) || !isfinite(rho)) {
                sc->status = PCG_NONFINITE;
                sc->done = 1;
            } else if (sc->resid <= d->tol) {
                sc->status = PCG_OK;
                sc->done = 1;
            } else if (sc->iter >= d->max_iter) {
                sc->status = PCG_MAXITER;
                sc->done = 1;
            } else if (!(alpha > 0.0)) {
                // v~ vanished: the Krylov space is exhausted, x is the solution
                sc->status = PCG_OK;
                sc->done = 1;
            }
        }
        if (use_cond) cudaGraphSetConditional(h_while, sc->done ? 0u : 1u);
    }
}

// The last pending x update, then beta = D x.
__global__ void __launch_bounds__(256) k_l_finish(const LsqrDesc *__restrict__ d, LsqrWs ws) {
    const LsqrScalars *sc = ws.sc;
    const bool pend = sc->pending != 0;
    const double phi_rho = sc->phi_rho;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d->p;
         j += (int64_t)gridDim.x * blockDim.x) {
        double x = ws.x[j];
        if (pend) x += phi_rho * ws.w[j];
        d->beta[j] = d->tau * d->lambda[j] * x;
    }
}

// ===========================================================================
// host side
// ===========================================================================

static int lsqr_group(double mean_len) {
    return mean_len < 6 ? 4 : mean_len < 20 ? 8 : mean_len < 56 ? 16 : 32;
}

// launches kernel template K at the lane-group width G
#define PCG_LSQR_G(G, K, ...)                                  \
    switch (G) {                                               \
        case 4: K<4> __VA_ARGS__; break;                       \
        case 8: K<8> __VA_ARGS__; break;                       \
        case 16: K<16> __VA_ARGS__; break;                     \
        default: K<32> __VA_ARGS__; break;                     \
    }

static void *rows_ptr(int G) {
    switch (G) {
        case 4: return (void *)k_l_rows<4>;
        case 8: return (void *)k_l_rows<8>;
        case 16: return (void *)k_l_rows<16>;
        default: return (void *)k_l_rows<32>;
    }
}
static void *cols_ptr(int G) {
    switch (G) {
        case 4: return (void *)k_l_cols<4>;
        case 8: return (void *)k_l_cols<8>;
        case 16: return (void *)k_l_cols<16>;
        default: return (void *)k_l_cols<32>;
    }
}

static pcg_status lsqr_workspace(pcg_ctx *ctx, int64_t n, int64_t p, LsqrWs *ws) {
    cudaError_t e;
    const size_t nn = (size_t)std::max<int64_t>(n, 1), np = (size_t)std::max<int64_t>(p, 1);
    double *bn = (double *)grow(ctx, "lsqr:n", sizeof(double) * 3 * nn, &e);
    double *bp = (double *)grow(ctx, "lsqr:p", sizeof(double) * 5 * np, &e);
    double *part = (double *)grow(ctx, "lsqr:partials", sizeof(double) * kMaxReduceBlocks, &e);
    unsigned *cnt = (unsigned *)grow(ctx, "lsqr:counters", sizeof(unsigned) * 4, &e);
    LsqrScalars *sc = (LsqrScalars *)grow(ctx, "lsqr:scalars", sizeof(LsqrScalars), &e);
    LsqrDesc *desc = (LsqrDesc *)grow(ctx, "lsqr:desc", sizeof(LsqrDesc), &e);
    if (!bn || !bp || !part || !cnt || !sc || !desc) return cuda_error(ctx, e, "allocating the LSQR workspace");
    ws->ut = bn;
    ws->qt = bn + nn;
    ws->sqw = bn + 2 * nn;
    ws->ub = bp;
    ws->vt = bp + np;
    ws->y = bp + 2 * np;
    ws->w = bp + 3 * np;
    ws->x = bp + 4 * np;
    ws->partials = part;
    ws->counters = cnt;
    ws->sc = sc;
    ws->desc = desc;
    return PCG_OK;
}

pcg_status run_lsqr(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                    const double *z, const double *lambda, double tau, const double *eta,
                    const double *delta, double tol, int max_iter, double *beta, int *iters,
                    double *resid) {
    LsqrWs ws{};
    pcg_status st = lsqr_workspace(ctx, Xr->n, Xr->p, &ws);
    if (st != PCG_OK) return st;
    cudaError_t e;
    LsqrDesc *hd = (LsqrDesc *)grow_host(ctx, "lsqr:hdesc", sizeof(LsqrDesc), &e);
    LsqrScalars *hs = (LsqrScalars *)grow_host(ctx, "lsqr:hsc", sizeof(LsqrScalars), &e);
    if (!hd || !hs) return cuda_error(ctx, e, "allocating pinned staging");
    LsqrDesc d{Xr->row_ptr, Xr->col_idx, Xc->col_ptr, Xc->row_idx, omega, z, lambda, eta, delta, beta,
               Xr->n, Xr->p, tau, tol, max_iter, ctx->opt.stop_rule};
    *hd = d;
    cudaStream_t s = ctx->stream;
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ws.desc, hd, sizeof(LsqrDesc), cudaMemcpyHostToDevice, s));
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(ws.counters, 0, sizeof(unsigned) * 4, s));
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(ws.sc, 0, sizeof(LsqrScalars), s));
    const int Gr = lsqr_group(d.n > 0 ? (double)Xr->nnz / d.n : 1.0);
    const int Gc = lsqr_group(d.p > 0 ? (double)Xr->nnz / d.p : 1.0);
    const int grid = std::min(ctx->num_sms * 8, kMaxReduceBlocks);
    const int grid_v = (int)std::max<int64_t>(1, std::min<int64_t>((d.p + 255) / 256, ctx->num_sms * 4));
    const LsqrDesc *dd = ws.desc;
    if (ctx->opt.use_graph && !ctx->opt.profile) {
        char key[160];
        snprintf(key, sizeof key, "lsqr:%d:%d:%d:%d:%p:%p", Gr, Gc, grid, grid_v, (void *)ws.ut, (void *)ws.ub);
        auto it = ctx->named_graphs.find(key);
        cudaGraphExec_t exec = nullptr;
        if (it == ctx->named_graphs.end()) {
            cudaGraph_t g = nullptr;
            PCG_CUDA_TRY(ctx, cudaGraphCreate(&g, 0));
            cudaGraphConditionalHandle hw{};
            int one = 1, zero = 0;
            cudaGraphNode_t n0, n1, nw, nr, nc, nf;
            auto add = [&](cudaGraph_t gg, cudaGraphNode_t *nd, const cudaGraphNode_t *dep, void *fn, int gr,
                           void **args) {
                cudaKernelNodeParams kp = {};
                kp.func = fn;
                kp.gridDim = dim3(gr);
                kp.blockDim = dim3(256);
                kp.kernelParams = args;
                return cudaGraphAddKernelNode(nd, gg, dep, dep ? 1 : 0, &kp);
            };
            void *a0[] = {(void *)&dd, &ws};
            e = add(g, &n0, nullptr, (void *)k_l_start, grid, a0);
            void *a1[] = {(void *)&dd, &ws, &one, &hw, &zero};
            if (e == cudaSuccess) e = add(g, &n1, &n0, cols_ptr(Gc), grid, a1);
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
            cudaGraph_t body = nullptr;
            if (e == cudaSuccess) {
                cudaGraphNodeParams cp = {};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = hw;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                e = cudaGraphAddNode(&nw, g, &n1, nullptr, 1, &cp);
                if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
            }
            void *ar[] = {(void *)&dd, &ws};
            if (e == cudaSuccess) e = add(body, &nr, nullptr, rows_ptr(Gr), grid, ar);
            void *ac[] = {(void *)&dd, &ws, &zero, &hw, &one};
            if (e == cudaSuccess) e = add(body, &nc, &nr, cols_ptr(Gc), grid, ac);
            void *af[] = {(void *)&dd, &ws};
            if (e == cudaSuccess) e = add(g, &nf, &nw, (void *)k_l_finish, grid_v, af);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_error(ctx, e, "building the LSQR graph");
            ctx->named_graphs[key] = exec;
        } else {
            exec = it->second;
        }
        PCG_CUDA_TRY(ctx, cudaGraphLaunch(exec, s));
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hs, ws.sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, s));
        PCG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        // start, first column pass, per trip a row and a column pass, finish
        ctx->last_launches += 3 + 2 * (int64_t)std::max(hs->iter, 1);
    } else {
        cudaGraphConditionalHandle none{};
        PCG_PROF(ctx, "l_start", k_l_start<<<grid, 256, 0, s>>>(dd, ws));
        PCG_PROF(ctx, "l_cols", PCG_LSQR_G(Gc, k_l_cols, <<<grid, 256, 0, s>>>(dd, ws, 1, none, 0)));
        for (int it = 0;; it += 8) {
            for (int k = 0; k < 8; ++k) {
                PCG_PROF(ctx, "l_rows", PCG_LSQR_G(Gr, k_l_rows, <<<grid, 256, 0, s>>>(dd, ws)));
                PCG_PROF(ctx, "l_cols", PCG_LSQR_G(Gc, k_l_cols, <<<grid, 256, 0, s>>>(dd, ws, 0, none, 0)));
            }
            PCG_CUDA_TRY(ctx, cudaGetLastError());
            PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hs, ws.sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, s));
            PCG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            prof_collect(ctx);
            if (hs->done) break;
            if (it > max_iter + 16) return set_error(ctx, PCG_TIMEOUT, "host loop ran past max_iter");
        }
        PCG_PROF(ctx, "l_finish", k_l_finish<<<grid_v, 256, 0, s>>>(dd, ws));
        PCG_CUDA_TRY(ctx, cudaGetLastError());
        PCG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        prof_collect(ctx);
    }
    *iters = hs->iter;
    *resid = hs->resid;
    if (hs->status == kRunning) return set_error(ctx, PCG_TIMEOUT, "LSQR did not finish");
    if (hs->status != PCG_OK) {
        const char *what = hs->status == PCG_MAXITER ? "max_iter reached before the stop rule"
                           : hs->status == PCG_BREAKDOWN ? "LSQR breakdown: alpha_1 or beta_1 is zero"
                                                         : "non-finite LSQR scalar";
        return set_error(ctx, (pcg_status)hs->status, what);
    }
    return PCG_OK;
}

}  // namespace pcg
