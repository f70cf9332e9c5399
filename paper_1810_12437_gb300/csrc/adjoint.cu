// Adjoint of the draw (not in the paper): implicit differentiation of
// beta = Phi^-1 b with Phi = X^T Omega X + diag(d), d_j = tau^-2 lambda_j^-2.
// With g = Phi^-1 (dL/dbeta) from one more prior-preconditioned CG solve:
//   dL/domega_i      = -(X g)_i (X beta)_i  [+ (X g)_i (z_i + eta_i / (2 sqrt omega_i))]
//   dL/dlog lambda_j =  2 d_j g_j beta_j    [- g_j delta_j / (tau lambda_j)]
//   dL/dlog tau      =  sum_j dL/dlog lambda_j
// where the bracketed terms enter when b is built by Eq. 2.3 from
// (z, eta, delta) inside the draw.  One CSR pass gathers both X g and
// X beta, reading the index stream once.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace pcg {

template <int G>
__global__ void __launch_bounds__(256) k_adj_omega(int64_t n, const int64_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci,
                                                   const double *__restrict__ g,
                                                   const double *__restrict__ beta,
                                                   const double *__restrict__ omega,
                                                   const double *__restrict__ z,
                                                   const double *__restrict__ eta, int draw,
                                                   double *__restrict__ g_omega) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    for (int64_t base = warp * gpw; base < n; base += nwarps * gpw) {
        const int64_t i = base + sub;
        double xg = 0.0, xb = 0.0;
        if (i < n) {
            const int64_t k1 = rp[i + 1];
            for (int64_t k = rp[i] + lane; k < k1; k += G) {
                const int32_t j = ld_stream(ci + k);
                xg += ld_gather(g + j);
                xb += ld_gather(beta + j);
            }
        }
        xg = group_sum<G>(xg);
        xb = group_sum<G>(xb);
        if (i < n && lane == 0) {
            double go = -xg * xb;
            if (draw) {
                const double o = omega[i];
                go += xg * (z[i] + eta[i] / (2.0 * sqrt(o)));
            }
            g_omega[i] = go;
        }
    }
}

__global__ void __launch_bounds__(256) k_adj_lambda(int64_t p, double tau,
                                                    const double *__restrict__ lambda,
                                                    const double *__restrict__ g,
                                                    const double *__restrict__ beta,
                                                    const double *__restrict__ delta, int draw,
                                                    double *__restrict__ g_loglambda,
                                                    double *partials, unsigned int *counter,
                                                    double *g_logtau_dev) {
    __shared__ double red[32];
    __shared__ double sums[1];
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double lam = lambda[j];
        double gl = 2.0 * prior_prec(tau, lam) * g[j] * beta[j];
        if (draw) gl -= g[j] * delta[j] / (tau * lam);
        g_loglambda[j] = gl;
        acc += gl;
    }
    const double tot = block_sum(acc, red);
    if (grid_reduce<1>(&tot, partials, counter, sums, red) && threadIdx.x == 0) *g_logtau_dev = sums[0];
}

pcg_status launch_adjoint_terms(pcg_ctx *ctx, const pcg_csr *Xr, const double *omega,
                                const double *z, const double *lambda, double tau,
                                const double *eta, const double *delta, const double *beta,
                                const double *g, int mode, double *g_omega, double *g_loglambda,
                                double *g_logtau) {
    cudaError_t e;
    char *scratch = (char *)grow(ctx, "adjoint", 256 + sizeof(double) * kMaxReduceBlocks, &e);
    if (!scratch) return cuda_error(ctx, e, "allocating adjoint scratch");
    double *tau_dev = (double *)scratch;
    unsigned int *counter = (unsigned int *)(scratch + 64);
    double *partials = (double *)(scratch + 256);
    double *h = (double *)grow_host(ctx, "adjoint_h", sizeof(double), &e);
    if (!h) return cuda_error(ctx, e, "allocating adjoint host scratch");
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(scratch, 0, 256, ctx->stream));
    const int draw = mode == PCG_ADJ_DRAW ? 1 : 0;
    const int grid = grid_for(ctx, 256, 8);
    const double mean_row = Xr->n > 0 ? (double)Xr->nnz / Xr->n : 1.0;
    const int G = mean_row < 6 ? 4 : mean_row < 20 ? 8 : mean_row < 56 ? 16 : 32;
    if (Xr->n > 0) {
        ++ctx->last_launches;
        switch (G) {
            case 4: k_adj_omega<4><<<grid, 256, 0, ctx->stream>>>(Xr->n, Xr->row_ptr, Xr->col_idx, g, beta, omega, z, eta, draw, g_omega); break;
            case 8: k_adj_omega<8><<<grid, 256, 0, ctx->stream>>>(Xr->n, Xr->row_ptr, Xr->col_idx, g, beta, omega, z, eta, draw, g_omega); break;
            case 16: k_adj_omega<16><<<grid, 256, 0, ctx->stream>>>(Xr->n, Xr->row_ptr, Xr->col_idx, g, beta, omega, z, eta, draw, g_omega); break;
            default: k_adj_omega<32><<<grid, 256, 0, ctx->stream>>>(Xr->n, Xr->row_ptr, Xr->col_idx, g, beta, omega, z, eta, draw, g_omega); break;
        }
    }
    const int gv = (int)std::max<int64_t>(1, std::min<int64_t>((Xr->p + 255) / 256, ctx->num_sms * 4));
    PCG_PROF(ctx, "adj_lambda", k_adj_lambda<<<gv, 256, 0, ctx->stream>>>(Xr->p, tau, lambda, g, beta, delta, draw, g_loglambda,
                                              partials, counter, tau_dev));
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(h, tau_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    *g_logtau = *h;
    return PCG_OK;
}

}  // namespace pcg
