// Single right-hand-side path: Prop. 2.1 right-hand side (Eq. 2.3) and
// prior-preconditioned CG (Sec. 2.4, Algorithm S1, stop rule Eq. S2) on
// Phi beta = b (Eq. 2.4), with Phi applied matrix-free as
// u = Omega (X s) (CSR pass) and v = X^T u + tau^-2 Lambda^-2 s (CSC pass).
//
// Kernels of one CG iteration (device-side while loop of a CUDA graph):
//   k_csr        u_i = omega_i sum_{j in row i} s_j
//   k_csc        v_j = sum_{i in col j} u_i + d_j s_j,   sigma = s.v,  alpha = rho/sigma
//   k_update     beta += alpha s, r -= alpha v, rho' = r.(m r); stop test; gamma
//   [if need_ru] k_csr on beta in float64, then k_true_resid: r = b - Phi beta,
//                rho = r.(m r)   (reliable update of the refined mode)
//   k_sdir       s = m r + gamma s   (and its float32 copy for the next gathers)
// with d = tau^-2 lambda^-2 and m = tau^2 lambda^2.  Every dot product and
// CG scalar is float64; the grid reductions are deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "device_common.cuh"
#include "df.cuh"
#include "internal.h"
#include "tiled.h"

namespace pcg {

__device__ __forceinline__ bool gate_closed(const int *done, const int *need) {
    return *(volatile const int *)done || (need && !*(volatile const int *)need);
}

// ---------------------------------------------------------------------------
// a1: w_i = omega_i z_i + sqrt(omega_i) eta_i (float64), and the float32 copy
// of omega used by the float32 products.
// ---------------------------------------------------------------------------
__global__ void k_rhs_w(const DrawDesc *__restrict__ d, double *__restrict__ w,
                        float *__restrict__ om32, int want_w, int want_om32,
                        double *__restrict__ om64, float2 *__restrict__ omdf) {
    const int64_t n = d->n;
    const double *__restrict__ om = d->omega;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double o = om[i];
        if (want_w) w[i] = o * d->z[i] + sqrt(o) * d->eta[i];
        if (want_om32) om32[i] = (float)o;
        if (om64) om64[i] = o;
        if (omdf) omdf[i] = df_from_double(o);
    }
}

// out = sum_t Pc[t] + d v (pcg_phi_mul through the tiled products)
template <typename T>
__global__ void k_t_fin_out(const DrawDesc *__restrict__ d, TiledArgs A, const double *__restrict__ v,
                            double *__restrict__ out) {
    const TiledPlan &P = A.plan;
    const int64_t p = d->p;
    const T *__restrict__ Pc = reinterpret_cast<const T *>(P.Pc);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const T acc = sum_strided(Pc + j, P.T_r, (size_t)p);
        out[j] = part_to_double(acc) + desc_d(d, j) * v[j];
    }
}

// ---------------------------------------------------------------------------
// a1 + a2: b_j = sum_{i in col j} w_i + delta_j / (tau lambda_j)  (or the given
// right-hand side), then beta = 0, r = b, z = M^-1 b, s = z, rho_0 = r.z, and
// the stop rule's reference rho_b = ||tau lambda (.) b||^2 (Eq. S2; equal to
// rho_0 under the prior preconditioner).  With a warm start (Sec. S4.1) only b
// and rho_b are formed here: k_warm_init sets r, s and rho from beta_0.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(256) k_rhs_init(const DrawDesc *__restrict__ d,
                                                  const double *__restrict__ w, SingleWs ws) {
    __shared__ double red[32];
    __shared__ double sums[2];
    const int64_t p = d->p;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    const bool warm = d->warm != 0;
    double rho = 0.0, rho_b = 0.0;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        double acc = 0.0;
        if (d->rhs == nullptr && j < p)
            acc = segment_partial<G, double>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], w, lane);
        acc = group_sum<G>(acc);
        if (j < p && lane == 0) {
            const double b = d->rhs ? d->rhs[j] : acc + desc_prior_term(d, j, d->delta[j]);
            const double tb = b * (desc_mstop(d, j) * b);
            ws.b[j] = b;
            rho_b += tb;
            if (!warm) {
                const double z = desc_m(d, j) * b;
                ws.r[j] = b;
                ws.s64[j] = z;
                ws.s32[j] = (float)z;
                if (d->df) ws.sdf[j] = df_from_double(z);
                d->beta[j] = 0.0;
                rho += d->mj ? b * z : tb;
            }
        }
    }
    double tot[2];
    tot[0] = block_sum(rho, red);
    tot[1] = block_sum(rho_b, red);
    if (grid_reduce<2>(tot, ws.partials, ws.counters + 0, sums, red) && threadIdx.x == 0) {
        CgScalars *sc = ws.sc;
        const double r0 = sums[0], rb = sums[1];
        sc->rho = r0;
        sc->rho0 = rb;
        sc->rho_prev = r0;
        sc->sigma = 0.0;
        sc->alpha = 0.0;
        sc->gamma = 0.0;
        sc->iter = 0;
        sc->need_ru = 0;
        sc->pending = 0;
        sc->ru_trips = 0;
        sc->resid = stop_quantity(d->stop_rule, rb, rb, p);
        if (!isfinite(rb) || !isfinite(r0)) {
            sc->status = PCG_NONFINITE;
            sc->done = 1;
        } else if (warm) {
            sc->status = kRunning;   // decided by k_warm_init
            sc->done = 0;
        } else if (stop_met(d->stop_rule, rb, rb, p, d->tol)) {
            sc->status = PCG_OK;
            sc->done = 1;
        } else if (d->max_iter <= 0) {
            sc->status = PCG_MAXITER;
            sc->done = 1;
        } else {
            sc->status = kRunning;
            sc->done = 0;
        }
    }
}

// Jacobi preconditioner (Sec. 2.4): M^-1_j = 1 / diag(Phi)_j with
// diag(Phi)_j = sum_{i in col j} omega_i + d_j for binary X (float64).
template <int G>
__global__ void __launch_bounds__(256) k_jacobi(const DrawDesc *__restrict__ d, double *__restrict__ mj) {
    const int64_t p = d->p;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        double acc = 0.0;
        if (j < p)
            acc = segment_partial<G, double>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], d->omega, lane);
        acc = group_sum<G>(acc);
        if (j < p && lane == 0) mj[j] = 1.0 / (acc + desc_d(d, j));
    }
}

// Warm start (Sec. S4.1): with u64 = Omega X beta_0 (float64), r_0 = b -
// (X^T u64 + d beta_0), z = M^-1 r_0, s = z, rho = r.z; stop test on
// ||tau lambda (.) r_0||^2 against rho_b (set by k_rhs_init).
template <int G>
__global__ void __launch_bounds__(256) k_warm_init(const DrawDesc *__restrict__ d,
                                                   const double *__restrict__ u64, SingleWs ws) {
    __shared__ double red[32];
    __shared__ double sums[2];
    CgScalars *sc = ws.sc;
    if (*(volatile const int *)&sc->done) return;
    const int64_t p = d->p;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    double rho = 0.0, rho_s = 0.0;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        double acc = 0.0;
        if (j < p)
            acc = segment_partial<G, double>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], u64, lane);
        acc = group_sum<G>(acc);
        if (j < p && lane == 0) {
            const double rj = ws.b[j] - (acc + desc_d(d, j) * d->beta[j]);
            const double z = desc_m(d, j) * rj;
            ws.r[j] = rj;
            ws.s64[j] = z;
            ws.s32[j] = (float)z;
            if (d->df) ws.sdf[j] = df_from_double(z);
            const double t = rj * z;
            rho += t;
            rho_s += d->mj ? rj * (desc_mstop(d, j) * rj) : t;
        }
    }
    double tot[2];
    tot[0] = block_sum(rho, red);
    tot[1] = block_sum(rho_s, red);
    if (grid_reduce<2>(tot, ws.partials, ws.counters + 4, sums, red) && threadIdx.x == 0) {
        const double r0 = sums[0], rs = sums[1];
        sc->rho = r0;
        sc->rho_prev = r0;
        sc->resid = stop_quantity(d->stop_rule, rs, sc->rho0, p);
        if (!isfinite(r0) || !isfinite(rs)) {
            sc->status = PCG_NONFINITE;
            sc->done = 1;
        } else if (stop_met(d->stop_rule, rs, sc->rho0, p, d->tol)) {
            sc->status = PCG_OK;
            sc->done = 1;
        } else if (d->max_iter <= 0) {
            sc->status = PCG_MAXITER;
            sc->done = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// a3: u_i = omega_i sum_{j in row i} s_j   (T = float: float32 gathers and sums)
// ---------------------------------------------------------------------------
template <typename T, int G>
__global__ void __launch_bounds__(256) k_csr(const DrawDesc *__restrict__ d,
                                             const T *__restrict__ s, const T *__restrict__ om,
                                             T *__restrict__ u, const int *done, const int *need) {
    if (gate_closed(done, need)) return;
    // float64 callers may pass NULL to read beta (s) or omega (om) from the
    // descriptor, so that cached graphs hold no caller pointer.
    const T *__restrict__ sv = s ? s : (const T *)d->beta;
    const T *__restrict__ omv = om ? om : (const T *)d->omega;
    const int64_t n = d->n;
    const int64_t *__restrict__ rp = d->row_ptr;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    for (int64_t base = warp * gpw; base < n; base += nwarps * gpw) {
        const int64_t i = base + sub;
        T acc = T(0);
        if (i < n)
            acc = segment_partial<G, T>(d->col_idx, rp[i], rp[i + 1], sv, lane);
        acc = group_sum<G>(acc);
        if (i < n && lane == 0) u[i] = omv[i] * acc;
    }
}

// ---------------------------------------------------------------------------
// a4 + a5: v_j = sum_{i in col j} u_i + d_j s_j (float64 out), sigma = s.v,
// alpha = rho / sigma.  With `out` set (pcg_phi_mul) it only writes out = v.
// ---------------------------------------------------------------------------
template <typename T, int G>
__global__ void __launch_bounds__(256) k_csc(const DrawDesc *__restrict__ d,
                                             const T *__restrict__ u, const double *__restrict__ sv,
                                             double *__restrict__ out, SingleWs ws, int reduce) {
    __shared__ double red[32];
    __shared__ double sums[1];
    if (reduce && *(volatile const int *)&ws.sc->done) return;
    const int64_t p = d->p;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    double sig = 0.0;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        T acc = T(0);
        if (j < p)
            acc = segment_partial<G, T>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], u, lane);
        acc = group_sum<G>(acc);
        if (j < p && lane == 0) {
            const double sj = sv[j];
            const double v = (double)acc + desc_d(d, j) * sj;
            out[j] = v;
            sig += sj * v;
        }
    }
    if (!reduce) return;
    const double tot = block_sum(sig, red);
    if (grid_reduce<1>(&tot, ws.partials, ws.counters + 1, sums, red) && threadIdx.x == 0) {
        CgScalars *sc = ws.sc;
        const double sigma = sums[0];
        sc->sigma = sigma;
        if (!isfinite(sigma)) {
            sc->status = PCG_NONFINITE;
            sc->done = 1;
        } else if (!(sigma > 0.0) || !(sc->rho > 0.0)) {
            sc->status = PCG_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->alpha = sc->rho / sigma;
        }
    }
}

// ---------------------------------------------------------------------------
// a6 + a7: beta += alpha s; r -= alpha v; rho' = r.(m r); stop test; gamma.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_update(const DrawDesc *__restrict__ d, SingleWs ws,
                                                cudaGraphConditionalHandle h_ru, int use_cond) {
    __shared__ double red[32];
    __shared__ double sums[2];
    CgScalars *sc = ws.sc;
    if (*(volatile const int *)&sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_ru, 0);
        return;
    }
    const int64_t p = d->p;
    const double alpha = sc->alpha;
    double rho = 0.0, rho_s = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double bj = d->beta[j] + alpha * ws.s64[j];
        const double rj = ws.r[j] - alpha * ws.v64[j];
        d->beta[j] = bj;
        ws.r[j] = rj;
        const double t = rj * (desc_m(d, j) * rj);
        rho += t;
        rho_s += d->mj ? rj * (desc_mstop(d, j) * rj) : t;
    }
    double tot[2];
    tot[0] = block_sum(rho, red);
    tot[1] = block_sum(rho_s, red);
    if (grid_reduce<2>(tot, ws.partials, ws.counters + 2, sums, red) && threadIdx.x == 0) {
        const double rn = sums[0], rs = sums[1];
        sc->iter += 1;
        if (!isfinite(rn) || !isfinite(rs)) {
            sc->status = PCG_NONFINITE;
            sc->done = 1;
            sc->need_ru = 0;
        } else {
            // the stop rule on ||tau lambda (.) r||^2 (Eq. S2), whatever M is
            const bool conv = stop_met(d->stop_rule, rs, sc->rho0, p, d->tol);
            sc->rho_prev = sc->rho;
            sc->rho = rn;
            sc->gamma = rn / sc->rho_prev;
            sc->resid = stop_quantity(d->stop_rule, rs, sc->rho0, p);
            if (d->refined) {
                const bool periodic = d->reliable_k > 0 && (sc->iter % d->reliable_k) == 0;
                sc->pending = conv ? 1 : 0;
                sc->need_ru = (conv || periodic) ? 1 : 0;
                if (!conv && sc->iter >= d->max_iter) {
                    sc->status = PCG_MAXITER;
                    sc->done = 1;
                    sc->need_ru = 0;
                }
            } else if (conv) {
                sc->status = PCG_OK;
                sc->done = 1;
            } else if (sc->iter >= d->max_iter) {
                sc->status = PCG_MAXITER;
                sc->done = 1;
            }
        }
        if (sc->need_ru && !sc->done) sc->ru_trips += 1;
        if (use_cond) cudaGraphSetConditional(h_ru, (sc->need_ru && !sc->done) ? 1u : 0u);
    }
}

// ---------------------------------------------------------------------------
// a8 (refined mode): r = b - (X^T u64 + d beta) with u64 = Omega X beta in
// float64; rho = r.(m r) replaces the recursion's value.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(256) k_true_resid(const DrawDesc *__restrict__ d,
                                                    const double *__restrict__ u64, SingleWs ws,
                                                    int gated) {
    __shared__ double red[32];
    __shared__ double sums[2];
    CgScalars *sc = ws.sc;
    if (gated && gate_closed(&sc->done, &sc->need_ru)) return;
    const int64_t p = d->p;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    double rho = 0.0, rho_s = 0.0;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        double acc = 0.0;
        if (j < p)
            acc = segment_partial<G, double>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], u64, lane);
        acc = group_sum<G>(acc);
        if (j < p && lane == 0) {
            const double bj = d->beta[j];
            const double rj = ws.b[j] - (acc + desc_d(d, j) * bj);
            ws.r[j] = rj;
            const double t = rj * (desc_m(d, j) * rj);
            rho += t;
            rho_s += d->mj ? rj * (desc_mstop(d, j) * rj) : t;
        }
    }
    double tot[2];
    tot[0] = block_sum(rho, red);
    tot[1] = block_sum(rho_s, red);
    if (grid_reduce<2>(tot, ws.partials, ws.counters + 3, sums, red) && threadIdx.x == 0) {
        const double rt = sums[0], rts = sums[1];
        sc->need_ru = 0;
        if (!isfinite(rt) || !isfinite(rts)) {
            sc->status = PCG_NONFINITE;
            sc->done = 1;
        } else {
            sc->rho = rt;
            sc->gamma = rt / sc->rho_prev;
            sc->resid = stop_quantity(d->stop_rule, rts, sc->rho0, p);
            if (sc->pending) {
                if (stop_met(d->stop_rule, rts, sc->rho0, p, d->tol)) {
                    sc->status = PCG_OK;
                    sc->done = 1;
                } else {
                    // the recursion met the rule but the float64 residual does
                    // not: restart from it (s = M^-1 r), i.e. refine the
                    // current beta instead of extending a stale direction
                    sc->pending = 0;
                    sc->gamma = 0.0;
                    if (sc->iter >= d->max_iter) {
                        sc->status = PCG_MAXITER;
                        sc->done = 1;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// s = m r + gamma s (float64 master and float32 gather copy); sets the while
// condition of the graph to "not done".
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sdir(const DrawDesc *__restrict__ d, SingleWs ws,
                                              cudaGraphConditionalHandle h_while, int use_cond) {
    CgScalars *sc = ws.sc;
    const int done = *(volatile const int *)&sc->done;
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional(h_while, done ? 0u : 1u);
    if (done) return;
    const int64_t p = d->p;
    const double gamma = sc->gamma;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double s = desc_m(d, j) * ws.r[j] + gamma * ws.s64[j];
        ws.s64[j] = s;
        ws.s32[j] = (float)s;
        if (d->df) ws.sdf[j] = df_from_double(s);
    }
}

// v (float64) -> double-float pairs (pcg_phi_mul in the DF32 mode)
__global__ void k_to_df(const double *__restrict__ x, float2 *__restrict__ y, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x)
        y[j] = df_from_double(x[j]);
}

// v (float64) -> float32 copy (pcg_phi_mul in the float32 modes)
__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x)
        y[j] = (float)x[j];
}

// b only (pcg_build_rhs): b_j = sum w_i + delta_j / (tau lambda_j)
template <int G>
__global__ void __launch_bounds__(256) k_rhs_b(const DrawDesc *__restrict__ d,
                                               const double *__restrict__ w, double *__restrict__ b) {
    const int64_t p = d->p;
    const int lane = threadIdx.x & (G - 1);
    const int64_t gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t sub = (threadIdx.x & 31) / G;
    for (int64_t base = warp * gpw; base < p; base += nwarps * gpw) {
        const int64_t j = base + sub;
        double acc = 0.0;
        if (j < p)
            acc = segment_partial<G, double>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], w, lane);
        acc = group_sum<G>(acc);
        if (j < p && lane == 0) b[j] = acc + desc_prior_term(d, j, d->delta[j]);
    }
}

// ===========================================================================
// host side
// ===========================================================================

static int pick_group(double mean_len) {
    if (mean_len < 6) return 4;
    if (mean_len < 20) return 8;
    if (mean_len < 56) return 16;
    return 32;
}

// Dispatch helpers: instantiate the kernels for the four group widths.
#define PCG_DISPATCH_G(G, ...)                         \
    switch (G) {                                       \
        case 4: { constexpr int GG = 4; __VA_ARGS__; } break;   \
        case 8: { constexpr int GG = 8; __VA_ARGS__; } break;   \
        case 16: { constexpr int GG = 16; __VA_ARGS__; } break; \
        default: { constexpr int GG = 32; __VA_ARGS__; } break; \
    }

template <typename T>
static void *csr_kernel_ptr(int G) {
    void *f = nullptr;
    PCG_DISPATCH_G(G, f = (void *)k_csr<T, GG>);
    return f;
}
template <typename T>
static void *csc_kernel_ptr(int G) {
    void *f = nullptr;
    PCG_DISPATCH_G(G, f = (void *)k_csc<T, GG>);
    return f;
}
static void *rhs_init_ptr(int G) {
    void *f = nullptr;
    PCG_DISPATCH_G(G, f = (void *)k_rhs_init<GG>);
    return f;
}
static void *true_resid_ptr(int G) {
    void *f = nullptr;
    PCG_DISPATCH_G(G, f = (void *)k_true_resid<GG>);
    return f;
}
static void *jacobi_ptr(int G) {
    void *f = nullptr;
    PCG_DISPATCH_G(G, f = (void *)k_jacobi<GG>);
    return f;
}
static void *warm_init_ptr(int G) {
    void *f = nullptr;
    PCG_DISPATCH_G(G, f = (void *)k_warm_init<GG>);
    return f;
}

pcg_status ensure_single_ws(pcg_ctx *ctx, int64_t n, int64_t p) {
    if (n <= ctx->cap_n && p <= ctx->cap_p && ctx->ws.sc) return PCG_OK;
    const int64_t cn = std::max<int64_t>(std::max<int64_t>(n, ctx->cap_n), 1);
    const int64_t cp = std::max<int64_t>(std::max<int64_t>(p, ctx->cap_p), 1);
    SingleWs &w = ctx->ws;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(w.b);
    cudaFree(w.u);
    w = SingleWs{};
    // cached graphs hold workspace pointers: drop the single-RHS ones
    for (auto it = ctx->named_graphs.begin(); it != ctx->named_graphs.end();) {
        if (it->first.rfind("single:", 0) == 0) {
            cudaGraphExecDestroy(it->second);
            it = ctx->named_graphs.erase(it);
        } else {
            ++it;
        }
    }
    // one allocation, carved into aligned pieces
    const size_t al = 256;
    auto up = [&](size_t x) { return (x + al - 1) / al * al; };
    const size_t szp64 = up(sizeof(double) * cp), szp32 = up(sizeof(float) * cp);
    const size_t szn32 = up(sizeof(float) * cn), szn64 = up(sizeof(double) * cn);
    const size_t szpart = up(sizeof(double) * kMaxReduceBlocks * 4);
    const size_t total = 6 * szp64 + szp32 + szn32 + 2 * szn64 + szpart + up(64 * sizeof(unsigned)) +
                         up(sizeof(CgScalars)) + up(sizeof(DrawDesc));
    char *base = nullptr;
    PCG_CUDA_TRY(ctx, cudaMalloc(&base, total));
    PCG_CUDA_TRY(ctx, cudaMalloc(&w.u, up(sizeof(double) * cn)));
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, total, ctx->stream));
    size_t off = 0;
    auto take = [&](size_t sz) { char *q = base + off; off += sz; return q; };
    w.b = (double *)take(szp64);
    w.r = (double *)take(szp64);
    w.s64 = (double *)take(szp64);
    w.v64 = (double *)take(szp64);
    w.s32 = (float *)take(szp32);
    w.sdf = (float2 *)take(szp64);
    w.om32 = (float *)take(szn32);
    w.om64 = (double *)take(szn64);
    w.omdf = (float2 *)take(szn64);
    w.mj = (double *)take(szp64);
    w.partials = (double *)take(szpart);
    w.counters = (unsigned *)take(up(64 * sizeof(unsigned)));
    w.sc = (CgScalars *)take(up(sizeof(CgScalars)));
    w.desc = (DrawDesc *)take(up(sizeof(DrawDesc)));
    ctx->cap_n = cn;
    ctx->cap_p = cp;
    if (!ctx->h_desc) PCG_CUDA_TRY(ctx, cudaMallocHost(&ctx->h_desc, sizeof(DrawDesc)));
    if (!ctx->h_sc) PCG_CUDA_TRY(ctx, cudaMallocHost(&ctx->h_sc, sizeof(CgScalars)));
    return PCG_OK;
}

struct SingleLaunch {
    int G_row, G_col;
    int grid_stream;   // streaming kernels
    int grid_vec;      // p-length vector kernels
    int threads;
};

static SingleLaunch single_launch(pcg_ctx *ctx, const DrawDesc &d) {
    SingleLaunch L;
    L.threads = 256;
    L.G_row = pick_group(d.n > 0 ? (double)d.nnz / (double)d.n : 1.0);
    L.G_col = pick_group(d.p > 0 ? (double)d.nnz / (double)d.p : 1.0);
    if (ctx->shape.csr_tpr > 0 && ctx->shape.blocks > 0) { /* tuned override, if any */ }
    const int per_sm = 8;   // 2048 resident threads per SM at 256 threads per block
    L.grid_stream = std::min(ctx->num_sms * per_sm, kMaxReduceBlocks);
    const int64_t need_vec = (d.p + L.threads - 1) / L.threads;
    L.grid_vec = (int)std::max<int64_t>(1, std::min<int64_t>(need_vec, ctx->num_sms * 4));
    return L;
}

// Adds one kernel node; args is the kernel's argument pointer array.
static cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *deps,
                              size_t ndeps, void *func, int grid, int block, void **args,
                              size_t smem = 0) {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

// Kernel argument values must outlive node creation; they are copied into the
// graph by cudaGraphAddKernelNode.
struct NodeArgs {
    const DrawDesc *d;
    SingleWs ws;
    const void *s_gather, *om, *u;
    const double *u64, *s64, *nulld;
    double *w64, *v64;
    float *om32;
    const int *done, *nulli;
    cudaGraphConditionalHandle h_ru, h_while;
    int one, zero, want_w, want_om32, use_cond_ru;
    TiledArgs ta;
    double *om64;
    float2 *omdf;
    const void *om_t, *s_t;
    void *pc;
    double *mj;
};

static pcg_status build_graph(pcg_ctx *ctx, const DrawDesc &d, int precision, const TiledPlan &tp,
                              cudaGraphExec_t *out) {
    const SingleLaunch L = single_launch(ctx, d);
    const bool tiled = tp.valid;
    // float32 gathers in the FP32 modes; float64 sources (s64, omega) in the
    // FP64 and DF32 modes (the DF32 tiled kernels split them on staging)
    TiledKernels TK{};
    if (tiled) {
        pcg_status st = tiled_prepare(ctx, tp, &TK);
        if (st != PCG_OK) return st;
    }
    const bool f32 = precision == PCG_PREC_FP32 || precision == PCG_PREC_FP32_REFINED;
    const bool refined = d.refined != 0;
    NodeArgs A{};
    A.d = ctx->ws.desc;
    A.ws = ctx->ws;
    A.done = &ctx->ws.sc->done;
    A.nulli = nullptr;
    A.nulld = nullptr;
    A.w64 = (double *)ctx->ws.u;
    A.om32 = ctx->ws.om32;
    A.want_w = d.rhs == nullptr ? 1 : 0;
    A.want_om32 = f32 ? 1 : 0;
    const bool df = prec_pairs(precision);
    A.s_gather = f32 ? (const void *)ctx->ws.s32 : (const void *)ctx->ws.s64;
    A.om = f32 ? (const void *)ctx->ws.om32 : nullptr;   // NULL: float64 omega from the descriptor
    A.u = ctx->ws.u;
    A.u64 = (const double *)ctx->ws.u;
    A.v64 = ctx->ws.v64;
    A.s64 = ctx->ws.s64;
    A.one = 1;
    A.zero = 0;
    A.use_cond_ru = refined ? 1 : 0;
    A.ta.plan = tp;
    A.om64 = (tiled && !f32 && !df) ? ctx->ws.om64 : nullptr;
    A.omdf = (tiled && df) ? ctx->ws.omdf : nullptr;
    // sources of the tiled products: float32, double-float pairs or float64
    A.om_t = f32 ? (const void *)ctx->ws.om32 : df ? (const void *)ctx->ws.omdf : (const void *)ctx->ws.om64;
    A.s_t = f32 ? (const void *)ctx->ws.s32 : df ? (const void *)ctx->ws.sdf : (const void *)ctx->ws.s64;
    A.pc = tp.Pc;

    cudaGraph_t g = nullptr;
    PCG_CUDA_TRY(ctx, cudaGraphCreate(&g, 0));
    cudaError_t e = cudaSuccess;
    cudaGraphNode_t n_w, n_init, n_while, n_csr, n_csc, n_upd, n_if, n_sdir, n_rcsr, n_tr;
    cudaGraph_t body = nullptr;
    {
        void *args[] = {&A.d, &A.w64, &A.om32, &A.want_w, &A.want_om32, &A.om64, &A.omdf};
        e = add_kernel(g, &n_w, nullptr, 0, (void *)k_rhs_w, L.grid_stream, L.threads, args);
    }
    cudaGraphNode_t pre = n_w;
    if (e == cudaSuccess && d.mj) {   // Jacobi preconditioner, before any use of M^-1
        cudaGraphNode_t n_j;
        A.mj = ctx->ws.mj;
        void *args[] = {&A.d, &A.mj};
        e = add_kernel(g, &n_j, &pre, 1, jacobi_ptr(L.G_col), L.grid_stream, L.threads, args);
        pre = n_j;
    }
    if (e == cudaSuccess) {
        void *args[] = {&A.d, &A.w64, &A.ws};
        e = add_kernel(g, &n_init, &pre, 1, rhs_init_ptr(L.G_col), L.grid_stream, L.threads, args);
    }
    if (e == cudaSuccess && d.warm) {   // r_0 = b - Phi beta_0 (float64 product on beta_0)
        cudaGraphNode_t n_wc = nullptr, n_wi = nullptr;
        void *a1[] = {&A.d, &A.nulld, &A.nulld, &A.w64, &A.done, &A.nulli};
        e = add_kernel(g, &n_wc, &n_init, 1, csr_kernel_ptr<double>(L.G_row), L.grid_stream, L.threads, a1);
        if (e == cudaSuccess) {
            void *a2[] = {&A.d, &A.u64, &A.ws};
            e = add_kernel(g, &n_wi, &n_wc, 1, warm_init_ptr(L.G_col), L.grid_stream, L.threads, a2);
        }
        n_init = n_wi;
    }
    if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&A.h_while, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = A.h_while;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&n_while, g, &n_init, nullptr, 1, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess && tiled) {
        // tiled products: CSR tiles -> u -> CSC strips -> finalize (sigma, alpha)
        cudaGraphNode_t n_tc, n_u;
        void *a1[] = {&A.ta, &A.s_t, &A.one, &A.zero, &A.done, &A.zero};
        e = add_kernel(body, &n_csr, nullptr, 0, TK.csr, tp.T_c * tp.csr_blocks, tp.threads, a1, tp.smem_c);
        if (e == cudaSuccess) {
            void *au[] = {&A.ta, &A.om_t, &A.one, &A.zero, &A.done, &A.zero};
            e = add_kernel(body, &n_u, &n_csr, 1, TK.u, tiled_u_blocks(tp, ctx->num_sms), 256, au);
        }
        if (e == cudaSuccess) {
            void *a2[] = {&A.ta, &A.pc, &A.one, &A.zero, &A.done, &A.zero};
            e = add_kernel(body, &n_tc, &n_u, 1, TK.csc, tp.T_r * tp.csc_chunks, tp.threads, a2, tp.smem_r);
        }
        if (e == cudaSuccess) {
            void *a3[] = {&A.d, &A.ta, &A.ws};
            e = add_kernel(body, &n_csc, &n_tc, 1, TK.fin1, L.grid_vec, L.threads, a3);
        }
    } else if (e == cudaSuccess) {
        void *args[] = {&A.d, &A.s_gather, &A.om, &A.u, &A.done, &A.nulli};
        e = add_kernel(body, &n_csr, nullptr, 0,
                       f32 ? csr_kernel_ptr<float>(L.G_row) : csr_kernel_ptr<double>(L.G_row),
                       L.grid_stream, L.threads, args);
        if (e == cudaSuccess) {
            void *a2[] = {&A.d, &A.u, &A.s64, &A.v64, &A.ws, &A.one};
            e = add_kernel(body, &n_csc, &n_csr, 1,
                           f32 ? csc_kernel_ptr<float>(L.G_col) : csc_kernel_ptr<double>(L.G_col),
                           L.grid_stream, L.threads, a2);
        }
    }
    if (e == cudaSuccess && refined)
        e = cudaGraphConditionalHandleCreate(&A.h_ru, body, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        void *args[] = {&A.d, &A.ws, &A.h_ru, &A.use_cond_ru};
        e = add_kernel(body, &n_upd, &n_csc, 1, (void *)k_update, L.grid_vec, L.threads, args);
    }
    cudaGraphNode_t last = n_upd;
    if (e == cudaSuccess && refined) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = A.h_ru;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&n_if, body, &n_upd, nullptr, 1, &cp);
        if (e == cudaSuccess) {
            cudaGraph_t ifb = cp.conditional.phGraph_out[0];
            // float64 product on beta: s and omega come from the descriptor (NULL)
            void *a1[] = {&A.d, &A.nulld, &A.nulld, &A.w64, &A.done, &A.nulli};
            e = add_kernel(ifb, &n_rcsr, nullptr, 0, csr_kernel_ptr<double>(L.G_row),
                           L.grid_stream, L.threads, a1);
            if (e == cudaSuccess) {
                void *a2[] = {&A.d, &A.u64, &A.ws, &A.zero};
                e = add_kernel(ifb, &n_tr, &n_rcsr, 1, true_resid_ptr(L.G_col), L.grid_stream,
                               L.threads, a2);
            }
            last = n_if;
        }
    }
    if (e == cudaSuccess) {
        void *args[] = {&A.d, &A.ws, &A.h_while, &A.one};
        e = add_kernel(body, &n_sdir, &last, 1, (void *)k_sdir, L.grid_vec, L.threads, args);
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "building the draw graph");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(ctx, e, "instantiating the draw graph");
    *out = exec;
    return PCG_OK;
}

// Plain launches (use_graph = 0): same kernels, host check every 8 iterations.
static pcg_status run_plain(pcg_ctx *ctx, const DrawDesc &d, int precision, const TiledPlan &tp) {
    const SingleLaunch L = single_launch(ctx, d);
    const char *csr_name = precision == PCG_PREC_DF32   ? "t_csr_df32"
                           : precision == PCG_PREC_FX64 ? "t_csr_fx64"
                           : precision == PCG_PREC_FP64 ? "t_csr_f64"
                                                        : "t_csr_f32";
    const char *csc_name = precision == PCG_PREC_DF32   ? "t_csc_df32"
                           : precision == PCG_PREC_FX64 ? "t_csc_fx64"
                           : precision == PCG_PREC_FP64 ? "t_csc_f64"
                                                        : "t_csc_f32";
    TiledKernels TK{};
    if (tp.valid) {
        pcg_status st = tiled_prepare(ctx, tp, &TK);
        if (st != PCG_OK) return st;
    }
    TiledArgs ta{tp};
    const bool f32 = precision == PCG_PREC_FP32 || precision == PCG_PREC_FP32_REFINED;
    SingleWs ws = ctx->ws;
    const DrawDesc *dd = ws.desc;
    cudaStream_t st = ctx->stream;
    const int B = L.threads;
    const bool df = prec_pairs(precision);
    PCG_PROF(ctx, "rhs_w", k_rhs_w<<<L.grid_stream, B, 0, st>>>(dd, (double *)ws.u, ws.om32, d.rhs == nullptr, f32,
                                                                (tp.valid && !f32 && !df) ? ws.om64 : nullptr,
                                                                (tp.valid && df) ? ws.omdf : nullptr));
    if (d.mj)
        PCG_PROF(ctx, "jacobi", PCG_DISPATCH_G(L.G_col, (k_jacobi<GG><<<L.grid_stream, B, 0, st>>>(dd, ws.mj))));
    PCG_PROF(ctx, "rhs_init", PCG_DISPATCH_G(L.G_col, (k_rhs_init<GG><<<L.grid_stream, B, 0, st>>>(dd, (const double *)ws.u, ws))));
    const int *done = &ws.sc->done, *need = &ws.sc->need_ru;
    if (d.warm) {
        PCG_PROF(ctx, "warm_csr_f64", PCG_DISPATCH_G(L.G_row, (k_csr<double, GG><<<L.grid_stream, B, 0, st>>>(
                                       dd, nullptr, nullptr, (double *)ws.u, done, nullptr))));
        PCG_PROF(ctx, "warm_init", PCG_DISPATCH_G(L.G_col, (k_warm_init<GG><<<L.grid_stream, B, 0, st>>>(
                                    dd, (const double *)ws.u, ws))));
    }
    for (int it = 0;; it += 8) {
        for (int k = 0; k < 8; ++k) {
            if (tp.valid) {
                const void *sg = f32 ? (const void *)ws.s32 : df ? (const void *)ws.sdf : (const void *)ws.s64;
                const void *omt = f32 ? (const void *)ws.om32 : df ? (const void *)ws.omdf : (const void *)ws.om64;
                int one = 1, zero = 0;
                void *a1[] = {&ta, (void *)&sg, &one, &zero, (void *)&done, &zero};
                void *au[] = {&ta, (void *)&omt, &one, &zero, (void *)&done, &zero};
                void *pc = tp.Pc;
                void *a2[] = {&ta, &pc, &one, &zero, (void *)&done, &zero};
                void *a3[] = {(void *)&dd, &ta, &ws};
                PCG_PROF(ctx, csr_name,
                         cudaLaunchKernel(TK.csr, dim3(tp.T_c * tp.csr_blocks), dim3(tp.threads), a1, tp.smem_c, st));
                PCG_PROF(ctx, "t_u", cudaLaunchKernel(TK.u, dim3(tiled_u_blocks(tp, ctx->num_sms)), dim3(256), au, 0, st));
                PCG_PROF(ctx, csc_name,
                         cudaLaunchKernel(TK.csc, dim3(tp.T_r * tp.csc_chunks), dim3(tp.threads), a2, tp.smem_r, st));
                PCG_PROF(ctx, "t_fin", cudaLaunchKernel(TK.fin1, dim3(L.grid_vec), dim3(B), a3, 0, st));
            } else if (f32) {
                PCG_PROF(ctx, "csr_f32", PCG_DISPATCH_G(L.G_row, (k_csr<float, GG><<<L.grid_stream, B, 0, st>>>(
                                            dd, ws.s32, ws.om32, (float *)ws.u, done, nullptr))));
                PCG_PROF(ctx, "csc_f32", PCG_DISPATCH_G(L.G_col, (k_csc<float, GG><<<L.grid_stream, B, 0, st>>>(
                                            dd, (const float *)ws.u, ws.s64, ws.v64, ws, 1))));
            } else {
                PCG_PROF(ctx, "csr_f64", PCG_DISPATCH_G(L.G_row, (k_csr<double, GG><<<L.grid_stream, B, 0, st>>>(
                                            dd, ws.s64, nullptr, (double *)ws.u, done, nullptr))));
                PCG_PROF(ctx, "csc_f64", PCG_DISPATCH_G(L.G_col, (k_csc<double, GG><<<L.grid_stream, B, 0, st>>>(
                                            dd, (const double *)ws.u, ws.s64, ws.v64, ws, 1))));
            }
            PCG_PROF(ctx, "update", k_update<<<L.grid_vec, B, 0, st>>>(dd, ws, 0, 0));
            if (d.refined) {
                PCG_PROF(ctx, "ru_csr_f64", PCG_DISPATCH_G(L.G_row, (k_csr<double, GG><<<L.grid_stream, B, 0, st>>>(
                                            dd, nullptr, nullptr, (double *)ws.u, done, need))));
                PCG_PROF(ctx, "ru_true_resid", PCG_DISPATCH_G(L.G_col, (k_true_resid<GG><<<L.grid_stream, B, 0, st>>>(
                                            dd, (const double *)ws.u, ws, 1))));
            }
            PCG_PROF(ctx, "sdir", k_sdir<<<L.grid_vec, B, 0, st>>>(dd, ws, 0, 0));
        }
        PCG_CUDA_TRY(ctx, cudaGetLastError());
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_sc, ws.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        PCG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        prof_collect(ctx);
        if (ctx->h_sc->done) break;
        if (it > d.max_iter + 16) return set_error(ctx, PCG_TIMEOUT, "host loop ran past max_iter");
    }
    return PCG_OK;
}

// The context's unshrunk coefficients (pcg_set_unshrunk) into a descriptor.
static pcg_status with_unshrunk(pcg_ctx *ctx, DrawDesc &d) {
    if (ctx->unshrunk_q1 > d.p)
        return set_error(ctx, PCG_BADARG, "more unshrunk coefficients (pcg_set_unshrunk) than columns of X");
    d.q1 = ctx->unshrunk_q1;
    d.ud = ctx->unshrunk_d;
    d.um = ctx->unshrunk_m;
    return PCG_OK;
}

pcg_status run_single(pcg_ctx *ctx, const DrawDesc &din, int precision, int mode, int *iters,
                      double *resid) {
    pcg_status st = ensure_single_ws(ctx, din.n, din.p);
    if (st != PCG_OK) return st;
    DrawDesc d = din;
    d.refined = (precision == PCG_PREC_FP32_REFINED) ? 1 : 0;
    d.reliable_k = ctx->opt.reliable_k;
    d.df = prec_pairs(precision) ? 1 : 0;
    d.mj = ctx->opt.preconditioner == PCG_PRECOND_JACOBI ? ctx->ws.mj : nullptr;
    st = with_unshrunk(ctx, d);
    if (st != PCG_OK) return st;
    *ctx->h_desc = d;
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws.desc, ctx->h_desc, sizeof(DrawDesc),
                                      cudaMemcpyHostToDevice, ctx->stream));
    TiledPlan tp{};
    if (ctx->tiled_enabled) {
        const pcg_csr xr{d.n, d.p, d.nnz, d.row_ptr, d.col_idx};
        const pcg_csc xc{d.n, d.p, d.nnz, d.col_ptr, d.row_idx};
        const int vt = tiled_vtype(precision);
        st = build_tiled_plan(ctx, "single", &xr, &xc, 1, vt, 1, true, &tp);
        if (st != PCG_OK) return st;
    }
    if (ctx->opt.use_graph && !ctx->opt.profile) {
        // The graph bakes in the workspace, the plan buffers and the launch
        // shapes (never a caller pointer: those are read from the descriptor).
        const SingleLaunch L = single_launch(ctx, d);
        char key[256];
        snprintf(key, sizeof key, "single:%d:%d:%d:%d:%d:%d:%d:%d:%d|%d:%016llx",
                 L.G_row, L.G_col, L.grid_stream, L.grid_vec, precision, d.refined, mode, d.mj ? 1 : 0,
                 d.warm, (int)tp.valid, (unsigned long long)(tp.valid ? plan_fingerprint(tp) : 0ull));
        // n and p enter through the plan only when it is valid
        std::string skey = std::string(key) + (tp.valid ? ":" + std::to_string(tp.n) + ":" + std::to_string(tp.p) : "");
        auto it = ctx->named_graphs.find(skey);
        cudaGraphExec_t exec = nullptr;
        if (it == ctx->named_graphs.end()) {
            st = build_graph(ctx, d, precision, tp, &exec);
            if (st != PCG_OK) return st;
            ctx->named_graphs[skey] = exec;
        } else {
            exec = it->second;
        }
        PCG_CUDA_TRY(ctx, cudaGraphLaunch(exec, ctx->stream));
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_sc, ctx->ws.sc, sizeof(CgScalars),
                                          cudaMemcpyDeviceToHost, ctx->stream));
        PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        // graph nodes that ran: 2 set-up kernels (+1 Jacobi, +2 warm start), per loop trip (at least one)
        // 4 (untiled) or 6 (tiled: csr, u, csc, finalize, update, direction),
        // 2 per float64 recomputation of r
        const CgScalars &h = *ctx->h_sc;
        ctx->last_launches += 2 + (d.mj ? 1 : 0) + (d.warm ? 2 : 0) +
                              (tp.valid ? 6 : 4) * (int64_t)std::max(h.iter, 1) + 2 * (int64_t)h.ru_trips;
    } else {
        st = run_plain(ctx, d, precision, tp);
        if (st != PCG_OK) return st;
    }
    const CgScalars &sc = *ctx->h_sc;
    *iters = sc.iter;
    *resid = sc.resid;
    if (sc.status == kRunning) return set_error(ctx, PCG_TIMEOUT, "draw did not finish");
    if (sc.status != PCG_OK) {
        const char *what = sc.status == PCG_MAXITER ? "max_iter reached before the stop rule"
                           : sc.status == PCG_BREAKDOWN ? "CG breakdown: s.Phi s <= 0 or rho <= 0"
                                                        : "non-finite CG scalar";
        return set_error(ctx, (pcg_status)sc.status, what);
    }
    return PCG_OK;
}

pcg_status launch_build_rhs(pcg_ctx *ctx, const pcg_csc *X, const double *omega, const double *z,
                            const double *lambda, double tau, const double *eta,
                            const double *delta, double *b) {
    pcg_status st = ensure_single_ws(ctx, X->n, X->p);
    if (st != PCG_OK) return st;
    DrawDesc d{};
    d.col_ptr = X->col_ptr;
    d.row_idx = X->row_idx;
    d.omega = omega;
    d.z = z;
    d.lambda = lambda;
    d.eta = eta;
    d.delta = delta;
    d.n = X->n;
    d.p = X->p;
    d.nnz = X->nnz;
    d.tau = tau;
    st = with_unshrunk(ctx, d);
    if (st != PCG_OK) return st;
    *ctx->h_desc = d;
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws.desc, ctx->h_desc, sizeof(DrawDesc),
                                      cudaMemcpyHostToDevice, ctx->stream));
    const int grid = std::min(ctx->num_sms * 8, kMaxReduceBlocks);
    const int G = pick_group(d.p > 0 ? (double)d.nnz / d.p : 1.0);
    PCG_PROF(ctx, "rhs_w", k_rhs_w<<<grid, 256, 0, ctx->stream>>>(ctx->ws.desc, (double *)ctx->ws.u, ctx->ws.om32, 1, 0, nullptr, nullptr));
    PCG_PROF(ctx, "rhs_b", PCG_DISPATCH_G(G, (k_rhs_b<GG><<<grid, 256, 0, ctx->stream>>>(ctx->ws.desc, (const double *)ctx->ws.u, b))));
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    return PCG_OK;
}

pcg_status launch_phi_mul(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const double *omega,
                          const double *lambda, double tau, const double *v, double *out) {
    pcg_status st = ensure_single_ws(ctx, Xr->n, Xr->p);
    if (st != PCG_OK) return st;
    DrawDesc d{};
    d.row_ptr = Xr->row_ptr;
    d.col_idx = Xr->col_idx;
    d.col_ptr = Xc->col_ptr;
    d.row_idx = Xc->row_idx;
    d.omega = omega;
    d.lambda = lambda;
    d.n = Xr->n;
    d.p = Xr->p;
    d.nnz = Xr->nnz;
    d.tau = tau;
    st = with_unshrunk(ctx, d);
    if (st != PCG_OK) return st;
    *ctx->h_desc = d;
    cudaStream_t s = ctx->stream;
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws.desc, ctx->h_desc, sizeof(DrawDesc),
                                      cudaMemcpyHostToDevice, s));
    // the gate flags of the iteration kernels must read "running"
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->ws.sc, 0, sizeof(CgScalars), s));
    const int grid = std::min(ctx->num_sms * 8, kMaxReduceBlocks);
    const int Gr = pick_group(d.n > 0 ? (double)d.nnz / d.n : 1.0);
    const int Gc = pick_group(d.p > 0 ? (double)d.nnz / d.p : 1.0);
    SingleWs ws = ctx->ws;
    const int *done = &ws.sc->done;
    const int prec = ctx->opt.precision;
    const bool f32 = prec == PCG_PREC_FP32 || prec == PCG_PREC_FP32_REFINED;
    TiledPlan tp{};
    if (ctx->tiled_enabled) {
        const int vt = tiled_vtype(prec);
        pcg_status st2 = build_tiled_plan(ctx, "single", Xr, Xc, 1, vt, 1, false, &tp);
        if (st2 != PCG_OK) return st2;
    }
    if (tp.valid) {
        TiledKernels TK{};
        pcg_status st2 = tiled_prepare(ctx, tp, &TK);
        if (st2 != PCG_OK) return st2;
        TiledArgs ta{tp};
        const bool df = prec_pairs(prec);
        if (f32) PCG_PROF(ctx, "to_f32", k_to_f32<<<grid, 256, 0, s>>>(v, ws.s32, d.p));
        if (df) PCG_PROF(ctx, "to_df", k_to_df<<<grid, 256, 0, s>>>(v, ws.sdf, d.p));
        PCG_PROF(ctx, "rhs_w", k_rhs_w<<<grid, 256, 0, s>>>(ws.desc, nullptr, ws.om32, 0, f32 ? 1 : 0,
                                                            (f32 || df) ? nullptr : ws.om64,
                                                            df ? ws.omdf : nullptr));
        const void *sg = f32 ? (const void *)ws.s32 : df ? (const void *)ws.sdf : (const void *)v;
        const void *omt = f32 ? (const void *)ws.om32 : df ? (const void *)ws.omdf : (const void *)ws.om64;
        int one = 1, zero = 0;
        void *a1[] = {&ta, (void *)&sg, &one, &zero, (void *)&done, &zero};
        void *au[] = {&ta, (void *)&omt, &one, &zero, (void *)&done, &zero};
        void *pc = tp.Pc;
        void *a2[] = {&ta, &pc, &one, &zero, (void *)&done, &zero};
        PCG_PROF(ctx, "t_csr", cudaLaunchKernel(TK.csr, dim3(tp.T_c * tp.csr_blocks), dim3(tp.threads), a1, tp.smem_c, s));
        PCG_PROF(ctx, "t_u", cudaLaunchKernel(TK.u, dim3(tiled_u_blocks(tp, ctx->num_sms)), dim3(256), au, 0, s));
        PCG_PROF(ctx, "t_csc", cudaLaunchKernel(TK.csc, dim3(tp.T_r * tp.csc_chunks), dim3(tp.threads), a2, tp.smem_r, s));
        if (f32) PCG_PROF(ctx, "t_fin_out", k_t_fin_out<float><<<grid, 256, 0, s>>>(ws.desc, ta, v, out));
        else if (df) PCG_PROF(ctx, "t_fin_out", k_t_fin_out<float2><<<grid, 256, 0, s>>>(ws.desc, ta, v, out));
        else PCG_PROF(ctx, "t_fin_out", k_t_fin_out<double><<<grid, 256, 0, s>>>(ws.desc, ta, v, out));
    } else if (f32) {
        PCG_PROF(ctx, "to_f32", k_to_f32<<<grid, 256, 0, s>>>(v, ws.s32, d.p));
        PCG_PROF(ctx, "rhs_w", k_rhs_w<<<grid, 256, 0, s>>>(ws.desc, nullptr, ws.om32, 0, 1, nullptr, nullptr));
        PCG_PROF(ctx, "csr_f32", PCG_DISPATCH_G(Gr, (k_csr<float, GG><<<grid, 256, 0, s>>>(ws.desc, ws.s32, ws.om32, (float *)ws.u, done, nullptr))));
        PCG_PROF(ctx, "csc_f32", PCG_DISPATCH_G(Gc, (k_csc<float, GG><<<grid, 256, 0, s>>>(ws.desc, (const float *)ws.u, v, out, ws, 0))));
    } else {
        PCG_PROF(ctx, "csr_f64", PCG_DISPATCH_G(Gr, (k_csr<double, GG><<<grid, 256, 0, s>>>(ws.desc, v, omega, (double *)ws.u, done, nullptr))));
        PCG_PROF(ctx, "csc_f64", PCG_DISPATCH_G(Gc, (k_csc<double, GG><<<grid, 256, 0, s>>>(ws.desc, (const double *)ws.u, v, out, ws, 0))));
    }
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    prof_collect(ctx);
    return PCG_OK;
}

}  // namespace pcg
