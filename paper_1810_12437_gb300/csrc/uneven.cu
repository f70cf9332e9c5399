// Uneven batch: independent draws (each with its own X, omega, lambda, tau,
// eta, delta, and its own n and p) solved by ONE persistent kernel.
//
// Each problem advances through phases, every phase split into tiles:
//   W  rows  w = omega z + sqrt(omega) eta                      (Eq. 2.3, first two terms)
//   I  cols  b = X^T w + delta / (tau lambda); beta = 0; r = b; s = m b; rho_0
//   A  rows  u = omega (.) X s                                   (CSR pass)
//   B  cols  v = X^T u + d s; sigma = s.v; alpha = rho / sigma   (CSC pass)
//   C  vec   beta += alpha s; r -= alpha v; rho' = r.(m r); stop test (Eq. S2)
//   D1 rows  u64 = omega (.) X beta in float64                   (refined mode, when asked)
//   D2 cols  r = b - (X^T u64 + d beta); rho = r.(m r)
//   E  vec   s = m r + gamma s
// then A again until the problem stops.  CTAs take (problem, phase, tile)
// items from a per-problem claim word that packs the current phase with a
// claim count; the CTA that completes the last tile of a phase reduces the
// tiles' partial sums in tile order (so results do not depend on scheduling),
// updates the problem's CG scalars and publishes the next phase.  No CTA ever
// waits for another: an idle CTA backs off and gives up, setting a timeout
// flag, if no tile anywhere completes for `idle_limit_ns`.
//
// Products: float64 (s64, u64, omega gathered), float32 (float copies) or
// double-float (float-pair copies summed with TwoSum, about 48 bits; the
// fixed-point mode runs as double-float here).  Vectors written inside the
// kernel are read through L2 (ld.global.cg), never through the non-coherent
// read-only path, because they change between phases.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <fstream>
#include <type_traits>
#include <sstream>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "df.cuh"
#include "internal.h"

namespace pcg {

enum : int { PH_W = 0, PH_I = 1, PH_A = 2, PH_B = 3, PH_C = 4, PH_D1 = 5, PH_D2 = 6, PH_E = 7, PH_TERM = 15 };

struct UProb {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *omega, *z, *lambda, *eta, *delta;
    double *beta;
    double tau;
    int64_t n, p;
    // workspace
    double *b, *r, *s64, *v64, *u64, *part;
    float *s32, *u32, *om32;
    int nt_row, nt_col, nt_vec;
    int rows_per_tile, cols_per_tile, vec_per_tile;
    int g_row, g_col;   // lanes per row / column (power of two <= 32)
    int df;             // double-float products: s32, u32, om32 hold float pairs
};

struct __align__(128) UState {
    unsigned long long claim;   // phase << 56 | claimed tiles
    unsigned int done;          // completed tiles of the current phase
    int pad0;
    CgScalars sc;
};

struct UGlobal {
    int finished;               // problems that reached PH_TERM
    int timeout;                // set when an idle CTA gave up
    unsigned long long progress;// completed tiles, all problems
    double tol;
    int max_iter, stop_rule, refined, reliable_k;
    long long idle_limit_ns;
};

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ntiles(const UProb &P, int ph) {
    switch (ph) {
        case PH_W: case PH_A: case PH_D1: return P.nt_row;
        case PH_I: case PH_B: case PH_D2: return P.nt_col;
        case PH_C: case PH_E: return P.nt_vec;
        default: return 0;
    }
}

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// coherent (L2) loads of data produced inside the kernel
template <typename T>
__device__ __forceinline__ T ldc(const T *p) { return __ldcg(p); }

// sum over a group of g lanes (g runtime, power of two); all lanes call it
template <typename T>
__device__ __forceinline__ T gsum(T v, int g) {
    for (int o = g >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// A double-float value (a float pair summed with TwoSum, about 48 bits):
// the gathered type of the double-float products of the persistent kernel.
struct DFv {
    float2 v;
    __device__ __forceinline__ DFv() : v(make_float2(0.f, 0.f)) {}
    __device__ __forceinline__ explicit DFv(int) : v(make_float2(0.f, 0.f)) {}
    __device__ __forceinline__ explicit DFv(float2 x) : v(x) {}
    __device__ __forceinline__ DFv operator+(const DFv &o) const { return DFv(df_add(v, o.v)); }
    __device__ __forceinline__ DFv &operator+=(const DFv &o) { v = df_add(v, o.v); return *this; }
    __device__ __forceinline__ DFv operator*(const DFv &o) const { return DFv(df_mul(v, o.v)); }
    __device__ __forceinline__ explicit operator double() const { return df_to_double(v); }
};

template <>
__device__ __forceinline__ DFv ldc<DFv>(const DFv *p) {
    return DFv(__ldcg(reinterpret_cast<const float2 *>(p)));
}

template <>
__device__ __forceinline__ DFv gsum<DFv>(DFv x, int g) {
    for (int o = g >> 1; o > 0; o >>= 1) {
        const float2 y = make_float2(__shfl_xor_sync(kFull, x.v.x, o), __shfl_xor_sync(kFull, x.v.y, o));
        x += DFv(y);
    }
    return x;
}

// Where each product type reads and writes its vectors: float32 copies,
// float64 originals, or float-pair copies (the float32 buffers, twice as long).
template <typename T> struct Src;
template <> struct Src<float> {
    __device__ static const float *s(const UProb &P) { return P.s32; }
    __device__ static float *u(const UProb &P) { return P.u32; }
    __device__ static const float *om(const UProb &P) { return P.om32; }
};
template <> struct Src<double> {
    __device__ static const double *s(const UProb &P) { return P.s64; }
    __device__ static double *u(const UProb &P) { return P.u64; }
    __device__ static const double *om(const UProb &P) { return P.omega; }
};
template <> struct Src<DFv> {
    __device__ static const DFv *s(const UProb &P) { return reinterpret_cast<const DFv *>(P.s32); }
    __device__ static DFv *u(const UProb &P) { return reinterpret_cast<DFv *>(P.u32); }
    __device__ static const DFv *om(const UProb &P) { return reinterpret_cast<const DFv *>(P.om32); }
};

// the float copy of a float64 value in the problem's gather format
__device__ __forceinline__ void store_copy(float *buf, int64_t i, double x, int df) {
    if (df) reinterpret_cast<float2 *>(buf)[i] = df_from_double(x);
    else buf[i] = (float)x;
}

// Tile loop helper: segments [s0, s1) handled by groups of g lanes over the CTA.
// For each segment calls body(seg, lane, active) uniformly across the warp.
template <typename F>
__device__ __forceinline__ void for_segments(int64_t s0, int64_t s1, int g, F body) {
    const int lane = threadIdx.x & (g - 1);
    const int gpw = 32 / g;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int sub = (threadIdx.x & 31) / g;
    for (int64_t base = s0 + (int64_t)warp * gpw; base < s1; base += (int64_t)nwarps * gpw) {
        const int64_t seg = base + sub;
        body(seg, lane, seg < s1);
    }
}

template <typename T>
__device__ __forceinline__ T seg_sum_coherent(const int32_t *__restrict__ idx, int64_t k0, int64_t k1,
                                              const T *x, int lane, int g) {
    T acc = T(0);
    int64_t k = k0 + lane;
    for (; k + 3 * g < k1; k += 4 * g) {
        const int32_t j0 = ld_stream(idx + k), j1 = ld_stream(idx + k + g);
        const int32_t j2 = ld_stream(idx + k + 2 * g), j3 = ld_stream(idx + k + 3 * g);
        acc += (ldc(x + j0) + ldc(x + j1)) + (ldc(x + j2) + ldc(x + j3));
    }
    for (; k < k1; k += g) acc += ldc(x + ld_stream(idx + k));
    return acc;
}

// ---------------------------------------------------------------------------
// tile bodies (whole CTA); partial sums go to P.part[t] (one per tile)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void tile_rows(const UProb &P, int ph, int t, const UState &S) {
    const int64_t r0 = (int64_t)t * P.rows_per_tile;
    const int64_t r1 = imin64(P.n, r0 + P.rows_per_tile);
    if (ph == PH_W) {
        const bool copy = !std::is_same<T, double>::value;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const double o = P.omega[i];
            P.u64[i] = o * P.z[i] + sqrt(o) * P.eta[i];
            if (copy) store_copy(P.om32, i, o, P.df);
        }
        return;
    }
    const int g = P.g_row;
    if (ph == PH_A) {
        const T *s = Src<T>::s(P);
        T *u = Src<T>::u(P);
        const T *om = Src<T>::om(P);
        for_segments(r0, r1, g, [&](int64_t i, int lane, bool act) {
            T acc = act ? seg_sum_coherent<T>(P.col_idx, P.row_ptr[i], P.row_ptr[i + 1], s, lane, g) : T(0);
            acc = gsum(acc, g);
            if (act && lane == 0) u[i] = ldc(om + i) * acc;
        });
    } else {   // PH_D1: float64 product on beta
        for_segments(r0, r1, g, [&](int64_t i, int lane, bool act) {
            double acc = act ? seg_sum_coherent<double>(P.col_idx, P.row_ptr[i], P.row_ptr[i + 1], P.beta, lane, g) : 0.0;
            acc = gsum(acc, g);
            if (act && lane == 0) P.u64[i] = P.omega[i] * acc;
        });
    }
}

template <typename T>
__device__ void tile_cols(const UProb &P, int ph, int t, const UState &S, double *red) {
    const int64_t c0 = (int64_t)t * P.cols_per_tile;
    const int64_t c1 = imin64(P.p, c0 + P.cols_per_tile);
    const int g = P.g_col;
    const double tau = P.tau;
    double part = 0.0;
    if (ph == PH_I) {
        for_segments(c0, c1, g, [&](int64_t j, int lane, bool act) {
            double acc = act ? seg_sum_coherent<double>(P.row_idx, P.col_ptr[j], P.col_ptr[j + 1], P.u64, lane, g) : 0.0;
            acc = gsum(acc, g);
            if (act && lane == 0) {
                const double lam = P.lambda[j];
                const double b = acc + P.delta[j] / (tau * lam);
                const double z = prior_var(tau, lam) * b;
                P.b[j] = b;
                P.r[j] = b;
                P.s64[j] = z;
                store_copy(P.s32, j, z, P.df);
                P.beta[j] = 0.0;
                part += b * z;
            }
        });
    } else if (ph == PH_B) {
        const T *u = Src<T>::u(P);
        for_segments(c0, c1, g, [&](int64_t j, int lane, bool act) {
            T acc = act ? seg_sum_coherent<T>(P.row_idx, P.col_ptr[j], P.col_ptr[j + 1], u, lane, g) : T(0);
            acc = gsum(acc, g);
            if (act && lane == 0) {
                const double sj = ldc(P.s64 + j);
                const double v = (double)acc + prior_prec(tau, P.lambda[j]) * sj;
                P.v64[j] = v;
                part += sj * v;
            }
        });
    } else {   // PH_D2
        for_segments(c0, c1, g, [&](int64_t j, int lane, bool act) {
            double acc = act ? seg_sum_coherent<double>(P.row_idx, P.col_ptr[j], P.col_ptr[j + 1], P.u64, lane, g) : 0.0;
            acc = gsum(acc, g);
            if (act && lane == 0) {
                const double lam = P.lambda[j];
                const double rj = ldc(P.b + j) - (acc + prior_prec(tau, lam) * ldc(P.beta + j));
                P.r[j] = rj;
                part += rj * (prior_var(tau, lam) * rj);
            }
        });
    }
    const double tot = block_sum(part, red);
    if (threadIdx.x == 0) P.part[t] = tot;
}

__device__ void tile_vec(const UProb &P, int ph, int t, const UState &S, double *red) {
    const int64_t a = (int64_t)t * P.vec_per_tile;
    const int64_t e = imin64(P.p, a + P.vec_per_tile);
    const double tau = P.tau;
    if (ph == PH_C) {
        const double alpha = ldc(&S.sc.alpha);
        double part = 0.0;
        for (int64_t j = a + threadIdx.x; j < e; j += blockDim.x) {
            const double bj = ldc(P.beta + j) + alpha * ldc(P.s64 + j);
            const double rj = ldc(P.r + j) - alpha * ldc(P.v64 + j);
            P.beta[j] = bj;
            P.r[j] = rj;
            part += rj * (prior_var(tau, P.lambda[j]) * rj);
        }
        const double tot = block_sum(part, red);
        if (threadIdx.x == 0) P.part[t] = tot;
    } else {   // PH_E
        const double gamma = ldc(&S.sc.gamma);
        for (int64_t j = a + threadIdx.x; j < e; j += blockDim.x) {
            const double s = prior_var(tau, P.lambda[j]) * ldc(P.r + j) + gamma * ldc(P.s64 + j);
            P.s64[j] = s;
            store_copy(P.s32, j, s, P.df);
        }
    }
}

// Sum of the tile partials in tile order (deterministic); valid in thread 0.
__device__ double reduce_parts(const UProb &P, int nt, double *red) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) acc += ldc(P.part + k);
    return block_sum(acc, red);
}

// Finalise phase `ph` of problem q (whole CTA calls; thread 0 decides) and
// publish the next phase.
__device__ void finalize(const UProb &P, UState &S, UGlobal &G, int ph, double *red) {
    double tot = 0.0;
    if (ph == PH_I || ph == PH_B || ph == PH_C || ph == PH_D2) tot = reduce_parts(P, ntiles(P, ph), red);
    if (threadIdx.x == 0) {
        // the scalars were last written by whichever CTA finalised the previous
        // phase, possibly on another SM: read them through L2, not L1
        CgScalars sc;
        constexpr int NW = sizeof(CgScalars) / sizeof(unsigned long long);
        static_assert(sizeof(CgScalars) % sizeof(unsigned long long) == 0, "CgScalars layout");
        unsigned long long *lw = reinterpret_cast<unsigned long long *>(&sc);
        unsigned long long *gw = reinterpret_cast<unsigned long long *>(&S.sc);
        for (int k = 0; k < NW; ++k) lw[k] = __ldcg(gw + k);
        const int64_t p = P.p;
        int nx = PH_TERM;
        switch (ph) {
            case PH_W: nx = PH_I; break;
            case PH_I: {
                sc.rho = sc.rho0 = sc.rho_prev = tot;
                sc.sigma = sc.alpha = sc.gamma = 0.0;
                sc.iter = 0;
                sc.need_ru = sc.pending = 0;
                sc.ru_trips = 0;
                sc.resid = stop_quantity(G.stop_rule, tot, tot, p);
                if (!isfinite(tot)) { sc.status = PCG_NONFINITE; }
                else if (stop_met(G.stop_rule, tot, tot, p, G.tol)) { sc.status = PCG_OK; }
                else if (G.max_iter <= 0) { sc.status = PCG_MAXITER; }
                else { sc.status = kRunning; nx = PH_A; }
                break;
            }
            case PH_A: nx = PH_B; break;
            case PH_B: {
                sc.sigma = tot;
                if (!isfinite(tot)) sc.status = PCG_NONFINITE;
                else if (!(tot > 0.0) || !(sc.rho > 0.0)) sc.status = PCG_BREAKDOWN;
                else { sc.alpha = sc.rho / tot; nx = PH_C; }
                break;
            }
            case PH_C: {
                const double rn = tot;
                sc.iter += 1;
                if (!isfinite(rn)) { sc.status = PCG_NONFINITE; break; }
                const bool conv = stop_met(G.stop_rule, rn, sc.rho0, p, G.tol);
                sc.rho_prev = sc.rho;
                sc.rho = rn;
                sc.gamma = rn / sc.rho_prev;
                sc.resid = stop_quantity(G.stop_rule, rn, sc.rho0, p);
                if (G.refined) {
                    const bool periodic = G.reliable_k > 0 && (sc.iter % G.reliable_k) == 0;
                    sc.pending = conv ? 1 : 0;
                    if (conv || periodic) { nx = PH_D1; sc.ru_trips += 1; }
                    else if (sc.iter >= G.max_iter) sc.status = PCG_MAXITER;
                    else nx = PH_E;
                } else if (conv) {
                    sc.status = PCG_OK;
                } else if (sc.iter >= G.max_iter) {
                    sc.status = PCG_MAXITER;
                } else {
                    nx = PH_E;
                }
                break;
            }
            case PH_D1: nx = PH_D2; break;
            case PH_D2: {
                const double rt = tot;
                if (!isfinite(rt)) { sc.status = PCG_NONFINITE; break; }
                sc.rho = rt;
                sc.gamma = rt / sc.rho_prev;
                sc.resid = stop_quantity(G.stop_rule, rt, sc.rho0, p);
                if (sc.pending && stop_met(G.stop_rule, rt, sc.rho0, p, G.tol)) {
                    sc.status = PCG_OK;
                } else if (sc.iter >= G.max_iter) {
                    sc.status = PCG_MAXITER;
                } else {
                    // float64 residual above the rule after the recursion met
                    // it: restart from the float64 residual
                    if (sc.pending) sc.gamma = 0.0;
                    sc.pending = 0;
                    nx = PH_E;
                }
                break;
            }
            case PH_E: nx = PH_A; break;
            default: break;
        }
        if (nx == PH_TERM) sc.done = 1;
        for (int k = 0; k < NW; ++k) __stcg(gw + k, lw[k]);
        S.done = 0u;
        __threadfence();
        atomicExch(&S.claim, (unsigned long long)nx << 56);
        if (nx == PH_TERM) atomicAdd(&G.finished, 1);
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_uneven(const UProb *__restrict__ probs, UState *st,
                                                UGlobal *g, int nprob) {
    __shared__ double red[32];
    __shared__ int s_q, s_ph, s_t, s_last;
    int q0 = blockIdx.x % nprob;          // thread 0 only
    unsigned long long idle_since = 0, seen = 0;
    while (true) {
        if (threadIdx.x == 0) {
            s_q = -1;
            if (*(volatile int *)&g->finished >= nprob || *(volatile int *)&g->timeout) {
                s_q = -2;
            } else {
                for (int k = 0; k < nprob; ++k) {
                    const int q = (q0 + k) % nprob;
                    const unsigned long long w = *(volatile unsigned long long *)&st[q].claim;
                    int ph = (int)(w >> 56);
                    if (ph == PH_TERM || (unsigned)(w & 0xffffffffull) >= (unsigned)ntiles(probs[q], ph)) continue;
                    const unsigned long long old = atomicAdd(&st[q].claim, 1ull);
                    ph = (int)(old >> 56);
                    const unsigned t = (unsigned)(old & 0xffffffffull);
                    if (ph != PH_TERM && t < (unsigned)ntiles(probs[q], ph)) {
                        s_q = q;
                        s_ph = ph;
                        s_t = (int)t;
                        q0 = q;
                        break;
                    }
                }
            }
            __threadfence();
        }
        __syncthreads();
        const int q = s_q;
        if (q == -2) break;
        if (q == -1) {
            if (threadIdx.x == 0) {
                const unsigned long long prog = *(volatile unsigned long long *)&g->progress;
                const unsigned long long now = globaltimer();
                if (prog != seen || idle_since == 0) {
                    seen = prog;
                    idle_since = now;
                } else if ((long long)(now - idle_since) > g->idle_limit_ns) {
                    atomicExch(&g->timeout, 1);
                }
                __nanosleep(200);
            }
            __syncthreads();
            continue;
        }
        idle_since = 0;
        const UProb &P = probs[q];
        const int ph = s_ph, t = s_t;
        switch (ph) {
            case PH_W: case PH_A: case PH_D1: tile_rows<T>(P, ph, t, st[q]); break;
            case PH_I: case PH_B: case PH_D2: tile_cols<T>(P, ph, t, st[q], red); break;
            default: tile_vec(P, ph, t, st[q], red); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned c = atomicAdd(&st[q].done, 1u);
            s_last = (c + 1 == (unsigned)ntiles(P, ph)) ? 1 : 0;
            atomicAdd(&g->progress, 1ull);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            finalize(P, st[q], *g, ph, red);
        }
    }
}

// ===========================================================================
// host side: workspace layout, autotuned tile shapes, graph with one node
// ===========================================================================
struct UTile {
    int rows, cols, vec, per_sm;
};

static int pick_g(double mean) { return mean < 6 ? 4 : mean < 20 ? 8 : mean < 56 ? 16 : 32; }

static std::string signature(int nprob, const pcg_problem *probs, int prec) {
    long long tn = 0, tp = 0, tz = 0;
    for (int q = 0; q < nprob; ++q) {
        tn += probs[q].X_csr.n;
        tp += probs[q].X_csr.p;
        tz += probs[q].X_csr.nnz;
    }
    char buf[128];
    snprintf(buf, sizeof buf, "uneven:%d:%lld:%lld:%lld:%d", nprob, tn, tp, tz, prec);
    return buf;
}

static bool load_cache(pcg_ctx *ctx, const std::string &key, UTile *t) {
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end() && it->second.size() == 4) {
        *t = {it->second[0], it->second[1], it->second[2], it->second[3]};
        return true;
    }
    if (!ctx->opt.autotune_cache) return false;
    std::ifstream f(ctx->opt.autotune_cache);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream ss(line);
        std::string k;
        UTile u{};
        if (ss >> k >> u.rows >> u.cols >> u.vec >> u.per_sm && k == key) {
            *t = u;
            ctx->tuned[key] = {u.rows, u.cols, u.vec, u.per_sm};
            return true;
        }
    }
    return false;
}

static void store_cache(pcg_ctx *ctx, const std::string &key, const UTile &t) {
    ctx->tuned[key] = {t.rows, t.cols, t.vec, t.per_sm};
    if (!ctx->opt.autotune_cache) return;
    std::ofstream f(ctx->opt.autotune_cache, std::ios::app);
    f << key << " " << t.rows << " " << t.cols << " " << t.vec << " " << t.per_sm << "\n";
}

struct UnevenPlan {
    UProb *d_probs = nullptr;
    UState *d_state = nullptr;
    UGlobal *d_glob = nullptr;
    std::vector<UProb> h_probs;
    int grid = 0;
};

// Product arithmetic of the persistent kernel: float64, float32, or double-float
// (float pairs summed with TwoSum; also serves PCG_PREC_FX64).
enum UKind { kU64 = 0, kU32 = 1, kUDF = 2 };

static UKind uneven_kind(int precision) {
    return precision == PCG_PREC_FP64 ? kU64 : prec_pairs(precision) ? kUDF : kU32;
}

static const void *uneven_kernel(UKind k) {
    return k == kU64 ? (const void *)k_uneven<double> : k == kUDF ? (const void *)k_uneven<DFv>
                                                                   : (const void *)k_uneven<float>;
}

static pcg_status plan_uneven(pcg_ctx *ctx, int nprob, const pcg_problem *probs, const UTile &tile,
                              UKind kind, UnevenPlan *pl) {
    const int fw = kind == kUDF ? 2 : 1;   // floats per copied value
    // workspace sizes
    size_t dbl = 0, flt = 0;
    std::vector<UProb> hp(nprob);
    int max_nt = 1;
    for (int q = 0; q < nprob; ++q) {
        const pcg_problem &pr = probs[q];
        const int64_t n = pr.X_csr.n, p = pr.X_csr.p;
        UProb &P = hp[q];
        P = UProb{};
        P.row_ptr = pr.X_csr.row_ptr;
        P.col_idx = pr.X_csr.col_idx;
        P.col_ptr = pr.X_csc.col_ptr;
        P.row_idx = pr.X_csc.row_idx;
        P.omega = pr.omega;
        P.z = pr.z;
        P.lambda = pr.lambda;
        P.eta = pr.eta;
        P.delta = pr.delta;
        P.beta = pr.beta;
        P.tau = pr.tau;
        P.n = n;
        P.p = p;
        P.rows_per_tile = tile.rows;
        P.cols_per_tile = tile.cols;
        P.vec_per_tile = tile.vec;
        P.nt_row = (int)((n + tile.rows - 1) / tile.rows);
        P.nt_col = (int)((p + tile.cols - 1) / tile.cols);
        P.nt_vec = (int)((p + tile.vec - 1) / tile.vec);
        if (P.nt_row == 0) P.nt_row = 1;   // empty phases still complete once
        if (P.nt_col == 0) P.nt_col = 1;
        if (P.nt_vec == 0) P.nt_vec = 1;
        P.g_row = pick_g(n > 0 ? (double)pr.X_csr.nnz / n : 1.0);
        P.g_col = pick_g(p > 0 ? (double)pr.X_csr.nnz / p : 1.0);
        max_nt = std::max({max_nt, P.nt_col, P.nt_vec});
        // exactly what the carving below takes (each array rounded up to 4 elements)
        auto r4 = [](int64_t x) { return (size_t)((x + 3) & ~int64_t(3)); };
        dbl += 4 * r4(p) + r4(n) + r4(std::max(P.nt_col, P.nt_vec));   // b r s64 v64, u64, part
        flt += fw * (r4(p) + 2 * r4(n));                                 // s32, u32, om32
        P.df = kind == kUDF ? 1 : 0;
    }
    cudaError_t e;
    char *wd = (char *)grow(ctx, "uneven_d", sizeof(double) * dbl + 256, &e);
    if (!wd) return cuda_error(ctx, e, "allocating the uneven workspace");
    char *wf = (char *)grow(ctx, "uneven_f", sizeof(float) * flt + 256, &e);
    if (!wf) return cuda_error(ctx, e, "allocating the uneven workspace");
    double *pd = (double *)wd;
    float *pf = (float *)wf;
    for (int q = 0; q < nprob; ++q) {
        UProb &P = hp[q];
        const int64_t n = P.n, p = P.p;
        auto a4 = [](int64_t x) { return (x + 3) & ~int64_t(3); };
        P.b = pd; pd += a4(p);
        P.r = pd; pd += a4(p);
        P.s64 = pd; pd += a4(p);
        P.v64 = pd; pd += a4(p);
        P.u64 = pd; pd += a4(n);
        P.part = pd; pd += a4(std::max(P.nt_col, P.nt_vec));
        P.s32 = pf; pf += fw * a4(p);
        P.u32 = pf; pf += fw * a4(n);
        P.om32 = pf; pf += fw * a4(n);
    }
    pl->d_probs = (UProb *)grow(ctx, "uneven_probs", sizeof(UProb) * nprob, &e);
    if (!pl->d_probs) return cuda_error(ctx, e, "allocating the uneven descriptors");
    pl->d_state = (UState *)grow(ctx, "uneven_state", sizeof(UState) * nprob, &e);
    if (!pl->d_state) return cuda_error(ctx, e, "allocating the uneven state");
    pl->d_glob = (UGlobal *)grow(ctx, "uneven_glob", sizeof(UGlobal), &e);
    if (!pl->d_glob) return cuda_error(ctx, e, "allocating the uneven state");
    pl->h_probs = hp;
    int occ = 0;
    PCG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, uneven_kernel(kind), 256, 0));
    pl->grid = ctx->num_sms * std::max(1, std::min(occ, tile.per_sm));
    return PCG_OK;
}

// One timed or real run of the persistent kernel through a one-node graph.
static pcg_status launch_uneven(pcg_ctx *ctx, int nprob, UnevenPlan &pl, UKind kind, double tol,
                                int max_iter, float *ms_out) {
    cudaError_t e;
    UProb *hp = (UProb *)grow_host(ctx, "uneven_hprobs", sizeof(UProb) * nprob, &e);
    UGlobal *hg = (UGlobal *)grow_host(ctx, "uneven_hglob", sizeof(UGlobal), &e);
    if (!hp || !hg) return cuda_error(ctx, e, "allocating pinned staging");
    std::copy(pl.h_probs.begin(), pl.h_probs.end(), hp);
    UGlobal G{};
    G.tol = tol;
    G.max_iter = max_iter;
    G.stop_rule = ctx->opt.stop_rule;
    // float64 recomputation of r: the float32-refined mode only
    G.refined = ctx->opt.precision == PCG_PREC_FP32_REFINED ? 1 : 0;
    G.reliable_k = ctx->opt.reliable_k;
    // give up after this long without any completed tile anywhere
    G.idle_limit_ns = (long long)llround(ctx->opt.idle_limit_s * 1e9);
    *hg = G;
    cudaStream_t s = ctx->stream;
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(pl.d_probs, hp, sizeof(UProb) * nprob, cudaMemcpyHostToDevice, s));
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(pl.d_glob, hg, sizeof(UGlobal), cudaMemcpyHostToDevice, s));
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(pl.d_state, 0, sizeof(UState) * nprob, s));   // all at PH_W, count 0
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        cudaError_t ce = cudaEventCreate(&e0);
        if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
        if (ce != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            return cuda_error(ctx, ce, "timing an autotune candidate");
        }
    }
    std::string key = std::string("uneven_graph:") + std::to_string((int)kind) + ":" + std::to_string(pl.grid) +
                      ":" + std::to_string(nprob) + ":" + std::to_string((uintptr_t)pl.d_probs) + ":" +
                      std::to_string((uintptr_t)pl.d_state) + ":" + std::to_string((uintptr_t)pl.d_glob);
    if (ctx->opt.use_graph && !ctx->opt.profile) {
        auto it = ctx->named_graphs.find(key);
        cudaGraphExec_t exec = nullptr;
        if (it == ctx->named_graphs.end()) {
            cudaGraph_t g = nullptr;
            PCG_CUDA_TRY(ctx, cudaGraphCreate(&g, 0));
            cudaKernelNodeParams kp = {};
            const UProb *a0 = pl.d_probs;
            UState *a1 = pl.d_state;
            UGlobal *a2 = pl.d_glob;
            int a3 = nprob;
            void *args[] = {&a0, &a1, &a2, &a3};
            kp.func = (void *)uneven_kernel(kind);
            kp.gridDim = dim3(pl.grid);
            kp.blockDim = dim3(256);
            kp.kernelParams = args;
            cudaGraphNode_t node;
            cudaError_t ee = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp);
            if (ee == cudaSuccess) ee = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (ee != cudaSuccess) return cuda_error(ctx, ee, "building the uneven-batch graph");
            ctx->named_graphs[key] = exec;
        } else {
            exec = it->second;
        }
        PCG_CUDA_TRY(ctx, cudaGraphLaunch(exec, s));
        ctx->last_launches += 1;
    } else {
        const UProb *a0 = pl.d_probs;
        UState *a1 = pl.d_state;
        UGlobal *a2 = pl.d_glob;
        int a3 = nprob;
        void *args[] = {&a0, &a1, &a2, &a3};
        PCG_PROF(ctx, "uneven_persistent",
                 cudaLaunchKernel(uneven_kernel(kind), dim3(pl.grid), dim3(256), args, 0, s));
    }
    cudaError_t le = cudaGetLastError();
    if (ms_out) {
        cudaError_t ce = le;
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms_out, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (ce != cudaSuccess) return cuda_error(ctx, ce, "timing an autotune candidate");
    }
    PCG_CUDA_TRY(ctx, le);
    return PCG_OK;
}

static pcg_status run_uneven_active(pcg_ctx *ctx, int nprob, const pcg_problem *probs, double tol,
                                    int max_iter, int *iters, double *resid, int *status);

pcg_status run_uneven(pcg_ctx *ctx, int nprob, const pcg_problem *probs, double tol, int max_iter,
                      int *iters, double *resid, int *status) {
    // problems with p = 0 have nothing to draw (and may carry NULL vectors):
    // they never enter the kernel
    std::vector<pcg_problem> act;
    std::vector<int> map;
    for (int q = 0; q < nprob; ++q) {
        iters[q] = 0;
        resid[q] = 0.0;
        status[q] = PCG_OK;
        if (probs[q].X_csr.p > 0) {
            act.push_back(probs[q]);
            map.push_back(q);
        }
    }
    if (act.empty()) return PCG_OK;
    std::vector<int> it(act.size()), stt(act.size());
    std::vector<double> rs(act.size());
    pcg_status st = run_uneven_active(ctx, (int)act.size(), act.data(), tol, max_iter, it.data(),
                                      rs.data(), stt.data());
    for (size_t k = 0; k < act.size(); ++k) {
        iters[map[k]] = it[k];
        resid[map[k]] = rs[k];
        status[map[k]] = stt[k];
    }
    return st;
}

static pcg_status run_uneven_active(pcg_ctx *ctx, int nprob, const pcg_problem *probs, double tol,
                                    int max_iter, int *iters, double *resid, int *status) {
    const UKind kind = uneven_kind(ctx->opt.precision);
    const std::string sig = signature(nprob, probs, ctx->opt.precision);
    UTile tile{};
    if (!load_cache(ctx, sig, &tile)) {
        // autotune: time the whole batch for each candidate tile shape and keep
        // the fastest (the candidates' results are recomputed below)
        const UTile cands[] = {{256, 64, 8192, 8},   {1024, 128, 8192, 8}, {4096, 512, 16384, 8},
                               {1024, 256, 16384, 4}, {512, 64, 4096, 6},  {2048, 256, 8192, 6},
                               {128, 32, 4096, 8},    {64, 16, 2048, 8}};
        float best = 1e30f;
        UTile bt = cands[1];
        for (const UTile &c : cands) {
            UnevenPlan pl;
            pcg_status st = plan_uneven(ctx, nprob, probs, c, kind, &pl);
            if (st != PCG_OK) return st;
            float ms = 0.f;
            st = launch_uneven(ctx, nprob, pl, kind, tol, max_iter, &ms);
            if (st != PCG_OK) return st;
            if (ms < best) {
                best = ms;
                bt = c;
            }
        }
        tile = bt;
        store_cache(ctx, sig, tile);
        ctx->last_launches = 0;
    }
    UnevenPlan pl;
    pcg_status st = plan_uneven(ctx, nprob, probs, tile, kind, &pl);
    if (st != PCG_OK) return st;
    st = launch_uneven(ctx, nprob, pl, kind, tol, max_iter, nullptr);
    if (st != PCG_OK) return st;
    cudaError_t e;
    UState *hs = (UState *)grow_host(ctx, "uneven_hstate", sizeof(UState) * nprob, &e);
    UGlobal *hg = (UGlobal *)grow_host(ctx, "uneven_hglob2", sizeof(UGlobal), &e);
    if (!hs || !hg) return cuda_error(ctx, e, "allocating pinned staging");
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hs, pl.d_state, sizeof(UState) * nprob, cudaMemcpyDeviceToHost, ctx->stream));
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hg, pl.d_glob, sizeof(UGlobal), cudaMemcpyDeviceToHost, ctx->stream));
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    pcg_status worst = PCG_OK;
    for (int q = 0; q < nprob; ++q) {
        iters[q] = hs[q].sc.iter;
        resid[q] = hs[q].sc.resid;
        int s = hs[q].sc.status;
        if (!hs[q].sc.done) s = PCG_TIMEOUT;
        status[q] = s;
        if (s > worst) worst = (pcg_status)s;
    }
    if (hg->timeout) return set_error(ctx, PCG_TIMEOUT, "uneven batch: an idle CTA gave up waiting for progress");
    if (worst != PCG_OK) return set_error(ctx, worst, "at least one problem did not converge (see status[])");
    return PCG_OK;
}

}  // namespace pcg
