// Batched draws sharing X: R chains, each with its own omega, lambda, tau,
// eta, delta and CG scalars, advanced together so that every iteration reads
// the index streams of X once for the whole block of right-hand sides:
//   U = Omega (.) (X S)           sparse times dense block (CSR pass)
//   V = X^T U + D (.) S           (CSC pass), sigma_r = S_r . V_r
// Vectors are interleaved [row][rhs] with the RHS count padded to RP (a power
// of two >= 4), so one nonzero gathers RP contiguous float32 values as RP/4
// float4 loads.  CG scalars, dot products, beta and r are float64; the
// refined mode recomputes r = b - Phi beta in float64 (Sec. 2.4 recursion,
// Eq. 2.3 right-hand sides, Eq. S2 stop rule per chain).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "device_common.cuh"
#include "df.cuh"
#include "internal.h"
#include "tiled.h"

namespace pcg {

struct BatchDesc {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *omega, *z, *lambda, *tau, *eta, *delta;   // caller, chain-major
    double *beta_out;                                     // caller, chain-major
    int64_t n, p, nnz;
    int R, RP;
    double tol;
    int max_iter, stop_rule, refined, reliable_k;
    int RG;   // right-hand sides per tiled product group (0: untiled products)
    int df;   // double-float products: s32 / om32 hold float pairs (float2)
    int tail; // a group-width-1 plan takes over the products when one chain is left
    // unshrunk coefficients 0 .. q1-1 of every chain (Sec. S4.3): prior precision
    // ud[j] (0: flat prior) and preconditioner variance um[j] = gamma_j^2
    int q1;
    const double *ud, *um;
};

// flags[] layout (kFlagInts ints, device):
//   [0] all chains done, [1] some chain needs the float64 recomputation,
//   [2] iterations that ran it, [3] a compaction was planned this iteration,
//   [4] active product groups, [5] compactions so far,
//   [6] 1 once the tail plan runs the products, [7] 0 while it runs (its gate),
//   [32 + s] chain held by slot s, [64 + s] old slot moved to slot s by the compaction,
//   [96 + g] 1 when product group g holds no live chain (its products are skipped).
constexpr int kFlagInts = 128;

struct BatchWs {
    double *b, *r, *s64, *v64, *beta, *m, *dg;   // p*RP each (interleaved)
    float *s32;                                  // p*RP floats, or p*RP float pairs (df)
    void *u;                                     // n*RP doubles (w64, then u32 / u64)
    double *om64;                                // n*RP
    float *om32;                                 // n*RP floats, or n*RP float pairs (df)
    float *s_tail, *om_tail;                     // the tail plan's chain (slot 0): s (p) and omega (n),
                                                 // contiguous, in the s32 / om32 element type
    double *partials;                            // kMaxReduceBlocks * 32
    unsigned int *counters;                      // 16
    CgScalars *sc;                               // 32
    int *flags;                                  // see the layout above
    BatchDesc *desc;
};

// Slots a per-element kernel must visit: those of the product groups still
// active (live chains sit in the low slots after compaction), rounded up to a
// power of two a2 <= RP so that a thread keeps one slot (threadIdx.x mod a2)
// and the rest of the grid covers the elements.  All RP slots before any
// compaction or in the untiled layout.
__device__ __forceinline__ int active_slots_pow2(const BatchDesc *__restrict__ d, const int *flags, int RP) {
    const int act = d->RG > 0 ? min(RP, flags[4] * d->RG) : RP;
    int a2 = 1;
    while (a2 < act) a2 <<= 1;
    return a2;
}

// Grid reduction of NV values per block held in shared memory (vals), summed
// in a fixed order.  Returns true in the last block, where sums[] holds the
// totals.
template <int NV>
__device__ bool grid_reduce_arr(const double *vals, double *partials, unsigned int *counter,
                                double *sums) {
    __shared__ bool am_last;
    __shared__ double tmp[256];
    __syncthreads();
    if (threadIdx.x < NV) partials[(size_t)blockIdx.x * NV + threadIdx.x] = vals[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    constexpr int NG = 256 / NV;
    const int k = threadIdx.x % NV, grp = threadIdx.x / NV;
    double a0 = 0.0, a1 = 0.0;
    if (grp < NG && threadIdx.x < 256) {
        unsigned b = grp;
        for (; b + NG < gridDim.x; b += 2 * NG) {
            a0 += __ldcg(partials + (size_t)b * NV + k);
            a1 += __ldcg(partials + (size_t)(b + NG) * NV + k);
        }
        if (b < gridDim.x) a0 += __ldcg(partials + (size_t)b * NV + k);
        tmp[threadIdx.x] = a0 + a1;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double a = 0.0;
        for (int g = 0; g < NG; ++g) a += tmp[g * NV + threadIdx.x];
        sums[threadIdx.x] = a;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4shfl_xor(float4 a, int o) {
    return make_float4(__shfl_xor_sync(kFull, a.x, o), __shfl_xor_sync(kFull, a.y, o),
                       __shfl_xor_sync(kFull, a.z, o), __shfl_xor_sync(kFull, a.w, o));
}
__device__ __forceinline__ double2 d2add(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 d2shfl_xor(double2 a, int o) {
    return make_double2(__shfl_xor_sync(kFull, a.x, o), __shfl_xor_sync(kFull, a.y, o));
}

// Sum over one CSR row / CSC column of the RP-wide float32 rows of x; lanes
// are (slot, chunk) with RP/4 chunks of 4 values.  Valid in slot-0 lanes.
template <int RP>
__device__ __forceinline__ float4 block_row_sum_f32(const int32_t *__restrict__ idx, int64_t k0,
                                                    int64_t k1, const float *__restrict__ x,
                                                    bool active) {
    constexpr int C = RP / 4, SL = 32 / C;
    const int lane = threadIdx.x & 31, c = lane % C, slot = lane / C;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
        int64_t k = k0 + slot;
        for (; k + SL < k1; k += 2 * SL) {
            const int32_t j0 = ld_stream(idx + k), j1 = ld_stream(idx + k + SL);
            const float4 a0 = __ldg(reinterpret_cast<const float4 *>(x + (size_t)j0 * RP) + c);
            const float4 a1 = __ldg(reinterpret_cast<const float4 *>(x + (size_t)j1 * RP) + c);
            acc = f4add(acc, f4add(a0, a1));
        }
        if (k < k1) {
            const int32_t j0 = ld_stream(idx + k);
            acc = f4add(acc, __ldg(reinterpret_cast<const float4 *>(x + (size_t)j0 * RP) + c));
        }
    }
#pragma unroll
    for (int o = 16; o >= C; o >>= 1) acc = f4add(acc, f4shfl_xor(acc, o));
    return acc;
}

// Same in float64 with RP/2 chunks of 2 values.
template <int RP>
__device__ __forceinline__ double2 block_row_sum_f64(const int32_t *__restrict__ idx, int64_t k0,
                                                     int64_t k1, const double *__restrict__ x,
                                                     bool active) {
    constexpr int C = RP / 2, SL = 32 / C;
    const int lane = threadIdx.x & 31, c = lane % C, slot = lane / C;
    double2 acc = make_double2(0.0, 0.0);
    if (active) {
        for (int64_t k = k0 + slot; k < k1; k += SL) {
            const int32_t j0 = ld_stream(idx + k);
            acc = d2add(acc, __ldg(reinterpret_cast<const double2 *>(x + (size_t)j0 * RP) + c));
        }
    }
#pragma unroll
    for (int o = 16; o >= C; o >>= 1) acc = d2add(acc, d2shfl_xor(acc, o));
    return acc;
}

// ---- right-hand sides -----------------------------------------------------
// w_{i,r} = omega z + sqrt(omega) eta; omega copies (float64 and float32),
// interleaved; padding columns are zero.
__global__ void k_b_prep(const BatchDesc *__restrict__ d, double *__restrict__ w,
                         double *__restrict__ om64, float *__restrict__ om32) {
    const int64_t n = d->n;
    const int R = d->R, RP = d->RP;
    const int64_t total = n * RP;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / n);
        const int64_t i = t - (int64_t)r * n;
        double wv = 0.0, o = 0.0;
        if (r < R) {
            o = d->omega[t];
            wv = o * d->z[t] + sqrt(o) * d->eta[t];
        }
        w[i * RP + r] = wv;
        om64[i * RP + r] = o;
        if (d->df) reinterpret_cast<float2 *>(om32)[i * RP + r] = df_from_double(o);
        else om32[i * RP + r] = (float)o;
    }
}

// b = X^T w + delta / (tau lambda); m, d; beta = 0, r = b, s = m b, rho_0.
template <int RP>
__global__ void __launch_bounds__(256) k_b_init(const BatchDesc *__restrict__ d,
                                                const double *__restrict__ w, BatchWs ws) {
    __shared__ double part[8][RP];
    __shared__ double vals[RP];
    __shared__ double sums[RP];
    constexpr int C = RP / 2;
    const int64_t p = d->p;
    const int R = d->R;
    const int lane = threadIdx.x & 31, c = lane % C, slot = lane / C, warp_in_blk = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double rho[2] = {0.0, 0.0};
    for (int64_t j = warp; j < p; j += nwarps) {
        const double2 acc = block_row_sum_f64<RP>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], w, true);
        if (slot == 0) {
            const double a[2] = {acc.x, acc.y};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int r = 2 * c + q;
                const size_t o = (size_t)j * RP + r;
                double b = 0.0, m = 0.0, dg = 0.0;
                if (r < R) {
                    const double tau = d->tau[r], lam = d->lambda[(size_t)r * p + j];
                    const bool un = j < d->q1;   // unshrunk coefficient
                    dg = un ? d->ud[j] : prior_prec(tau, lam);
                    m = un ? d->um[j] : prior_var(tau, lam);
                    const double dl = d->delta[(size_t)r * p + j];
                    b = a[q] + (un ? dl * sqrt(dg) : dl / (tau * lam));
                }
                const double zz = m * b;
                ws.b[o] = b;
                ws.r[o] = b;
                ws.m[o] = m;
                ws.dg[o] = dg;
                ws.s64[o] = zz;
                if (d->df) reinterpret_cast<float2 *>(ws.s32)[o] = df_from_double(zz);
                else ws.s32[o] = (float)zz;
                ws.beta[o] = 0.0;
                rho[q] += b * zz;
            }
        }
    }
    if (slot == 0) {
        part[warp_in_blk][2 * c] = rho[0];
        part[warp_in_blk][2 * c + 1] = rho[1];
    }
    __syncthreads();
    if (threadIdx.x < RP) {
        double a = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) a += part[w2][threadIdx.x];
        vals[threadIdx.x] = a;
    }
    if (grid_reduce_arr<RP>(vals, ws.partials, ws.counters + 0, sums)) {
        const int r = threadIdx.x;
        if (r < R) {
            CgScalars *sc = ws.sc + r;
            const double r0 = sums[r];
            sc->rho = r0;
            sc->rho0 = r0;
            sc->rho_prev = r0;
            sc->sigma = sc->alpha = sc->gamma = 0.0;
            sc->iter = 0;
            sc->need_ru = 0;
            sc->pending = 0;
            sc->resid = stop_quantity(d->stop_rule, r0, r0, p);
            if (!isfinite(r0)) { sc->status = PCG_NONFINITE; sc->done = 1; }
            else if (stop_met(d->stop_rule, r0, r0, p, d->tol)) { sc->status = PCG_OK; sc->done = 1; }
            else if (d->max_iter <= 0) { sc->status = PCG_MAXITER; sc->done = 1; }
            else { sc->status = kRunning; sc->done = 0; }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int q = 0; q < R; ++q) all &= ws.sc[q].done ? 1 : 0;
            ws.flags[0] = all;
            ws.flags[1] = 0;
            ws.flags[2] = 0;
            ws.flags[3] = 0;
            ws.flags[4] = d->RG > 0 ? RP / d->RG : 1;
            ws.flags[5] = 0;
            ws.flags[6] = 0;
            ws.flags[7] = 1;
        }
        if (threadIdx.x < 32) {
            ws.flags[96 + threadIdx.x] = 0;
            ws.flags[32 + threadIdx.x] = threadIdx.x;
            ws.flags[64 + threadIdx.x] = threadIdx.x;
        }
    }
}

// ---- per-iteration products -------------------------------------------------
template <int RP>
__global__ void __launch_bounds__(256) k_b_csr(const BatchDesc *__restrict__ d,
                                               const float *__restrict__ S,
                                               const float *__restrict__ om,
                                               float *__restrict__ U, const int *done_all) {
    if (*(volatile const int *)done_all) return;
    constexpr int C = RP / 4;
    const int64_t n = d->n;
    const int64_t *__restrict__ rp = d->row_ptr;
    const int lane = threadIdx.x & 31, c = lane % C, slot = lane / C;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const float4 acc = block_row_sum_f32<RP>(d->col_idx, rp[i], rp[i + 1], S, true);
        if (slot == 0) {
            const float4 w = reinterpret_cast<const float4 *>(om + (size_t)i * RP)[c];
            reinterpret_cast<float4 *>(U + (size_t)i * RP)[c] =
                make_float4(acc.x * w.x, acc.y * w.y, acc.z * w.z, acc.w * w.w);
        }
    }
}

// float64 product on beta (refined mode): U64 = Omega (.) X beta
template <int RP>
__global__ void __launch_bounds__(256) k_b_csr64(const BatchDesc *__restrict__ d,
                                                 const double *__restrict__ B,
                                                 const double *__restrict__ om,
                                                 double *__restrict__ U, const int *flags) {
    if (*(volatile const int *)&flags[0] || !*(volatile const int *)&flags[1]) return;
    constexpr int C = RP / 2;
    const int64_t n = d->n;
    const int64_t *__restrict__ rp = d->row_ptr;
    const int lane = threadIdx.x & 31, c = lane % C, slot = lane / C;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const double2 acc = block_row_sum_f64<RP>(d->col_idx, rp[i], rp[i + 1], B, true);
        if (slot == 0) {
            const double2 w = reinterpret_cast<const double2 *>(om + (size_t)i * RP)[c];
            reinterpret_cast<double2 *>(U + (size_t)i * RP)[c] = make_double2(acc.x * w.x, acc.y * w.y);
        }
    }
}

template <int RP>
__global__ void __launch_bounds__(256) k_b_csc(const BatchDesc *__restrict__ d,
                                               const float *__restrict__ U, BatchWs ws) {
    __shared__ double part[8][RP];
    __shared__ double vals[RP];
    __shared__ double sums[RP];
    if (*(volatile const int *)&ws.flags[0]) return;
    constexpr int C = RP / 4;
    const int64_t p = d->p;
    const int R = d->R;
    const int lane = threadIdx.x & 31, c = lane % C, slot = lane / C, wib = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double sg[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t j = warp; j < p; j += nwarps) {
        const float4 acc = block_row_sum_f32<RP>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], U, true);
        if (slot == 0) {
            const float a[4] = {acc.x, acc.y, acc.z, acc.w};
            const size_t o = (size_t)j * RP + 4 * c;
            const double2 s01 = reinterpret_cast<const double2 *>(ws.s64 + o)[0];
            const double2 s23 = reinterpret_cast<const double2 *>(ws.s64 + o)[1];
            const double2 d01 = reinterpret_cast<const double2 *>(ws.dg + o)[0];
            const double2 d23 = reinterpret_cast<const double2 *>(ws.dg + o)[1];
            const double s[4] = {s01.x, s01.y, s23.x, s23.y};
            const double dd[4] = {d01.x, d01.y, d23.x, d23.y};
            double v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[q] = (double)a[q] + dd[q] * s[q];
                sg[q] += s[q] * v[q];
            }
            reinterpret_cast<double2 *>(ws.v64 + o)[0] = make_double2(v[0], v[1]);
            reinterpret_cast<double2 *>(ws.v64 + o)[1] = make_double2(v[2], v[3]);
        }
    }
    if (slot == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) part[wib][4 * c + q] = sg[q];
    }
    __syncthreads();
    if (threadIdx.x < RP) {
        double a = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) a += part[w2][threadIdx.x];
        vals[threadIdx.x] = a;
    }
    if (grid_reduce_arr<RP>(vals, ws.partials, ws.counters + 1, sums)) {
        const int r = threadIdx.x;
        if (r < R) {
            CgScalars *sc = ws.sc + r;
            if (!sc->done) {
                const double sigma = sums[r];
                sc->sigma = sigma;
                if (!isfinite(sigma)) { sc->status = PCG_NONFINITE; sc->done = 1; }
                else if (!(sigma > 0.0) || !(sc->rho > 0.0)) { sc->status = PCG_BREAKDOWN; sc->done = 1; }
                else sc->alpha = sc->rho / sigma;
            }
        }
    }
}

// Tiled products: v = sum_t Pc[t] + d s (float64), sigma per chain, alpha.
// FUSED (the single-pass update of k_b_update_fused): also r.(M^-1 v) and
// v.(M^-1 v), from which the last block forms the next direction's weight
// gamma = rho'/rho before the update pass, by the identity
//   rho' = (r - alpha v).M^-1 (r - alpha v) = rho - 2 alpha r.M^-1 v + alpha^2 v.M^-1 v
// (Chronopoulos and Gear); the update pass then computes rho' itself for the
// stop test and the next alpha.
template <int RP, typename PT, bool FUSED>
__global__ void __launch_bounds__(256) k_b_fin(const BatchDesc *__restrict__ d, const PT *__restrict__ Pc_main,
                                               int T_main, const PT *__restrict__ Pc_tail, int T_tail,
                                               BatchWs ws) {
    constexpr int NV = FUSED ? 3 * RP : RP;
    __shared__ double part[8][NV];
    __shared__ double vals[NV];
    __shared__ double sums[NV];
    if (*(volatile const int *)&ws.flags[0]) return;
    const bool tail = ws.flags[6] != 0;
    const PT *__restrict__ Pc = tail ? Pc_tail : Pc_main;
    const int T_r = tail ? T_tail : T_main;
    const int64_t p = d->p;
    const int R = d->R;
    // only the slots of active product groups (the others' partials are not read)
    const int a2 = active_slots_pow2(d, ws.flags, RP);
    const int lg2 = __ffs(a2) - 1;
    const int r = threadIdx.x & (a2 - 1);    // fixed per thread: the stride is a multiple of a2
    double sg = 0.0, rmv = 0.0, vmv = 0.0;
    const int64_t total = p * RP;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (p << lg2);
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = (q >> lg2) * RP + r;
        // the tail plan's partials are one chain's, contiguous: [T_tail][p]
        const PT acc = tail ? (r == 0 ? sum_strided(Pc + (q >> lg2), T_r, (size_t)p) : PT{})
                            : sum_strided(Pc + t, T_r, (size_t)total);
        const double s = ws.s64[t];
        const double v = part_to_double(acc) + ws.dg[t] * s;
        ws.v64[t] = v;
        sg += s * v;
        if (FUSED) {
            const double mv = ws.m[t] * v;
            rmv += ws.r[t] * mv;
            vmv += v * mv;
        }
    }
    for (int o = 16; o >= a2; o >>= 1) {
        sg += __shfl_xor_sync(kFull, sg, o);
        if (FUSED) {
            rmv += __shfl_xor_sync(kFull, rmv, o);
            vmv += __shfl_xor_sync(kFull, vmv, o);
        }
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane < RP) {
        part[wib][lane] = lane < a2 ? sg : 0.0;
        if (FUSED) {
            part[wib][RP + lane] = lane < a2 ? rmv : 0.0;
            part[wib][2 * RP + lane] = lane < a2 ? vmv : 0.0;
        }
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double a = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) a += part[w2][threadIdx.x];
        vals[threadIdx.x] = a;
    }
    if (grid_reduce_arr<NV>(vals, ws.partials, ws.counters + 1, sums)) {
        const int q = threadIdx.x;
        if (q < R) {
            CgScalars *sc = ws.sc + q;
            if (!sc->done) {
                const double sigma = sums[q];
                sc->sigma = sigma;
                if (!isfinite(sigma)) { sc->status = PCG_NONFINITE; sc->done = 1; }
                else if (!(sigma > 0.0) || !(sc->rho > 0.0)) { sc->status = PCG_BREAKDOWN; sc->done = 1; }
                else {
                    const double alpha = sc->rho / sigma;
                    sc->alpha = alpha;
                    if (FUSED) {
                        const double rho_next = sc->rho - 2.0 * alpha * sums[RP + q] + alpha * alpha * sums[2 * RP + q];
                        sc->gamma = rho_next / sc->rho;
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int k = 0; k < R; ++k) all &= ws.sc[k].done ? 1 : 0;
            ws.flags[0] = all;
        }
    }
}

// The single-pass CG update (after k_b_fin<..., true>): beta += alpha s,
// r -= alpha v, z = M^-1 r, s = z + gamma s with gamma from the finalize, and
// rho' = r.z, in one pass over the grid; the last block applies the stop
// tests and sets the graph's while condition.  (Modes without the float64
// recomputation of r; the refined mode runs k_b_update, the recomputation,
// then k_b_sdir.)
template <int RP>
__global__ void __launch_bounds__(256) k_b_update_fused(const BatchDesc *__restrict__ d, BatchWs ws,
                                                        cudaGraphConditionalHandle h_while, int use_cond) {
    __shared__ double part[8][RP];
    __shared__ double vals[RP];
    __shared__ double sums[RP];
    if (*(volatile const int *)&ws.flags[0]) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_while, 0u);
        return;
    }
    const int64_t p = d->p;
    const int R = d->R;
    const int a2 = active_slots_pow2(d, ws.flags, RP);
    const int lg2 = __ffs(a2) - 1;
    const int r = threadIdx.x & (a2 - 1);    // fixed per thread: the stride is a multiple of a2
    const bool live = r < R && !ws.sc[r].done;
    const double alpha = live ? ws.sc[r].alpha : 0.0;
    const double gamma = live ? ws.sc[r].gamma : 0.0;
    const bool df = d->df != 0;
    const bool tail = ws.flags[6] != 0;
    double rho = 0.0;
    if (live) {
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (p << lg2);
             q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t t = (q >> lg2) * RP + r;
            const double s = ws.s64[t];
            const double rj = ws.r[t] - alpha * ws.v64[t];
            const double z = ws.m[t] * rj;
            const double sn = z + gamma * s;
            ws.beta[t] += alpha * s;
            ws.r[t] = rj;
            ws.s64[t] = sn;
            if (df) reinterpret_cast<float2 *>(ws.s32)[t] = df_from_double(sn);
            else ws.s32[t] = (float)sn;
            if (tail && r == 0) {   // the tail plan gathers a contiguous copy
                if (df) reinterpret_cast<float2 *>(ws.s_tail)[q >> lg2] = df_from_double(sn);
                else ws.s_tail[q >> lg2] = (float)sn;
            }
            rho += rj * z;
        }
    }
    for (int o = 16; o >= a2; o >>= 1) rho += __shfl_xor_sync(kFull, rho, o);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (RP <= 32 && lane < RP) part[wib][lane] = lane < a2 ? rho : 0.0;
    __syncthreads();
    if (threadIdx.x < RP) {
        double a = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) a += part[w2][threadIdx.x];
        vals[threadIdx.x] = a;
    }
    if (grid_reduce_arr<RP>(vals, ws.partials, ws.counters + 2, sums)) {
        const int q = threadIdx.x;
        if (q < R) {
            CgScalars *sc = ws.sc + q;
            if (!sc->done) {
                const double rn = sums[q];
                sc->iter += 1;
                if (!isfinite(rn)) {
                    sc->status = PCG_NONFINITE;
                    sc->done = 1;
                } else {
                    sc->rho_prev = sc->rho;
                    sc->rho = rn;
                    sc->resid = stop_quantity(d->stop_rule, rn, sc->rho0, p);
                    if (stop_met(d->stop_rule, rn, sc->rho0, p, d->tol)) {
                        sc->status = PCG_OK;
                        sc->done = 1;
                    } else if (sc->iter >= d->max_iter) {
                        sc->status = PCG_MAXITER;
                        sc->done = 1;
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int k = 0; k < R; ++k) all &= ws.sc[k].done ? 1 : 0;
            ws.flags[0] = all;
            ws.flags[1] = 0;
            if (use_cond) cudaGraphSetConditional(h_while, all ? 0u : 1u);
        }
    }
}

// beta += alpha s, r -= alpha v, rho' per chain; stop tests and bookkeeping.
template <int RP>
__global__ void __launch_bounds__(256) k_b_update(const BatchDesc *__restrict__ d, BatchWs ws,
                                                  cudaGraphConditionalHandle h_ru, int use_cond) {
    __shared__ double part[8][RP];
    __shared__ double vals[RP];
    __shared__ double sums[RP];
    if (*(volatile const int *)&ws.flags[0]) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_ru, 0);
        return;
    }
    const int64_t p = d->p;
    const int R = d->R;
    const int a2 = active_slots_pow2(d, ws.flags, RP);
    const int lg2 = __ffs(a2) - 1;
    const int r = threadIdx.x & (a2 - 1);    // fixed per thread: the stride is a multiple of a2
    const bool live = r < R && !ws.sc[r].done;
    const double alpha = live ? ws.sc[r].alpha : 0.0;
    double rho = 0.0;
    if (live) {
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (p << lg2);
             q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t t = (q >> lg2) * RP + r;
            const double bj = ws.beta[t] + alpha * ws.s64[t];
            const double rj = ws.r[t] - alpha * ws.v64[t];
            ws.beta[t] = bj;
            ws.r[t] = rj;
            rho += rj * (ws.m[t] * rj);
        }
    }
    // lanes with equal r: xor over the lane bits above a2
    for (int o = 16; o >= a2; o >>= 1) rho += __shfl_xor_sync(kFull, rho, o);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (RP <= 32 && lane < RP) part[wib][lane] = lane < a2 ? rho : 0.0;
    __syncthreads();
    if (threadIdx.x < RP) {
        double a = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) a += part[w2][threadIdx.x];
        vals[threadIdx.x] = a;
    }
    if (grid_reduce_arr<RP>(vals, ws.partials, ws.counters + 2, sums)) {
        const int q = threadIdx.x;
        if (q < R) {
            CgScalars *sc = ws.sc + q;
            if (!sc->done) {
                const double rn = sums[q];
                sc->iter += 1;
                if (!isfinite(rn)) {
                    sc->status = PCG_NONFINITE;
                    sc->done = 1;
                    sc->need_ru = 0;
                } else {
                    const bool conv = stop_met(d->stop_rule, rn, sc->rho0, p, d->tol);
                    sc->rho_prev = sc->rho;
                    sc->rho = rn;
                    sc->gamma = rn / sc->rho_prev;
                    sc->resid = stop_quantity(d->stop_rule, rn, sc->rho0, p);
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
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1, any = 0;
            for (int k = 0; k < R; ++k) {
                all &= ws.sc[k].done ? 1 : 0;
                any |= (ws.sc[k].need_ru && !ws.sc[k].done) ? 1 : 0;
            }
            ws.flags[0] = all;
            ws.flags[1] = any;
            if (any && !all) ws.flags[2] += 1;
            if (use_cond) cudaGraphSetConditional(h_ru, (any && !all) ? 1u : 0u);
        }
    }
}

// r = b - (X^T U64 + d beta) for the chains that asked for it.
template <int RP>
__global__ void __launch_bounds__(256) k_b_true_resid(const BatchDesc *__restrict__ d,
                                                      const double *__restrict__ U, BatchWs ws) {
    __shared__ double part[8][RP];
    __shared__ double vals[RP];
    __shared__ double sums[RP];
    if (*(volatile const int *)&ws.flags[0] || !*(volatile const int *)&ws.flags[1]) return;
    constexpr int C = RP / 2;
    const int64_t p = d->p;
    const int R = d->R;
    const int lane = threadIdx.x & 31, c = lane % C, slot = lane / C, wib = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool want[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int r = 2 * c + q;
        want[q] = r < R && ws.sc[r].need_ru && !ws.sc[r].done;
    }
    double rho[2] = {0.0, 0.0};
    for (int64_t j = warp; j < p; j += nwarps) {
        const double2 acc = block_row_sum_f64<RP>(d->row_idx, d->col_ptr[j], d->col_ptr[j + 1], U, true);
        if (slot == 0) {
            const double a[2] = {acc.x, acc.y};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!want[q]) continue;
                const size_t o = (size_t)j * RP + 2 * c + q;
                const double rj = ws.b[o] - (a[q] + ws.dg[o] * ws.beta[o]);
                ws.r[o] = rj;
                rho[q] += rj * (ws.m[o] * rj);
            }
        }
    }
    if (slot == 0) {
        part[wib][2 * c] = rho[0];
        part[wib][2 * c + 1] = rho[1];
    }
    __syncthreads();
    if (threadIdx.x < RP) {
        double a = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) a += part[w2][threadIdx.x];
        vals[threadIdx.x] = a;
    }
    if (grid_reduce_arr<RP>(vals, ws.partials, ws.counters + 3, sums)) {
        const int q = threadIdx.x;
        if (q < R) {
            CgScalars *sc = ws.sc + q;
            if (sc->need_ru && !sc->done) {
                const double rt = sums[q];
                sc->need_ru = 0;
                if (!isfinite(rt)) {
                    sc->status = PCG_NONFINITE;
                    sc->done = 1;
                } else {
                    sc->rho = rt;
                    sc->gamma = rt / sc->rho_prev;
                    sc->resid = stop_quantity(d->stop_rule, rt, sc->rho0, p);
                    if (sc->pending) {
                        if (stop_met(d->stop_rule, rt, sc->rho0, p, d->tol)) {
                            sc->status = PCG_OK;
                            sc->done = 1;
                        } else {
                            // float64 residual above the rule: restart from it
                            sc->pending = 0;
                            sc->gamma = 0.0;
                            if (sc->iter >= d->max_iter) { sc->status = PCG_MAXITER; sc->done = 1; }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int k = 0; k < R; ++k) all &= ws.sc[k].done ? 1 : 0;
            ws.flags[0] = all;
            ws.flags[1] = 0;
        }
    }
}

// s = m r + gamma s for live chains; sets the while condition.
template <int RP>
__global__ void __launch_bounds__(256) k_b_sdir(const BatchDesc *__restrict__ d, BatchWs ws,
                                                cudaGraphConditionalHandle h_while, int use_cond) {
    const int all = *(volatile const int *)&ws.flags[0];
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_while, all ? 0u : 1u);
    if (all) return;
    const int a2 = active_slots_pow2(d, ws.flags, RP);
    const int lg2 = __ffs(a2) - 1;
    const int r = threadIdx.x & (a2 - 1);    // fixed per thread: the stride is a multiple of a2
    if (r >= d->R || ws.sc[r].done) return;
    const double gamma = ws.sc[r].gamma;
    const bool df = d->df != 0;
    const bool tail = ws.flags[6] != 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (d->p << lg2);
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = (q >> lg2) * RP + r;
        const double s = ws.m[t] * ws.r[t] + gamma * ws.s64[t];
        ws.s64[t] = s;
        if (df) reinterpret_cast<float2 *>(ws.s32)[t] = df_from_double(s);
        else ws.s32[t] = (float)s;
        if (tail && r == 0) {   // the tail plan gathers a contiguous copy
            if (df) reinterpret_cast<float2 *>(ws.s_tail)[q >> lg2] = df_from_double(s);
            else ws.s_tail[q >> lg2] = (float)s;
        }
    }
}

// Compaction (tiled products only): when the live chains fit in fewer product
// groups than are active, move them to the lowest slots (finished chains keep
// their state in the slots after them) and switch the freed groups off.  One
// block decides; k_b_compact_apply then permutes every per-chain row.
template <int RP>
__global__ void k_b_compact_plan(const BatchDesc *__restrict__ d, BatchWs ws) {
    __shared__ CgScalars tmp[RP];
    __shared__ int perm[RP], chain[RP], go;
    const int R = d->R, RG = d->RG;
    if (threadIdx.x == 0) {
        go = 0;
        if (RG > 0 && !ws.flags[0]) {
            int live = 0;
            for (int s = 0; s < R; ++s) live += ws.sc[s].done ? 0 : 1;
            const int need = (live + RG - 1) / RG;
            // one chain left: the group-width-1 plan takes over (the chain moves to slot 0)
            const bool to_tail = d->tail && live == 1 && !ws.flags[6];
            if (to_tail) {
                ws.flags[6] = 1;
                ws.flags[7] = 0;
            }
            if (need < ws.flags[4] || to_tail) {
                int k = 0;
                for (int s = 0; s < R; ++s)
                    if (!ws.sc[s].done) perm[k++] = s;
                for (int s = 0; s < R; ++s)
                    if (ws.sc[s].done) perm[k++] = s;
                for (int s = R; s < RP; ++s) perm[s] = s;
                go = 1;
                ws.flags[4] = need;
                ws.flags[5] += 1;
            }
        }
        ws.flags[3] = go;
    }
    __syncthreads();
    if (!go) return;
    const int s = threadIdx.x;
    if (s < RP) {
        tmp[s] = ws.sc[perm[s]];
        chain[s] = ws.flags[32 + perm[s]];
    }
    __syncthreads();
    if (s < RP) {
        ws.sc[s] = tmp[s];
        ws.flags[32 + s] = chain[s];
        ws.flags[64 + s] = perm[s];
    }
    if (s < 32) ws.flags[96 + s] = (ws.flags[6] || s >= ws.flags[4]) ? 1 : 0;
}

template <int RP, typename V>
__device__ __forceinline__ void permute_row(V *row, const int *perm) {
    V v[RP];
#pragma unroll
    for (int s = 0; s < RP; ++s) v[s] = row[s];
#pragma unroll
    for (int s = 0; s < RP; ++s) row[s] = v[perm[s]];
}

template <int RP>
__global__ void __launch_bounds__(256) k_b_compact_apply(const BatchDesc *__restrict__ d, BatchWs ws) {
    __shared__ int perm[RP];
    if (!*(volatile const int *)&ws.flags[3]) return;
    if (threadIdx.x < RP) perm[threadIdx.x] = ws.flags[64 + threadIdx.x];
    __syncthreads();
    const int64_t p = d->p, n = d->n;
    const bool tail = ws.flags[6] != 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const size_t o = (size_t)j * RP;
        permute_row<RP>(ws.b + o, perm);
        permute_row<RP>(ws.r + o, perm);
        permute_row<RP>(ws.s64 + o, perm);
        permute_row<RP>(ws.beta + o, perm);
        permute_row<RP>(ws.m + o, perm);
        permute_row<RP>(ws.dg + o, perm);
        if (d->df) permute_row<RP>(reinterpret_cast<float2 *>(ws.s32) + o, perm);
        else permute_row<RP>(ws.s32 + o, perm);
        if (tail) {   // the tail plan's chain now sits in slot 0
            if (d->df) reinterpret_cast<float2 *>(ws.s_tail)[j] = reinterpret_cast<const float2 *>(ws.s32)[o];
            else ws.s_tail[j] = ws.s32[o];
        }
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const size_t o = (size_t)i * RP;
        if (d->df) permute_row<RP>(reinterpret_cast<float2 *>(ws.om32) + o, perm);
        else permute_row<RP>(ws.om32 + o, perm);
        permute_row<RP>(ws.om64 + o, perm);
        if (tail) {
            if (d->df) reinterpret_cast<float2 *>(ws.om_tail)[i] = reinterpret_cast<const float2 *>(ws.om32)[o];
            else ws.om_tail[i] = ws.om32[o];
        }
    }
}

// Graph mode with a tail plan: picks this iteration's products (the tail
// plan's once one chain is left, else the main plan's) for the if/else node
// that follows.
__global__ void k_b_tail_cond(const int *__restrict__ flags, cudaGraphConditionalHandle h_tail) {
    if (threadIdx.x == 0) cudaGraphSetConditional(h_tail, flags[6] ? 1u : 0u);
}

// interleaved beta -> caller's chain-major beta
__global__ void k_b_out(const BatchDesc *__restrict__ d, const double *__restrict__ beta,
                        const int *__restrict__ flags) {
    const int64_t p = d->p;
    const int R = d->R, RP = d->RP;
    const int64_t total = p * R;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(t / p);
        const int64_t j = t - (int64_t)s * p;
        d->beta_out[(int64_t)flags[32 + s] * p + j] = beta[j * RP + s];
    }
}

// ===========================================================================
// host side
// ===========================================================================

static cudaError_t add_node(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *deps,
                            size_t ndeps, void *func, dim3 grid, int block, void **args,
                            size_t smem = 0) {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

struct BatchKernels {
    void *init, *csr, *csr64, *csc, *fin, *update, *true_resid, *sdir, *cplan, *capply;
    void *fin_fused, *update_fused;
};

template <int RP>
static BatchKernels batch_kernels(bool df) {
    return {(void *)k_b_init<RP>,         (void *)k_b_csr<RP>,          (void *)k_b_csr64<RP>,
            (void *)k_b_csc<RP>,
            df ? (void *)k_b_fin<RP, float2, false> : (void *)k_b_fin<RP, float, false>,
            (void *)k_b_update<RP>,
            (void *)k_b_true_resid<RP>,   (void *)k_b_sdir<RP>,         (void *)k_b_compact_plan<RP>,
            (void *)k_b_compact_apply<RP>,
            df ? (void *)k_b_fin<RP, float2, true> : (void *)k_b_fin<RP, float, true>,
            (void *)k_b_update_fused<RP>};
}

// The single-pass update (k_b_fin<..., true> + k_b_update_fused) can serve
// the tiled products of the modes without the float64 recomputation of r when
// the environment variable PCG_BETA_FUSED_UPDATE=1 asks for it.  It is off by
// default: on the half-Cauchy systems of the benchmark the recurrence for rho'
// loses enough accuracy to cost 12 % more iterations in all (one chain 33 %)
// and 9 % of the draw rate, more than the kernel it saves.
static bool fused_update(bool refined, int RG) {
    const char *env = getenv("PCG_BETA_FUSED_UPDATE");
    return !refined && RG > 0 && env && env[0] == '1';
}

static BatchKernels kernels_for(int RP, bool df = false) {
    switch (RP) {
        case 4: return batch_kernels<4>(df);
        case 8: return batch_kernels<8>(df);
        case 16: return batch_kernels<16>(df);
        default: return batch_kernels<32>(df);
    }
}

// How the products of one iteration run: untiled (RG = 0) or tiled in
// RP / RG groups of RG right-hand sides.
struct BatchProducts {
    int RG = 0;
    bool df = false;           // float-pair sources and partials (double-float or fixed-point products)
    bool fx = false;           // fixed-point products
    TiledPlan plan{};
    TiledKernels tk{};
    void *pc_all = nullptr;    // [T_r][p][RP] partials (float, or float pairs with df)
    // tail plan: group width 1 over slot 0, for the last live chain (RG >= 2 only)
    bool tail = false;
    TiledPlan plan1{};
    TiledKernels tk1{};
    void *pc1 = nullptr;       // [T_r1][p][RP] partials of the tail plan
};

struct BatchNodeArgs {
    const BatchDesc *d;
    BatchWs ws;
    double *w64;
    double *om64;
    float *om32;
    const float *s32;
    float *u32;
    const double *u64c;
    double *u64;
    const double *beta;
    const int *flag0;
    const int *flags;
    cudaGraphConditionalHandle h_while, h_ru, h_tail;
    int one, zero, use_ru, RPv, T_r;
    TiledArgs ta;
    void *pc_all;
    const void *s_src, *om_src;
    const int *gate_base;          // product group g is skipped when gate_base[g] != 0
    int u_blocks;                  // grid of the u kernel per group
    // tail plan (group width 1, slot 0), gated by flags[7]
    TiledArgs ta1;
    void *pc1;
    const int *gate_tail;
    int u_blocks1, T_r1;
    const void *s_tail, *om_tail;  // the tail chain's contiguous s and omega
};

// Adds the products of one iteration to `body` after `dep`; returns the last node.
static cudaError_t add_products(cudaGraph_t body, const cudaGraphNode_t *dep, int ndep,
                                BatchNodeArgs &A, const BatchKernels &K, const BatchProducts &bp,
                                int RP, int grid, int gvec, cudaGraphNode_t *last) {
    cudaError_t e = cudaSuccess;
    if (bp.RG == 0) {
        cudaGraphNode_t n1;
        void *a1[] = {&A.d, &A.s32, &A.om32, &A.u32, &A.flag0};
        e = add_node(body, &n1, dep, ndep, K.csr, grid, 256, a1);
        if (e != cudaSuccess) return e;
        void *a2[] = {&A.d, &A.u32, &A.ws};
        return add_node(body, last, &n1, 1, K.csc, grid, 256, a2);
    }
    const TiledPlan &P = bp.plan;
    // the main plan's products: every RHS group in one launch (blockIdx.y);
    // finished groups exit at once
    auto add_main = [&](cudaGraph_t gph, const cudaGraphNode_t *d0, int nd0, cudaGraphNode_t *out) {
        cudaGraphNode_t nc, nu;
        void *a1[] = {&A.ta, &A.s_src, &A.RPv, &A.zero, &A.gate_base, &A.zero};
        cudaError_t r = add_node(gph, &nc, d0, d0 ? nd0 : 0, bp.tk.csr, dim3(P.T_c * P.csr_blocks, RP / bp.RG),
                                 P.threads, a1, P.smem_c);
        if (r != cudaSuccess) return r;
        void *au[] = {&A.ta, &A.om_src, &A.RPv, &A.zero, &A.gate_base, &A.zero};
        r = add_node(gph, &nu, &nc, 1, bp.tk.u, dim3(A.u_blocks, RP / bp.RG), 256, au);
        if (r != cudaSuccess) return r;
        void *a2[] = {&A.ta, &A.pc_all, &A.RPv, &A.zero, &A.gate_base, &A.zero};
        return add_node(gph, out, &nu, 1, bp.tk.csc, dim3(P.T_r * P.csc_chunks, RP / bp.RG), P.threads, a2,
                        P.smem_r);
    };
    // the tail plan's products (group width 1, the chain in slot 0)
    auto add_tail = [&](cudaGraph_t gph, const cudaGraphNode_t *d0, int nd0, cudaGraphNode_t *out) {
        const TiledPlan &Q = bp.plan1;
        cudaGraphNode_t t1, tu;
        void *b1[] = {&A.ta1, &A.s_tail, &A.one, &A.zero, &A.gate_tail, &A.zero};
        cudaError_t r = add_node(gph, &t1, d0, d0 ? nd0 : 0, bp.tk1.csr, dim3(Q.T_c * Q.csr_blocks, 1), Q.threads,
                                 b1, Q.smem_c);
        if (r != cudaSuccess) return r;
        void *bu[] = {&A.ta1, &A.om_tail, &A.one, &A.zero, &A.gate_tail, &A.zero};
        r = add_node(gph, &tu, &t1, 1, bp.tk1.u, dim3(A.u_blocks1, 1), 256, bu);
        if (r != cudaSuccess) return r;
        void *b2[] = {&A.ta1, &A.pc1, &A.one, &A.zero, &A.gate_tail, &A.zero};
        return add_node(gph, out, &tu, 1, bp.tk1.csc, dim3(Q.T_r * Q.csc_chunks, 1), Q.threads, b2, Q.smem_r);
    };
    cudaGraphNode_t prev;
    if (!bp.tail) {
        e = add_main(body, dep, ndep, &prev);
    } else {
        // one set of products per iteration: an if/else node on the tail flag
        // (set by a one-thread kernel), so the plan not in use launches nothing
        cudaGraphNode_t nsel;
        void *as[] = {&A.flags, &A.h_tail};
        e = add_node(body, &nsel, dep, dep ? ndep : 0, (void *)k_b_tail_cond, dim3(1), 32, as);
        if (e != cudaSuccess) return e;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = A.h_tail;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 2;   // [0]: taken when the value is nonzero, [1]: otherwise
        e = cudaGraphAddNode(&prev, body, &nsel, nullptr, 1, &cp);
        if (e != cudaSuccess) return e;
        cudaGraphNode_t last_t, last_m;
        e = add_tail(cp.conditional.phGraph_out[0], nullptr, 0, &last_t);
        if (e != cudaSuccess) return e;
        e = add_main(cp.conditional.phGraph_out[1], nullptr, 0, &last_m);
    }
    if (e != cudaSuccess) return e;
    void *a3[] = {&A.d, &A.pc_all, &A.T_r, &A.pc1, &A.T_r1, &A.ws};
    return add_node(body, last, &prev, 1, K.fin, gvec, 256, a3);
}

static pcg_status build_batch_graph(pcg_ctx *ctx, const BatchWs &ws, int RP, bool refined,
                                    const BatchProducts &bp, cudaGraphExec_t *out) {
    BatchKernels K = kernels_for(RP, bp.df);
    const bool fused = fused_update(refined, bp.RG);
    if (fused) K.fin = K.fin_fused;
    const int grid = grid_for(ctx, 256, 8);
    const int gvec = grid_for(ctx, 256, 4);
    BatchNodeArgs A{};
    A.d = ws.desc;
    A.ws = ws;
    A.w64 = (double *)ws.u;
    A.om64 = ws.om64;
    A.om32 = ws.om32;
    A.s32 = ws.s32;
    A.u32 = (float *)ws.u;
    A.u64 = (double *)ws.u;
    A.u64c = (const double *)ws.u;
    A.beta = ws.beta;
    A.flag0 = ws.flags;
    A.flags = ws.flags;
    A.one = 1;
    A.zero = 0;
    A.use_ru = refined ? 1 : 0;
    A.RPv = RP;
    A.ta.plan = bp.plan;
    A.pc_all = bp.pc_all;
    A.s_src = ws.s32;    // float32 values, or float pairs in the double-float mode
    A.om_src = ws.om32;
    A.T_r = bp.plan.T_r;
    A.gate_base = ws.flags + 96;
    A.u_blocks = bp.RG > 0 ? tiled_u_blocks(bp.plan, ctx->num_sms) : 1;
    A.ta1.plan = bp.plan1;
    A.pc1 = bp.tail ? bp.pc1 : bp.pc_all;
    A.gate_tail = ws.flags + 7;
    A.s_tail = ws.s_tail;
    A.om_tail = ws.om_tail;
    A.u_blocks1 = bp.tail ? tiled_u_blocks(bp.plan1, ctx->num_sms) : 1;
    A.T_r1 = bp.tail ? bp.plan1.T_r : bp.plan.T_r;
    cudaGraph_t g = nullptr;
    PCG_CUDA_TRY(ctx, cudaGraphCreate(&g, 0));
    cudaError_t e;
    cudaGraphNode_t n_prep, n_init, n_while, n_prod, n_upd, n_if, n_sdir, n_r1, n_r2, n_out;
    {
        void *a[] = {&A.d, &A.w64, &A.om64, &A.om32};
        e = add_node(g, &n_prep, nullptr, 0, (void *)k_b_prep, grid, 256, a);
    }
    if (e == cudaSuccess) {
        void *a[] = {&A.d, &A.w64, &A.ws};
        e = add_node(g, &n_init, &n_prep, 1, K.init, grid, 256, a);
    }
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&A.h_while, g, 1, cudaGraphCondAssignDefault);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = A.h_while;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&n_while, g, &n_init, nullptr, 1, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess && bp.tail) e = cudaGraphConditionalHandleCreate(&A.h_tail, body, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = add_products(body, nullptr, 0, A, K, bp, RP, grid, gvec, &n_prod);
    if (e == cudaSuccess && refined) e = cudaGraphConditionalHandleCreate(&A.h_ru, body, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess && fused) {
        void *a[] = {&A.d, &A.ws, &A.h_while, &A.one};
        e = add_node(body, &n_upd, &n_prod, 1, K.update_fused, gvec, 256, a);
    } else if (e == cudaSuccess) {
        void *a[] = {&A.d, &A.ws, &A.h_ru, &A.use_ru};
        e = add_node(body, &n_upd, &n_prod, 1, K.update, gvec, 256, a);
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
            void *a1[] = {&A.d, &A.beta, &A.om64, &A.u64, &A.flags};
            e = add_node(ifb, &n_r1, nullptr, 0, K.csr64, grid, 256, a1);
            if (e == cudaSuccess) {
                void *a2[] = {&A.d, &A.u64c, &A.ws};
                e = add_node(ifb, &n_r2, &n_r1, 1, K.true_resid, grid, 256, a2);
            }
            last = n_if;
        }
    }
    if (e == cudaSuccess && fused) {
        n_sdir = n_upd;   // the fused update already formed s
    } else if (e == cudaSuccess) {
        void *a[] = {&A.d, &A.ws, &A.h_while, &A.one};
        e = add_node(body, &n_sdir, &last, 1, K.sdir, gvec, 256, a);
    }
    if (e == cudaSuccess && bp.RG > 0) {
        cudaGraphNode_t n_cp, n_ca;
        void *a1[] = {&A.d, &A.ws};
        e = add_node(body, &n_cp, &n_sdir, 1, K.cplan, 1, 32, a1);
        if (e == cudaSuccess) e = add_node(body, &n_ca, &n_cp, 1, K.capply, gvec, 256, a1);
    }
    if (e == cudaSuccess) {
        void *a[] = {&A.d, &A.beta, &A.flags};
        e = add_node(g, &n_out, &n_while, 1, (void *)k_b_out, gvec, 256, a);
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "building the batched graph");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(ctx, e, "instantiating the batched graph");
    *out = exec;
    return PCG_OK;
}

template <int RP>
static void launch_batch_plain_iter(pcg_ctx *ctx, const BatchWs &ws, bool refined, int grid, int gvec,
                                    const BatchProducts &bp) {
    cudaStream_t st = ctx->stream;
    if (bp.RG == 0) {
        PCG_PROF(ctx, "b_csr_f32", k_b_csr<RP><<<grid, 256, 0, st>>>(ws.desc, ws.s32, ws.om32, (float *)ws.u, ws.flags));
        PCG_PROF(ctx, "b_csc_f32", k_b_csc<RP><<<grid, 256, 0, st>>>(ws.desc, (const float *)ws.u, ws));
    } else {
        const TiledPlan &P = bp.plan;
        TiledArgs ta{P};
        int rp = RP, zero = 0, T_r = P.T_r;
        const void *s32 = ws.s32;    // float32 values, or float pairs in the double-float mode
        const void *om32 = ws.om32;
        void *pc = bp.pc_all;
        const int *flags = ws.flags;
        const BatchDesc *dd = ws.desc;
        BatchWs wsv = ws;
        const int *gate = flags + 96;
        void *a1[] = {&ta, (void *)&s32, &rp, &zero, (void *)&gate, &zero};
        void *au[] = {&ta, (void *)&om32, &rp, &zero, (void *)&gate, &zero};
        void *a2[] = {&ta, &pc, &rp, &zero, (void *)&gate, &zero};
        const dim3 gc(P.T_c * P.csr_blocks, RP / bp.RG), gr(P.T_r * P.csc_chunks, RP / bp.RG);
        const dim3 gu(tiled_u_blocks(P, ctx->num_sms), RP / bp.RG);
        PCG_PROF(ctx, bp.fx ? "bt_csr_fx64" : bp.df ? "bt_csr_df32" : "bt_csr_f32", cudaLaunchKernel(bp.tk.csr, gc, dim3(P.threads), a1, P.smem_c, st));
        PCG_PROF(ctx, "bt_u", cudaLaunchKernel(bp.tk.u, gu, dim3(256), au, 0, st));
        PCG_PROF(ctx, bp.fx ? "bt_csc_fx64" : bp.df ? "bt_csc_df32" : "bt_csc_f32", cudaLaunchKernel(bp.tk.csc, gr, dim3(P.threads), a2, P.smem_r, st));
        void *pc1 = bp.tail ? bp.pc1 : bp.pc_all;
        int T_r1 = bp.tail ? bp.plan1.T_r : P.T_r;
        if (bp.tail) {
            const TiledPlan &Q = bp.plan1;
            TiledArgs ta1{Q};
            const int *gt = flags + 7;
            const void *stl = ws.s_tail, *omt = ws.om_tail;
            int one = 1;
            void *b1[] = {&ta1, (void *)&stl, &one, &zero, (void *)&gt, &zero};
            void *bu[] = {&ta1, (void *)&omt, &one, &zero, (void *)&gt, &zero};
            void *b2[] = {&ta1, &pc1, &one, &zero, (void *)&gt, &zero};
            PCG_PROF(ctx, bp.fx ? "bt1_csr_fx64" : bp.df ? "bt1_csr_df32" : "bt1_csr_f32",
                     cudaLaunchKernel(bp.tk1.csr, dim3(Q.T_c * Q.csr_blocks, 1), dim3(Q.threads), b1, Q.smem_c, st));
            PCG_PROF(ctx, "bt1_u", cudaLaunchKernel(bp.tk1.u, dim3(tiled_u_blocks(Q, ctx->num_sms), 1), dim3(256), bu, 0, st));
            PCG_PROF(ctx, bp.fx ? "bt1_csc_fx64" : bp.df ? "bt1_csc_df32" : "bt1_csc_f32",
                     cudaLaunchKernel(bp.tk1.csc, dim3(Q.T_r * Q.csc_chunks, 1), dim3(Q.threads), b2, Q.smem_r, st));
        }
        void *a3[] = {(void *)&dd, &pc, &T_r, &pc1, &T_r1, &wsv};
        void *fin = fused_update(refined, bp.RG)
                        ? (bp.df ? (void *)k_b_fin<RP, float2, true> : (void *)k_b_fin<RP, float, true>)
                        : (bp.df ? (void *)k_b_fin<RP, float2, false> : (void *)k_b_fin<RP, float, false>);
        PCG_PROF(ctx, "bt_fin", cudaLaunchKernel(fin, dim3(gvec), dim3(256), a3, 0, st));
    }
    if (fused_update(refined, bp.RG)) {
        PCG_PROF(ctx, "b_update_fused", k_b_update_fused<RP><<<gvec, 256, 0, st>>>(ws.desc, ws, 0, 0));
    } else {
        PCG_PROF(ctx, "b_update", k_b_update<RP><<<gvec, 256, 0, st>>>(ws.desc, ws, 0, 0));
        if (refined) {
            PCG_PROF(ctx, "b_ru_csr_f64", k_b_csr64<RP><<<grid, 256, 0, st>>>(ws.desc, ws.beta, ws.om64, (double *)ws.u, ws.flags));
            PCG_PROF(ctx, "b_ru_true_resid", k_b_true_resid<RP><<<grid, 256, 0, st>>>(ws.desc, (const double *)ws.u, ws));
        }
        PCG_PROF(ctx, "b_sdir", k_b_sdir<RP><<<gvec, 256, 0, st>>>(ws.desc, ws, 0, 0));
    }
    if (bp.RG > 0) {
        PCG_PROF(ctx, "b_compact_plan", k_b_compact_plan<RP><<<1, 32, 0, st>>>(ws.desc, ws));
        PCG_PROF(ctx, "b_compact_apply", k_b_compact_apply<RP><<<gvec, 256, 0, st>>>(ws.desc, ws));
    }
}

template <int RP>
static void launch_batch_plain_init(pcg_ctx *ctx, const BatchWs &ws, int grid) {
    PCG_PROF(ctx, "b_prep", k_b_prep<<<grid, 256, 0, ctx->stream>>>(ws.desc, (double *)ws.u, ws.om64, ws.om32));
    PCG_PROF(ctx, "b_init", k_b_init<RP><<<grid, 256, 0, ctx->stream>>>(ws.desc, (const double *)ws.u, ws));
}

// Tiled products for a group width RG (0: untiled).
static pcg_status make_products(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, int RP, int RG,
                                BatchProducts *bp, bool with_tail) {
    *bp = BatchProducts{};
    const bool df = prec_pairs(ctx->opt.precision);
    const bool fx = ctx->opt.precision == PCG_PREC_FX64;
    if ((RG == 0 || !ctx->tiled_enabled) && !df) return PCG_OK;
    if (RG == 0) RG = 1;   // double-float products exist only in tiled form
    char tag[32];
    snprintf(tag, sizeof tag, "batch%d%s", RG, fx ? "x" : df ? "d" : "");
    const int vt = tiled_vtype(ctx->opt.precision);
    pcg_status st = build_tiled_plan(ctx, tag, Xr, Xc, RG, vt, RP / RG, true, &bp->plan);
    if (st != PCG_OK) return st;
    if (!bp->plan.valid) return PCG_OK;
    st = tiled_prepare(ctx, bp->plan, &bp->tk);
    if (st != PCG_OK) return st;
    cudaError_t e;
    bp->pc_all = grow(ctx, std::string(tag) + ":pc_all",
                      (df ? sizeof(double) : sizeof(float)) * (size_t)bp->plan.T_r * bp->plan.p * RP, &e);
    if (!bp->pc_all) return cuda_error(ctx, e, "allocating the batched partials");
    bp->RG = RG;
    bp->df = df;
    bp->fx = fx;
    // PCG_BETA_BATCH_TAIL=0 in the environment keeps the main plan to the end
    const char *tail_env = getenv("PCG_BETA_BATCH_TAIL");
    if (with_tail && RG >= 2 && !(tail_env && tail_env[0] == '0')) {
        // group width 1 for the last live chain: half the staged bytes per
        // gather of the main plan's width-RG groups
        char tag1[32];
        snprintf(tag1, sizeof tag1, "batchtail%s", fx ? "x" : df ? "d" : "");
        st = build_tiled_plan(ctx, tag1, Xr, Xc, 1, vt, 1, true, &bp->plan1);
        if (st != PCG_OK) return st;
        if (bp->plan1.valid) {
            st = tiled_prepare(ctx, bp->plan1, &bp->tk1);
            if (st != PCG_OK) return st;
            bp->pc1 = grow(ctx, std::string(tag1) + ":pc1",
                           (df ? sizeof(double) : sizeof(float)) * (size_t)bp->plan1.T_r * bp->plan1.p * RP, &e);
            if (!bp->pc1) return cuda_error(ctx, e, "allocating the batched partials");
            bp->tail = true;
        }
    }
    return PCG_OK;
}

static pcg_status batched_once(pcg_ctx *ctx, const BatchWs &ws, int RP, bool refined, int nrhs,
                               int max_iter, const BatchProducts &bp, CgScalars *hsc, int *hflags) {
    const int grid = grid_for(ctx, 256, 8), gvec = grid_for(ctx, 256, 4);
    if (ctx->opt.use_graph && !ctx->opt.profile) {
        char key[256];
        const bool fused = fused_update(refined, bp.RG);
        snprintf(key, sizeof key, "batch:%d:%d:%d:%d:%p:%p:%p:%p:%p|%d%s%s%s:%016llx:%016llx:%p:%p",
                 RP, (int)refined, grid, gvec, (void *)ws.b, ws.u, (void *)ws.om64, (void *)ws.om32, (void *)ws.flags,
                 bp.RG, bp.df ? "d" : "", bp.tail ? "t" : "", fused ? "f" : "",
                 (unsigned long long)plan_fingerprint(bp.plan),
                 (unsigned long long)(bp.tail ? plan_fingerprint(bp.plan1) : 0ull), bp.pc_all, bp.pc1);
        auto it = ctx->named_graphs.find(key);
        cudaGraphExec_t exec = nullptr;
        if (it == ctx->named_graphs.end()) {
            pcg_status st = build_batch_graph(ctx, ws, RP, refined, bp, &exec);
            if (st != PCG_OK) return st;
            ctx->named_graphs[key] = exec;
        } else {
            exec = it->second;
        }
        PCG_CUDA_TRY(ctx, cudaGraphLaunch(exec, ctx->stream));
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hsc, ws.sc, sizeof(CgScalars) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hflags, ws.flags, sizeof(int) * kFlagInts, cudaMemcpyDeviceToHost, ctx->stream));
        PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        // graph nodes that ran: prep, init and the output transpose; per loop
        // trip (at least one) the products (one plan's three; with a tail plan
        // also the kernel that picks the plan), the finalize, the update (one
        // fused kernel, or update and direction) and compaction; 2 per float64
        // recomputation of r
        int trips = 1;
        for (int r = 0; r < nrhs; ++r) trips = std::max(trips, hsc[r].iter);
        const int per_trip = (bp.RG ? 3 + (bp.tail ? 1 : 0) + 1 + 2 : 2) + (fused ? 1 : 2);
        ctx->last_launches += 3 + (int64_t)per_trip * trips + 2 * (int64_t)hflags[2];
        return PCG_OK;
    }
    switch (RP) {
        case 4: launch_batch_plain_init<4>(ctx, ws, grid); break;
        case 8: launch_batch_plain_init<8>(ctx, ws, grid); break;
        case 16: launch_batch_plain_init<16>(ctx, ws, grid); break;
        default: launch_batch_plain_init<32>(ctx, ws, grid); break;
    }
    for (int it = 0;; it += 8) {
        for (int k = 0; k < 8; ++k) {
            switch (RP) {
                case 4: launch_batch_plain_iter<4>(ctx, ws, refined, grid, gvec, bp); break;
                case 8: launch_batch_plain_iter<8>(ctx, ws, refined, grid, gvec, bp); break;
                case 16: launch_batch_plain_iter<16>(ctx, ws, refined, grid, gvec, bp); break;
                default: launch_batch_plain_iter<32>(ctx, ws, refined, grid, gvec, bp); break;
            }
        }
        PCG_CUDA_TRY(ctx, cudaGetLastError());
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hflags, ws.flags, sizeof(int) * kFlagInts, cudaMemcpyDeviceToHost, ctx->stream));
        PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        prof_collect(ctx);
        if (hflags[0]) break;
        if (it > max_iter + 16) return set_error(ctx, PCG_TIMEOUT, "host loop ran past max_iter");
    }
    PCG_PROF(ctx, "b_out", k_b_out<<<gvec, 256, 0, ctx->stream>>>(ws.desc, ws.beta, ws.flags));
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hsc, ws.sc, sizeof(CgScalars) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hflags, ws.flags, sizeof(int) * kFlagInts, cudaMemcpyDeviceToHost, ctx->stream));
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    return PCG_OK;
}

// RHS-group width for this design and block: cached per (n, p, nnz, RP)
// in the context and the autotune file; otherwise every candidate runs a few
// iterations and the fastest per iteration wins.
static pcg_status choose_rg(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, const BatchWs &ws,
                            BatchDesc &d, BatchDesc *hd, int RP, bool refined, int nrhs,
                            CgScalars *hsc, int *hflags, int *rg_out) {
    // PCG_BETA_BATCH_RG in the environment forces the width (tests use it to
    // cover every width); 0 selects the untiled products
    const char *force = getenv("PCG_BETA_BATCH_RG");
    if (force && force[0]) {
        const int v = atoi(force);
        *rg_out = (v == 1 || v == 2 || v == 4 || v == 8) && v <= RP ? v : 0;
        if (prec_pairs(ctx->opt.precision) && *rg_out == 0) *rg_out = 4 <= RP ? 4 : RP;   // float pairs: tiled only
        return PCG_OK;
    }
    char key[128];
    snprintf(key, sizeof key, "batch_rg:%lld:%lld:%lld:%d:%d", (long long)Xr->n, (long long)Xr->p,
             (long long)Xr->nnz, RP, ctx->opt.precision);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end() && !it->second.empty()) {
        *rg_out = it->second[0];
        return PCG_OK;
    }
    if (ctx->opt.autotune_cache) {
        FILE *f = fopen(ctx->opt.autotune_cache, "r");
        if (f) {
            char k[128];
            int v;
            while (fscanf(f, "%127s %d%*[^\n]", k, &v) == 2) {
                if (strcmp(k, key) == 0) {
                    fclose(f);
                    ctx->tuned[key] = {v};
                    *rg_out = v;
                    return PCG_OK;
                }
            }
            fclose(f);
        }
    }
    int best_rg = 0;
    if (ctx->tiled_enabled) {
        const int saved_iter = d.max_iter;
        const double saved_tol = d.tol;
        d.max_iter = 12;   // a short, fixed number of iterations per candidate
        d.tol = 0.0;
        *hd = d;
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ws.desc, hd, sizeof(BatchDesc), cudaMemcpyHostToDevice, ctx->stream));
        float best = 1e30f;
        const int cands[] = {0, 1, 2, 4, 8};
        const bool df = prec_pairs(ctx->opt.precision);
        for (int rg : cands) {
            if (rg > RP || (df && rg == 0)) continue;   // float-pair products exist tiled only
            BatchProducts bp;
            pcg_status st = make_products(ctx, Xr, Xc, RP, rg, &bp, false);
            if (st != PCG_OK) return st;
            if (rg && !bp.RG) continue;
            d.RG = bp.RG;
            d.tail = 0;
            *hd = d;
            PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ws.desc, hd, sizeof(BatchDesc), cudaMemcpyHostToDevice, ctx->stream));
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {   // the first run builds the graph
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                cudaError_t ce = cudaEventCreate(&e0);
                if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
                if (ce == cudaSuccess) ce = cudaEventRecord(e0, ctx->stream);
                if (ce == cudaSuccess) st = batched_once(ctx, ws, RP, refined, nrhs, 12, bp, hsc, hflags);
                if (ce == cudaSuccess && st == PCG_OK) ce = cudaEventRecord(e1, ctx->stream);
                if (ce == cudaSuccess && st == PCG_OK) ce = cudaEventSynchronize(e1);
                if (ce == cudaSuccess && st == PCG_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
                if (st != PCG_OK) return st;
                if (ce != cudaSuccess) return cuda_error(ctx, ce, "timing an autotune candidate");
            }
            if (ms < best) {
                best = ms;
                best_rg = rg;
            }
        }
        d.max_iter = saved_iter;
        d.tol = saved_tol;
        *hd = d;
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ws.desc, hd, sizeof(BatchDesc), cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->tuned[key] = {best_rg};
    if (ctx->opt.autotune_cache) {
        FILE *f = fopen(ctx->opt.autotune_cache, "a");
        if (f) {
            fprintf(f, "%s %d\n", key, best_rg);
            fclose(f);
        }
    }
    *rg_out = best_rg;
    return PCG_OK;
}

pcg_status run_batched(pcg_ctx *ctx, const pcg_csr *Xr, const pcg_csc *Xc, int nrhs,
                       const double *omega, const double *z, const double *lambda,
                       const double *tau, const double *eta, const double *delta, double tol,
                       int max_iter, double *beta, int *iters, double *resid, int *status) {
    if (ctx->opt.precision == PCG_PREC_FP64)
        return set_error(ctx, PCG_BADARG, "the batched path computes its products in float32 arithmetic: use PCG_PREC_FP32_REFINED, PCG_PREC_FP32, PCG_PREC_DF32 or PCG_PREC_FX64");
    int RP = 4;
    while (RP < nrhs) RP *= 2;
    const int64_t n = std::max<int64_t>(Xr->n, 1), p = std::max<int64_t>(Xr->p, 1);
    const size_t vp = sizeof(double) * (size_t)p * RP;
    const size_t al = 256;
    auto up = [&](size_t x) { return (x + al - 1) / al * al; };
    // one block for the p-sized vectors and the small state
    const size_t total_p = 7 * up(vp) + up(sizeof(float2) * (size_t)p * RP) + up(sizeof(float2) * (size_t)p) +
                           up(sizeof(double) * kMaxReduceBlocks * 32) + up(64 * sizeof(unsigned)) +
                           up(sizeof(CgScalars) * kMaxBatch) + up(sizeof(int) * kFlagInts) + up(sizeof(BatchDesc));
    cudaError_t e;
    char *bp_mem = (char *)grow(ctx, "batch_p", total_p, &e);
    if (!bp_mem) return cuda_error(ctx, e, "allocating the batched workspace");
    void *bu = grow(ctx, "batch_u", sizeof(double) * (size_t)n * RP, &e);
    if (!bu) return cuda_error(ctx, e, "allocating the batched workspace");
    double *bom64 = (double *)grow(ctx, "batch_om64", sizeof(double) * (size_t)n * RP, &e);
    if (!bom64) return cuda_error(ctx, e, "allocating the batched workspace");
    float *bom32 = (float *)grow(ctx, "batch_om32", sizeof(float2) * (size_t)n * RP, &e);
    if (!bom32) return cuda_error(ctx, e, "allocating the batched workspace");
    float *bomt = (float *)grow(ctx, "batch_omtail", sizeof(float2) * (size_t)n, &e);
    if (!bomt) return cuda_error(ctx, e, "allocating the batched workspace");
    BatchWs ws{};
    size_t off = 0;
    auto take = [&](size_t sz) { char *q = bp_mem + off; off += up(sz); return q; };
    ws.b = (double *)take(vp);
    ws.r = (double *)take(vp);
    ws.s64 = (double *)take(vp);
    ws.v64 = (double *)take(vp);
    ws.beta = (double *)take(vp);
    ws.m = (double *)take(vp);
    ws.dg = (double *)take(vp);
    ws.s32 = (float *)take(sizeof(float2) * (size_t)p * RP);
    ws.s_tail = (float *)take(sizeof(float2) * (size_t)p);
    ws.partials = (double *)take(sizeof(double) * kMaxReduceBlocks * 32);
    ws.counters = (unsigned *)take(64 * sizeof(unsigned));
    ws.sc = (CgScalars *)take(sizeof(CgScalars) * kMaxBatch);
    ws.flags = (int *)take(sizeof(int) * kFlagInts);
    ws.desc = (BatchDesc *)take(sizeof(BatchDesc));
    ws.u = bu;
    ws.om64 = bom64;
    ws.om32 = bom32;
    ws.om_tail = bomt;
    // counters must start at zero; the rest is written before it is read
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(ws.counters, 0, 64 * sizeof(unsigned), ctx->stream));

    BatchDesc *hd = (BatchDesc *)grow_host(ctx, "batch_desc", sizeof(BatchDesc), &e);
    CgScalars *hsc = (CgScalars *)grow_host(ctx, "batch_sc", sizeof(CgScalars) * kMaxBatch, &e);
    int *hflags = (int *)grow_host(ctx, "batch_flags", sizeof(int) * kFlagInts, &e);
    if (!hd || !hsc || !hflags) return cuda_error(ctx, e, "allocating pinned staging");
    BatchDesc d{};
    d.row_ptr = Xr->row_ptr;
    d.col_idx = Xr->col_idx;
    d.col_ptr = Xc->col_ptr;
    d.row_idx = Xc->row_idx;
    d.omega = omega;
    d.z = z;
    d.lambda = lambda;
    d.tau = tau;
    d.eta = eta;
    d.delta = delta;
    d.beta_out = beta;
    d.n = Xr->n;
    d.p = Xr->p;
    d.nnz = Xr->nnz;
    d.R = nrhs;
    d.RP = RP;
    d.tol = tol;
    d.max_iter = max_iter;
    d.stop_rule = ctx->opt.stop_rule;
    d.refined = ctx->opt.precision == PCG_PREC_FP32_REFINED ? 1 : 0;
    d.reliable_k = ctx->opt.reliable_k;
    d.df = prec_pairs(ctx->opt.precision) ? 1 : 0;
    if (ctx->unshrunk_q1 > Xr->p)
        return set_error(ctx, PCG_BADARG, "more unshrunk coefficients (pcg_set_unshrunk) than columns of X");
    d.q1 = ctx->unshrunk_q1;
    d.ud = ctx->unshrunk_d;
    d.um = ctx->unshrunk_m;
    const bool refined = d.refined != 0;
    int RG = 0;
    pcg_status st = choose_rg(ctx, Xr, Xc, ws, d, hd, RP, refined, nrhs, hsc, hflags, &RG);
    if (st != PCG_OK) return st;
    BatchProducts bp;
    st = make_products(ctx, Xr, Xc, RP, RG, &bp, true);
    if (st != PCG_OK) return st;
    // float pairs exist only in the tiled products (the untiled kernels read
    // float32 copies; with no nonzero they gather nothing)
    if (prec_pairs(ctx->opt.precision) && !bp.RG && Xr->nnz > 0)
        return set_error(ctx, PCG_BADARG, "PCG_PREC_DF32 and PCG_PREC_FX64 need the tiled products, which do not "
                                          "apply to this design (too large for their 32-bit positions): use "
                                          "PCG_PREC_FP32_REFINED");
    ctx->last_launches = 0;
    d.RG = bp.RG;
    d.tail = bp.tail ? 1 : 0;
    *hd = d;
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(ws.desc, hd, sizeof(BatchDesc), cudaMemcpyHostToDevice, ctx->stream));
    st = batched_once(ctx, ws, RP, refined, nrhs, max_iter, bp, hsc, hflags);
    if (st != PCG_OK) return st;
    pcg_status worst = PCG_OK;
    for (int s = 0; s < nrhs; ++s) {   // slot s holds chain flags[32 + s] after compactions
        const int r = hflags[32 + s];
        iters[r] = hsc[s].iter;
        resid[r] = hsc[s].resid;
        status[r] = hsc[s].status == kRunning ? PCG_TIMEOUT : hsc[s].status;
        if (status[r] > worst) worst = (pcg_status)status[r];
    }
    if (worst != PCG_OK) return set_error(ctx, worst, "at least one chain did not converge (see status[])");
    return PCG_OK;
}

}  // namespace pcg
