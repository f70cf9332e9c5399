// Device helpers shared by the kernels: warp/group sums, the deterministic
// last-block grid reduction, and the CG stop rule.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace pcg {

constexpr unsigned kFull = 0xffffffffu;

// Sum over aligned groups of G lanes (G a power of two <= 32); every lane of
// the warp must call it.  The result is valid in every lane of the group.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Block-wide sum of one value per thread; result valid in thread 0.
// `red` must hold blockDim.x / 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = group_sum<32>(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
        t = group_sum<32>(t);
    }
    return t;
}

// Deterministic grid reduction of NV doubles.  Every block calls it with its
// block totals in thread 0 (vals[0..NV-1]).  Returns true in all threads of
// the one block that finishes last; there, sums[0..NV-1] (shared memory,
// valid in every thread after the call) hold the totals summed in block
// order, so the result does not depend on scheduling.  The counter is reset
// for the next use.
template <int NV>
__device__ bool grid_reduce(const double *vals, double *partials, unsigned int *counter,
                            double *sums, double *red) {
    __shared__ bool am_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[(size_t)blockIdx.x * NV + k] = vals[k];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        // each thread sums a strided subset in block order; block_sum combines
        // the per-thread sums in a fixed tree, so the order is deterministic.
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            acc += __ldcg(partials + (size_t)b * NV + k);
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) sums[k] = acc;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// Stop quantity and rule (Eq. S2): rho = ||tau lambda (.) r||^2.
__device__ __forceinline__ double stop_quantity(int rule, double rho, double rho0, int64_t p) {
    if (rule == PCG_STOP_RELATIVE) return rho0 > 0.0 ? sqrt(rho / rho0) : 0.0;
    return p > 0 ? sqrt(rho / (double)p) : 0.0;
}

__device__ __forceinline__ bool stop_met(int rule, double rho, double rho0, int64_t p, double tol) {
    return stop_quantity(rule, rho, rho0, p) <= tol;
}

// Prior precision d_j = tau^-2 lambda_j^-2 and its inverse m_j = tau^2 lambda_j^2
// (Eq. 1.2 and Sec. 2.4).
__device__ __forceinline__ double prior_prec(double tau, double lam) {
    const double t = tau * lam;
    return 1.0 / (t * t);
}
__device__ __forceinline__ double prior_var(double tau, double lam) {
    const double t = tau * lam;
    return t * t;
}

// The same per coefficient of a single-RHS draw: d_j, m_j and the prior term
// sqrt(d_j) delta_j of Eq. 2.3, with the unshrunk coefficients j < q1 (Sec. S4.3)
// taking their prior precision sigma_j^-2 and preconditioner variance gamma_j^2.
__device__ __forceinline__ double desc_d(const DrawDesc *d, int64_t j) {
    return j < d->q1 ? d->ud[j] : prior_prec(d->tau, d->lambda[j]);
}
// m_j of the stop rule (Eq. S2, and Sec. S4.3's M for the unshrunk ones) ...
__device__ __forceinline__ double desc_mstop(const DrawDesc *d, int64_t j) {
    return j < d->q1 ? d->um[j] : prior_var(d->tau, d->lambda[j]);
}
// ... and M^-1 of the preconditioner: the same, or the Jacobi 1 / diag(Phi)_j.
__device__ __forceinline__ double desc_m(const DrawDesc *d, int64_t j) {
    return d->mj ? d->mj[j] : desc_mstop(d, j);
}
__device__ __forceinline__ double desc_prior_term(const DrawDesc *d, int64_t j, double delta) {
    return j < d->q1 ? delta * sqrt(d->ud[j]) : delta / (d->tau * d->lambda[j]);
}

// Streaming loads of index arrays (read once per pass: keep them out of L1
// and mark them first to evict from L2), and cached loads of gathered vectors.
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ int4 ld_stream4(const int4 *p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ T ld_gather(const T *p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// lane-partial gather-sum of one CSR row / CSC column by a group of G lanes;
// the caller combines the group with group_sum outside any divergent branch.
// ---------------------------------------------------------------------------
template <int G, typename T>
__device__ __forceinline__ T segment_partial(const int32_t *__restrict__ idx, int64_t k0,
                                                int64_t k1, const T *__restrict__ x, int lane) {
    T acc = T(0);
    int64_t k = k0 + lane;
    for (; k + 3 * G < k1; k += 4 * G) {
        const int32_t j0 = ld_stream(idx + k), j1 = ld_stream(idx + k + G);
        const int32_t j2 = ld_stream(idx + k + 2 * G), j3 = ld_stream(idx + k + 3 * G);
        const T a0 = ld_gather(x + j0), a1 = ld_gather(x + j1);
        const T a2 = ld_gather(x + j2), a3 = ld_gather(x + j3);
        acc += (a0 + a1) + (a2 + a3);
    }
    for (; k < k1; k += G) acc += ld_gather(x + ld_stream(idx + k));
    return acc;
}

}  // namespace pcg
