// Double-float ("DF") arithmetic: a value is an unevaluated pair hi + lo of
// floats (about 48 significant bits), added with Knuth's error-free TwoSum and
// multiplied with an FMA-based TwoProduct (Dekker 1971; Knuth, TAOCP vol. 2,
// Sec. 4.2.2).  GB300 runs float64 at a small fraction of its float32 rate, so
// the tiled products keep DF values in float arithmetic end to end; only the
// vector kernels convert to and from float64, once per element.
#pragma once

#include <cuda_runtime.h>

namespace pcg {

// a + b = t + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float &t, float &e) {
    t = __fadd_rn(a, b);
    const float bv = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bv)), __fsub_rn(b, bv));
}

__device__ __forceinline__ float2 df_norm(float hi, float lo) {
    float t, e;
    two_sum(hi, lo, t, e);
    return make_float2(t, e);
}

__device__ __forceinline__ float2 df_from_double(double x) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}

__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float t, e;
    two_sum(a.x, b.x, t, e);
    return df_norm(t, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return df_norm(p, e);
}

// Two independent TwoSums on packed pairs (sm_100 FADD2 / FFMA2: one
// instruction per two lanes of work); x - y is formed as fma(y, -1, x), whose
// product is exact, so it rounds exactly as the subtraction.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &t, float2 &e) {
    const float2 m1 = make_float2(-1.f, -1.f);
    t = __fadd2_rn(a, b);
    const float2 bv = __ffma2_rn(a, m1, t);    // t - a
    const float2 tb = __ffma2_rn(bv, m1, t);   // t - bv
    e = __fadd2_rn(__ffma2_rn(tb, m1, a), __ffma2_rn(bv, m1, b));   // (a - tb) + (b - bv)
}

// generic helpers over the partial-sum types of the tiled products
__device__ __forceinline__ float part_add(float a, float b) { return a + b; }
__device__ __forceinline__ double part_add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 part_add(float2 a, float2 b) { return df_add(a, b); }
__device__ __forceinline__ double part_to_double(float a) { return (double)a; }
__device__ __forceinline__ double part_to_double(double a) { return a; }
__device__ __forceinline__ double part_to_double(float2 a) { return df_to_double(a); }

// sum_{k < K} x[k * stride] in a fixed order: x0, then blocks of eight added
// as a tree ((x1 + x2) + (x3 + x4)) + ((x5 + x6) + (x7 + x8)), then the rest
// one by one; the eight loads of a block are issued together (K is a runtime
// count of tile or strip partials)
template <typename PT>
__device__ __forceinline__ PT sum_strided(const PT *__restrict__ x, int K, size_t stride) {
    PT acc = __ldg(x);
    int k = 1;
    for (; k + 8 <= K; k += 8) {
        PT v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(x + (size_t)(k + u) * stride);
        const PT lo = part_add(part_add(v[0], v[1]), part_add(v[2], v[3]));
        const PT hi = part_add(part_add(v[4], v[5]), part_add(v[6], v[7]));
        acc = part_add(acc, part_add(lo, hi));
    }
    for (; k < K; ++k) acc = part_add(acc, __ldg(x + (size_t)k * stride));
    return acc;
}

}  // namespace pcg
