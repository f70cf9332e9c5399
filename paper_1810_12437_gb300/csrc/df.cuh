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

// generic helpers over the partial-sum types of the tiled products
__device__ __forceinline__ float part_add(float a, float b) { return a + b; }
__device__ __forceinline__ double part_add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 part_add(float2 a, float2 b) { return df_add(a, b); }
__device__ __forceinline__ double part_to_double(float a) { return (double)a; }
__device__ __forceinline__ double part_to_double(double a) { return a; }
__device__ __forceinline__ double part_to_double(float2 a) { return df_to_double(a); }

}  // namespace pcg
