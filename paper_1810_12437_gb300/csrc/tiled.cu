// Shared-memory tiled products for u = Omega X s and v = X^T u + d s.
//
// Both passes are sparse gathers.  Gathering 4-byte values straight from L2
// costs a 32-byte sector per nonzero, which bounds the plain kernels far below
// HBM bandwidth; here the gathered vector is staged in shared memory instead:
//
//   CSR pass  X split into column tiles of W_c columns.  A CTA stages the
//             tile's slice of s (W_c x RG values, up to ~220 KB) in shared
//             memory, then sums its rows' nonzeros inside the tile, gathering
//             from shared memory; it writes per-tile row partials Pr[c][i].
//   CSC pass  rows split into strips of W_r rows.  A CTA stages
//             u_i = omega_i * sum_c Pr[c][i] for the strip's rows in shared
//             memory, then sums its columns' nonzeros inside the strip;
//             it writes per-strip column partials Pc[t][j].
//   finalize  v_j = sum_t Pc[t][j] + d_j s_j, sigma = s.v (float64).
//
// A per-call plan rewrites the indices as 16-bit offsets inside their tile or
// strip (half the index bytes of int32), tile by tile, each row's (column's)
// run padded to whole 8-index chunks whose pad slots point at a zero slot in
// shared memory, so the inner loop has no per-entry tests.  RG values are
// gathered per nonzero (RG right-hand sides of a batch at once; RG = 1 for
// one draw).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>

#include <cub/cub.cuh>

#include "device_common.cuh"
#include "internal.h"
#include "tiled.h"

namespace pcg {

// ---------------------------------------------------------------------------
// plan building
// ---------------------------------------------------------------------------

// bounds[t * nseg + s] = first position in segment s whose index is >= t * W,
// for t = 0..T (t = 0 gives the segment start, t = T its end).
__global__ void k_plan_bounds(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                              int64_t nseg, int W, int T, uint32_t *__restrict__ bounds) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = ptr[s], b = ptr[s + 1];
        bounds[s] = (uint32_t)a;
        int64_t lo = a;
        for (int t = 1; t < T; ++t) {
            const int64_t key = (int64_t)t * W;
            int64_t l = lo, h = b;   // first position in [lo, b) with idx >= key
            while (l < h) {
                const int64_t m = (l + h) >> 1;
                if (idx[m] < key) l = m + 1;
                else h = m;
            }
            bounds[(int64_t)t * nseg + s] = (uint32_t)l;
            lo = l;
        }
        bounds[(int64_t)T * nseg + s] = (uint32_t)b;
    }
}

// chunks[t * nseg + s] = number of 8-index chunks of segment s in tile t
// (its entries rounded up to a multiple of 8); chunks[T * nseg] = 0.
__global__ void k_plan_chunks(const uint32_t *__restrict__ bounds, int64_t nseg, int T,
                              uint32_t *__restrict__ chunks) {
    const int64_t total = (int64_t)T * nseg;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q <= total;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q == total) {
            chunks[q] = 0u;
        } else {
            const int64_t t = q / nseg, s = q - t * nseg;
            const uint32_t len = bounds[(t + 1) * nseg + s] - bounds[t * nseg + s];
            chunks[q] = (len + 7u) >> 3;
        }
    }
}

// Writes each (tile t, segment s) run of indices, as offsets inside the tile,
// to its own whole chunks starting at chunk cstart[t * nseg + s]; the slots
// after the run are filled with the sentinel W (a zero slot in shared memory).
__global__ void k_plan_fill(const int32_t *__restrict__ idx, const uint32_t *__restrict__ bounds,
                            const uint32_t *__restrict__ cstart, int64_t nseg, int T, int W,
                            uint16_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = (int64_t)T * nseg;
    for (int64_t q = warp; q < total; q += nwarps) {
        const int64_t t = q / nseg, s = q - t * nseg;
        const uint32_t a = bounds[t * nseg + s], b = bounds[(t + 1) * nseg + s];
        const uint32_t len = b - a, padded = (len + 7u) & ~7u;
        const uint64_t dst = (uint64_t)cstart[q] * 8u;
        const int base = (int)(t * W);
        for (uint32_t e = lane; e < padded; e += 32)
            out[dst + e] = e < len ? (uint16_t)(idx[a + e] - base) : (uint16_t)W;
    }
}

__global__ void k_plan_order_keys(const int64_t *__restrict__ col_ptr, int64_t p,
                                  int32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        keys[j] = (int32_t)(col_ptr[j + 1] - col_ptr[j]);
        vals[j] = (int32_t)j;
    }
}

static int pick_lanes(double mean_chunks) {
    // about four chunks per lane, many segments in flight per warp
    if (mean_chunks >= 128) return 32;
    if (mean_chunks >= 48) return 16;
    if (mean_chunks >= 20) return 8;
    return 4;
}

// Builds one side of the plan: padded tile-major indices and chunk bounds.
static pcg_status plan_side(pcg_ctx *ctx, const std::string &tag, const int64_t *ptr,
                            const int32_t *idx, int64_t nseg, int64_t nnz, int W, int T,
                            uint16_t **out_idx, uint32_t **out_cb, double *mean_chunks) {
    cudaError_t e;
    const int64_t nb = (int64_t)(T + 1) * nseg;
    uint32_t *bounds = (uint32_t *)grow(ctx, tag + ":bounds", sizeof(uint32_t) * nb, &e);
    if (!bounds) return cuda_error(ctx, e, "allocating the tiled plan");
    const int64_t nc = (int64_t)T * nseg + 1;
    uint32_t *chunks = (uint32_t *)grow(ctx, tag + ":chunks", sizeof(uint32_t) * nc, &e);
    if (!chunks) return cuda_error(ctx, e, "allocating the tiled plan");
    uint32_t *cb = (uint32_t *)grow(ctx, tag + ":cb", sizeof(uint32_t) * nc, &e);
    if (!cb) return cuda_error(ctx, e, "allocating the tiled plan");
    // at most 7 pad slots per segment
    const int64_t cap = nnz + 7 * (int64_t)T * nseg + 8;
    uint16_t *pidx = (uint16_t *)grow(ctx, tag + ":idx", sizeof(uint16_t) * cap, &e);
    if (!pidx) return cuda_error(ctx, e, "allocating the tiled plan");
    size_t tmp_bytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, chunks, cb, (int)nc, ctx->stream);
    void *tmp = grow(ctx, "plan:scan_tmp", tmp_bytes + 256, &e);
    if (!tmp) return cuda_error(ctx, e, "allocating the plan scan");
    const int grid = grid_for(ctx, 256, 8);
    cudaStream_t s = ctx->stream;
    PCG_PROF(ctx, "plan_bounds", k_plan_bounds<<<grid, 256, 0, s>>>(ptr, idx, nseg, W, T, bounds));
    PCG_PROF(ctx, "plan_chunks", k_plan_chunks<<<grid, 256, 0, s>>>(bounds, nseg, T, chunks));
    PCG_CUDA_TRY(ctx, cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, chunks, cb, (int)nc, s));
    PCG_PROF(ctx, "plan_fill", k_plan_fill<<<grid, 256, 0, s>>>(idx, bounds, cb, nseg, T, W, pidx));
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    *out_idx = pidx;
    *out_cb = cb;
    *mean_chunks = (double)(nnz + 3.5 * (double)T * nseg) / 8.0 / ((double)T * nseg);
    return PCG_OK;
}

pcg_status build_tiled_plan(pcg_ctx *ctx, const char *tag, const pcg_csr *Xr, const pcg_csc *Xc,
                            int RG, int vtype, TiledPlan *pl) {
    *pl = TiledPlan{};
    const int vsize = vtype == kVtF32 ? 4 : 8;   // staged bytes per value (DF: two floats)
    pl->vtype = vtype;
    const int64_t n = Xr->n, p = Xr->p, nnz = Xr->nnz;
    // positions are 32-bit inside the kernels (padding included)
    if (n <= 0 || p <= 0 || nnz <= 0 || nnz + 8 * (n + p) * 4 >= (int64_t)0xfffffff0ll) return PCG_OK;
    int64_t w = (kTileSmemBytes - RG * vsize) / (RG * vsize);   // one slot is the zero sentinel
    w = std::min<int64_t>(w, 65528);
    w &= ~int64_t(7);
    pl->RG = RG;
    pl->vsize = vsize;
    pl->n = n;
    pl->p = p;
    pl->nnz = nnz;
    pl->W_c = (int)std::min<int64_t>(w, p);
    pl->T_c = (int)((p + pl->W_c - 1) / pl->W_c);
    pl->W_r = (int)std::min<int64_t>(w, n);
    pl->T_r = (int)((n + pl->W_r - 1) / pl->W_r);
    std::string t(tag);
    double mc_r = 0, mc_c = 0;
    pcg_status st = plan_side(ctx, t + ":csr", Xr->row_ptr, Xr->col_idx, n, nnz, pl->W_c, pl->T_c,
                              &pl->col16, &pl->rt, &mc_r);
    if (st != PCG_OK) return st;
    st = plan_side(ctx, t + ":csc", Xc->col_ptr, Xc->row_idx, p, nnz, pl->W_r, pl->T_r, &pl->row16,
                   &pl->cs, &mc_c);
    if (st != PCG_OK) return st;
    cudaError_t e;
    {
        // column order by decreasing length for the CSC pass
        int32_t *keys = (int32_t *)grow(ctx, t + ":ord_keys", sizeof(int32_t) * 2 * p, &e);
        if (!keys) return cuda_error(ctx, e, "allocating the column order");
        int32_t *vals = (int32_t *)grow(ctx, t + ":ord_vals", sizeof(int32_t) * 2 * p, &e);
        if (!vals) return cuda_error(ctx, e, "allocating the column order");
        pl->col_order = vals + p;
        const int grid = grid_for(ctx, 256, 4);
        PCG_PROF(ctx, "plan_order", k_plan_order_keys<<<grid, 256, 0, ctx->stream>>>(Xc->col_ptr, p, keys, vals));
        size_t tb = 0;
        cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, keys, keys + p, vals, vals + p, (int)p, 0, 32,
                                                  ctx->stream);
        void *tmp = grow(ctx, "plan:sort_tmp", tb + 256, &e);
        if (!tmp) return cuda_error(ctx, e, "allocating the column sort");
        PCG_CUDA_TRY(ctx, cub::DeviceRadixSort::SortPairsDescending(tmp, tb, keys, keys + p, vals, vals + p,
                                                                    (int)p, 0, 32, ctx->stream));
    }
    // partial sums: float for float values, double otherwise (DF included)
    pl->Pr = grow(ctx, t + ":Pr", (size_t)vsize * RG * (size_t)pl->T_c * n, &e);
    if (!pl->Pr) return cuda_error(ctx, e, "allocating the tiled partials");
    pl->Pc = grow(ctx, t + ":Pc", (size_t)vsize * RG * (size_t)pl->T_r * p, &e);
    if (!pl->Pc) return cuda_error(ctx, e, "allocating the tiled partials");
    // launch shapes: one wave of CTAs, rows and columns split evenly (their
    // nonzero counts then differ by a few percent for these designs)
    const size_t smem_c = (size_t)(pl->W_c + 1) * RG * vsize, smem_r = (size_t)(pl->W_r + 1) * RG * vsize;
    const int occ_c = std::max(1, std::min(4, (int)(kSmemPerSm / (smem_c + 4096))));
    const int occ_r = std::max(1, std::min(4, (int)(kSmemPerSm / (smem_r + 4096))));
    // one CTA per SM when the staged slice fills its shared memory: give it
    // 1024 threads so that enough index loads are in flight
    pl->threads = (occ_c == 1 || occ_r == 1) ? 1024 : 512;
    pl->csr_blocks = std::max(1, ctx->num_sms * occ_c / pl->T_c);
    pl->csr_blocks = (int)std::min<int64_t>(pl->csr_blocks, (n + 31) / 32);
    pl->csc_chunks = std::max(1, ctx->num_sms * occ_r / pl->T_r);
    pl->csc_chunks = (int)std::min<int64_t>(pl->csc_chunks, std::max<int64_t>(1, p / 32));
    pl->G_row = pick_lanes(mc_r);
    pl->G_col = pick_lanes(mc_c);
    pl->smem_c = smem_c;
    pl->smem_r = smem_r;
    pl->valid = true;
    return PCG_OK;
}

// ---------------------------------------------------------------------------
// value types.  float and double are gathered and summed as themselves.  DF
// ("double-float") holds each value as an unevaluated pair hi + lo of floats
// (about 48 significant bits) and sums with the error-free TwoSum, so float
// arithmetic reaches float64-like accuracy (GB300 runs float64 at a small
// fraction of its float32 rate).
// ---------------------------------------------------------------------------
template <typename T>
struct Tr;
template <>
struct Tr<float> {
    using smem = float;    // staged value
    using part = float;    // tile / strip partial sums
    using src = float;     // gather source in global memory
};
template <>
struct Tr<double> {
    using smem = double;
    using part = double;
    using src = double;
};
template <>
struct Tr<DF> {
    using smem = float2;
    using part = double;
    using src = double;
};

template <typename T>
__device__ __forceinline__ typename Tr<T>::smem to_smem(typename Tr<T>::src x) { return x; }
template <>
__device__ __forceinline__ float2 to_smem<DF>(double x) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}
template <typename T>
__device__ __forceinline__ typename Tr<T>::smem smem_zero() { return typename Tr<T>::smem(0); }
template <>
__device__ __forceinline__ float2 smem_zero<DF>() { return make_float2(0.f, 0.f); }

// s + x = t + e exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &t, float &e) {
    t = __fadd_rn(a, b);
    const float bv = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bv)), __fsub_rn(b, bv));
}

template <typename T, int RG>
struct Vec {
    T v[RG];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < RG; ++r) v[r] = T(0);
    }
    __device__ __forceinline__ void add_smem(const T *base) {   // base: shared memory
        if constexpr (sizeof(T) == 4 && RG % 4 == 0) {
#pragma unroll
            for (int r = 0; r < RG; r += 4) {
                const float4 x = *reinterpret_cast<const float4 *>(base + r);
                v[r] += x.x; v[r + 1] += x.y; v[r + 2] += x.z; v[r + 3] += x.w;
            }
        } else if constexpr (sizeof(T) == 4 && RG == 2) {
            const float2 x = *reinterpret_cast<const float2 *>(base);
            v[0] += x.x; v[1] += x.y;
        } else if constexpr (sizeof(T) == 8 && RG % 2 == 0) {
#pragma unroll
            for (int r = 0; r < RG; r += 2) {
                const double2 x = *reinterpret_cast<const double2 *>(base + r);
                v[r] += x.x; v[r + 1] += x.y;
            }
        } else {
#pragma unroll
            for (int r = 0; r < RG; ++r) v[r] += base[r];
        }
    }
    template <int G>
    __device__ __forceinline__ void reduce() {
#pragma unroll
        for (int r = 0; r < RG; ++r) v[r] = group_sum<G>(v[r]);
    }
    __device__ __forceinline__ T out(int r) const { return v[r]; }
};

template <int RG>
struct Vec<DF, RG> {
    float s[RG], c[RG];   // running sum and its accumulated rounding errors
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < RG; ++r) s[r] = c[r] = 0.f;
    }
    __device__ __forceinline__ void add1(int r, float2 x) {
        float t, e;
        two_sum(s[r], x.x, t, e);
        s[r] = t;
        c[r] += e + x.y;
    }
    __device__ __forceinline__ void add_smem(const float2 *base) {
        if constexpr (RG % 2 == 0) {
#pragma unroll
            for (int r = 0; r < RG; r += 2) {
                const float4 x = *reinterpret_cast<const float4 *>(base + r);
                add1(r, make_float2(x.x, x.y));
                add1(r + 1, make_float2(x.z, x.w));
            }
        } else {
#pragma unroll
            for (int r = 0; r < RG; ++r) add1(r, base[r]);
        }
    }
    template <int G>
    __device__ __forceinline__ void reduce() {
#pragma unroll
        for (int r = 0; r < RG; ++r) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                const float os = __shfl_xor_sync(kFull, s[r], o), oc = __shfl_xor_sync(kFull, c[r], o);
                float t, e;
                two_sum(s[r], os, t, e);
                s[r] = t;
                c[r] += oc + e;
            }
        }
    }
    __device__ __forceinline__ double out(int r) const { return (double)s[r] + (double)c[r]; }
};

// Adds the gathered values of one whole chunk of 8 indices (pad slots point
// at the zero sentinel, so every entry is added unconditionally).
template <typename T, int RG>
__device__ __forceinline__ void chunk_add(const uint4 w, const typename Tr<T>::smem *__restrict__ sv,
                                          Vec<T, RG> &acc) {
    const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        acc.add_smem(sv + (wd[h] & 0xffffu) * RG);
        acc.add_smem(sv + (wd[h] >> 16) * RG);
    }
}

// Chunks [q0, q1) of one padded segment by a group of G lanes, four 16-byte
// chunk loads in flight per lane.  Every lane of the warp runs the same number
// of rounds (the most any group of the warp needs), the surplus chunks masked,
// so groups never split the warp into separate paths.  All 32 lanes must call
// it (an idle group passes q0 = q1).
template <typename T, int RG, int G>
__device__ __forceinline__ void segment_smem_sum(const uint16_t *__restrict__ idx16, uint32_t q0,
                                                 uint32_t q1, const typename Tr<T>::smem *__restrict__ sv,
                                                 Vec<T, RG> &acc, int lane) {
    const uint4 *__restrict__ w4 = reinterpret_cast<const uint4 *>(idx16);
    const uint32_t rounds = (q1 - q0 + G - 1) / G;
    const uint32_t wr = __reduce_max_sync(kFull, rounds);
    uint32_t q = q0 + lane;
    for (uint32_t t = 0; t < wr; t += 4, q += 4 * G) {
        const bool va = q < q1, vb = q + G < q1, vc = q + 2 * G < q1, vd = q + 3 * G < q1;
        uint4 a = {}, b = {}, c = {}, d = {};
        if (va) a = __ldcs(w4 + q);
        if (vb) b = __ldcs(w4 + q + G);
        if (vc) c = __ldcs(w4 + q + 2 * G);
        if (vd) d = __ldcs(w4 + q + 3 * G);
        if (va) chunk_add<T, RG>(a, sv, acc);
        if (vb) chunk_add<T, RG>(b, sv, acc);
        if (vc) chunk_add<T, RG>(c, sv, acc);
        if (vd) chunk_add<T, RG>(d, sv, acc);
    }
}

// ---------------------------------------------------------------------------
// CSR pass: blockIdx.x = c * csr_blocks + b
// S: global gather source, element (j, r) at S[j * s_stride + s_off + r]
// ---------------------------------------------------------------------------
template <typename T, int RG, int G>
__global__ void __launch_bounds__(1024) k_t_csr(TiledArgs A, const typename Tr<T>::src *__restrict__ S,
                                               int s_stride, int s_off, const int *gate, int gate_need) {
    using SM = typename Tr<T>::smem;
    using PT = typename Tr<T>::part;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (gate && (*(volatile const int *)gate) != gate_need) return;
    SM *sS = reinterpret_cast<SM *>(smem_raw);
    const TiledPlan &P = A.plan;
    const int c = blockIdx.x / P.csr_blocks, b = blockIdx.x % P.csr_blocks;
    const int64_t j0 = (int64_t)c * P.W_c;
    const int64_t ext = min((int64_t)P.W_c, P.p - j0);
    for (int64_t t = threadIdx.x; t < ext * RG; t += blockDim.x) {
        const int64_t j = t / RG;
        const int r = (int)(t - j * RG);
        sS[t] = to_smem<T>(S[(j0 + j) * s_stride + s_off + r]);
    }
    if (threadIdx.x < RG) sS[(size_t)P.W_c * RG + threadIdx.x] = smem_zero<T>();   // pad sentinel
    __syncthreads();
    const int64_t n = P.n;
    const int64_t i0 = n * b / P.csr_blocks, i1 = n * (b + 1) / P.csr_blocks;
    const int lane = threadIdx.x & (G - 1);
    const int gpw = 32 / G;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sub = (threadIdx.x & 31) / G;
    // chunk bounds of tile c: row i's chunks are [rb[i], rb[i + 1])
    const uint32_t *__restrict__ rb = P.rt + (size_t)c * n;
    PT *__restrict__ Pr = reinterpret_cast<PT *>(P.Pr) + (size_t)c * n * RG;
    const int64_t step = (int64_t)nw * gpw;
    int64_t base = i0 + (int64_t)warp * gpw;
    int64_t i = base + sub;
    uint32_t a0 = i < i1 ? __ldg(rb + i) : 0u, a1 = i < i1 ? __ldg(rb + i + 1) : 0u;
    for (; base < i1; base += step) {
        // bounds of this group's next row, loaded while this row is summed
        const int64_t in = i + step;
        const uint32_t b0 = in < i1 ? __ldg(rb + in) : 0u, b1 = in < i1 ? __ldg(rb + in + 1) : 0u;
        Vec<T, RG> acc;
        acc.zero();
        segment_smem_sum<T, RG, G>(P.col16, i < i1 ? a0 : 0u, i < i1 ? a1 : 0u, sS, acc, lane);
        acc.template reduce<G>();
        if (i < i1 && lane == 0) {
#pragma unroll
            for (int r = 0; r < RG; ++r) Pr[(size_t)i * RG + r] = acc.out(r);
        }
        i = in;
        a0 = b0;
        a1 = b1;
    }
}

// ---------------------------------------------------------------------------
// CSC pass: blockIdx.x = t * csc_chunks + h.  Stages u = om (.) sum_c Pr[c]
// for the strip's rows; om element (i, r) at om[i * om_stride + om_off + r].
// Column partial (t, j, r) goes to pc_out[(t * p + j) * pc_stride + pc_off + r].
// ---------------------------------------------------------------------------
template <typename T, int RG, int G>
__global__ void __launch_bounds__(1024) k_t_csc(TiledArgs A, const typename Tr<T>::src *__restrict__ om,
                                               int om_stride, int om_off,
                                               typename Tr<T>::part *__restrict__ pc_out, int pc_stride,
                                               int pc_off, const int *gate, int gate_need) {
    using SM = typename Tr<T>::smem;
    using PT = typename Tr<T>::part;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (gate && (*(volatile const int *)gate) != gate_need) return;
    SM *sU = reinterpret_cast<SM *>(smem_raw);
    const TiledPlan &P = A.plan;
    const int t = blockIdx.x / P.csc_chunks, h = blockIdx.x % P.csc_chunks;
    const int64_t n = P.n, p = P.p;
    const int64_t r0 = (int64_t)t * P.W_r;
    const int64_t ext = min((int64_t)P.W_r, n - r0);
    const PT *__restrict__ Pr = reinterpret_cast<const PT *>(P.Pr);
    for (int64_t q = threadIdx.x; q < ext * RG; q += blockDim.x) {
        const int64_t i = r0 + q / RG;
        const int r = (int)(q % RG);
        PT acc = Pr[(size_t)i * RG + r];
        for (int c = 1; c < P.T_c; ++c) acc += Pr[((size_t)c * n + i) * RG + r];
        sU[q] = to_smem<T>(om[i * om_stride + om_off + r] * acc);
    }
    if (threadIdx.x < RG) sU[(size_t)P.W_r * RG + threadIdx.x] = smem_zero<T>();   // pad sentinel
    __syncthreads();
    // the strip's columns in order of decreasing length; this CTA takes every
    // csc_chunks-th of them, so each CTA gets a mix of lengths and the lane
    // groups of a warp get columns of similar length
    const int64_t jA = 0, jB = (p - h + P.csc_chunks - 1) / P.csc_chunks;   // positions h + k * chunks
    const int lane = threadIdx.x & (G - 1);
    const int gpw = 32 / G;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sub = (threadIdx.x & 31) / G;
    // chunk bounds of strip t: column j's chunks are [cb[j], cb[j + 1])
    const uint32_t *__restrict__ cb = P.cs + (size_t)t * p;
    const int32_t *__restrict__ order = P.col_order;
    PT *__restrict__ Pc = pc_out + (size_t)t * p * pc_stride + pc_off;
    const int64_t step = (int64_t)nw * gpw;
    int64_t base = jA + (int64_t)warp * gpw;
    int64_t k = base + sub;
    int32_t j = k < jB ? __ldg(order + h + k * P.csc_chunks) : 0;
    uint32_t a0 = k < jB ? __ldg(cb + j) : 0u, a1 = k < jB ? __ldg(cb + j + 1) : 0u;
    for (; base < jB; base += step) {
        const int64_t kn = k + step;
        const int32_t jn = kn < jB ? __ldg(order + h + kn * P.csc_chunks) : 0;
        const uint32_t b0 = kn < jB ? __ldg(cb + jn) : 0u, b1 = kn < jB ? __ldg(cb + jn + 1) : 0u;
        Vec<T, RG> acc;
        acc.zero();
        segment_smem_sum<T, RG, G>(P.row16, k < jB ? a0 : 0u, k < jB ? a1 : 0u, sU, acc, lane);
        acc.template reduce<G>();
        if (k < jB && lane == 0) {
#pragma unroll
            for (int r = 0; r < RG; ++r) Pc[(size_t)j * pc_stride + r] = acc.out(r);
        }
        k = kn;
        j = jn;
        a0 = b0;
        a1 = b1;
    }
}

// ---------------------------------------------------------------------------
// single-RHS finalize: v = sum_t Pc[t] + d s (float64), sigma = s.v, alpha
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_t_fin1(const DrawDesc *__restrict__ d, TiledArgs A,
                                                SingleWs ws) {
    __shared__ double red[32];
    __shared__ double sums[1];
    if (*(volatile const int *)&ws.sc->done) return;
    const TiledPlan &P = A.plan;
    const int64_t p = d->p;
    const double tau = d->tau;
    const T *__restrict__ Pc = reinterpret_cast<const T *>(P.Pc);
    double sig = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        T acc = Pc[j];
        for (int t = 1; t < P.T_r; ++t) acc += Pc[(size_t)t * p + j];
        const double sj = ws.s64[j];
        const double v = (double)acc + prior_prec(tau, d->lambda[j]) * sj;
        ws.v64[j] = v;
        sig += sj * v;
    }
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
// host: kernel pointers and shared-memory attributes
// ---------------------------------------------------------------------------
template <typename T, int RG>
static void *csr_ptr(int G) {
    switch (G) {
        case 4: return (void *)k_t_csr<T, RG, 4>;
        case 8: return (void *)k_t_csr<T, RG, 8>;
        case 16: return (void *)k_t_csr<T, RG, 16>;
        default: return (void *)k_t_csr<T, RG, 32>;
    }
}
template <typename T, int RG>
static void *csc_ptr(int G) {
    switch (G) {
        case 4: return (void *)k_t_csc<T, RG, 4>;
        case 8: return (void *)k_t_csc<T, RG, 8>;
        case 16: return (void *)k_t_csc<T, RG, 16>;
        default: return (void *)k_t_csc<T, RG, 32>;
    }
}

template <typename T>
static void *csr_ptr_rg(int RG, int G) {
    switch (RG) {
        case 1: return csr_ptr<T, 1>(G);
        case 2: return csr_ptr<T, 2>(G);
        case 4: return csr_ptr<T, 4>(G);
        default: return csr_ptr<T, 8>(G);
    }
}
template <typename T>
static void *csc_ptr_rg(int RG, int G) {
    switch (RG) {
        case 1: return csc_ptr<T, 1>(G);
        case 2: return csc_ptr<T, 2>(G);
        case 4: return csc_ptr<T, 4>(G);
        default: return csc_ptr<T, 8>(G);
    }
}

TiledKernels tiled_kernels(const TiledPlan &pl) {
    TiledKernels k{};
    if (pl.vtype == kVtF32) {
        k.csr = csr_ptr_rg<float>(pl.RG, pl.G_row);
        k.csc = csc_ptr_rg<float>(pl.RG, pl.G_col);
        k.fin1 = (void *)k_t_fin1<float>;
    } else if (pl.vtype == kVtDF) {
        k.csr = csr_ptr_rg<DF>(pl.RG, pl.G_row);
        k.csc = csc_ptr_rg<DF>(pl.RG, pl.G_col);
        k.fin1 = (void *)k_t_fin1<double>;
    } else {
        k.csr = csr_ptr_rg<double>(pl.RG, pl.G_row);
        k.csc = csc_ptr_rg<double>(pl.RG, pl.G_col);
        k.fin1 = (void *)k_t_fin1<double>;
    }
    return k;
}

pcg_status tiled_prepare(pcg_ctx *ctx, const TiledPlan &pl, TiledKernels *k) {
    *k = tiled_kernels(pl);
    PCG_CUDA_TRY(ctx, cudaFuncSetAttribute(k->csr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem_c));
    PCG_CUDA_TRY(ctx, cudaFuncSetAttribute(k->csc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem_r));
    return PCG_OK;
}

}  // namespace pcg
