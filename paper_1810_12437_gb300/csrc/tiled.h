// Plan and launch interface of the shared-memory tiled products (tiled.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace pcg {

constexpr int kTileSmemBytes = 220 * 1024;   // staged slice of the gathered vector

// value types of the tiled products
constexpr int kVtF32 = 0;   // float values, float sums
constexpr int kVtF64 = 1;   // double values, double sums
constexpr int kVtDF = 2;    // double-float pairs summed with TwoSum (float arithmetic)
constexpr int kVtFX = 3;    // float pairs staged as 64-bit fixed point per tile, integer sums
struct DF {};
struct FX {};

// value type of the tiled products for a precision (PCG_PREC_*)
inline int tiled_vtype(int precision) {
    return precision == PCG_PREC_FP64 ? kVtF64
         : precision == PCG_PREC_DF32 ? kVtDF
         : precision == PCG_PREC_FX64 ? kVtFX
                                      : kVtF32;
}
constexpr size_t kSmemPerSm = 228 * 1024;     // shared memory of one SM
// threads of a tiled-product CTA (one CTA per SM): 24 warps, or 16 when a
// gathered value is wider than 16 bytes (more registers per thread)
constexpr int tiled_threads(int value_bytes) { return value_bytes > 16 ? 512 : 768; }
constexpr int kBlk = 4;                       // chunks a lane reads per block (two blocks in flight)
constexpr uint32_t kSegCost = 2;              // work split: cost of a segment in chunks

struct TiledPlan {
    bool valid;
    int RG, vsize, vtype;     // values gathered per nonzero, staged bytes per value, kVt*
    int ngroups;              // RHS groups sharing the plan (blockIdx.y of the products)
    int64_t n, p, nnz;
    int W_c, T_c;             // column tile width and count (CSR pass)
    int W_r, T_r;             // row strip height and count (CSC pass)
    uint16_t *col16;          // tile-major column offsets inside the tile, each tile's rows by
                              // decreasing length in the tile (row_keys), each row's run padded to
                              // whole 8-entry chunks with the sentinel W_c
    uint16_t *row16;          // strip-major row offsets inside the strip, each strip's columns by
                              // decreasing length in the strip (col_keys), padded likewise (W_r)
    uint32_t *rt;             // rt[c * n + k]: first chunk of row row_keys[c * n + k] in tile c (T_c * n + 1)
    uint32_t *cs;             // cs[t * p + k]: first chunk of column col_keys[t * p + k] in strip t (T_r * p + 1)
    int32_t *row_keys;        // [T_c][n]: the rows of each tile in the CSR pass's segment order
    int32_t *col_keys;        // [T_r][p]: the columns of each strip in the CSC pass's segment order
    int32_t *split_r;         // [T_c][csr_blocks * nw + 1]: first row position of each warp of a column tile
    int32_t *split_c;         // [T_r][csc_chunks * nw + 1]: first column position of each warp of a strip
    // The lane-major copy of col16 that the CSR pass reads: the chunks of warp w
    // of tile c are rows [wrow_r[c * nwt + w], wrow_r[c * nwt + w + 1]) of 32
    // chunks each (nwt = csr_blocks * nw warps per tile), row j of a round
    // holding chunk j of every lane, so that one index load of the warp reads
    // 512 contiguous bytes.  A lane whose segment has no chunk j holds a
    // sentinel chunk there; row lm_sent_r is all sentinel chunks (read past a
    // warp's last round).  The CSC pass reads row16 as stored.
    const uint4 *lm_r;
    uint32_t *wrow_r;   // [T_c * nwt + 1]
    uint32_t lm_sent_r;
    void *Pr;                 // row partials [ngroups][T_c][n][RG]
    void *Pc;                 // column partials [T_r][p][RG] (one group)
    void *U;                  // u = omega (.) sum_c Pr in the staged type: [ngroups][u_stride]
    int64_t u_stride;         // values per group in U (n * RG, padded to 256 bytes)
    int csr_blocks, csc_chunks, threads, nw;
    uint32_t sent_r, sent_c;  // the sentinel chunk (8 zero-slot entries) of each index array
    int *maxch;               // device, [2]: most chunks of one segment in one tile (CSR, CSC pass)
    size_t smem_c, smem_r;    // dynamic shared memory of the two passes
};

struct TiledArgs {
    TiledPlan plan;
};

struct TiledKernels {
    void *csr, *u, *csc, *fin1;
};

// grid of the u kernel (k_t_u, a grid-stride loop): blocks of 256 threads per
// RHS group, at most 8 per SM over all groups and at least 2 per SM and group
// (a launch whose groups are all gated off then schedules few blocks)
inline int tiled_u_blocks(const TiledPlan &pl, int num_sms) {
    const int64_t need = (pl.n * pl.RG + 255) / 256;
    const int per_sm = pl.ngroups >= 4 ? 2 : 8 / (pl.ngroups > 0 ? pl.ngroups : 1);
    const int64_t cap = (int64_t)num_sms * per_sm;
    return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

// Tile widths and counts of the tiled products for a design of this shape
// (RG values of vsize bytes staged per column or row); false when the tiled
// products do not apply: empty X, or more padded positions or segments than
// the plan's 32-bit positions and int counts hold.
bool tiled_geometry(int64_t n, int64_t p, int64_t nnz, int RG, int vsize, int *W_c, int *T_c, int *W_r,
                    int *T_r);

// Builds (on the context stream) the 16-bit index copies, tile bounds and
// per-warp work split of X for RG values of type vtype per gather and
// `ngroups` RHS groups; with many_products also the bank-aware entry order
// (worth its cost only when the plan serves many products).  Leaves
// pl->valid false when the tiled products do not apply (tiled_geometry).
pcg_status build_tiled_plan(pcg_ctx *ctx, const char *tag, const pcg_csr *Xr, const pcg_csc *Xc,
                            int RG, int vtype, int ngroups, bool many_products, TiledPlan *pl);
TiledKernels tiled_kernels(const TiledPlan &pl);
// A hash of every field of the plan (its buffers and shapes): cached graphs
// bake the plan into their kernel parameters, so their keys include it.
uint64_t plan_fingerprint(const TiledPlan &pl);
// kernel pointers plus their dynamic shared-memory attributes
pcg_status tiled_prepare(pcg_ctx *ctx, const TiledPlan &pl, TiledKernels *k);

}  // namespace pcg
