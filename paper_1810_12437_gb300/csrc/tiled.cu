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
#include <string.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include <cub/cub.cuh>

#include "device_common.cuh"
#include "df.cuh"
#include "internal.h"
#include "tiled.h"

namespace pcg {

// ---------------------------------------------------------------------------
// plan building
// ---------------------------------------------------------------------------

// bounds[t * nseg + s] = first position in segment s whose index is >= t * W,
// for t = 0..T (t = 0 gives the segment start, t = T its end).
__global__ void k_plan_bounds(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t nseg,
                              int W, int T, uint32_t *__restrict__ bounds) {
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

// Sort keys of the per-tile segment order: tile ascending, then chunk count
// descending (key = t << 32 | ~chunks), value = the segment.
__global__ void k_plan_tile_keys(const uint32_t *__restrict__ bounds, int64_t nseg, int T,
                                 uint64_t *__restrict__ keys, int32_t *__restrict__ vals) {
    const int64_t total = (int64_t)T * nseg;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = q / nseg, s = q - t * nseg;
        const uint32_t ch = (bounds[(t + 1) * nseg + s] - bounds[t * nseg + s] + 7u) >> 3;
        keys[q] = ((uint64_t)t << 32) | (uint64_t)(~ch);
        vals[q] = (int32_t)s;
    }
}

// chunks[t * nseg + k] = number of 8-index chunks (entries rounded up to a
// multiple of 8) of segment order[t * nseg + k] in tile t; chunks[T * nseg] = 0.
__global__ void k_plan_chunks_sorted(const uint32_t *__restrict__ bounds, const int32_t *__restrict__ order,
                                     int64_t nseg, int T, uint32_t *__restrict__ chunks) {
    const int64_t total = (int64_t)T * nseg;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q <= total;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q == total) {
            chunks[q] = 0u;
        } else {
            const int64_t t = q / nseg, s = order[q];
            chunks[q] = (bounds[(t + 1) * nseg + s] - bounds[t * nseg + s] + 7u) >> 3;
        }
    }
}

// Writes the run of indices of the k-th segment of tile t (segment
// order[t * nseg + k]), as offsets inside the tile, to its own whole chunks
// starting at chunk cstart[t * nseg + k]; the slots after the run are filled
// with the sentinel W (a zero slot in shared memory).
__global__ void k_plan_fill_sorted(const int32_t *__restrict__ idx, const uint32_t *__restrict__ bounds,
                                   const int32_t *__restrict__ order, const uint32_t *__restrict__ cstart,
                                   int64_t nseg, int T, int W, uint16_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = (int64_t)T * nseg;
    for (int64_t q = warp; q < total; q += nwarps) {
        const int64_t t = q / nseg, s = order[q];
        const uint32_t a = bounds[t * nseg + s], b = bounds[(t + 1) * nseg + s];
        const uint32_t len = b - a, padded = (len + 7u) & ~7u;
        const uint64_t dst = (uint64_t)cstart[q] * 8u;
        const int base = (int)(t * W);
        for (uint32_t e = lane; e < padded; e += 32)
            out[dst + e] = e < len ? (uint16_t)(idx[a + e] - base) : (uint16_t)W;
    }
}

// The sentinel chunk: 8 copies of W (every entry reads the zero slot), read by
// lanes whose segment has no chunk left.
__global__ void k_plan_sentinel(uint16_t *__restrict__ chunk, int W) {
    if (threadIdx.x < 8) chunk[threadIdx.x] = (uint16_t)W;
}

// *out = max(*out, most chunks of one segment in one tile) (bounds the number
// of values a fixed-point segment sum adds; *out starts at 0)
__global__ void k_plan_maxch(const uint32_t *__restrict__ chunks, int64_t nts, int *__restrict__ out) {
    uint32_t m = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nts; q += (int64_t)gridDim.x * blockDim.x)
        m = max(m, chunks[q]);
    m = __reduce_max_sync(kFull, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, (int)min(m, (uint32_t)INT32_MAX));
}

// Work split: split[t * (nwt + 1) + k] = first segment of the k-th of nwt
// warps in tile t, chosen so that the warps get equal costs, a segment's cost
// being its chunks plus kSegCost (its bounds, reduction and output)
// (split[.. + 0] = 0 and split[.. + nwt] = nseg, so every segment, empty ones
// included, belongs to exactly one warp).
__global__ void k_plan_split(const uint32_t *__restrict__ cb, int64_t nseg, int T, int nwt,
                             int32_t *__restrict__ split) {
    const int64_t total = (int64_t)T * (nwt + 1);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = q / (nwt + 1);
        const int k = (int)(q - t * (nwt + 1));
        int64_t s;
        if (k == 0) {
            s = 0;
        } else if (k == nwt) {
            s = nseg;
        } else {
            const uint64_t c0 = cb[t * nseg];
            const uint64_t total = (uint64_t)cb[(t + 1) * nseg] - c0 + (uint64_t)kSegCost * (uint64_t)nseg;
            const uint64_t target = total * (uint64_t)k / (uint64_t)nwt;
            int64_t l = 0, h = nseg;   // first segment whose cost prefix reaches the target
            while (l < h) {
                const int64_t m = (l + h) >> 1;
                if ((uint64_t)cb[t * nseg + m] - c0 + (uint64_t)kSegCost * (uint64_t)m < target) l = m + 1;
                else h = m;
            }
            s = l;
        }
        split[q] = (int32_t)s;
    }
}

// lanes per segment (log2) for a warp whose segments hold `chunks` chunks in
// all: one lane when they average at most kLaneChunks chunks (adjacent lanes
// then read adjacent segments), else the fewest lanes (at least two, so that a
// group reads whole sectors) that cover a typical segment with kRoundBlocks
// blocks each.  Longer rounds spread a round's fixed work (bounds, lane
// reduction, output) over more chunks; measured on GB300, two blocks per lane
// beat one by 6-17 % per product, and one lane up to 4 chunks beat up to 2 by
// 3 % on the column pass.
constexpr uint32_t kRoundBlocks = 2;
constexpr uint32_t kLaneChunks = 4;
__device__ __forceinline__ int lanes_log2(uint32_t chunks, uint32_t nseg) {
    if (chunks <= kLaneChunks * nseg) return 0;
    const uint32_t mean = (chunks + nseg - 1) / nseg;
    int lg = 1;
    while (lg < 5 && ((uint32_t)(kRoundBlocks * kBlk) << lg) < mean) ++lg;
    return lg;
}

// Bank-aware entry order.  In the products (warp_segments) each lane walks
// every G-th chunk of its segment in blocks of kBlk, and the k-th shared-memory
// load of a block (chunk k / 8 of the lane's block, entry k % 8) is one
// instruction over the warp whose cost is the largest number of distinct words
// any bank serves.  Entries of one segment can be placed in any of its load
// slots without changing the sum.  This kernel replays the products' schedule
// (the same work split, lanes per segment, rounds and blocks) and, slot by
// slot, lets the lanes of each bank phase claim entries of their block in
// distinct banks: kPermRounds rounds of proposals (each lane proposes a bank
// it still holds, rotated per lane and slot; the lowest lane of a collision
// wins), then the rest take any entry they hold.
// A local search then refines that order (refine_banks).
// nb = banks one load instruction spreads over (128 / bytes per gathered
// value, at least 2); phase = lanes per bank phase (128 / min(bytes, 16)).
constexpr int kPermRounds = 4;
constexpr int kPermWarps = 8;
constexpr int kPermChunks = kBlk;   // chunks per lane and block: 32 entries, one bit each
// the entry sets below are 32-bit masks (one bit per entry of a lane's block)
static_assert(kPermChunks * 8 <= 32, "the bank-order kernel tracks a block's entries in 32-bit masks");
constexpr int kRefineIters = 64;    // swap attempts per bank phase and block

// Largest load of one slot's bank phase (cnt: its non-pad entries per bank;
// z: lanes reading the zero slot, one word in bank bw however many read it)
// and the first bank that carries it.
__device__ __forceinline__ void slot_load(const unsigned char *cnt, int z, int nb, int bw, int &mx, int &mb) {
    mx = 0;
    mb = 0;
    for (int b = 0; b < nb; ++b) {
        const int c = cnt[b] + (b == bw && z > 0);
        if (c > mx) {
            mx = c;
            mb = b;
        }
    }
}

// Local search over one block's order (E[lane][slot], all 32 lanes, after the
// greedy pass).  The cost of a slot in a bank phase is its largest number of
// distinct words one bank serves; pad entries and lanes past their segment's
// end all read the zero slot W, which counts as one word.  For each phase,
// up to kRefineIters times: take a slot whose cost is above one (rotating
// over such slots), one lane's entry in that slot's fullest bank, and let
// every lane of the warp price the swap of that entry with the same lane's
// entry in one other slot (lane s prices slot s); the cheapest swap is taken
// when it does not raise the summed cost of the two slots.  A swap keeps every
// entry in its lane's block, so the products only change in rounding.
// scratch: 1280 bytes of this warp's shared memory.
__device__ void refine_banks(uint16_t (*E)[kPermChunks * 8], unsigned char *scratch, uint32_t vmask, int lane,
                             int nb, int phase, uint32_t W) {
    const int nph = 32 / phase;
    unsigned char *cnt = scratch;                                   // [nph][32 slots][nb]
    unsigned char *zs = scratch + 1024;                             // [nph][32 slots]
    uint32_t *vm = reinterpret_cast<uint32_t *>(scratch + 1152);   // per lane: valid chunks
    __syncwarp();
    vm[lane] = vmask;
    const uint32_t run = __reduce_or_sync(kFull, vmask);   // chunks the warp executes
    const int bw = (int)(W & (uint32_t)(nb - 1));
    const int s = lane;                                     // the slot this lane counts and prices
    const bool exe = (run >> (s >> 3)) & 1u;
    __syncwarp();
    for (int p = 0; p < nph; ++p) {
        unsigned char *row = cnt + (p * 32 + s) * nb;
        for (int b = 0; b < nb; ++b) row[b] = 0;
        int z = 0;
        if (exe) {
            for (int q = 0; q < phase; ++q) {
                const int l = p * phase + q;
                if ((vm[l] >> (s >> 3)) & 1u) {
                    const uint32_t x = E[l][s];
                    if (x == W) ++z;
                    else ++row[x & (uint32_t)(nb - 1)];
                } else {
                    ++z;
                }
            }
        }
        zs[p * 32 + s] = (unsigned char)z;
    }
    __syncwarp();
    for (int p = 0; p < nph; ++p) {
        for (int it = 0; it < kRefineIters; ++it) {
            int mx = 0, mb = 0;
            if (exe) slot_load(cnt + (p * 32 + s) * nb, zs[p * 32 + s], nb, bw, mx, mb);
            const unsigned conf = __ballot_sync(kFull, mx >= 2);
            if (!conf) break;
            const int rot = (it * 13 + p * 7) & 31;
            const int s1 = (__ffs(__funnelshift_r(conf, conf, rot)) - 1 + rot) & 31;
            const int b1 = __shfl_sync(kFull, mb, s1);
            const int m1 = __shfl_sync(kFull, mx, s1);
            bool cand = false;   // lane q of the phase holds a non-pad entry of bank b1 in slot s1
            if (lane < phase) {
                const int l = p * phase + lane;
                if ((vm[l] >> (s1 >> 3)) & 1u) {
                    const uint32_t x = E[l][s1];
                    cand = x != W && (int)(x & (uint32_t)(nb - 1)) == b1;
                }
            }
            const unsigned cm = __ballot_sync(kFull, cand);
            if (!cm) continue;
            const int qr = (it * 5) & (phase - 1);
            const int l = p * phase + ((__ffs(__funnelshift_r(cm, cm, qr)) - 1 + qr) & 31);
            const uint32_t x1 = E[l][s1];
            int delta = 1 << 16;
            uint32_t x2 = 0;
            int b2 = -1;
            if (s != s1 && exe && ((vm[l] >> (s >> 3)) & 1u)) {
                x2 = E[l][s];
                b2 = x2 == W ? -1 : (int)(x2 & (uint32_t)(nb - 1));
                if (b2 != b1) {
                    const unsigned char *r1 = cnt + (p * 32 + s1) * nb, *r2 = cnt + (p * 32 + s) * nb;
                    const int z1 = zs[p * 32 + s1] + (b2 < 0), z2 = zs[p * 32 + s] - (b2 < 0);
                    int n1 = 0, n2 = 0;
                    for (int b = 0; b < nb; ++b) {
                        const int c1 = r1[b] - (b == b1) + (b == b2) + (b == bw && z1 > 0);
                        const int c2 = r2[b] - (b == b2) + (b == b1) + (b == bw && z2 > 0);
                        n1 = max(n1, c1);
                        n2 = max(n2, c2);
                    }
                    delta = n1 + n2 - m1 - mx;
                }
            }
            const unsigned key = ((unsigned)(delta + 16) << 5) | (unsigned)((s - rot) & 31);
            const unsigned best = __reduce_min_sync(kFull, key);
            if ((int)(best >> 5) - 16 <= 0 && key == best) {
                unsigned char *r1 = cnt + (p * 32 + s1) * nb, *r2 = cnt + (p * 32 + s) * nb;
                E[l][s1] = (uint16_t)x2;
                E[l][s] = (uint16_t)x1;
                --r1[b1];
                ++r2[b1];
                if (b2 < 0) {
                    ++zs[p * 32 + s1];
                    --zs[p * 32 + s];
                } else {
                    ++r1[b2];
                    --r2[b2];
                }
            }
            __syncwarp();
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kPermWarps * 32)
    k_plan_permute(uint16_t *__restrict__ idx16, const uint32_t *__restrict__ cb_all,
                   const int32_t *__restrict__ split, int64_t nseg, int T, int nwt, int nb, int phase,
                   uint32_t W) {
    __shared__ uint16_t ent_s[kPermWarps][32][kPermChunks * 8];
    __shared__ uint32_t bm_s[kPermWarps][32][32];   // per lane and bank: unplaced entries (bit i = ent[i])
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kPermWarps + wl;   // simulated warp: tile t, warp k
    if (gw >= (int64_t)T * nwt) return;
    const int t = (int)(gw / nwt), k = (int)(gw - (int64_t)t * nwt);
    const int sA = split[(int64_t)t * (nwt + 1) + k], sB = split[(int64_t)t * (nwt + 1) + k + 1];
    const uint32_t *__restrict__ cb = cb_all + (int64_t)t * nseg;
    uint4 *__restrict__ w4 = reinterpret_cast<uint4 *>(idx16);
    const unsigned phase_lanes = phase >= 32 ? kFull : (((1u << phase) - 1u) << (lane & ~(phase - 1)));
    uint16_t *ent = ent_s[wl][lane];
    uint32_t *bm = bm_s[wl][lane];
    if (sA >= sB) return;
    const int lg = lanes_log2(cb[sB] - cb[sA], (uint32_t)(sB - sA));
    const int spr = 32 >> lg, sub = lane >> lg, ln = lane & ((1 << lg) - 1);
    for (int base = sA; base < sB; base += spr) {
        const int seg = base + sub;
        const uint32_t q0 = seg < sB ? cb[seg] : 0u, q1 = seg < sB ? cb[seg + 1] : 0u;
        const uint32_t m = __reduce_max_sync(kFull, q1 - q0);
        const uint32_t nch = (m + (1u << lg) - 1) >> lg;   // chunks per lane
        const uint32_t nwin = (nch + kPermChunks - 1) / kPermChunks;
        for (uint32_t win = 0; win < nwin; ++win) {
            // the lane's chunk u of this block: q + u G
            const uint32_t q = q0 + (uint32_t)ln + ((win * kPermChunks) << lg);
            unsigned vmask = 0;   // valid chunk slots u of this window
#pragma unroll
            for (int u = 0; u < kPermChunks; ++u) {
                const uint32_t c = q + ((uint32_t)u << lg);
                if (c < q1) {
                    vmask |= 1u << u;
                    const uint4 w = w4[c];
                    const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        ent[u * 8 + 2 * h] = (uint16_t)(wd[h] & 0xffffu);
                        ent[u * 8 + 2 * h + 1] = (uint16_t)(wd[h] >> 16);
                    }
                }
            }
            for (int b = 0; b < nb; ++b) bm[b] = 0u;
            uint32_t rem = 0;   // entries not yet placed (bit i = ent[i])
#pragma unroll
            for (int u = 0; u < kPermChunks; ++u)
                if (vmask >> u & 1u) rem |= 0xffu << (u * 8);
            uint32_t have = 0;   // banks this lane still holds
            for (int i = 0; i < kPermChunks * 8; ++i) {
                if (rem >> i & 1u) {
                    const int b = ent[i] & (nb - 1);
                    bm[b] |= 1u << i;
                    have |= 1u << b;
                }
            }
            uint16_t placed[kPermChunks * 8];
            for (int slot = 0; slot < kPermChunks * 8; ++slot) {
                const int u = slot >> 3;
                const bool part = (vmask >> u) & 1u;
                if (!__any_sync(kFull, part)) continue;
                bool done = !part;
                int pick = -1;
                uint32_t taken = 0;   // banks claimed in this lane's phase
                for (int r = 0; r < kPermRounds; ++r) {
                    int prop = -1;
                    const uint32_t av = have & ~taken;
                    if (!done && av) {
                        const int rot = (lane * 7 + slot * 3 + r * 5) & (nb - 1);
                        // first bank at or after rot (cyclically) among av
                        const uint32_t hi = av & (~0u << rot), lo = av & ~(~0u << rot);
                        prop = hi ? (__ffs(hi) - 1) : (__ffs(lo) - 1);
                    }
                    const unsigned same = __match_any_sync(kFull, prop < 0 ? -1 - lane : prop);
                    const unsigned peers = same & phase_lanes;
                    const bool win_ = prop >= 0 && (__ffs(peers) - 1) == lane;
                    uint32_t claim = win_ ? (1u << prop) : 0u;
                    for (int o = phase >> 1; o > 0; o >>= 1) claim |= __shfl_xor_sync(kFull, claim, o);
                    taken |= claim;
                    if (win_) {
                        done = true;
                        pick = prop;
                    }
                }
                if (part) {
                    const int b0 = pick >= 0 ? pick : (ent[__ffs(rem) - 1] & (nb - 1));
                    const int i = __ffs(bm[b0]) - 1;
                    bm[b0] &= ~(1u << i);
                    if (!bm[b0]) have &= ~(1u << b0);
                    rem &= ~(1u << i);
                    placed[slot] = ent[i];
                }
            }
            __syncwarp();   // every lane is done with its greedy pass (ent, bm)
#pragma unroll
            for (int i = 0; i < kPermChunks * 8; ++i) ent[i] = (vmask >> (i >> 3) & 1u) ? placed[i] : (uint16_t)W;
            refine_banks(ent_s[wl], reinterpret_cast<unsigned char *>(bm_s[wl]), vmask, lane, nb, phase, W);
#pragma unroll
            for (int u = 0; u < kPermChunks; ++u) {
                if (vmask >> u & 1u) {
                    uint4 w;
                    w.x = (uint32_t)ent[u * 8 + 0] | ((uint32_t)ent[u * 8 + 1] << 16);
                    w.y = (uint32_t)ent[u * 8 + 2] | ((uint32_t)ent[u * 8 + 3] << 16);
                    w.z = (uint32_t)ent[u * 8 + 4] | ((uint32_t)ent[u * 8 + 5] << 16);
                    w.w = (uint32_t)ent[u * 8 + 6] | ((uint32_t)ent[u * 8 + 7] << 16);
                    w4[q + ((uint32_t)u << lg)] = w;
                }
            }
            __syncwarp();   // ent and bm are rewritten by the next block
        }
    }
}

// Lane-major layout.  Warp w of tile t (item q = t * nwt + w) sums the
// segments [split[t][w], split[t][w + 1]) in rounds of 32 >> lg segments, a
// round running nch chunk rows (nch: the round's longest segment in chunks,
// divided by the 2^lg lanes per segment and rounded up); in row j lane l reads
// chunk ln + j 2^lg of its segment (l = sub 2^lg + ln), or the sentinel chunk
// past the segment's end.  k_plan_lm_rows counts each item's rows (rows[q];
// rows[T * nwt] = 0), k_plan_lm_fill copies the chunks to their rows starting
// at row wrow[q] (the exclusive sum of rows), one warp per item, so the
// products read in row j exactly the chunk they would have read before.
__device__ __forceinline__ int lm_item(const uint32_t *__restrict__ cb, const int32_t *__restrict__ split,
                                       int64_t nseg, int nwt, int64_t q, const uint32_t **cbt, int *sA, int *sB) {
    const int64_t t = q / nwt;
    const int w = (int)(q - t * nwt);
    const int32_t *sp = split + t * (nwt + 1) + w;
    *sA = sp[0];
    *sB = sp[1];
    *cbt = cb + t * nseg;
    return *sA < *sB ? lanes_log2((*cbt)[*sB] - (*cbt)[*sA], (uint32_t)(*sB - *sA)) : 0;
}

__global__ void k_plan_lm_rows(const uint32_t *__restrict__ cb, const int32_t *__restrict__ split, int64_t nseg,
                               int T, int nwt, uint32_t *__restrict__ rows) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)T * nwt;
    if (warp == 0 && lane == 0) rows[items] = 0u;
    for (int64_t q = warp; q < items; q += nwarps) {
        const uint32_t *cbt;
        int sA, sB;
        const int lg = lm_item(cb, split, nseg, nwt, q, &cbt, &sA, &sB);
        const int spr = 32 >> lg, sub = lane >> lg;
        uint32_t r = 0;
        for (int base = sA; base < sB; base += spr) {
            const int seg = base + sub;
            const uint32_t len = seg < sB ? cbt[seg + 1] - cbt[seg] : 0u;
            r += (__reduce_max_sync(kFull, len) + (1u << lg) - 1) >> lg;
        }
        if (lane == 0) rows[q] = r;
    }
}

__global__ void k_plan_lm_fill(const uint4 *__restrict__ src, const uint32_t *__restrict__ cb,
                               const int32_t *__restrict__ split, int64_t nseg, int T, int nwt,
                               const uint32_t *__restrict__ wrow, uint32_t sent, uint4 *__restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)T * nwt;
    const uint4 pad = src[sent];
    if (warp == 0) dst[((size_t)wrow[items] << 5) + lane] = pad;   // the all-sentinel row
    for (int64_t q = warp; q < items; q += nwarps) {
        const uint32_t *cbt;
        int sA, sB;
        const int lg = lm_item(cb, split, nseg, nwt, q, &cbt, &sA, &sB);
        const int spr = 32 >> lg, sub = lane >> lg, ln = lane & ((1 << lg) - 1);
        size_t row = wrow[q];
        for (int base = sA; base < sB; base += spr) {
            const int seg = base + sub;
            const uint32_t q0 = seg < sB ? cbt[seg] : 0u, q1 = seg < sB ? cbt[seg + 1] : 0u;
            const uint32_t nch = (__reduce_max_sync(kFull, q1 - q0) + (1u << lg) - 1) >> lg;
            for (uint32_t j = 0; j < nch; ++j) {
                const uint32_t c = q0 + (uint32_t)ln + (j << lg);
                dst[((row + j) << 5) + lane] = c < q1 ? src[c] : pad;
            }
            row += nch;
        }
    }
}

// Builds one side of the plan: padded tile-major indices, chunk bounds and
// the per-warp work split.
static pcg_status plan_side(pcg_ctx *ctx, const std::string &tag, const int64_t *ptr,
                            const int32_t *idx, int64_t nseg, int64_t nnz, int W, int T, int nwt,
                            int value_bytes, bool bank_order, uint16_t **out_idx, uint32_t **out_cb,
                            int32_t **out_split, uint32_t *out_sent, int32_t **out_keys, int *out_maxch,
                            bool lane_major, const uint4 **out_lm, uint32_t **out_wrow, uint32_t *out_lm_sent,
                            bool *fits) {
    *fits = false;
    cudaError_t e;
    const int64_t nb = (int64_t)(T + 1) * nseg;
    const int64_t nts = (int64_t)T * nseg;
    uint32_t *bounds = (uint32_t *)grow(ctx, tag + ":bounds", sizeof(uint32_t) * nb, &e);
    if (!bounds) return cuda_error(ctx, e, "allocating the tiled plan");
    const int64_t nc = nts + 1;
    uint32_t *chunks = (uint32_t *)grow(ctx, tag + ":chunks", sizeof(uint32_t) * nc, &e);
    if (!chunks) return cuda_error(ctx, e, "allocating the tiled plan");
    uint32_t *cb = (uint32_t *)grow(ctx, tag + ":cb", sizeof(uint32_t) * nc, &e);
    if (!cb) return cuda_error(ctx, e, "allocating the tiled plan");
    int32_t *split = (int32_t *)grow(ctx, tag + ":split", sizeof(int32_t) * (size_t)T * (nwt + 1), &e);
    if (!split) return cuda_error(ctx, e, "allocating the tiled plan");
    uint64_t *skeys = (uint64_t *)grow(ctx, tag + ":sort_keys", sizeof(uint64_t) * 2 * nts, &e);
    if (!skeys) return cuda_error(ctx, e, "allocating the tiled plan");
    int32_t *svals = (int32_t *)grow(ctx, tag + ":sort_vals", sizeof(int32_t) * 2 * nts, &e);
    if (!svals) return cuda_error(ctx, e, "allocating the tiled plan");
    // at most 7 pad slots per segment, then the sentinel chunk
    const int64_t cap = ((nnz + 7 * nts + 7) & ~int64_t(7)) + 8;
    uint16_t *pidx = (uint16_t *)grow(ctx, tag + ":idx", sizeof(uint16_t) * cap, &e);
    if (!pidx) return cuda_error(ctx, e, "allocating the tiled plan");
    const int64_t items = (int64_t)T * nwt;   // (tile, warp) pairs of the lane-major layout
    uint32_t *lrows = (uint32_t *)grow(ctx, tag + ":lm_rows", sizeof(uint32_t) * (items + 1), &e);
    if (!lrows) return cuda_error(ctx, e, "allocating the tiled plan");
    uint32_t *wrow = (uint32_t *)grow(ctx, tag + ":wrow", sizeof(uint32_t) * (items + 1), &e);
    if (!wrow) return cuda_error(ctx, e, "allocating the tiled plan");
    size_t scan_bytes = 0, sort_bytes = 0, lm_scan_bytes = 0;
    int tbits = 1;
    while ((1 << tbits) < T) ++tbits;
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, chunks, cb, (int)nc, ctx->stream);
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, skeys, skeys + nts, svals, svals + nts, (int)nts, 0,
                                    32 + tbits, ctx->stream);
    cub::DeviceScan::ExclusiveSum(nullptr, lm_scan_bytes, lrows, wrow, (int)(items + 1), ctx->stream);
    void *tmp = grow(ctx, "plan:tmp", std::max(std::max(scan_bytes, sort_bytes), lm_scan_bytes) + 256, &e);
    if (!tmp) return cuda_error(ctx, e, "allocating the plan scratch");
    const int grid = grid_for(ctx, 256, 8);
    cudaStream_t s = ctx->stream;
    int32_t *order = svals + nts;
    // segment bounds per tile in the stored order, then every tile's segments
    // by decreasing chunk count (stable: ties keep the stored order), so the
    // segments a round of a warp holds have nearly equal lengths
    PCG_PROF(ctx, "plan_bounds", k_plan_bounds<<<grid, 256, 0, s>>>(ptr, idx, nseg, W, T, bounds));
    PCG_PROF(ctx, "plan_order", k_plan_tile_keys<<<grid, 256, 0, s>>>(bounds, nseg, T, skeys, svals));
    PCG_CUDA_TRY(ctx, cub::DeviceRadixSort::SortPairs(tmp, sort_bytes, skeys, skeys + nts, svals, order, (int)nts,
                                                      0, 32 + tbits, s));
    PCG_PROF(ctx, "plan_chunks", k_plan_chunks_sorted<<<grid, 256, 0, s>>>(bounds, order, nseg, T, chunks));
    PCG_CUDA_TRY(ctx, cub::DeviceScan::ExclusiveSum(tmp, scan_bytes, chunks, cb, (int)nc, s));
    k_plan_maxch<<<grid, 256, 0, s>>>(chunks, nts, out_maxch);
    PCG_PROF(ctx, "plan_fill", k_plan_fill_sorted<<<grid, 256, 0, s>>>(idx, bounds, order, cb, nseg, T, W, pidx));
    const uint32_t sent = (uint32_t)(cap / 8 - 1);
    k_plan_sentinel<<<1, 32, 0, s>>>(pidx + (size_t)sent * 8, W);
    PCG_PROF(ctx, "plan_split", k_plan_split<<<grid_for(ctx, 256, 1), 256, 0, s>>>(cb, nseg, T, nwt, split));
    if (bank_order) {
        const int nb = std::max(2, 128 / value_bytes), phase = 128 / std::min(value_bytes, 16);
        const int64_t sim = (int64_t)T * nwt;
        const int blocks = (int)((sim + kPermWarps - 1) / kPermWarps);
        PCG_PROF(ctx, "plan_permute",
                 k_plan_permute<<<blocks, kPermWarps * 32, 0, s>>>(pidx, cb, split, nseg, T, nwt, nb, phase,
                                                                    (uint32_t)W));
    }
    *out_idx = pidx;
    *out_cb = cb;
    *out_split = split;
    *out_sent = sent;
    *out_keys = order;
    if (!lane_major) {
        PCG_CUDA_TRY(ctx, cudaGetLastError());
        *fits = true;
        return PCG_OK;
    }
    // the lane-major copy: rows per (tile, warp), their exclusive sum, then
    // the copy into (total + 1) rows of 32 chunks
    k_plan_lm_rows<<<grid, 256, 0, s>>>(cb, split, nseg, T, nwt, lrows);
    PCG_CUDA_TRY(ctx, cub::DeviceScan::ExclusiveSum(tmp, lm_scan_bytes, lrows, wrow, (int)(items + 1), s));
    uint32_t *htot = (uint32_t *)grow_host(ctx, tag + ":lm_total", sizeof(uint32_t), &e);
    if (!htot) return cuda_error(ctx, e, "allocating the tiled plan");
    PCG_CUDA_TRY(ctx, cudaMemcpyAsync(htot, wrow + items, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PCG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const uint64_t rows = *htot;
    if ((rows + 1) * 32u >= (uint64_t)UINT32_MAX) return PCG_OK;   // chunk positions must fit 32 bits
    uint4 *lm = (uint4 *)grow(ctx, tag + ":lm", sizeof(uint4) * (size_t)(rows + 1) * 32u, &e);
    if (!lm) return cuda_error(ctx, e, "allocating the lane-major index copy");
    PCG_PROF(ctx, "plan_lane_major",
             k_plan_lm_fill<<<grid, 256, 0, s>>>(reinterpret_cast<const uint4 *>(pidx), cb, split, nseg, T, nwt,
                                                 wrow, sent, lm));
    PCG_CUDA_TRY(ctx, cudaGetLastError());
    *out_lm = lm;
    *out_wrow = wrow;
    *out_lm_sent = (uint32_t)rows;
    *fits = true;
    return PCG_OK;
}

// splitmix64's finalizer
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// *out += a position-dependent hash of every entry of the design's four index
// arrays (a sum of mixed (array, position, value) words, so the order in which
// threads add does not matter; *out starts at 0)
__global__ void k_design_hash(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const int64_t *__restrict__ cp, const int32_t *__restrict__ ri, int64_t n,
                              int64_t p, int64_t nnz, unsigned long long *__restrict__ out) {
    unsigned long long h = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = tid; i < nnz; i += stride) {
        const unsigned long long q = (unsigned long long)i << 2;
        h += mix64(((unsigned long long)(uint32_t)__ldg(ci + i) << 32) ^ (q | 0ull) ^ 0x9e3779b97f4a7c15ull);
        h += mix64(((unsigned long long)(uint32_t)__ldg(ri + i) << 32) ^ (q | 1ull) ^ 0xc2b2ae3d27d4eb4full);
    }
    for (int64_t i = tid; i <= n; i += stride)
        h += mix64(mix64((unsigned long long)__ldg(rp + i)) ^ (((unsigned long long)i << 2) | 2ull));
    for (int64_t i = tid; i <= p; i += stride)
        h += mix64(mix64((unsigned long long)__ldg(cp + i)) ^ (((unsigned long long)i << 2) | 3ull));
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(kFull, h, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, h);
}

// A cached plan: valid while the design's pointers, sizes and content (hash)
// and the plan's parameters are those it was built for.
struct PlanCacheEntry {
    uint64_t key, content;
    TiledPlan plan;
};

static uint64_t fnv_mix(uint64_t h, uint64_t v) {
    for (int k = 0; k < 8; ++k) {
        h ^= (v >> (8 * k)) & 0xffu;
        h *= 1099511628211ull;
    }
    return h;
}

bool tiled_geometry(int64_t n, int64_t p, int64_t nnz, int RG, int vsize, int *W_c, int *T_c, int *W_r,
                    int *T_r) {
    if (n <= 0 || p <= 0 || nnz <= 0 || RG <= 0 || vsize <= 0) return false;
    if (n >= (int64_t)INT32_MAX || p >= (int64_t)INT32_MAX) return false;
    int64_t w = (kTileSmemBytes - RG * vsize) / (RG * vsize);   // one slot is the zero sentinel
    w = std::min<int64_t>(w, 65528);
    w &= ~int64_t(7);
    if (w < 8) return false;
    // as few tiles (strips) as fit, then equal widths (a multiple of 8), so that
    // the last one is not a small remainder whose CTAs idle while the others work
    auto balanced = [&](int64_t len, int *W, int *T) {
        const int64_t t = (len + std::min(w, len) - 1) / std::min(w, len);
        *T = (int)t;
        *W = (int)(t == 1 ? len : std::min<int64_t>(w, ((len + t - 1) / t + 7) & ~int64_t(7)));
    };
    balanced(p, W_c, T_c);
    balanced(n, W_r, T_r);
    // Each side keeps every entry's padded position in 32 bits (at most 7 pad
    // slots for each of the T x nseg segments, the sentinel chunk after them:
    // the allocation plan_side makes) and counts its segments, and one bound
    // per segment and tile boundary, in int (the sorts and scans).
    auto fits = [&](int64_t T, int64_t nseg) {
        const int64_t nts = T * nseg;
        const int64_t cap = ((nnz + 7 * nts + 7) & ~int64_t(7)) + 8;
        return (T + 1) * nseg < (int64_t)INT32_MAX && cap < (int64_t)0xfffffff0ll;
    };
    return fits(*T_c, n) && fits(*T_r, p);
}

pcg_status build_tiled_plan(pcg_ctx *ctx, const char *tag, const pcg_csr *Xr, const pcg_csc *Xc,
                            int RG, int vtype, int ngroups, bool many_products, TiledPlan *pl) {
    *pl = TiledPlan{};
    const int vsize = vtype == kVtF32 ? 4 : 8;   // staged bytes per value (DF: two floats; FX: int64)
    pl->vtype = vtype;
    const int64_t n = Xr->n, p = Xr->p, nnz = Xr->nnz;
    int Wc = 0, Tc = 0, Wr = 0, Tr = 0;
    if (!tiled_geometry(n, p, nnz, RG, vsize, &Wc, &Tc, &Wr, &Tr)) return PCG_OK;   // untiled products
    // A plan depends on the design alone (and on RG, the value type and the
    // groups): reuse the one built for this tag when nothing it depends on has
    // changed, the design's content included (hashed on the device: about one
    // read of the index arrays, instead of the plan's sorts and bank order).
    uint64_t key = 1469598103934665603ull, content = 0;
    if (ctx->plan_cache_enabled) {
        const uint64_t vals[] = {(uint64_t)(uintptr_t)Xr->row_ptr, (uint64_t)(uintptr_t)Xr->col_idx,
                                 (uint64_t)(uintptr_t)Xc->col_ptr, (uint64_t)(uintptr_t)Xc->row_idx,
                                 (uint64_t)n, (uint64_t)p, (uint64_t)nnz, (uint64_t)RG, (uint64_t)vtype,
                                 (uint64_t)ngroups, (uint64_t)(many_products && ctx->bank_permute),
                                 (uint64_t)ctx->num_sms};
        for (uint64_t v : vals) key = fnv_mix(key, v);
        for (const char *c = tag; *c; ++c) key = fnv_mix(key, (uint64_t)(unsigned char)*c);
        cudaError_t e;
        unsigned long long *dh = (unsigned long long *)grow(ctx, "plan:hash", sizeof(unsigned long long), &e);
        if (!dh) return cuda_error(ctx, e, "allocating the design hash");
        unsigned long long *hh =
            (unsigned long long *)grow_host(ctx, "plan:hash", sizeof(unsigned long long), &e);
        if (!hh) return cuda_error(ctx, e, "allocating the design hash");
        PCG_CUDA_TRY(ctx, cudaMemsetAsync(dh, 0, sizeof(unsigned long long), ctx->stream));
        k_design_hash<<<grid_for(ctx, 256, 8), 256, 0, ctx->stream>>>(Xr->row_ptr, Xr->col_idx, Xc->col_ptr,
                                                                     Xc->row_idx, n, p, nnz, dh);
        PCG_CUDA_TRY(ctx, cudaGetLastError());
        PCG_CUDA_TRY(ctx, cudaMemcpyAsync(hh, dh, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
        PCG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        content = *hh;
        auto it = ctx->plan_cache.find(tag);
        if (it != ctx->plan_cache.end() && it->second.size() == sizeof(PlanCacheEntry)) {
            PlanCacheEntry ent;
            memcpy(&ent, it->second.data(), sizeof ent);
            if (ent.key == key && ent.content == content) {
                *pl = ent.plan;
                return PCG_OK;
            }
        }
        ctx->plan_cache.erase(tag);   // rebuilt below under the same buffer names
    }
    pl->RG = RG;
    pl->vsize = vsize;
    pl->ngroups = std::max(1, ngroups);
    pl->n = n;
    pl->p = p;
    pl->nnz = nnz;
    pl->W_c = Wc;
    pl->T_c = Tc;
    pl->W_r = Wr;
    pl->T_r = Tr;
    // launch shapes: per group one wave of CTAs over the tiles (strips)
    const size_t smem_c = (size_t)(pl->W_c + 1) * RG * vsize, smem_r = (size_t)(pl->W_r + 1) * RG * vsize;
    const int occ_c = std::max(1, std::min(2, (int)(kSmemPerSm / (smem_c + 2048))));
    const int occ_r = std::max(1, std::min(2, (int)(kSmemPerSm / (smem_r + 2048))));
    pl->threads = tiled_threads(RG * vsize);
    pl->nw = pl->threads / 32;
    pl->csr_blocks = std::max(1, ctx->num_sms * occ_c / pl->T_c);
    pl->csr_blocks = (int)std::min<int64_t>(pl->csr_blocks, std::max<int64_t>(1, n / (2 * pl->nw)));
    pl->csc_chunks = std::max(1, ctx->num_sms * occ_r / pl->T_r);
    pl->csc_chunks = (int)std::min<int64_t>(pl->csc_chunks, std::max<int64_t>(1, p / (2 * pl->nw)));
    pl->smem_c = smem_c;
    pl->smem_r = smem_r;
    std::string t(tag);
    // the bank-aware entry order costs tens of products' time: only for plans
    // that serve a whole solve
    const bool bank_order = ctx->bank_permute && many_products;
    cudaError_t e;
    pl->maxch = (int *)grow(ctx, t + ":maxch", 2 * sizeof(int), &e);
    if (!pl->maxch) return cuda_error(ctx, e, "allocating the tiled plan");
    PCG_CUDA_TRY(ctx, cudaMemsetAsync(pl->maxch, 0, 2 * sizeof(int), ctx->stream));
    bool fits_r = false, fits_c = false;
    pcg_status st = plan_side(ctx, t + ":csr", Xr->row_ptr, Xr->col_idx, n, nnz, pl->W_c, pl->T_c,
                              pl->csr_blocks * pl->nw, RG * vsize, bank_order, &pl->col16, &pl->rt,
                              &pl->split_r, &pl->sent_r, &pl->row_keys, pl->maxch, true, &pl->lm_r,
                              &pl->wrow_r, &pl->lm_sent_r, &fits_r);
    if (st != PCG_OK) return st;
    if (!fits_r) return PCG_OK;   // untiled products (pl->valid stays false)
    st = plan_side(ctx, t + ":csc", Xc->col_ptr, Xc->row_idx, p, nnz, pl->W_r, pl->T_r, pl->csc_chunks * pl->nw,
                   RG * vsize, bank_order, &pl->row16, &pl->cs, &pl->split_c, &pl->sent_c, &pl->col_keys,
                   pl->maxch + 1, false, nullptr, nullptr, nullptr, &fits_c);
    if (st != PCG_OK) return st;
    if (!fits_c) return PCG_OK;
    // partial sums: float for float values, double otherwise (DF included);
    // row partials per group, column partials of one group (callers with
    // several groups pass their own column-partial array)
    pl->Pr = grow(ctx, t + ":Pr", (size_t)vsize * RG * (size_t)pl->T_c * n * pl->ngroups, &e);
    if (!pl->Pr) return cuda_error(ctx, e, "allocating the tiled partials");
    pl->Pc = grow(ctx, t + ":Pc", (size_t)vsize * RG * (size_t)pl->T_r * p, &e);
    if (!pl->Pc) return cuda_error(ctx, e, "allocating the tiled partials");
    // u of every group, each group's slice padded to 256 bytes
    pl->u_stride = (((int64_t)vsize * RG * n + 255) & ~int64_t(255)) / vsize;
    pl->U = grow(ctx, t + ":U", (size_t)vsize * pl->u_stride * pl->ngroups, &e);
    if (!pl->U) return cuda_error(ctx, e, "allocating the tiled u");
    pl->valid = true;
    if (ctx->plan_cache_enabled) {
        PlanCacheEntry ent{key, content, *pl};
        std::vector<unsigned char> bytes(sizeof ent);
        memcpy(bytes.data(), &ent, sizeof ent);
        ctx->plan_cache[tag] = std::move(bytes);
    }
    return PCG_OK;
}

// ---------------------------------------------------------------------------
// value types.  float and double are gathered and summed as themselves.  DF
// ("double-float", df.cuh) holds each value as a pair hi + lo of floats and
// sums with TwoSum, so float arithmetic reaches float64-like accuracy; its
// sources (s, omega), staged values and partial sums are all float pairs, so
// the products run no float64 instruction.
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
    using part = float2;
    using src = float2;
};
template <>
struct Tr<FX> {
    using smem = long long;   // the value times 2^k, rounded (k: the tile's scale exponent)
    using part = float2;
    using src = float2;
};

template <typename T>
__device__ __forceinline__ typename Tr<T>::smem smem_zero() { return typename Tr<T>::smem(0); }
template <>
__device__ __forceinline__ float2 smem_zero<DF>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ long long smem_zero<FX>() { return 0ll; }
template <typename T>
__device__ __forceinline__ typename Tr<T>::src src_zero() { return typename Tr<T>::src(0); }
template <>
__device__ __forceinline__ float2 src_zero<DF>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ float2 src_zero<FX>() { return make_float2(0.f, 0.f); }

// ---------------------------------------------------------------------------
// Fixed point (FX).  A CTA stages its tile of float pairs (hi + lo), takes the
// largest |hi| of each right-hand side r over the tile, and picks k_r so that
// every value of r times 2^k_r stays below 2^(61 - hb), where a segment of the
// pass adds fewer than 2^hb values (hb: bits of 8 x the plan's most chunks in
// one segment and tile).  Each value becomes round(hi 2^k) + round(lo 2^k) as
// a 64-bit integer, so every segment sum is exact and below 2^61; the grid
// step 2^-k_r is 2^(hb - 60) of r's largest value in the tile or less.  A sum
// is returned as a float pair times 2^-k_r.  The conversions use integer and
// float32 instructions only (GB300 runs 64-bit float/integer conversions at
// the float64 rate).
// ---------------------------------------------------------------------------
constexpr int kFxNonFinite = INT32_MIN;   // scale of a tile holding NaN or Inf

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }   // -126 <= e <= 127

// k for a tile whose largest |hi| has float bits mb
__device__ __forceinline__ int fx_scale(uint32_t mb, int maxch) {
    if (mb >= 0x7f800000u) return kFxNonFinite;
    if (mb == 0u) return 0;
    const int e = max(1, (int)(mb >> 23));                   // |value| < 2^(e - 126)
    const int hb = 32 - __clz(8 * max(1, maxch));            // a segment adds fewer than 2^hb values
    return 187 - hb - e;                                     // 61 - hb - (e - 126)
}

// round(x 2^k) for |x 2^k| < 2^58, from the bits of x: x = m 2^E with an
// integer mantissa m < 2^24, so x 2^k = m 2^s, shifted left, or right with
// rounding to nearest (halves away from zero)
__device__ __forceinline__ long long fx_round(float x, int k) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu);
    const uint32_t m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int s = (e ? e : 1) - 150 + k;
    long long q;
    if (s >= 0) q = (long long)((unsigned long long)m << s);
    else if (s >= -24) q = (long long)((m + (1u << (-s - 1))) >> (-s));
    else q = 0;
    return (b >> 31) ? -q : q;
}

__device__ __forceinline__ long long fx_from_pair(float2 v, int k) {
    if (k == kFxNonFinite) return 0ll;
    return fx_round(v.x, k) + fx_round(v.y, k);
}

// q 2^-k as a float pair: q = p2 2^42 + p1 2^21 + p0 with pieces of at most 21
// bits (each an exact float), summed with TwoSum; |k| <= 187 applied as two
// exact power-of-two products
__device__ __forceinline__ float2 fx_to_pair(long long q, int k) {
    if (k == kFxNonFinite) return make_float2(__int_as_float(0x7fc00000), 0.f);
    const int p2 = (int)(q >> 42);                                     // |p2| < 2^20 (|q| < 2^62)
    const uint32_t r = (uint32_t)((((unsigned long long)q) >> 21) & 0x1fffffull);        // bits 21..41
    const uint32_t p0 = (uint32_t)q & 0x1fffffu;
    const float a = __int2float_rn(p2) * 4398046511104.f;             // 2^42
    const float b = __uint2float_rn(r) * 2097152.f;                    // 2^21
    float t, e, t2, e2;
    two_sum(a, b, t, e);
    two_sum(t, __uint2float_rn(p0), t2, e2);
    const float2 d = df_norm(t2, __fadd_rn(e, e2));
    const float t1 = pow2f(-(k >> 1)), t3 = pow2f(-(k - (k >> 1)));
    return make_float2(d.x * t1 * t3, d.y * t1 * t3);
}

// Per right-hand side scales of a CTA: thread values m0 (for r0) and m1 (for
// r0 + 1, when two == true) are the largest |hi| bits it staged; every thread
// of a warp with the same lane % span holds the same r0.  Writes k_r to
// sk[0..RG) (red: 32 * 8 words of shared memory); ends with a barrier.
template <int RG>
__device__ __forceinline__ void fx_scales(uint32_t m0, uint32_t m1, bool two, int span, int maxch,
                                          uint32_t *red, int *sk) {
    for (int o = 16; o >= span; o >>= 1) {
        m0 = max(m0, __shfl_xor_sync(kFull, m0, o));
        m1 = max(m1, __shfl_xor_sync(kFull, m1, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane < span) {
        if (two) {
            red[w * RG + 2 * lane] = m0;
            red[w * RG + 2 * lane + 1] = m1;
        } else {
            red[w * RG + lane] = m0;
        }
    }
    __syncthreads();
    if (threadIdx.x < RG) {
        uint32_t M = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) M = max(M, red[q * RG + threadIdx.x]);
        sk[threadIdx.x] = fx_scale(M, maxch);
    }
    __syncthreads();
}

// u = omega * (sum of row partials), in the staged type
__device__ __forceinline__ float scale_part(float o, float a) { return o * a; }
__device__ __forceinline__ double scale_part(double o, double a) { return o * a; }
__device__ __forceinline__ float2 scale_part(float2 o, float2 a) { return df_mul(o, a); }

// Accumulators of RG sums, in two independent sets (entries alternate between
// them, so consecutive additions do not wait on each other).  Even RG sums
// run as packed pairs (FADD2).
template <typename T, int RG>
struct Vec {
    T v[2][RG];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int r = 0; r < RG; ++r) v[k][r] = T(0);
    }
    __device__ __forceinline__ void bind(const int *) {}
    template <int K>
    __device__ __forceinline__ void add_smem(const T *base) {   // base: shared memory
        if constexpr (sizeof(T) == 4 && RG % 4 == 0) {
#pragma unroll
            for (int r = 0; r < RG; r += 4) {
                const float4 x = *reinterpret_cast<const float4 *>(base + r);
                add2<K>(r, make_float2(x.x, x.y));
                add2<K>(r + 2, make_float2(x.z, x.w));
            }
        } else if constexpr (sizeof(T) == 4 && RG == 2) {
            add2<K>(0, *reinterpret_cast<const float2 *>(base));
        } else if constexpr (sizeof(T) == 8 && RG % 2 == 0) {
#pragma unroll
            for (int r = 0; r < RG; r += 2) {
                const double2 x = *reinterpret_cast<const double2 *>(base + r);
                v[K][r] += x.x;
                v[K][r + 1] += x.y;
            }
        } else {
#pragma unroll
            for (int r = 0; r < RG; ++r) v[K][r] += base[r];
        }
    }
    template <int K>
    __device__ __forceinline__ void add2(int r, float2 x) {   // float only: v[K][r..r+1] += x
        const float2 s = __fadd2_rn(make_float2(v[K][r], v[K][r + 1]), x);
        v[K][r] = s.x;
        v[K][r + 1] = s.y;
    }
    // merges the two sets, then sums over aligned groups of 2^lg lanes
    // (every lane of the warp calls it)
    __device__ __forceinline__ void reduce(int lg) {
#pragma unroll
        for (int r = 0; r < RG; ++r) v[0][r] += v[1][r];
        for (int o = (1 << lg) >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int r = 0; r < RG; ++r) v[0][r] += __shfl_xor_sync(kFull, v[0][r], o);
        }
    }
    __device__ __forceinline__ T out(int r) const { return v[0][r]; }
};

// One right-hand side: the two accumulator sets (entries alternate between
// them) live in the x and y halves of one float pair, so the two entries of
// an index word take one packed TwoSum (the same roundings as two scalar ones).
template <>
struct Vec<DF, 1> {
    float2 S, C;   // S.x, C.x: set 0's sum and accumulated errors; S.y, C.y: set 1's
    __device__ __forceinline__ void bind(const int *) {}
    __device__ __forceinline__ void zero() { S = C = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add_word(const float2 *b0, const float2 *b1) {
        const float2 x0 = *b0, x1 = *b1;   // (hi, lo) of the word's two entries
        float2 t, e;
        two_sum2(S, make_float2(x0.x, x1.x), t, e);
        S = t;
        C = __fadd2_rn(C, __fadd2_rn(e, make_float2(x0.y, x1.y)));
    }
    __device__ __forceinline__ static void merge2(float &s0, float &c0, float s1, float c1) {
        float t, e;
        two_sum(s0, s1, t, e);
        s0 = t;
        c0 += c1 + e;
    }
    __device__ __forceinline__ void reduce(int lg) {
        merge2(S.x, C.x, S.y, C.y);
        for (int o = (1 << lg) >> 1; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(kFull, S.x, o), oc = __shfl_xor_sync(kFull, C.x, o);
            merge2(S.x, C.x, os, oc);
        }
    }
    __device__ __forceinline__ float2 out(int) const { return df_norm(S.x, C.x); }
};

// Double-float sums, RG >= 2 (RG = 1: the specialization above).  A staged
// row holds RG values as [hi_0 .. hi_{RG-1}, lo_0 .. lo_{RG-1}] (for RG = 1
// simply (hi, lo)), so that the his and los of two right-hand sides are
// adjacent pairs and their TwoSums run packed (two_sum2).  s: running sums,
// c: their accumulated rounding errors.
template <int RG>
struct Vec<DF, RG> {
    static_assert(RG >= 2, "one right-hand side uses Vec<DF, 1>");
    static constexpr int NP = RG / 2;   // packed pairs
    float2 s[2][NP], c[2][NP];
    __device__ __forceinline__ void bind(const int *) {}
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int q = 0; q < NP; ++q) s[k][q] = c[k][q] = make_float2(0.f, 0.f);
    }
    template <int K>
    __device__ __forceinline__ void add_smem(const float2 *base) {
        const float *f = reinterpret_cast<const float *>(base);
        if constexpr (RG == 2) {
            const float4 x = *reinterpret_cast<const float4 *>(f);   // hi0 hi1 lo0 lo1
            add_pair<K>(0, make_float2(x.x, x.y), make_float2(x.z, x.w));
        } else {
#pragma unroll
            for (int q = 0; q < NP; q += 2) {
                const float4 h = *reinterpret_cast<const float4 *>(f + 2 * q);
                const float4 l = *reinterpret_cast<const float4 *>(f + RG + 2 * q);
                add_pair<K>(q, make_float2(h.x, h.y), make_float2(l.x, l.y));
                add_pair<K>(q + 1, make_float2(h.z, h.w), make_float2(l.z, l.w));
            }
        }
    }
    template <int K>
    __device__ __forceinline__ void add_pair(int q, float2 hi, float2 lo) {
        float2 t, e;
        two_sum2(s[K][q], hi, t, e);
        s[K][q] = t;
        c[K][q] = __fadd2_rn(c[K][q], __fadd2_rn(e, lo));
    }
    __device__ __forceinline__ static void merge2(float &s0, float &c0, float s1, float c1) {
        float t, e;
        two_sum(s0, s1, t, e);
        s0 = t;
        c0 += c1 + e;
    }
    __device__ __forceinline__ void reduce(int lg) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            merge2(s[0][q].x, c[0][q].x, s[1][q].x, c[1][q].x);
            merge2(s[0][q].y, c[0][q].y, s[1][q].y, c[1][q].y);
        }
        for (int o = (1 << lg) >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float os = __shfl_xor_sync(kFull, s[0][q].x, o), oc = __shfl_xor_sync(kFull, c[0][q].x, o);
                merge2(s[0][q].x, c[0][q].x, os, oc);
                os = __shfl_xor_sync(kFull, s[0][q].y, o);
                oc = __shfl_xor_sync(kFull, c[0][q].y, o);
                merge2(s[0][q].y, c[0][q].y, os, oc);
            }
        }
    }
    __device__ __forceinline__ float2 out(int r) const {
        const float2 sq = s[0][r >> 1], cq = c[0][r >> 1];
        return (r & 1) ? df_norm(sq.y, cq.y) : df_norm(sq.x, cq.x);
    }
};

// Fixed-point sums (see FX above): exact integer additions in two sets.
template <int RG>
struct Vec<FX, RG> {
    long long a[2][RG];
    int k[RG];   // the tile's scale exponent of each right-hand side
    __device__ __forceinline__ void bind(const int *sk) {
#pragma unroll
        for (int r = 0; r < RG; ++r) k[r] = sk[r];
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < RG; ++r) a[j][r] = 0ll;
    }
    template <int K>
    __device__ __forceinline__ void add_smem(const long long *base) {
        if constexpr (RG == 1) {
            a[K][0] += base[0];
        } else {
#pragma unroll
            for (int r = 0; r < RG; r += 2) {
                const longlong2 x = *reinterpret_cast<const longlong2 *>(base + r);
                a[K][r] += x.x;
                a[K][r + 1] += x.y;
            }
        }
    }
    __device__ __forceinline__ void reduce(int lg) {
#pragma unroll
        for (int r = 0; r < RG; ++r) a[0][r] += a[1][r];
        for (int o = (1 << lg) >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int r = 0; r < RG; ++r) a[0][r] += __shfl_xor_sync(kFull, a[0][r], o);
        }
    }
    __device__ __forceinline__ float2 out(int r) const { return fx_to_pair(a[0][r], k[r]); }
};

// Writes value r of a staged row (the split layout above for double-float;
// fixed point stages each value as its float pair, converted in place later).
template <typename T, int RG, typename V>
__device__ __forceinline__ void store_staged(typename Tr<T>::smem *row, int r, V v) {
    if constexpr (std::is_same<T, DF>::value) {
        float *f = reinterpret_cast<float *>(row);
        f[r] = v.x;
        f[RG + r] = v.y;
    } else if constexpr (std::is_same<T, FX>::value) {
        reinterpret_cast<float2 *>(row)[r] = v;
    } else {
        row[r] = v;
    }
}

// Fixed point: converts the CTA's staged float pairs [0, nvals) (value t
// belongs to right-hand side t % RG) to int64 in place with the scales sk.
// blockDim.x is a multiple of RG, so a thread's values share one r.
template <int RG>
__device__ __forceinline__ void fx_convert(long long *sv, int64_t nvals, const int *sk) {
    const int k = sk[threadIdx.x % RG];
    float2 *f = reinterpret_cast<float2 *>(sv);
    for (int64_t t = threadIdx.x; t < nvals; t += blockDim.x) sv[t] = fx_from_pair(f[t], k);
}

// Adds the gathered values of one whole chunk of 8 indices (pad slots point
// at the zero sentinel, so every entry is added unconditionally).
template <typename T, int RG>
__device__ __forceinline__ void chunk_add(const uint4 w, const typename Tr<T>::smem *__restrict__ sv,
                                          Vec<T, RG> &acc) {
    const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        if constexpr (std::is_same<T, DF>::value && RG == 1) {
            acc.add_word(sv + (wd[h] & 0xffffu), sv + (wd[h] >> 16));   // both entries in one packed TwoSum
        } else {
            acc.template add_smem<0>(sv + (wd[h] & 0xffffu) * RG);
            acc.template add_smem<1>(sv + (wd[h] >> 16) * RG);
        }
    }
}

// One warp sums the segments [sA, sB) of a tile (rows of a column tile, or
// columns of a row strip, in their stored order), G lanes per segment: lane
// ln of a group reads the segment's chunks ln + G j and adds the staged values
// their entries name; the group's lanes are summed at the end.  G (1 to 32)
// is chosen per warp so that a typical segment of its range takes
// kRoundBlocks blocks of kBlk chunks per lane.  The warp runs in rounds of
// 32 / G consecutive segments; in a round every group runs the same number of
// chunks (the round's longest segment: the CSR rows have similar lengths and
// the CSC columns are stored by decreasing length), a lane past its
// segment's end reading a sentinel chunk (all zero values).  The next block
// (of this round, or the first of the next round) is loaded before the
// current one is summed, so 2 kBlk chunks per lane are in flight.  Segment s's
// chunks are [cb[s], cb[s + 1]); its sum goes to out[(keys ? keys[s] : s) *
// ostride + r].  fxk: the tile's fixed-point scale exponent of each
// right-hand side (FX only).
//
// Two index layouts (LM): the stored one, where chunk c of the tile-major
// stream w4 is w4[c] and `sent` is the sentinel chunk, or the plan's
// lane-major copy, where the warp's rows start at row `row0`, row j of a round
// holds chunk j of every lane (one index load of the warp is 512 contiguous
// bytes) and row `sent` is all sentinel chunks.  Measured on GB300 at n = 5e5,
// p = 5e4: the lane-major copy makes the CSR pass 8-12 % faster and the CSC
// pass 3-5 % slower, so the CSR pass reads it and the CSC pass the stored one.
struct SegRound {
    uint32_t q0, q1;   // this lane's segment's chunks (lane-major: 0 and its chunk count)
    int64_t key;
    uint32_t nch;      // chunks per lane in this round (uniform over the warp)
};

template <bool LM>
__device__ __forceinline__ SegRound load_round(const uint32_t *__restrict__ cb, const int32_t *__restrict__ keys,
                                               int base, int sB, int sub) {
    SegRound R;
    const int seg = base + sub;
    R.q0 = R.q1 = 0;
    R.key = seg;
    if (seg < sB) {
        if constexpr (LM) {
            R.q1 = __ldg(cb + seg + 1) - __ldg(cb + seg);
        } else {
            R.q0 = __ldg(cb + seg);
            R.q1 = __ldg(cb + seg + 1);
        }
        if (keys) R.key = __ldg(keys + seg);
    }
    R.nch = 0;
    return R;
}

__device__ __forceinline__ uint32_t round_chunks(const SegRound &R, int lg) {
    const uint32_t m = __reduce_max_sync(kFull, R.q1 - R.q0);
    return (m + (1u << lg) - 1) >> lg;
}

// stored layout: chunks q0 + ln + G (j + u) of this lane's segment
__device__ __forceinline__ void load_block(uint4 (&A)[kBlk], const uint4 *__restrict__ w4, const SegRound &R,
                                           uint32_t j, int ln, int lg, uint32_t sent) {
#pragma unroll
    for (int u = 0; u < kBlk; ++u) {
        const uint32_t c = R.q0 + (uint32_t)ln + ((j + (uint32_t)u) << lg);
        A[u] = w4[c < R.q1 ? c : sent];
    }
}

// lane-major layout: rows [row, row + kBlk), this lane's chunk of each; rows
// at or past `rend` read the sentinel row
__device__ __forceinline__ void load_rows(uint4 (&A)[kBlk], const uint4 *__restrict__ w4, uint32_t row,
                                          uint32_t rend, uint32_t sent_row, int lane) {
#pragma unroll
    for (int u = 0; u < kBlk; ++u) {
        const uint32_t r = row + (uint32_t)u;
        A[u] = w4[((r < rend ? r : sent_row) << 5) + (uint32_t)lane];
    }
}

template <typename T, int RG, bool LM>
__device__ __forceinline__ void warp_segments(const uint4 *__restrict__ w4, uint32_t row0, uint32_t sent,
                                              const uint32_t *__restrict__ cb, int sA, int sB,
                                              const typename Tr<T>::smem *__restrict__ sv,
                                              const int32_t *__restrict__ keys,
                                              typename Tr<T>::part *__restrict__ out, int64_t ostride,
                                              const int *fxk) {
    if (sA >= sB) return;
    const int lane = threadIdx.x & 31;
    const int lg = lanes_log2(__ldg(cb + sB) - __ldg(cb + sA), (uint32_t)(sB - sA));
    const int spr = 32 >> lg, sub = lane >> lg, ln = lane & ((1 << lg) - 1);
    SegRound cur = load_round<LM>(cb, keys, sA, sB, sub);
    cur.nch = round_chunks(cur, lg);
    SegRound nxt = load_round<LM>(cb, keys, sA + spr, sB, sub);
    int base = sA;
    uint32_t j = 0, rb = row0;   // rb (lane-major): the current round's first row
    uint4 A[kBlk];
    if constexpr (LM) load_rows(A, w4, rb, rb + cur.nch, sent, lane);
    else load_block(A, w4, cur, 0, ln, lg, sent);
    Vec<T, RG> acc;
    acc.bind(fxk);
    acc.zero();
    for (;;) {
        // the block after this one: in this round, or the first of the next
        const bool last = j + kBlk >= cur.nch;
        if (last && base + spr < sB) nxt.nch = round_chunks(nxt, lg);
        uint4 B[kBlk];
        if constexpr (LM) {
            if (!last) load_rows(B, w4, rb + j + kBlk, rb + cur.nch, sent, lane);
            else load_rows(B, w4, rb + cur.nch, rb + cur.nch + nxt.nch, sent, lane);
        } else {
            if (!last) load_block(B, w4, cur, j + kBlk, ln, lg, sent);
            else load_block(B, w4, nxt, 0, ln, lg, sent);
        }
#pragma unroll
        for (int u = 0; u < kBlk; ++u)
            if (j + (uint32_t)u < cur.nch) chunk_add<T, RG>(A[u], sv, acc);
        if (last) {
            acc.reduce(lg);
            if (base + sub < sB && ln == 0) {
#pragma unroll
                for (int r = 0; r < RG; ++r) out[cur.key * ostride + r] = acc.out(r);
            }
            acc.zero();
            base += spr;
            if (base >= sB) break;
            rb += cur.nch;
            cur = nxt;
            nxt = load_round<LM>(cb, keys, base + spr, sB, sub);
            j = 0;
        } else {
            j += kBlk;
        }
#pragma unroll
        for (int u = 0; u < kBlk; ++u) A[u] = B[u];
    }
}

// ---------------------------------------------------------------------------
// CSR pass: block (x, g) of group_block(), x = c * csr_blocks + b, g the RHS group.
// S: global gather source, element (j, r) of group g at
// S[j * s_stride + s_off + g * RG + r].  Skipped when gate[g] != gate_need.
// Writes the row partials of tile c: Pr[g][c][i][r].
// ---------------------------------------------------------------------------
constexpr int kStageUnroll = 16;   // staging: loads in flight per thread (8: 0.4 % slower per draw)

// (slice x, RHS group g) of a product block, for launches whose gridDim.y is
// the group count.  The blocks are numbered with the group varying fastest
// (linear id = x * groups + g), so the blocks of every group over one slice of
// X are dispatched together and the slice's index stream, read by each of
// them, comes from DRAM once and from L2 for the other groups (numbered group
// by group, each group would stream all of X's indices from DRAM again).
struct GroupBlock {
    int x, g;
};
__device__ __forceinline__ GroupBlock group_block() {
    if (gridDim.y == 1) return {(int)blockIdx.x, 0};
    const unsigned lin = blockIdx.x + blockIdx.y * gridDim.x;
    return {(int)(lin / gridDim.y), (int)(lin % gridDim.y)};
}

template <typename T, int RG>
__global__ void __launch_bounds__(tiled_threads(sizeof(typename Tr<T>::smem) * RG), 1)
    k_t_csr(TiledArgs A, const typename Tr<T>::src *__restrict__ S, int s_stride, int s_off, const int *gate,
            int gate_need) {
    using SM = typename Tr<T>::smem;
    using PT = typename Tr<T>::part;
    using SRC = typename Tr<T>::src;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GroupBlock gb = group_block();
    const int g = gb.g;
    if (gate && (*(volatile const int *)(gate + g)) != gate_need) return;
    SM *sS = reinterpret_cast<SM *>(smem_raw);
    const TiledPlan &P = A.plan;
    const int c = gb.x / P.csr_blocks, b = gb.x % P.csr_blocks;
    const int64_t j0 = (int64_t)c * P.W_c;
    const int64_t total = min((int64_t)P.W_c, P.p - j0) * RG;
    const int off = s_off + g * RG;
    constexpr bool fx = std::is_same<T, FX>::value;
    uint32_t mb = 0;   // fixed point: largest |hi| this thread staged (float bits)
    bool direct = false;
    if constexpr (!fx && (std::is_same<T, float>::value || std::is_same<T, double>::value ||
                          (std::is_same<T, DF>::value && RG == 1))) {
        // The staged layout is the source's here.  When the slice is
        // contiguous in global memory (one group: s_stride == RG) and 16-byte
        // aligned, copy it with cp.async: the whole slice in flight and no
        // registers held (one CTA per SM: nothing else hides the latency).
        const SRC *src = S + j0 * RG + off;
        direct = s_stride == RG && (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
        if (direct) {
            const int64_t words = (total * (int64_t)sizeof(SRC)) >> 4;
            const uint32_t sdst = (uint32_t)__cvta_generic_to_shared(sS);
            const uint4 *src4 = reinterpret_cast<const uint4 *>(src);
            for (int64_t w = threadIdx.x; w < words; w += blockDim.x)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst + (uint32_t)(w << 4)),
                             "l"(src4 + w)
                             : "memory");
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            // values past the last whole 16-byte word
            for (int64_t t = ((words << 4) / (int64_t)sizeof(SRC)) + threadIdx.x; t < total; t += blockDim.x)
                sS[t] = __ldg(src + t);
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        }
    }
    // otherwise stage the tile's slice of s through registers, kStageUnroll
    // loads in flight per thread
    for (int64_t t0 = threadIdx.x; !direct && t0 < total; t0 += (int64_t)kStageUnroll * blockDim.x) {
        SRC v[kStageUnroll];
#pragma unroll
        for (int k = 0; k < kStageUnroll; ++k) {
            const int64_t t = t0 + (int64_t)k * blockDim.x;
            v[k] = t < total ? __ldg(S + (j0 + t / RG) * s_stride + off + (int)(t % RG)) : src_zero<T>();
        }
#pragma unroll
        for (int k = 0; k < kStageUnroll; ++k) {
            const int64_t t = t0 + (int64_t)k * blockDim.x;
            if (t < total) store_staged<T, RG>(sS + (t / RG) * RG, (int)(t % RG), v[k]);
            if constexpr (fx) mb = max(mb, __float_as_uint(fabsf(v[k].x)));   // zero past the end
        }
    }
    if (threadIdx.x < RG) sS[(size_t)P.W_c * RG + threadIdx.x] = smem_zero<T>();   // pad sentinel
    __shared__ int fxk[8];
    if constexpr (fx) {
        __shared__ uint32_t red[32 * 8];
        fx_scales<RG>(mb, 0u, false, RG, __ldg(P.maxch), red, fxk);   // thread's values: r = tid % RG
        fx_convert<RG>(sS, total, fxk);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int wt = b * P.nw + warp;   // this warp's index within the tile
    const int32_t *__restrict__ sp = P.split_r + (size_t)c * (P.csr_blocks * P.nw + 1) + wt;
    const int sA = __ldg(sp), sB = __ldg(sp + 1);
    const uint32_t row0 = __ldg(P.wrow_r + (size_t)c * (P.csr_blocks * P.nw) + wt);
    PT *__restrict__ Pr = reinterpret_cast<PT *>(P.Pr) + ((size_t)g * P.T_c + c) * (size_t)P.n * RG;
    warp_segments<T, RG, true>(P.lm_r, row0, P.lm_sent_r, P.rt + (size_t)c * P.n, sA, sB, sS,
                               P.row_keys + (size_t)c * P.n, Pr, RG, fxk);
}

// ---------------------------------------------------------------------------
// u = om (.) sum_c Pr[g][c], once per iteration, in the staged value type:
// U[g][i][r] (group stride P.u_stride values).  blockIdx.y = RHS group g; om
// element (i, r) of group g at om[i * om_stride + om_off + g * RG + r].
// ---------------------------------------------------------------------------
template <typename T, int RG>
__global__ void __launch_bounds__(256) k_t_u(TiledArgs A, const typename Tr<T>::src *__restrict__ om,
                                             int om_stride, int om_off, const int *gate, int gate_need) {
    using PT = typename Tr<T>::part;
    using SM = typename Tr<T>::smem;
    const int g = blockIdx.y;
    if (gate && (*(volatile const int *)(gate + g)) != gate_need) return;
    const TiledPlan &P = A.plan;
    const int64_t n = P.n, total = n * RG;
    const PT *__restrict__ Pr = reinterpret_cast<const PT *>(P.Pr) + (size_t)g * P.T_c * (size_t)total;
    SM *__restrict__ U = reinterpret_cast<SM *>(P.U) + (size_t)g * P.u_stride;
    const int ooff = om_off + g * RG;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / RG;
        const int r = (int)(q % RG);
        const PT acc = sum_strided(Pr + q, P.T_c, (size_t)total);
        store_staged<T, RG>(U + i * RG, r, scale_part(__ldg(om + i * om_stride + ooff + r), acc));
    }
}

// ---------------------------------------------------------------------------
// CSC pass: block (x, g) of group_block(), x = t * csc_chunks + h, g the RHS group.
// Stages the strip's rows of U[g] (a contiguous copy, 16 bytes per load) and
// sums its columns' entries.  Column partial (t, j, r) goes to
// pc_out[(t * p + j) * pc_stride + pc_off + g * RG + r].
// ---------------------------------------------------------------------------
template <typename T, int RG>
__global__ void __launch_bounds__(tiled_threads(sizeof(typename Tr<T>::smem) * RG), 1)
    k_t_csc(TiledArgs A, typename Tr<T>::part *__restrict__ pc_out, int pc_stride, int pc_off, const int *gate,
            int gate_need) {
    using SM = typename Tr<T>::smem;
    using PT = typename Tr<T>::part;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GroupBlock gb = group_block();
    const int g = gb.g;
    if (gate && (*(volatile const int *)(gate + g)) != gate_need) return;
    SM *sU = reinterpret_cast<SM *>(smem_raw);
    const TiledPlan &P = A.plan;
    const int t = gb.x / P.csc_chunks, h = gb.x % P.csc_chunks;
    const int64_t n = P.n, p = P.p;
    const int64_t r0 = (int64_t)t * P.W_r;
    // bytes of the strip's slice, rounded up to whole 16-byte words (the
    // group's U is padded; the strip start is 32-byte aligned since W_r is a
    // multiple of 8)
    const int64_t bytes = min((int64_t)P.W_r, n - r0) * RG * (int64_t)sizeof(SM);
    const int64_t words = (bytes + 15) >> 4;
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(
        reinterpret_cast<const SM *>(P.U) + (size_t)g * P.u_stride + (size_t)r0 * RG);
    uint4 *dst = reinterpret_cast<uint4 *>(smem_raw);
    constexpr bool fx = std::is_same<T, FX>::value;
    const int64_t nvals = min((int64_t)P.W_r, n - r0) * RG;
    uint32_t mb = 0, mb1 = 0;   // fixed point: largest |hi| of the even and odd values this thread copied
    if constexpr (!fx) {
        // asynchronous 16-byte copies straight into shared memory: every word
        // of the slice in flight at once and no registers held (one CTA per
        // SM, so the copy's latency is not hidden by another CTA's work)
        const uint32_t sdst = (uint32_t)__cvta_generic_to_shared(dst);
        for (int64_t w = threadIdx.x; w < words; w += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst + (uint32_t)(w << 4)),
                         "l"(src + w)
                         : "memory");
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    // fixed point reads every value it copies (its tile scale): 16-byte words
    // through registers, half the float-pair unroll
    constexpr int kWordUnroll = kStageUnroll / 2;
    for (int64_t w0 = threadIdx.x; fx && w0 < words; w0 += (int64_t)kWordUnroll * blockDim.x) {
        uint4 v[kWordUnroll];
#pragma unroll
        for (int k = 0; k < kWordUnroll; ++k) {
            const int64_t w = w0 + (int64_t)k * blockDim.x;
            if (w < words) v[k] = __ldg(src + w);
        }
#pragma unroll
        for (int k = 0; k < kWordUnroll; ++k) {
            const int64_t w = w0 + (int64_t)k * blockDim.x;
            if (w < words) {
                dst[w] = v[k];
                if constexpr (fx) {   // |hi| of values 2w and 2w + 1 (the last word may run past the strip)
                    mb = max(mb, v[k].x & 0x7fffffffu);
                    if (2 * w + 1 < nvals) mb1 = max(mb1, v[k].z & 0x7fffffffu);
                }
            }
        }
    }
    __shared__ int fxk[8];
    if constexpr (fx) {
        // a thread's words hold values 2w, 2w + 1 with w = tid (mod 2), so
        // r0 = 2 tid % RG, and r0 + 1 for RG >= 2; fx_scales ends with a barrier
        __shared__ uint32_t red[32 * 8];
        if constexpr (RG == 1) fx_scales<RG>(max(mb, mb1), 0u, false, 1, __ldg(P.maxch + 1), red, fxk);
        else fx_scales<RG>(mb, mb1, true, RG / 2, __ldg(P.maxch + 1), red, fxk);
        fx_convert<RG>(sU, nvals, fxk);
    } else {
        __syncthreads();   // the pad sentinel may share the last copied word
    }
    if (threadIdx.x < RG) sU[(size_t)P.W_r * RG + threadIdx.x] = smem_zero<T>();
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int wt = h * P.nw + warp;   // this warp's index within the strip
    const int32_t *__restrict__ sp = P.split_c + (size_t)t * (P.csc_chunks * P.nw + 1) + wt;
    const int sA = __ldg(sp), sB = __ldg(sp + 1);
    PT *__restrict__ Pc = pc_out + (size_t)t * p * pc_stride + pc_off + g * RG;
    warp_segments<T, RG, false>(reinterpret_cast<const uint4 *>(P.row16), 0u, P.sent_c, P.cs + (size_t)t * p, sA,
                                sB, sU, P.col_keys + (size_t)t * p, Pc, pc_stride, fxk);
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
        const T acc = sum_strided(Pc + j, P.T_r, (size_t)p);
        const double sj = ws.s64[j];
        const double v = part_to_double(acc) + desc_d(d, j) * sj;
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
template <typename T>
static void *csr_ptr_rg(int RG) {
    switch (RG) {
        case 1: return (void *)k_t_csr<T, 1>;
        case 2: return (void *)k_t_csr<T, 2>;
        case 4: return (void *)k_t_csr<T, 4>;
        default: return (void *)k_t_csr<T, 8>;
    }
}
template <typename T>
static void *u_ptr_rg(int RG) {
    switch (RG) {
        case 1: return (void *)k_t_u<T, 1>;
        case 2: return (void *)k_t_u<T, 2>;
        case 4: return (void *)k_t_u<T, 4>;
        default: return (void *)k_t_u<T, 8>;
    }
}
template <typename T>
static void *csc_ptr_rg(int RG) {
    switch (RG) {
        case 1: return (void *)k_t_csc<T, 1>;
        case 2: return (void *)k_t_csc<T, 2>;
        case 4: return (void *)k_t_csc<T, 4>;
        default: return (void *)k_t_csc<T, 8>;
    }
}

uint64_t plan_fingerprint(const TiledPlan &pl) {
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the fields
    auto mix = [&](uint64_t v) {
        for (int k = 0; k < 8; ++k) {
            h ^= (v >> (8 * k)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    const void *ptrs[] = {pl.col16, pl.row16, pl.rt, pl.cs, pl.row_keys, pl.col_keys, pl.split_r, pl.split_c,
                          pl.Pr, pl.Pc, pl.U, pl.maxch, pl.lm_r, pl.wrow_r};
    for (const void *q : ptrs) mix((uint64_t)(uintptr_t)q);
    const int64_t vals[] = {pl.valid, pl.RG, pl.vsize, pl.vtype, pl.ngroups, pl.n, pl.p, pl.nnz, pl.W_c, pl.T_c,
                            pl.W_r, pl.T_r, pl.u_stride, pl.csr_blocks, pl.csc_chunks, pl.threads, pl.nw,
                            pl.sent_r, pl.sent_c, (int64_t)pl.smem_c, (int64_t)pl.smem_r, pl.lm_sent_r};
    for (int64_t v : vals) mix((uint64_t)v);
    return h;
}

TiledKernels tiled_kernels(const TiledPlan &pl) {
    TiledKernels k{};
    if (pl.vtype == kVtF32) {
        k.csr = csr_ptr_rg<float>(pl.RG);
        k.u = u_ptr_rg<float>(pl.RG);
        k.csc = csc_ptr_rg<float>(pl.RG);
        k.fin1 = (void *)k_t_fin1<float>;
    } else if (pl.vtype == kVtDF) {
        k.csr = csr_ptr_rg<DF>(pl.RG);
        k.u = u_ptr_rg<DF>(pl.RG);
        k.csc = csc_ptr_rg<DF>(pl.RG);
        k.fin1 = (void *)k_t_fin1<float2>;
    } else if (pl.vtype == kVtFX) {
        k.csr = csr_ptr_rg<FX>(pl.RG);
        k.u = u_ptr_rg<FX>(pl.RG);
        k.csc = csc_ptr_rg<FX>(pl.RG);
        k.fin1 = (void *)k_t_fin1<float2>;
    } else {
        k.csr = csr_ptr_rg<double>(pl.RG);
        k.u = u_ptr_rg<double>(pl.RG);
        k.csc = csc_ptr_rg<double>(pl.RG);
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
