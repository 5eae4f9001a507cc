// divas_fuse.cu -- kernels and C ABI of the depth-weighted voxel fusion.
//
// Data layout in device memory (one context = one occupied set):
//   occ_bits[ceil(g^3/32)]     occupancy prior as a bitfield, bit lin of the grid
//   item_pref, tile_count,     the compaction's counts: per tile of 1024 words
//   tile_offset, done          its count and exclusive prefix, per item of 8
//                              words its offset inside the tile; a done counter
//   active[cap]                occupied voxels in ascending linear index, stored as
//                              packed coordinates i | j << 10 | k << 20
//   W[cap], Z[cap], bits[cap]  accumulators of Eq. vmask, structure of arrays
//   seg_bits[words]            segmentation bitfield B^seg of the last finalize
//
// Kernels: a two-launch compaction (occupancy -> bits and tile counts, the
// last CTA scanning the counts; then the entries; sparse grids scatter their
// coordinates into the bits first) builds the active list (the active-voxel
// list of Sec. 3.5 / Appendix B.1); the fusion kernel walks the active list with a
// grid-stride loop and folds up to 32 views per launch; finalize writes the
// dense score grid with 128-bit stores (or the per-active scores), the seg
// bitfield with warp-assembled words and the view masks; labels look points up
// in the seg bitfield (Eq. pass1); the adjoint recomputes every vote and
// scatters its derivatives into pixel rasters.
#include "divas_fuse.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <utility>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fuse_math.cuh"
#include "cull.cuh"

using namespace divas;

namespace {

constexpr int kThreads = 256;
constexpr int32_t kStatusBadCoord = 1;
constexpr int32_t kStatusCapacity = 2;

struct BackPtrs {
    float* gm[kMaxViews];
    float* gd[kMaxViews];
};

// ---------------------------------------------------------------------------
// compaction
// ---------------------------------------------------------------------------
// The brick-major layout: 8^3 bricks in linear brick order (x fastest), cells
// inside a brick in linear order (x fastest), so a 32-bit word is an 8 x 4
// patch of one brick slice (g a multiple of 8).

// word and bit of coordinate (i, j, k) in the linear or brick-major layout
// (at most 2^30 cells: 32-bit positions); word ~0u for a coordinate outside the
// grid (negative values wrap above g), which also sets kStatusBadCoord
template <bool kBrick>
__device__ __forceinline__ void coord_bit(int32_t si, int32_t sj, int32_t sk, uint32_t ug,
                                          int32_t* __restrict__ status, uint32_t& word,
                                          uint32_t& bit) {
    const uint32_t i = (uint32_t)si, j = (uint32_t)sj, k = (uint32_t)sk;
    word = 0xffffffffu;
    bit = 0u;
    if (i >= ug || j >= ug || k >= ug) {
        atomicOr(status, kStatusBadCoord);
        return;
    }
    const uint32_t nb = ug >> 3;
    const uint32_t lin = kBrick ? (((k >> 3) * nb + (j >> 3)) * nb + (i >> 3)) * 512u +
                                      (((k & 7u) * 8u + (j & 7u)) * 8u + (i & 7u))
                                : (k * ug + j) * ug + i;
    word = lin >> 5;
    bit = 1u << (lin & 31u);
}

// This lane's run of consecutive lanes holding the same word (from the last
// head at or below the lane to the next head): its first lane and its end
// (exclusive).  Warp-uniform call.
__device__ __forceinline__ void word_run(uint32_t word, int& first, int& end) {
    const int lane = threadIdx.x & 31;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, word, 1);
    const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || prev != word);
    first = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const uint32_t after = heads & ~(0xffffffffu >> (31 - lane));
    end = after ? __ffs(after) - 1 : 32;
}

// OR of v over lanes [lane, end) by doubling steps (after the step of offset o
// a lane holds the OR over [lane, min(lane + 2 o, end))), so a run's first lane
// gets the run's OR: shuffles with the full mask, no per-run masks.
// Warp-uniform call.
__device__ __forceinline__ uint32_t run_suffix_or(uint32_t v, int end) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + o < end) v |= y;
    }
    return v;
}

// OR of bit over this lane's run of equal words among consecutive lanes (valid
// on the run's first lane), and whether the lane is the run's first.
// Warp-uniform call.
__device__ __forceinline__ uint32_t run_or(uint32_t word, uint32_t bit, bool& first_of_run) {
    int first, end;
    word_run(word, first, end);
    first_of_run = (int)(threadIdx.x & 31) == first;
    return run_suffix_or(bit, end);
}

// sparse coordinates -> bitfield (atomic OR; duplicates merge), in linear or
// brick-major layout.  A warp takes 128 consecutive coordinates per round, 4
// per lane (three 16-byte loads when the array is 16-byte aligned); a lane's
// coordinates that fall in the same 32-bit word are OR-ed together, then the
// lanes' k-th such runs that share a word with their neighbours' (one pass per
// k), so a sorted or spatially coherent set costs about one atomic per word
// and warp round instead of one per coordinate.
template <bool kBrick>
__global__ void __launch_bounds__(kThreads) k_scatter_coords(const int32_t* __restrict__ coords,
                                                             int64_t n, int32_t g,
                                                             uint32_t* __restrict__ bits,
                                                             int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const uint32_t ug = (uint32_t)g;
    const bool vec = (reinterpret_cast<uintptr_t>(coords) & 15) == 0;
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t wb = ((int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 128; wb < n;
         wb += n_warps * 128) {
        const int64_t q0 = wb + 4 * lane;
        int32_t v[12];
        if (vec && q0 + 4 <= n) {
            const uint4* p = reinterpret_cast<const uint4*>(coords + 3 * q0);
            const uint4 a = __ldcs(p), b = __ldcs(p + 1), c = __ldcs(p + 2);
            v[0] = (int32_t)a.x; v[1] = (int32_t)a.y; v[2] = (int32_t)a.z; v[3] = (int32_t)a.w;
            v[4] = (int32_t)b.x; v[5] = (int32_t)b.y; v[6] = (int32_t)b.z; v[7] = (int32_t)b.w;
            v[8] = (int32_t)c.x; v[9] = (int32_t)c.y; v[10] = (int32_t)c.z; v[11] = (int32_t)c.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = q0 + u < n;
#pragma unroll
                for (int d = 0; d < 3; ++d) v[3 * u + d] = in ? __ldcs(coords + 3 * (q0 + u) + d) : 0;
            }
        }
        uint32_t w[4], acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint32_t bit = 0u;
            w[u] = 0xffffffffu;
            if (q0 + u < n) coord_bit<kBrick>(v[3 * u], v[3 * u + 1], v[3 * u + 2], ug, status, w[u], bit);
            acc[u] = bit | (u > 0 && w[u] == w[u > 0 ? u - 1 : 0] ? acc[u > 0 ? u - 1 : 0] : 0u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // the lane's run ends at coordinate u: its word and bits take part in pass u
            const bool ends = u == 3 || w[u] != w[u < 3 ? u + 1 : 3];
            const uint32_t word = ends ? w[u] : 0xffffffffu;
            bool first;
            const uint32_t orv = run_or(word, ends ? acc[u] : 0u, first);
            if (word != 0xffffffffu && first) atomicOr(bits + word, orv);
        }
    }
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < kThreads / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t warp_off = warp > 0 ? warp_sums[warp - 1] : 0u;
    if (total) *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

// ---------------------------------------------------------------------------
// compaction in two launches, neither of which waits on another CTA.  A group
// is 32 consecutive occupancy words (1024 cells), held one word per lane; an
// item is 8 words (256 cells); a tile is the 32 groups of one k_tile_count CTA.
//   k_tile_count  per warp 4 groups: the uint8 prior is read with fully
//                 coalesced 16-byte loads (lane l: cells 16 l .. 16 l + 15 of
//                 a 512-cell half group), turned into 16-bit halves and paired
//                 across lanes into words (dense), or the words are read
//                 (sparse); item popcounts -> each item's offset inside its
//                 tile, and the tile's count.  The CTA that finishes last
//                 (ticket of a done counter, after a fence) scans the tile
//                 counts into tile_offset, writes the total and n_active, flags
//                 overflow and rearms the counter.
//   k_tile_emit   one warp per group (grid-stride), slot = group offset + word
//                 prefix + the word's set bits below the bit.  Scattered bits
//                 (largest word popcount <= number of non-empty words): every
//                 lane walks its own word; dense words: one round per
//                 non-empty word in which lane b writes bit b (consecutive
//                 slots per store).  Packed coordinates come from the word's
//                 first cell plus the bit while the word stays on one row.
// ---------------------------------------------------------------------------
constexpr int kGroupsPerWarp = 4;
constexpr int kTileGroups = (kThreads / 32) * kGroupsPerWarp;  // 32
constexpr int kTileSpan = kTileGroups * 32;                     // words per tile
constexpr int kItemWords = 8;
constexpr int kTileItems = kTileSpan / kItemWords;              // 128

// 16 occupancy bytes -> 16 bits (bit t = byte t != 0)
__device__ __forceinline__ uint32_t bytes_nonzero16(uint4 v) {
    const uint32_t x[4] = {v.x, v.y, v.z, v.w};
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // 0x01 in every nonzero byte, then gather the four byte-LSBs into a
        // nibble with one multiply (partial products land on distinct bits)
        const uint32_t m = __vcmpne4(x[k], 0u) & 0x01010101u;
        r |= ((m * 0x01020408u) >> 24) << (4 * k);
    }
    return r;
}

// 8 occupancy bytes -> 8 bits (bit t = byte t != 0)
__device__ __forceinline__ uint32_t bytes_nonzero8(uint2 v) {
    const uint32_t x[2] = {v.x, v.y};
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const uint32_t m = __vcmpne4(x[k], 0u) & 0x01010101u;
        r |= ((m * 0x01020408u) >> 24) << (4 * k);
    }
    return r;
}

// The brick-major words of one tile (64 bricks of 8^3 cells, 1024 words) from
// the uint8 prior (g a multiple of 8): thread t reads the 8-byte row segments
// of slices 2 (t & 3) and 2 (t & 3) + 1 of brick t >> 2 (lanes 4 apart hold
// neighbouring bricks, so a load instruction covers 64 contiguous bytes of 4
// rows) and packs them into that brick's words 4 (t & 3) .. + 3, which it
// writes to the bitfield and to sw (the tile's words in shared memory); with
// score_zero, the cells' dense scores are zeroed on the way.
__device__ __forceinline__ void brick_words_from_bytes(const uint8_t* __restrict__ occ, int32_t g,
                                                       const FastDiv& bdiv, int64_t n_words,
                                                       uint32_t* __restrict__ bits,
                                                       float* __restrict__ score_zero,
                                                       uint32_t* sw) {
    const int t = threadIdx.x;
    const int64_t b = (int64_t)blockIdx.x * 64 + (t >> 2);
    const int rg = t & 3;
    uint32_t wv[4] = {0u, 0u, 0u, 0u};
    if ((b + 1) * 16 <= n_words) {
        const uint32_t r = fast_div((uint32_t)b, bdiv), bk = fast_div(r, bdiv);
        const uint32_t bi = (uint32_t)b - r * bdiv.d, bj = r - bk * bdiv.d;
        uint2 raw[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {  // slice 2 rg + (q >> 3), row q & 7
            const int64_t row = ((int64_t)(bk * 8 + 2 * rg + (q >> 3)) * g + (bj * 8 + (q & 7))) * g;
            raw[q] = __ldcs(reinterpret_cast<const uint2*>(occ + row + bi * 8));
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) wv[q >> 2] |= bytes_nonzero8(raw[q]) << (8 * (q & 3));
        if (score_zero) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int64_t row =
                    ((int64_t)(bk * 8 + 2 * rg + (q >> 3)) * g + (bj * 8 + (q & 7))) * g + bi * 8;
                __stcs(reinterpret_cast<float4*>(score_zero + row), z);
                __stcs(reinterpret_cast<float4*>(score_zero + row) + 1, z);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) bits[b * 16 + 4 * rg + k] = wv[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) sw[(t >> 2) * 16 + 4 * rg + k] = wv[k];
    __syncthreads();
}

// kMode: 0 dense prior (linear words), 1 words already in the bitfield
// (sparse, either layout), 2 dense prior into brick-major words
template <int kMode>
__global__ void __launch_bounds__(kThreads) k_tile_count(
    const uint8_t* __restrict__ occ, uint32_t* __restrict__ bits, int64_t n_cells, int64_t n_words,
    int64_t cap, uint32_t* __restrict__ item_pref, uint32_t* __restrict__ tile_count,
    uint32_t* __restrict__ tile_offset, uint32_t* __restrict__ done, int32_t n_tiles,
    int32_t* __restrict__ d_n, int64_t* __restrict__ d_total, int32_t* __restrict__ status,
    int32_t g, FastDiv bdiv, float* __restrict__ score_zero) {
    __shared__ bool s_last;
    __shared__ uint32_t sw[kMode == 2 ? kTileSpan : 1];
    allow_dependents();  // the emit may be scheduled now; it waits for this grid's end
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g0 = (int64_t)blockIdx.x * kTileGroups + warp * kGroupsPerWarp;
    uint32_t word[kGroupsPerWarp];
    if (kMode == 2) {
        brick_words_from_bytes(occ, g, bdiv, n_words, bits, score_zero, sw);
#pragma unroll
        for (int q = 0; q < kGroupsPerWarp; ++q)
            word[q] = sw[(warp * kGroupsPerWarp + q) * 32 + lane];
    } else if (kMode == 1) {
#pragma unroll
        for (int q = 0; q < kGroupsPerWarp; ++q) {
            const int64_t w = (g0 + q) * 32 + lane;
            word[q] = w < n_words ? __ldcg(bits + w) : 0u;
        }
    } else {
        const bool vec = (reinterpret_cast<uintptr_t>(occ) & 15) == 0;
        uint4 raw[2 * kGroupsPerWarp];
#pragma unroll
        for (int q = 0; q < 2 * kGroupsPerWarp; ++q) {  // all loads in flight first
            const int64_t c = (g0 * 64 + q * 32 + lane) * 16;  // first cell of this lane's 16
            raw[q] = make_uint4(0u, 0u, 0u, 0u);
            if (vec && c + 16 <= n_cells) {
                raw[q] = __ldcs(reinterpret_cast<const uint4*>(occ + c));
            } else {
                uint32_t b[4] = {0u, 0u, 0u, 0u};
                for (int t = 0; t < 16 && c + t < n_cells; ++t)
                    b[t >> 2] |= (uint32_t)occ[c + t] << (8 * (t & 3));
                raw[q] = make_uint4(b[0], b[1], b[2], b[3]);
            }
        }
#pragma unroll
        for (int q = 0; q < kGroupsPerWarp; ++q) {
            // half group 2q covers words 0..15 of group q, half 2q + 1 words 16..31;
            // word m of a half = lanes 2m (low bits) and 2m + 1 (high bits)
            const uint32_t h0 = bytes_nonzero16(raw[2 * q]);
            const uint32_t h1 = bytes_nonzero16(raw[2 * q + 1]);
            const int src = 2 * (lane & 15);
            const uint32_t a0 = __shfl_sync(0xffffffffu, h0, src);
            const uint32_t b0 = __shfl_sync(0xffffffffu, h0, src + 1);
            const uint32_t a1 = __shfl_sync(0xffffffffu, h1, src);
            const uint32_t b1 = __shfl_sync(0xffffffffu, h1, src + 1);
            word[q] = lane < 16 ? (a0 | (b0 << 16)) : (a1 | (b1 << 16));
            const int64_t w = (g0 + q) * 32 + lane;
            if (w < n_words) bits[w] = word[q];
        }
    }
    // item counts (8 lanes each) -> the warp's 16 item counts, in item order
    uint32_t ic[kGroupsPerWarp], wsum = 0;
#pragma unroll
    for (int q = 0; q < kGroupsPerWarp; ++q) {
        uint32_t v = __popc(word[q]);
#pragma unroll
        for (int o = 1; o < kItemWords; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        ic[q] = v;  // the count of item (lane / 8) of group q, on every lane of that item
        wsum += __shfl_sync(0xffffffffu, v, 0) + __shfl_sync(0xffffffffu, v, 8) +
                __shfl_sync(0xffffffffu, v, 16) + __shfl_sync(0xffffffffu, v, 24);
    }
    uint32_t total;
    const uint32_t wex = block_exclusive_scan(lane == 0 ? wsum : 0u, &total);
    const uint32_t wbase = __shfl_sync(0xffffffffu, wex, 0);
    // lane 8 j + 0 writes item j of group q; prefix = wbase + items before it
    {
        uint32_t run = wbase;
#pragma unroll
        for (int q = 0; q < kGroupsPerWarp; ++q) {
            const uint32_t c0 = __shfl_sync(0xffffffffu, ic[q], 0);
            const uint32_t c1 = __shfl_sync(0xffffffffu, ic[q], 8);
            const uint32_t c2 = __shfl_sync(0xffffffffu, ic[q], 16);
            const uint32_t c3 = __shfl_sync(0xffffffffu, ic[q], 24);
            const int j = lane >> 3;
            const uint32_t before = (j > 0 ? c0 : 0u) + (j > 1 ? c1 : 0u) + (j > 2 ? c2 : 0u);
            if ((lane & 7) == 0) item_pref[(g0 + q) * (32 / kItemWords) + j] = run + before;
            run += c0 + c1 + c2 + c3;
        }
    }
    if (threadIdx.x == 0) {
        tile_count[blockIdx.x] = total;
        __threadfence();
        s_last = atomicAdd(done, 1u) == (uint32_t)(n_tiles - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // the last CTA: every tile count is visible (each was fenced before its ticket)
    __threadfence();
    const int32_t per = (n_tiles + kThreads - 1) / kThreads;
    const int32_t beg = min(n_tiles, (int32_t)threadIdx.x * per), end = min(n_tiles, beg + per);
    uint32_t run = 0;
    for (int32_t i = beg; i < end; ++i) run += __ldcg(tile_count + i);
    uint32_t all;
    uint32_t ex = block_exclusive_scan(run, &all);
    for (int32_t i = beg; i < end; ++i) {
        const uint32_t v = __ldcg(tile_count + i);
        tile_offset[i] = ex;
        ex += v;
    }
    if (threadIdx.x == 0) {
        *d_total = (int64_t)all;
        *d_n = (int32_t)((int64_t)all < cap ? (int64_t)all : cap);
        if ((int64_t)all > cap) atomicOr(status, kStatusCapacity);
        *done = 0u;  // rearmed for the next launch
    }
}

// packed coordinates i | j << 10 | k << 20 of linear cell lin
__device__ __forceinline__ uint32_t pack_lin(uint32_t lin, const FastDiv& gdiv) {
    const uint32_t r = fast_div(lin, gdiv);
    const uint32_t k = fast_div(r, gdiv);
    return (lin - r * gdiv.d) | ((r - k * gdiv.d) << 10) | (k << 20);
}

// The active-list entries of one group of 32 occupancy words (lane = word
// x of cell word w, the group g): slot = base + the word prefix + the word's
// set bits below the bit.  Scattered bits (largest word popcount <= number of
// non-empty words): every lane walks its own word; dense words: one round per
// non-empty word in which lane b writes bit b (consecutive slots per store).
// Packed coordinates come from the word's first cell plus the bit while the
// word stays on one row.  Warp-uniform: every lane of the warp calls it.
//
// Brick-major layout (kBrick; div divides by the bricks per side): word w is
// rows 4 (w & 1) .. + 3 of slice (w & 15) >> 1 of brick w >> 4, bit b the
// cell (b & 7, b >> 3) of that patch.
__device__ __forceinline__ uint32_t brick_word_p0(uint32_t w, const FastDiv& bdiv) {
    const uint32_t b = w >> 4, sl = w & 15u;
    const uint32_t r = fast_div(b, bdiv), bk = fast_div(r, bdiv);
    const uint32_t bi = b - r * bdiv.d, bj = r - bk * bdiv.d;
    return (bi << 3) | (((bj << 3) + ((sl & 1u) << 2)) << 10) | (((bk << 3) + (sl >> 1)) << 20);
}

// position of set bit number k of a byte (0 past its last set bit), for every
// byte and k < 8: entry 8 byte + k (built at compile time)
struct NthBitTable {
    uint8_t v[256 * 8];
};
constexpr NthBitTable make_nth_bit_table() {
    NthBitTable t{};
    for (int byte = 0; byte < 256; ++byte) {
        int seen = 0;
        for (int b = 0; b < 8; ++b)
            if ((byte >> b) & 1) t.v[8 * byte + seen++] = (uint8_t)b;
    }
    return t;
}
__device__ const NthBitTable kNthBit = make_nth_bit_table();

// position of set bit number n (from 0) of v, for n < popc(v); always in [0, 31]:
// the byte that holds it by two popcount halvings, the bit inside that byte
// from the table (a 2 KB global array, read through the L1 cache)
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t v, uint32_t n) {
    uint32_t sh = 0;
    const uint32_t lo16 = __popc(v & 0xffffu);
    if (n >= lo16) {
        n -= lo16;
        sh = 16;
    }
    const uint32_t lo8 = __popc((v >> sh) & 0xffu);
    if (n >= lo8) {
        n -= lo8;
        sh += 8;
    }
    return sh + __ldg(&kNthBit.v[(((v >> sh) & 0xffu) << 3) | (n & 7u)]);
}

template <bool kBrick>
__device__ __forceinline__ void emit_group(uint32_t x, int64_t w, int64_t g, int64_t base,
                                           int64_t cap, const FastDiv& gdiv,
                                           uint32_t* __restrict__ active) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t nz = __ballot_sync(0xffffffffu, x != 0u);
    if (nz == 0u) return;  // warp-uniform
    const uint32_t c = __popc(x);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t ex = inc - c;
    // this lane's word, bit 0
    const uint32_t p0 = kBrick ? brick_word_p0((uint32_t)w, gdiv) : pack_lin((uint32_t)(w * 32), gdiv);
    if (kBrick) {
        // brick words: rounds of 32 consecutive slots (coalesced stores, at most
        // as many rounds as non-empty words); slot s belongs to the last lane o
        // whose prefix ex_o <= s (its word holds it: ex_o + c_o > s) and is bit
        // number s - ex_o of that word
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        for (uint32_t s0 = 0; s0 < total; s0 += 32) {
            const uint32_t sl = s0 + lane;
            int o = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                if (__shfl_sync(0xffffffffu, ex, o + step) <= sl) o += step;
            const uint32_t xo = __shfl_sync(0xffffffffu, x, o);
            const uint32_t eo = __shfl_sync(0xffffffffu, ex, o);
            const uint32_t po = __shfl_sync(0xffffffffu, p0, o);
            const uint32_t b = nth_set_bit(xo, sl - eo);
            if (sl < total && base + sl < cap)
                active[base + sl] = po + (b & 7u) + ((b >> 3) << 10);
        }
        return;
    }
    const uint32_t max_c = __reduce_max_sync(0xffffffffu, c);
    if (max_c <= (uint32_t)__popc(nz)) {
        // scattered bits: every lane walks its own word (rounds = the largest popcount)
        uint32_t xb = x;
        int64_t slot = base + ex;
        const bool row = (p0 & 1023u) + 31u < gdiv.d;  // the word stays on one row
        while (xb) {
            const uint32_t b = __ffs(xb) - 1;
            xb &= xb - 1u;
            if (slot < cap)
                active[slot] = kBrick ? p0 + (b & 7u) + ((b >> 3) << 10)
                                      : (row ? p0 + b : pack_lin((uint32_t)(w * 32) + b, gdiv));
            ++slot;
        }
        return;
    }
    // dense words: one round per non-empty word, in which lane b writes bit b
    while (nz) {
        const int src = __ffs(nz) - 1;
        nz &= nz - 1u;
        const uint32_t xs = __shfl_sync(0xffffffffu, x, src);
        const uint32_t off = __shfl_sync(0xffffffffu, ex, src);
        const uint32_t ps = __shfl_sync(0xffffffffu, p0, src);
        if ((xs >> lane) & 1u) {
            const int64_t slot = base + off + __popc(xs & lt);
            if (slot < cap) {
                // same row as the word's bit 0 unless the row wraps inside the word
                active[slot] = kBrick ? ps + (lane & 7) + ((uint32_t)(lane >> 3) << 10)
                               : (ps & 1023u) + lane < gdiv.d
                                   ? ps + lane
                                   : pack_lin((uint32_t)((g * 32 + src) * 32 + lane), gdiv);
            }
        }
    }
}

// seg_zero / seg_zero2 (nullable): seg bitfields whose words are cleared on
// the way (the one-call step)
template <bool kBrick>
__global__ void __launch_bounds__(kThreads) k_tile_emit(
    const uint32_t* __restrict__ bits, int64_t n_words, int64_t cap, FastDiv gdiv,
    const uint32_t* __restrict__ item_pref, const uint32_t* __restrict__ tile_offset,
    uint32_t* __restrict__ active, uint32_t* __restrict__ seg_zero,
    uint32_t* __restrict__ seg_zero2) {
    wait_for_producer();  // the counts and prefixes of k_tile_count
    allow_dependents();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_groups = (n_words + 31) / 32;
    const int64_t n_warps = (int64_t)gridDim.x * (kThreads / 32);
    // the group's slot base and words (one round trip), loaded for the next
    // group of this warp while the current one is emitted
    auto fetch = [&](int64_t g, uint32_t& base, uint32_t& x) {
        base = 0u;
        x = 0u;
        if (g >= n_groups) return;
        const int64_t w = g * 32 + lane;
        base = __ldg(tile_offset + g / kTileGroups) + __ldg(item_pref + g * (32 / kItemWords));
        if (w < n_words) x = __ldcg(bits + w);
    };
    int64_t g = (int64_t)blockIdx.x * (kThreads / 32) + warp;
    uint32_t base, x;
    fetch(g, base, x);
    while (g < n_groups) {
        const int64_t gn = g + n_warps;
        uint32_t base_n, x_n;
        fetch(gn, base_n, x_n);
        const int64_t w = g * 32 + lane;
        if (w < n_words) {
            if (seg_zero) seg_zero[w] = 0u;
            if (seg_zero2) seg_zero2[w] = 0u;
        }
        emit_group<kBrick>(x, w, g, (int64_t)base, cap, gdiv, active);
        g = gn;
        base = base_n;
        x = x_n;
    }
}

// ---------------------------------------------------------------------------
// fusion
// ---------------------------------------------------------------------------
template <bool kAccumulate, bool kContracted, int kChunks>
__global__ void __launch_bounds__(kThreads) k_fuse(const uint32_t* __restrict__ active,
                                                   const int32_t* __restrict__ d_n, GridC G,
                                                   FuseC F, const __grid_constant__ ViewBatch VB,
                                                   float* __restrict__ W,
                                                   float* __restrict__ Z,
                                                   uint32_t* __restrict__ bits) {
    const int32_t n = *d_n;
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const VoxelGeom vg = voxel_geom<kContracted>(__ldg(active + a), G, F.gamma);
        float w = 0.f, z = 0.f;
        uint32_t b = 0;
        if (kAccumulate) {
            w = W[a];
            z = Z[a];
            b = bits[a];
        }
        if (vg.ok) fold_views<kContracted, kChunks>(VB, vg, F, w, z, b);
        W[a] = w;
        Z[a] = z;
        bits[a] = b;
    }
}

// launch k_fuse with the chunk count as a compile-time constant
template <bool kAccumulate, bool kContracted, int kChunks = 1>
cudaError_t launch_fuse_chunks(int chunks, int blocks, cudaStream_t s, const uint32_t* active,
                               const int32_t* d_n, const GridC& G, const FuseC& F,
                               const ViewBatch& vb, float* W, float* Z, uint32_t* bits) {
    if constexpr (kChunks < kMaxViews / kViewChunk) {
        if (chunks > kChunks)
            return launch_fuse_chunks<kAccumulate, kContracted, kChunks + 1>(
                chunks, blocks, s, active, d_n, G, F, vb, W, Z, bits);
    }
    k_fuse<kAccumulate, kContracted, kChunks><<<blocks, kThreads, 0, s>>>(active, d_n, G, F, vb,
                                                                          W, Z, bits);
    return cudaGetLastError();
}

// zeros of a dense score grid's unoccupied cells for the groups of 32
// occupancy words (1024 cells) g = gw, gw + nw, ...: one coalesced pass of
// 16-byte stores per group and warp (x_first: the first group's word, already
// loaded by this lane, or ~0u to load it here)
__device__ __forceinline__ void zero_unoccupied_groups(const uint32_t* __restrict__ occ_bits,
                                                       int64_t n_words, int64_t n_cells,
                                                       float* __restrict__ score_out, int64_t gw,
                                                       int64_t nw, uint32_t x_first,
                                                       bool have_first) {
    const int lane = threadIdx.x & 31;
    const int64_t n_groups = (n_words + 31) / 32;
    const bool vec = (reinterpret_cast<uintptr_t>(score_out) & 15) == 0;
    for (int64_t g = gw; g < n_groups; g += nw) {
        const int64_t w = g * 32 + lane;
        const uint32_t x = (g == gw && have_first) ? x_first
                                                   : (w < n_words ? __ldg(occ_bits + w) : 0u);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int f4 = q * 32 + lane;  // float4 index inside the group
            const uint32_t xw = __shfl_sync(0xffffffffu, x, f4 >> 3);
            const uint32_t nib = (xw >> ((f4 & 7) * 4)) & 0xfu;
            const int64_t cell = g * 1024 + 4 * f4;
            if (nib == 0u && vec && cell + 4 <= n_cells) {
                __stcs(reinterpret_cast<float4*>(score_out + cell), make_float4(0.f, 0.f, 0.f, 0.f));
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (!((nib >> k) & 1u) && cell + k < n_cells) score_out[cell + k] = 0.f;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// finalize
// ---------------------------------------------------------------------------
// seg bits of one warp's 32 voxels (active slots base .. base + 31): runs of
// consecutive lanes that share a 32-bit word (the active list is ascending, so
// a word's voxels are one run) are grouped, their set bits OR-ed in and -- for
// a bitfield that may hold an earlier seg of the same voxels -- their unset
// bits AND-ed out, one atomic per run and bitfield.  Every bit belongs to
// exactly one voxel, so the result does not depend on the order of the
// atomics (nor on a word's voxels forming one run).
__device__ __forceinline__ void seg_epilogue(bool live, bool seg, int64_t lin,
                                             uint32_t* __restrict__ seg_bits, bool clear_bits,
                                             uint32_t* __restrict__ seg_out, bool clear_out) {
    const int lane = threadIdx.x & 31;
    const uint32_t word = live ? (uint32_t)(lin >> 5) : 0xffffffffu;
    const uint32_t bit = live ? 1u << (lin & 31) : 0u;
    const bool clearing = clear_bits || (seg_out && clear_out);  // warp-uniform
    if (!clearing) {  // only bits to set: one atomic per seg voxel, no run merging
        if (live && seg) {
            atomicOr(seg_bits + word, bit);
            if (seg_out) atomicOr(seg_out + word, bit);
        }
        return;
    }
    int first, end;
    word_run(word, first, end);
    const uint32_t set = run_suffix_or(seg ? bit : 0u, end);
    const uint32_t clr = run_suffix_or(seg ? 0u : bit, end);
    if (!live || lane != first) return;
    if (set) atomicOr(seg_bits + word, set);
    if (clr && clear_bits) atomicAnd(seg_bits + word, ~clr);
    if (seg_out) {
        if (set) atomicOr(seg_out + word, set);
        if (clr && clear_out) atomicAnd(seg_out + word, ~clr);
    }
}

// normalise + threshold, one thread per active voxel: P = W / Z, seg = P >=
// tau_cons; the score goes to its dense or active-list position (the caller
// zeroed a dense grid's other cells).  The context's seg bitfield holds no bit
// of an unoccupied voxel (set_occupancy clears it), so its bits are set and
// cleared in place; seg_out (zeroed by the caller) only gets its set bits.
__global__ void __launch_bounds__(kThreads) k_finalize(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, int32_t g,
    int32_t dense, const float* __restrict__ W, const float* __restrict__ Z,
    const uint32_t* __restrict__ bits, float eps, float tau_cons, float* __restrict__ score_out,
    uint32_t* __restrict__ seg_bits, uint32_t* __restrict__ seg_out,
    uint32_t* __restrict__ vmask_out, unsigned long long* __restrict__ d_nseg) {
    const int32_t n = *d_n;
    const int lane = threadIdx.x & 31;
    const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
    for (int32_t base = gw * 32; base < n; base += nw * 32) {
        const int32_t a = base + lane;
        const bool live = a < n;
        bool seg = false;
        int64_t lin = 0;
        if (live) {
            const float w = __ldcs(W + a), z = __ldcs(Z + a);
            const float p = z > eps ? __fdiv_rn(w, z) : 0.f;
            seg = p >= tau_cons;
            lin = packed_lin(__ldg(active + a), g);
            if (score_out) score_out[dense ? lin : (int64_t)a] = p;
            if (vmask_out) vmask_out[a] = seg ? bits[a] : 0u;
        }
        seg_epilogue(live, seg, lin, seg_bits, true, seg_out, false);
        if (d_nseg) {
            const uint32_t cnt = __popc(__ballot_sync(0xffffffffu, seg));
            if (lane == 0 && cnt) atomicAdd(d_nseg, (unsigned long long)cnt);
        }
    }
}

// ---------------------------------------------------------------------------
// fusion + finalize in one pass (the one-call step and the incremental
// update): fold the batch's views (into fresh accumulators, or onto the
// stored ones with kAccumulate), store W, Z, bits, then P = W / Z, seg =
// P >= tau_cons, the score to its dense or active-list position and the seg
// bits (seg_epilogue; clear_bits / clear_out when the bitfield may hold an
// earlier seg of these voxels); with zero_unoccupied, a dense score grid then
// gets the zeros of its unoccupied cells.  Per voxel the arithmetic is that of
// k_fuse followed by k_finalize.
// ---------------------------------------------------------------------------
template <bool kAccumulate, bool kContracted, int kChunks, bool kF16Full = false>
__global__ void __launch_bounds__(kThreads, kContracted ? 5 : 6) k_fuse_fin(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, GridC G, FuseC F,
    const __grid_constant__ ViewBatch VB, float* __restrict__ W, float* __restrict__ Z,
    uint32_t* __restrict__ bits, int32_t dense, float* __restrict__ score_out,
    uint32_t* __restrict__ seg_bits, int32_t clear_bits, uint32_t* __restrict__ seg_out,
    int32_t clear_out, const uint32_t* __restrict__ occ_bits, int64_t n_words, int64_t n_cells,
    int32_t zero_unoccupied) {
    wait_for_producer();  // the active list and its length
    const int lane = threadIdx.x & 31;
    const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
    const int64_t n_groups = (n_words + 31) / 32;
    // occupancy word of the first group this warp zero-fills, fetched now and
    // used after the fusion loop
    uint32_t x_first = 0;
    if (zero_unoccupied && gw < n_groups && (int64_t)gw * 32 + lane < n_words)
        x_first = __ldg(occ_bits + (int64_t)gw * 32 + lane);
    const int32_t n = *d_n;
    for (int32_t base = gw * 32; base < n; base += nw * 32) {
        const int32_t a = base + lane;
        const bool live = a < n;
        bool seg = false;
        int64_t lin = 0;
        if (live) {
            const uint32_t pk = __ldg(active + a);
            const VoxelGeom vg = voxel_geom<kContracted>(pk, G, F.gamma);
            float w = 0.f, z = 0.f;
            uint32_t b = 0;
            if (kAccumulate) {
                w = W[a];
                z = Z[a];
                b = bits[a];
            }
            if (vg.ok) fold_views<kContracted, kChunks, kF16Full>(VB, vg, F, w, z, b);
            W[a] = w;
            Z[a] = z;
            bits[a] = b;
            const float p = z > F.eps ? __fdiv_rn(w, z) : 0.f;
            seg = p >= F.tau_cons;
            lin = packed_lin(pk, G.g);
            if (score_out) score_out[dense ? lin : (int64_t)a] = p;
        }
        seg_epilogue(live, seg, lin, seg_bits, clear_bits != 0, seg_out, clear_out != 0);
    }
    if (zero_unoccupied)
        zero_unoccupied_groups(occ_bits, n_words, n_cells, score_out, gw, nw, x_first, true);
}

// ---------------------------------------------------------------------------
// fusion + finalize with warp-level view culling (brick-ordered active lists):
// per warp of 32 voxels, the views that no brick of the warp's voxels may vote
// in (k_brick_views) are skipped; the kept views are folded in view order with
// the arithmetic of k_fuse_fin, so every result is bitwise that of k_fuse_fin.
// kMT: the batch's mask type when all views carry binary16 masks, else -1.
// ---------------------------------------------------------------------------
template <bool kAccumulate, bool kContracted, int kMT>
__global__ void __launch_bounds__(kThreads, kContracted ? 5 : 6) k_fuse_fin_cull(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, GridC G, FuseC F,
    const ViewC* __restrict__ views, int32_t n_views, const uint32_t* __restrict__ brick_keep,
    float* __restrict__ W, float* __restrict__ Z, uint32_t* __restrict__ bits, int32_t dense,
    float* __restrict__ score_out, int32_t score_zeroed, uint32_t* __restrict__ seg_bits,
    int32_t clear_bits, uint32_t* __restrict__ seg_out, int32_t clear_out) {
    __shared__ __align__(16) ViewC sv[kMaxViews];
    wait_for_producer();  // the active list, its length, the views and the bricks' kept views
    {  // the batch's view constants into shared memory (16-byte words)
        const uint4* src = reinterpret_cast<const uint4*>(views);
        uint4* dst = reinterpret_cast<uint4*>(sv);
        for (int k = threadIdx.x; k < n_views * (int)(sizeof(ViewC) / 16); k += blockDim.x)
            dst[k] = __ldg(src + k);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
    const int32_t n = *d_n;
    const uint32_t nb = (uint32_t)G.g >> 3;
    for (int32_t base = gw * 32; base < n; base += nw * 32) {
        const int32_t a = base + lane;
        const bool live = a < n;
        const uint32_t pk = live ? __ldg(active + a) : 0u;
        const uint32_t bk_index =
            (((pk >> 23) * nb + ((pk >> 13) & 127u)) * nb + ((pk & 1023u) >> 3));
        const uint32_t mine = live ? __ldg(brick_keep + bk_index) : 0u;
        // only the batch's views, whatever the masks hold
        const uint32_t keep = __reduce_or_sync(0xffffffffu, mine) &
                              (n_views >= 32 ? 0xffffffffu : (1u << n_views) - 1u);
        if (!kAccumulate && keep == 0u && !clear_bits) {
            // no view can vote for any voxel of the warp: zero accumulators and
            // P = 0 (a zeroed score grid holds it already), no seg bit to set or
            // clear
            if (live) {
                W[a] = 0.f;
                Z[a] = 0.f;
                bits[a] = 0u;
                if (score_out && !score_zeroed)
                    score_out[dense ? packed_lin(pk, G.g) : (int64_t)a] = 0.f;
            }
            continue;
        }
        const VoxelGeom vg = voxel_geom<kContracted>(pk, G, F.gamma);
        bool seg = false;
        int64_t lin = 0;
        if (live) {
            float w = 0.f, z = 0.f;
            uint32_t b = 0;
            if (kAccumulate) {
                w = W[a];
                z = Z[a];
                b = bits[a];
            }
            if (vg.ok) fold_views_kept<kContracted, kMT>(sv, keep, vg, F, w, z, b);
            W[a] = w;
            Z[a] = z;
            bits[a] = b;
            const float p = z > F.eps ? __fdiv_rn(w, z) : 0.f;
            seg = p >= F.tau_cons;
            lin = packed_lin(pk, G.g);
            // a zeroed score grid keeps its +0 where P = +0
            if (score_out && !(score_zeroed && __float_as_uint(p) == 0u))
                score_out[dense ? lin : (int64_t)a] = p;
        }
        seg_epilogue(live, seg, lin, seg_bits, clear_bits != 0, seg_out, clear_out != 0);
    }
}

// ---------------------------------------------------------------------------
// labels (Eq. pass1)
// ---------------------------------------------------------------------------
// floor of hi + lo (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ float floor_df(float hi, float lo) {
    const float f = floorf(hi);
    return (f == hi && lo < 0.f) ? f - 1.f : f;
}

// label of one point (x, y, z) against a seg bitfield
// the cell idx of point a (exact floor of (x - origin) / h, through the
// contraction for contracted grids); false outside the grid or for NaN
__device__ __forceinline__ bool point_cell(const float* __restrict__ xyz, int64_t a, const GridC& G,
                                           int32_t (&idx)[3]) {
    float xh[3] = {xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
    float xl[3] = {0.f, 0.f, 0.f};
    bool inside = false;
    if (!(isnan(xh[0]) || isnan(xh[1]) || isnan(xh[2]))) {
        if (G.contracted) {
            // r^2 = |x|^2 as hi + lo
            float s = 0.f, e = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float p, pe, t;
                two_prod(xh[q], xh[q], p, pe);
                two_sum(s, p, s, t);
                e = __fadd_rn(e, __fadd_rn(t, pe));
            }
            float n2h, n2l;
            two_sum(s, e, n2h, n2l);
            if ((n2h > 1.f) || (n2h == 1.f && n2l > 0.f)) {
                if (n2h > 1e30f) {  // |x| beyond 1e15: contract(x) = 2 x / |x| in FP32
                    const float inv = __frsqrt_rn(n2h);
                    // not reached by finite scenes; keeps the arithmetic finite
#pragma unroll
                    for (int q = 0; q < 3; ++q) { xh[q] = 2.f * xh[q] * inv; xl[q] = 0.f; }
                } else {
                    const float rh = __fsqrt_rn(n2h);
                    const float rl =
                        __fdiv_rn(__fadd_rn(__fmaf_rn(-rh, rh, n2h), n2l), __fmul_rn(2.f, rh));
                    // ir = 1 / r
                    const float ih = __frcp_rn(rh);
                    const float il = __fmul_rn(
                        ih, __fsub_rn(__fmaf_rn(-ih, rh, 1.f), __fmul_rn(ih, rl)));
                    // tt = 2 - ir
                    float th, tl;
                    two_sum(2.f, -ih, th, tl);
                    tl = __fsub_rn(tl, il);
                    two_sum(th, tl, th, tl);
                    // sc = tt * ir
                    float sh, sl;
                    two_prod(th, ih, sh, sl);
                    sl = __fadd_rn(sl, __fadd_rn(__fmul_rn(th, il), __fmul_rn(tl, ih)));
                    two_sum(sh, sl, sh, sl);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        float qh, ql;
                        two_prod(xh[q], sh, qh, ql);
                        ql = __fadd_rn(ql, __fmul_rn(xh[q], sl));
                        two_sum(qh, ql, xh[q], xl[q]);
                    }
                }
            }
        }
        inside = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            // s = (x - origin) / h as hi + lo
            float dh, dl;
            two_sum(xh[q], -G.origin[q], dh, dl);
            dl = __fadd_rn(dl, xl[q]);
            float sh, sl;
            if (G.inv_h != 0.f) {  // power-of-two edge: scaling is exact
                sh = __fmul_rn(dh, G.inv_h);
                sl = __fmul_rn(dl, G.inv_h);
            } else {
                sh = __fdiv_rn(dh, G.h);
                sl = __fdiv_rn(__fadd_rn(__fmaf_rn(-sh, G.h, dh), dl), G.h);
            }
            const float f = floor_df(sh, sl);
            if (!(f >= 0.f && f < (float)G.g)) inside = false;
            idx[q] = inside ? (int32_t)f : 0;
        }
    }
    return inside;
}

__device__ __forceinline__ uint8_t label_one(const float* __restrict__ xyz, int64_t a,
                                             const GridC& G,
                                             const uint32_t* __restrict__ seg_bits) {
    int32_t idx[3];
    if (!point_cell(xyz, a, G, idx)) return 0;
    const int64_t lin = ((int64_t)idx[2] * G.g + idx[1]) * G.g + idx[0];
    return (uint8_t)((__ldg(seg_bits + (lin >> 5)) >> (lin & 31)) & 1u);
}

// label of one point of a plain grid whose edge h is a power of two (G.inv_h
// != 0): s = fl(x - o) / h is exact scaling of the rounded difference, and
// rounding to nearest never crosses the representable k h, so floor(s) is the
// exact floor unless s is an integer -- only then is the rounding error of the
// difference (two_sum) needed to decide (the compensated path of label_one)
__device__ __forceinline__ uint8_t label_plain_pow2(float x, float y, float z, const GridC& G,
                                                   const uint32_t* __restrict__ seg_bits) {
    const float p[3] = {x, y, z};
    uint32_t idx[3];
    bool inside = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float dh = __fsub_rn(p[q], G.origin[q]);
        const float sh = __fmul_rn(dh, G.inv_h);
        float f = floorf(sh);
        if (f == sh) {  // on a cell boundary: the sign of the rounding error decides
            float h2, l2;
            two_sum(p[q], -G.origin[q], h2, l2);
            if (l2 < 0.f) f = __fsub_rn(f, 1.f);
        }
        inside = inside && f >= 0.f && f < (float)G.g;  // false for NaN
        idx[q] = inside ? (uint32_t)f : 0u;
    }
    if (!inside) return 0;
    const uint32_t g = (uint32_t)G.g;
    const uint32_t lin = (idx[2] * g + idx[1]) * g + idx[0];  // < 2^30
    return (uint8_t)((__ldg(seg_bits + (lin >> 5)) >> (lin & 31)) & 1u);
}

// four points per thread: their 48 bytes come in three 128-bit loads (when the
// array is 16-byte aligned) so that every thread has all its loads in flight
template <bool kPlainPow2>
__global__ void __launch_bounds__(kThreads) k_label(const float* __restrict__ xyz, int64_t n,
                                                    GridC G, const uint32_t* __restrict__ seg_bits,
                                                    uint8_t* __restrict__ labels) {
    wait_for_producer();  // the seg bitfield of the fusion
    const bool vec = (reinterpret_cast<uintptr_t>(xyz) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(labels) & 3) == 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 4 * q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = 4 * q;
        if (vec && a + 4 <= n) {
            const float4* p4 = reinterpret_cast<const float4*>(xyz + 3 * a);
            const float4 f0 = __ldcs(p4), f1 = __ldcs(p4 + 1), f2 = __ldcs(p4 + 2);
            const float pts[12] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y,
                                   f1.z, f1.w, f2.x, f2.y, f2.z, f2.w};
            uint32_t packed = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint8_t lab =
                    kPlainPow2 ? label_plain_pow2(pts[3 * k], pts[3 * k + 1], pts[3 * k + 2], G,
                                                  seg_bits)
                               : label_one(pts + 3 * k, 0, G, seg_bits);
                packed |= (uint32_t)lab << (8 * k);
            }
            *reinterpret_cast<uint32_t*>(labels + a) = packed;
        } else {
            for (int64_t b = a; b < a + 4 && b < n; ++b)
                labels[b] = kPlainPow2 ? label_plain_pow2(xyz[3 * b], xyz[3 * b + 1],
                                                          xyz[3 * b + 2], G, seg_bits)
                                       : label_one(xyz, b, G, seg_bits);
        }
    }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
template <bool kContracted, int kChunks>
__global__ void __launch_bounds__(kThreads) k_backward(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, GridC G, FuseC F,
    const __grid_constant__ ViewBatch VB, const __grid_constant__ BackPtrs BP,
    const float* __restrict__ W, const float* __restrict__ Z,
    const float* __restrict__ grad_score, int32_t dense) {
    const int32_t n = *d_n;
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const uint32_t pk = __ldg(active + a);
        const float gP = __ldg(grad_score + (dense ? packed_lin(pk, G.g) : (int64_t)a));
        const float z = Z[a];
        if (gP == 0.f || !(z > F.eps)) continue;
        const float P = __fdiv_rn(W[a], z);
        const VoxelGeom vg = voxel_geom<kContracted>(pk, G, F.gamma);
        if (!vg.ok) continue;
        const float gz = __fdiv_rn(gP, z);
        const float k2 = __fmul_rn(__fmul_rn(2.f, F.alpha1), __fmul_rn(vg.invDelta, vg.invDelta));
#pragma unroll
        for (int v = 0; v < kChunks * kViewChunk; ++v) {
            if (v >= VB.n) break;
            Vote vt;
            if (!eval_vote<kContracted>(VB.v[v], vg, F, vt)) continue;
            if (BP.gm[v]) {
                float dm = __fmul_rn(gz, vt.w);
                if (VB.v[v].mask_type == kMaskLogit)
                    dm = __fmul_rn(dm, __fmul_rn(vt.m, __fsub_rn(1.f, vt.m)));
                atomicAdd(BP.gm[v] + vt.pix, dm);
            }
            if (BP.gd[v]) {
                const float dw = __fmul_rn(__fmul_rn(vt.w, k2), vt.e);
                atomicAdd(BP.gd[v] + vt.pix, __fmul_rn(__fmul_rn(gz, __fsub_rn(vt.m, P)), dw));
            }
        }
    }
}

template <bool kContracted, int kChunks = 1>
cudaError_t launch_backward_chunks(int chunks, int blocks, cudaStream_t s, const uint32_t* active,
                                   const int32_t* d_n, const GridC& G, const FuseC& F,
                                   const ViewBatch& vb, const BackPtrs& bp, const float* W,
                                   const float* Z, const float* grad_score, int32_t dense) {
    if constexpr (kChunks < kMaxViews / kViewChunk) {
        if (chunks > kChunks)
            return launch_backward_chunks<kContracted, kChunks + 1>(
                chunks, blocks, s, active, d_n, G, F, vb, bp, W, Z, grad_score, dense);
    }
    k_backward<kContracted, kChunks><<<blocks, kThreads, 0, s>>>(active, d_n, G, F, vb, bp, W, Z,
                                                                 grad_score, dense);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// misc
// ---------------------------------------------------------------------------
template <bool kContracted>
__global__ void k_debug_project(const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n,
                                GridC G, FuseC F, ViewC V, int32_t* __restrict__ pix_out) {
    const int32_t n = *d_n;
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const VoxelGeom vg = voxel_geom<kContracted>(__ldg(active + a), G, F.gamma);
        float ph, pl;
        pix_out[a] = vg.ok ? project<kContracted>(V, vg, F.z_near, ph, pl) : -1;
    }
}

__global__ void k_debug_rcp(const float* __restrict__ x, int64_t n, float* __restrict__ nr,
                            float* __restrict__ ieee) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        nr[a] = rcp_nr(x[a]);
        ieee[a] = __frcp_rn(x[a]);
    }
}

__global__ void k_active_coords(const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n,
                                int32_t g, int32_t* __restrict__ out) {
    const int32_t n = *d_n;
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        int32_t i, j, k;
        unpack(active[a], i, j, k);
        out[3 * a] = i;
        out[3 * a + 1] = j;
        out[3 * a + 2] = k;
    }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
struct divas_ctx {
    divas_grid grid;
    divas_params params;
    GridC G;
    FuseC F;
    int64_t n_cells = 0, n_words = 0;
    int64_t cap = 0;
    int64_t n_active = 0;
    int32_t n_views = 0;
    int32_t sm_count = 148;
    uint32_t* occ_bits = nullptr;
    uint32_t* item_pref = nullptr;    // compaction: item offsets inside their tile
    uint32_t* tile_count = nullptr;   // compaction: active voxels per tile of 1024 words
    uint32_t* tile_offset = nullptr;  // exclusive prefix of tile_count
    uint32_t* done = nullptr;         // k_tile_count's done counter (rearmed by its last CTA)
    int32_t n_tiles = 0;
    uint32_t* seg_bits = nullptr;
    uint32_t* active = nullptr;
    FastDiv gdiv;  // division by g
    bool brick = false;  // DIVAS_ORDER_BRICKS: brick-major bitfield and active list
    FastDiv bdiv;        // division by g / 8 (brick order)
    float* pyr = nullptr;  // brick order: mask max pyramids of a view batch
    int64_t pyr_cap = 0;   // its capacity in floats
    uint32_t* brick_keep = nullptr;  // brick order: per brick, the views it may vote in
    CullView* cull_views = nullptr;  // brick order: the batch's views for the brick test
    ViewC* fold_views = nullptr;     // brick order: the batch's views for the culled fusion
    cudaStream_t aux = nullptr;      // brick order: the culling kernels' branch of a step
    cudaEvent_t fork[3] = {};        // brick order: start, occupancy bits ready, culling done
    void* sat = nullptr;   // tuple mode: integral-image scratch, grown on demand
    size_t sat_bytes = 0;
    void* wt = nullptr;    // depth weighting: selection state and histograms, grown on demand
    size_t wt_bytes = 0;
    float* W = nullptr;
    float* Z = nullptr;
    uint32_t* bits = nullptr;
    int32_t* d_n = nullptr;
    int32_t* d_status = nullptr;
    int64_t* d_total = nullptr;
    unsigned long long* d_nseg = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_init_error;

divas_status fail(divas_ctx* c, divas_status st, const std::string& msg) {
    if (c)
        c->err = msg;
    else
        g_init_error = msg;
    return st;
}

divas_status cuda_fail(divas_ctx* c, cudaError_t e, const char* where) {
    return fail(c, e == cudaErrorMemoryAllocation ? DIVAS_E_OOM : DIVAS_E_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define DIVAS_CUDA(ctx, call)                                   \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

#define DIVAS_LAUNCHED(ctx, what)                                  \
    do {                                                           \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what);    \
    } while (0)

inline cudaStream_t S(void* s) {
    // a launch is checked with cudaGetLastError, so first drop any stale,
    // non-sticky error that an earlier unchecked runtime call left behind
    (void)cudaGetLastError();
    return reinterpret_cast<cudaStream_t>(s);
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

int grid_for(int64_t items, int32_t sm_count, int per_sm = 16) {
    int64_t b = (items + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

bool finite_pos(float x) { return x > 0.f && x <= FLT_MAX; }

// launch with programmatic stream serialization (the kernel calls
// wait_for_producer before reading its predecessor's results)
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*f)(KArgs...), int blocks, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, std::forward<Args>(args)...);
}

// A plain grid's depth tolerance Delta = fl(gamma h) and its derived
// constants, as the kernels would round them: the single-precision product and
// quotient here round to nearest like __fmul_rn and __frcp_rn; Delta (1 +
// 2^-20) is exact in double and rounded up to float.
void set_tolerances(GridC& G, float gamma) {
    const float delta = gamma * G.h;
    G.delta = delta;
    G.inv_delta = 1.0f / delta;
    const double ds = (double)delta * (1.0 + 0x1p-20);
    float f = (float)ds;
    if ((double)f < ds) f = nextafterf(f, INFINITY);
    G.delta_s = f;
    G.pad2 = 0;
}

// Argument checks shared by every entry point that takes a grid, fusion
// parameters or a camera: nullptr when the argument is valid, else the reason.
const char* grid_problem(const divas_grid* grid, int32_t g_max) {
    if (!grid) return "grid is NULL";
    if (grid->g < 1 || grid->g > g_max) return "g out of range";
    if (!finite_pos(grid->h)) return "h must be finite and > 0";
    for (int q = 0; q < 3; ++q)
        if (!(fabsf(grid->origin[q]) <= FLT_MAX)) return "origin not finite";
    return nullptr;
}

// multiply-shift divider for d >= 1 (l = ceil(log2 d), m = 2^32 (2^l - d) / d + 1)
FastDiv make_fast_div(uint32_t d) {
    FastDiv f;
    int32_t l = 0;
    while ((1ull << l) < d) ++l;
    f.d = d;
    f.l = l;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.pad = 0;
    return f;
}

const char* params_problem(const divas_params* p) {
    if (!p) return "params is NULL";
    if (!(p->gamma > 0.f && p->gamma <= FLT_MAX) || !(p->alpha1 >= 0.f) ||
        !(p->alpha1 <= FLT_MAX) || !(p->eps >= 0.f) || !(p->tau_mask == p->tau_mask) ||
        !(p->tau_cons == p->tau_cons) || !(p->z_near == p->z_near))
        return "params out of range";
    if (p->flags & ~DIVAS_ORDER_BRICKS) return "unknown params flags";
    return nullptr;
}

const char* camera_problem(const divas_camera* cam) {
    if (!cam) return "camera is NULL";
    if (cam->W <= 0 || cam->H <= 0 || cam->W > 65535 || cam->H > 65535 ||
        (int64_t)cam->W * cam->H > INT32_MAX)
        return "camera W/H must be in 1..65535 with W*H < 2^31";
    for (int q = 0; q < 9; ++q)
        if (!(fabsf(cam->R[q]) <= FLT_MAX)) return "camera R not finite";
    for (int q = 0; q < 3; ++q)
        if (!(fabsf(cam->t[q]) <= FLT_MAX)) return "camera t not finite";
    if (!(fabsf(cam->fx) <= FLT_MAX && fabsf(cam->fy) <= FLT_MAX && fabsf(cam->cx) <= FLT_MAX &&
          fabsf(cam->cy) <= FLT_MAX))
        return "camera intrinsics not finite";
    return nullptr;
}

divas_status check_camera(divas_ctx* c, const divas_camera* cam) {
    if (const char* why = camera_problem(cam)) return fail(c, DIVAS_E_INVALID, why);
    return DIVAS_OK;
}

// Per-view constants.  Plain grids: lattice form p = T + M n, n = 2 idx + 1,
// T = R o + t, M = (h/2) R, each split into an exact hi part (multiples of a
// power of two 2^q with |T| + sum |M| (2g - 1) < 2^(q+24), so that the device
// FMA chain over hi parts is exact) and a lo remainder.
// Contracted grids: the fusion's rows (folded = true) or the camera's R and t
// as given (folded = false: the depth-tuple and NeRF modes, which form their
// own rows and intrinsics).
ViewC make_view(const divas_camera& cam, const GridC& G, const float* depth, const void* mask,
                int32_t mask_type, int32_t index, bool folded = true) {
    ViewC v;
    memset(&v, 0, sizeof(v));
    if (G.contracted && !folded) {
        memcpy(v.A, cam.R, sizeof(cam.R));
        memcpy(v.C, cam.t, sizeof(cam.t));
    } else if (G.contracted) {
        // intrinsics folded into the pixel rows (in double, rounded once); the
        // depth row as given
        for (int j = 0; j < 3; ++j) {
            v.A[j] = (float)((double)cam.fx * cam.R[j] + (double)cam.cx * cam.R[6 + j]);
            v.A[3 + j] = (float)((double)cam.fy * cam.R[3 + j] + (double)cam.cy * cam.R[6 + j]);
            v.A[6 + j] = cam.R[6 + j];
        }
        v.C[0] = (float)((double)cam.fx * cam.t[0] + (double)cam.cx * cam.t[2]);
        v.C[1] = (float)((double)cam.fy * cam.t[1] + (double)cam.cy * cam.t[2]);
        v.C[2] = cam.t[2];
        // the depth screen's bound 2^-19 (max_j |R_zj| n1 + |t_z|): powers of two
        // scale exactly; the coefficient is rounded up
        const float rz = std::max(fabsf(cam.R[6]), std::max(fabsf(cam.R[7]), fabsf(cam.R[8])));
        v.B[0] = nextafterf(ldexpf(rz, -19), INFINITY);
        v.E = ldexpf(fabsf(cam.t[2]), -19);
    } else {
        // camera coordinates of the lattice point n: p = T + M n, T = R o + t,
        // M = (h / 2) R (in double)
        const double hh = 0.5 * (double)G.h;
        const double nmax = 2.0 * G.g;  // centres n <= 2g - 1, corners n + 1 <= 2g
        double T[3], M[3][3];
        for (int r = 0; r < 3; ++r) {
            T[r] = (double)cam.t[r];
            for (int j = 0; j < 3; ++j) {
                T[r] += (double)cam.R[3 * r + j] * (double)G.origin[j];
                M[r][j] = hh * (double)cam.R[3 * r + j];
            }
        }
        // depth row: hi parts on a power-of-two quantum, so that the FMA chain
        // over them is exact, plus the lo remainders
        double bmax = fabs(T[2]);
        for (int j = 0; j < 3; ++j) bmax += fabs(M[2][j]) * nmax;
        int ex = 0;
        frexp(bmax * 1.001 + 1e-300, &ex);  // bmax * 1.001 < 2^ex
        const double quantum = ldexp(1.0, ex - 24);
        for (int j = 0; j < 3; ++j) {
            const double hi = rint(M[2][j] / quantum) * quantum;
            v.A[6 + j] = (float)hi;
            v.B[j] = (float)(M[2][j] - hi);
        }
        const double thi = rint(T[2] / quantum) * quantum;
        v.C[2] = (float)thi;
        v.E = (float)(T[2] - thi);
        // pixel rows: u p_z = (fx M_0 + cx M_2) n + (fx T_0 + cx T_2), likewise v
        for (int j = 0; j < 3; ++j) {
            v.A[j] = (float)((double)cam.fx * M[0][j] + (double)cam.cx * M[2][j]);
            v.A[3 + j] = (float)((double)cam.fy * M[1][j] + (double)cam.cy * M[2][j]);
        }
        v.C[0] = (float)((double)cam.fx * T[0] + (double)cam.cx * T[2]);
        v.C[1] = (float)((double)cam.fy * T[1] + (double)cam.cy * T[2]);
        if (folded) {
            // the plain depth row (rounded to float) and the depth screen's
            // slack 2^-20 b_max, rounded up
            for (int j = 0; j < 3; ++j) v.K[j] = (float)M[2][j];
            v.K[3] = nextafterf((float)ldexp(bmax, -20), INFINITY);
        }
    }
    if (G.contracted || !folded) {
        v.K[0] = cam.fx;
        v.K[1] = cam.fy;
        v.K[2] = cam.cx;
        v.K[3] = cam.cy;
    }
    v.W = cam.W;
    v.H = cam.H;
    v.mask_type = mask_type;
    v.bit = index < 32 ? (1u << index) : 0u;
    v.depth = depth;
    v.mask = mask;
    return v;
}

float logit_threshold(float tau) {
    if (!(tau > 0.f)) return -INFINITY;
    if (!(tau < 1.f)) return INFINITY;
    return (float)log((double)tau / (1.0 - (double)tau));
}

// launch k_fuse_fin with the chunk count as a compile-time constant; batches
// whose views all carry binary16 masks and fill their chunks exactly take the
// kF16Full instance
template <bool kAccumulate, bool kContracted, int kChunks = 1>
cudaError_t launch_fuse_fin_chunks(int chunks, int blocks, cudaStream_t s, const divas_ctx* c,
                                   const ViewBatch& vb, float* score_out, bool clear_bits,
                                   uint32_t* seg_out, bool clear_out, bool zero) {
    if constexpr (kChunks < kMaxViews / kViewChunk) {
        if (chunks > kChunks)
            return launch_fuse_fin_chunks<kAccumulate, kContracted, kChunks + 1>(
                chunks, blocks, s, c, vb, score_out, clear_bits, seg_out, clear_out, zero);
    }
    bool f16_full = vb.n == kChunks * kViewChunk;
    for (int32_t i = 0; i < vb.n && f16_full; ++i) f16_full = vb.v[i].mask_type == kMaskF16;
#define DIVAS_FUSE_FIN(F16)                                                                        \
    e = launch_dependent(k_fuse_fin<kAccumulate, kContracted, kChunks, F16>, blocks, s,           \
        (const uint32_t*)c->active, (const int32_t*)c->d_n, c->G, c->F, vb, c->W, c->Z, c->bits,   \
        (int32_t)(c->grid.kind == 0 ? 1 : 0), score_out, c->seg_bits,                              \
        (int32_t)(clear_bits ? 1 : 0), seg_out, (int32_t)(clear_out ? 1 : 0),                      \
        (const uint32_t*)c->occ_bits, c->n_words, c->n_cells, (int32_t)(zero ? 1 : 0))
    cudaError_t e;
    if (f16_full) DIVAS_FUSE_FIN(true);
    else DIVAS_FUSE_FIN(false);
#undef DIVAS_FUSE_FIN
    return e != cudaSuccess ? e : cudaGetLastError();
}

// zero: also write the zeros of a dense score_out's unoccupied cells
// floats of one view's mask pyramid (levels kPyrL0 .. kPyrL0 + kPyrLevels - 1)
int64_t pyramid_floats(int32_t W, int32_t H) {
    int64_t f = 0;
    for (int l = 0; l < kPyrLevels; ++l) {
        const int L = kPyrL0 + l;
        f += (int64_t)((W + (1 << L) - 1) >> L) * ((H + (1 << L) - 1) >> L);
    }
    return f;
}

// the cull constants of a view batch; false when the pyramids do not fit the
// context's buffer (the batch is then fused without culling)
bool make_cull(const divas_ctx* c, const ViewBatch& vb, CullBatch& cb) {
    memset(&cb, 0, sizeof(cb));
    cb.pyr = c->pyr;
    cb.n = vb.n;
    int64_t off = 0;
    for (int32_t k = 0; k < vb.n; ++k) {
        const ViewC& V = vb.v[k];
        CullC& C = cb.v[k];
        C.thr = V.mask_type == kMaskLogit ? c->F.logit_tau : c->F.tau_m;
        // row magnitudes for the rectangle's error margin (rounded up)
        float* sums[3] = {&C.su, &C.sv, &C.sz};
        float* cons[3] = {&C.cu, &C.cv, &C.cz};
        for (int r = 0; r < 3; ++r) {
            double a = 0.0;
            for (int j = 0; j < 3; ++j) a += fabs((double)V.A[3 * r + j]);
            *sums[r] = nextafterf((float)(a * (1.0 + 1e-6)), INFINITY);
            *cons[r] = fabsf(V.C[r]);
        }
        C.W = V.W;
        C.H = V.H;
        for (int l = 0; l < kPyrLevels; ++l) {
            const int L = kPyrL0 + l;
            C.lw[l] = (V.W + (1 << L) - 1) >> L;
            C.lh[l] = (V.H + (1 << L) - 1) >> L;
            C.off[l] = (int32_t)off;
            off += (int64_t)C.lw[l] * C.lh[l];
        }
        if (off > c->pyr_cap) return false;
    }
    return true;
}

template <bool kAccumulate, bool kContracted>
cudaError_t launch_fuse_fin_cull(const divas_ctx* c, const ViewBatch& vb, int blocks,
                                 cudaStream_t s, float* score_out, bool score_zeroed,
                                 bool clear_bits, uint32_t* seg_out, bool clear_out) {
    bool f16 = true;
    for (int32_t i = 0; i < vb.n && f16; ++i) f16 = vb.v[i].mask_type == kMaskF16;
#define DIVAS_FUSE_CULL(MT)                                                                       \
    launch_dependent(k_fuse_fin_cull<kAccumulate, kContracted, MT>, blocks, s,                    \
                     (const uint32_t*)c->active, (const int32_t*)c->d_n, c->G, c->F,              \
                     (const ViewC*)c->fold_views, vb.n, (const uint32_t*)c->brick_keep,            \
                     c->W, c->Z, c->bits, (int32_t)(c->grid.kind == 0 ? 1 : 0), score_out,        \
                     (int32_t)(score_zeroed ? 1 : 0), c->seg_bits, (int32_t)(clear_bits ? 1 : 0), \
                     seg_out, (int32_t)(clear_out ? 1 : 0))
    const cudaError_t e = f16 ? DIVAS_FUSE_CULL(kMaskF16) : DIVAS_FUSE_CULL(-1);
#undef DIVAS_FUSE_CULL
    return e != cudaSuccess ? e : cudaGetLastError();
}

// the mask pyramids of a batch (programmatic: a dependent launch -- the kernel
// reads the masks only, and waits for its predecessor before it ends -- else
// plain stream order)
cudaError_t launch_pyramid(const divas_ctx* c, const ViewBatch& vb, const CullBatch& cb,
                           cudaStream_t s, bool programmatic = true) {
    int32_t wmax = 1, hmax = 1;
    for (int32_t k = 0; k < vb.n; ++k) {
        wmax = std::max(wmax, vb.v[k].W);
        hmax = std::max(hmax, vb.v[k].H);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((wmax + kPyrTile - 1) / kPyrTile),
                       (unsigned)((hmax + kPyrTile - 1) / kPyrTile), (unsigned)vb.n);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = programmatic ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_mask_pyramid, vb, cb, c->cull_views, c->fold_views);
}

// the bricks' kept views: several bricks per warp, one wave of CTAs
cudaError_t launch_brick_views(const divas_ctx* c, const ViewBatch& vb, cudaStream_t s,
                               bool programmatic = true) {
    const int64_t n_bricks = c->n_words / 16;
    const int64_t per_warp = std::min<int64_t>(8, 32 / std::max(1, vb.n));
    const int64_t warps = (n_bricks + per_warp - 1) / per_warp;
    const int blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)c->sm_count * 8));
    if (!programmatic) {
        k_brick_views<<<blocks, kThreads, 0, s>>>(
            (const CullView*)c->cull_views, vb.n, (const float*)c->pyr, c->G, c->bdiv,
            (const uint32_t*)c->occ_bits, n_bricks, c->brick_keep);
        return cudaGetLastError();
    }
    return launch_dependent(k_brick_views, blocks, s, (const CullView*)c->cull_views, vb.n,
                            (const float*)c->pyr, c->G, c->bdiv, (const uint32_t*)c->occ_bits,
                            n_bricks, c->brick_keep);
}

// the culling fusion (the bricks' kept views are in place)
cudaError_t launch_culled_fuse(const divas_ctx* c, bool accumulate, const ViewBatch& vb,
                               cudaStream_t s, float* score_out, bool score_zeroed,
                               bool clear_bits, uint32_t* seg_out, bool clear_out) {
    const int blocks = grid_for(c->cap, c->sm_count);
    if (c->G.contracted)
        return accumulate ? launch_fuse_fin_cull<true, true>(
                   c, vb, blocks, s, score_out, score_zeroed, clear_bits, seg_out, clear_out)
                          : launch_fuse_fin_cull<false, true>(
                   c, vb, blocks, s, score_out, score_zeroed, clear_bits, seg_out, clear_out);
    return accumulate ? launch_fuse_fin_cull<true, false>(
                   c, vb, blocks, s, score_out, score_zeroed, clear_bits, seg_out, clear_out)
                      : launch_fuse_fin_cull<false, false>(
                   c, vb, blocks, s, score_out, score_zeroed, clear_bits, seg_out, clear_out);
}

// fewest views in a batch for which culling pays: below it the pyramid and brick
// test launches cost more than the views they skip (measured on the served
// session mix, where updates carry one view)
constexpr int32_t kCullMinViews = 4;

// whether a batch on this context is fused with culling (then cb holds its constants)
bool culling(const divas_ctx* c, const ViewBatch& vb, CullBatch& cb) {
    return c->brick && c->pyr && c->brick_keep && c->cull_views && c->fold_views && c->aux &&
           vb.n >= kCullMinViews && make_cull(c, vb, cb);
}

// score_zeroed: score_out holds +0 at every active voxel (brick contexts skip
// storing a P of +0 there)
// prepared: the batch's pyramids and the bricks' kept views were launched with
// the compaction (one-call step)
cudaError_t launch_fuse_fin(const divas_ctx* c, bool accumulate, const ViewBatch& vb,
                            cudaStream_t s, float* score_out, bool clear_bits, uint32_t* seg_out,
                            bool clear_out, bool zero, bool score_zeroed = false,
                            bool prepared = false) {
    CullBatch cb;
    if (prepared || culling(c, vb, cb)) {
        if (!prepared) {
            cudaError_t e = launch_pyramid(c, vb, cb, s);
            if (e == cudaSuccess) e = launch_brick_views(c, vb, s);
            if (e != cudaSuccess) return e;
        }
        return launch_culled_fuse(c, accumulate, vb, s, score_out, score_zeroed, clear_bits,
                                  seg_out, clear_out);
    }
    const int chunks = (vb.n + kViewChunk - 1) / kViewChunk;
    const int blocks = grid_for(zero ? std::max<int64_t>(c->cap, c->n_words) : c->cap, c->sm_count);
    if (c->G.contracted)
        return accumulate ? launch_fuse_fin_chunks<true, true>(chunks, blocks, s, c, vb, score_out,
                                                               clear_bits, seg_out, clear_out, zero)
                          : launch_fuse_fin_chunks<false, true>(chunks, blocks, s, c, vb,
                                                                score_out, clear_bits, seg_out,
                                                                clear_out, zero);
    return accumulate ? launch_fuse_fin_chunks<true, false>(chunks, blocks, s, c, vb, score_out,
                                                            clear_bits, seg_out, clear_out, zero)
                      : launch_fuse_fin_chunks<false, false>(chunks, blocks, s, c, vb, score_out,
                                                             clear_bits, seg_out, clear_out, zero);
}

// k_tile_emit grid: one group per warp, at most 16 CTAs per SM
int emit_blocks(int64_t n_words, int32_t sm_count) {
    const int64_t groups = (n_words + 31) / 32;
    const int64_t want = (groups + kThreads / 32 - 1) / (kThreads / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count * 16));
}

// occupancy -> bits -> tile counts -> active list (no allocation); seg_zero /
// seg_zero2 (nullable) are seg bitfields to clear on the way
// the culling branch of a brick-ordered one-call step: once the occupancy bits
// are complete on s, the helper stream (which already builds the pyramids)
// tests the bricks; fork[2] marks its end
divas_status fork_brick_views(divas_ctx* c, const ViewBatch& vb, cudaStream_t s) {
    DIVAS_CUDA(c, cudaEventRecord(c->fork[1], s));
    DIVAS_CUDA(c, cudaStreamWaitEvent(c->aux, c->fork[1], 0));
    const cudaError_t e = launch_brick_views(c, vb, c->aux, false);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_brick_views");
    DIVAS_CUDA(c, cudaEventRecord(c->fork[2], c->aux));
    return DIVAS_OK;
}

divas_status build_counts(divas_ctx* c, const uint8_t* occ, const int32_t* coords,
                          int64_t n_coords, cudaStream_t s, float* score_zero = nullptr,
                          const ViewBatch* fork_vb = nullptr) {
    if (c->grid.kind == 0) {
        if (c->brick && (reinterpret_cast<uintptr_t>(occ) & 7))
            return fail(c, DIVAS_E_INVALID, "brick order needs an 8-byte aligned dense prior");
        if (c->brick)
            k_tile_count<2><<<c->n_tiles, kThreads, 0, s>>>(
                occ, c->occ_bits, c->n_cells, c->n_words, c->cap, c->item_pref, c->tile_count,
                c->tile_offset, c->done, c->n_tiles, c->d_n, c->d_total, c->d_status, c->grid.g,
                c->bdiv, score_zero);
        else
            k_tile_count<0><<<c->n_tiles, kThreads, 0, s>>>(
                occ, c->occ_bits, c->n_cells, c->n_words, c->cap, c->item_pref, c->tile_count,
                c->tile_offset, c->done, c->n_tiles, c->d_n, c->d_total, c->d_status, c->grid.g,
                c->bdiv, nullptr);
        DIVAS_LAUNCHED(c, "k_tile_count");
        if (fork_vb) return fork_brick_views(c, *fork_vb, s);
    } else {
        DIVAS_CUDA(c, cudaMemsetAsync(c->occ_bits, 0, c->n_words * 4, s));
        if (n_coords > 0) {
            if (c->brick)
                k_scatter_coords<true><<<grid_for(n_coords, c->sm_count, 32), kThreads, 0, s>>>(
                    coords, n_coords, c->grid.g, c->occ_bits, c->d_status);
            else
                k_scatter_coords<false><<<grid_for(n_coords, c->sm_count, 32), kThreads, 0, s>>>(
                    coords, n_coords, c->grid.g, c->occ_bits, c->d_status);
            DIVAS_LAUNCHED(c, "k_scatter_coords");
        }
        if (fork_vb) {
            const divas_status st = fork_brick_views(c, *fork_vb, s);
            if (st != DIVAS_OK) return st;
        }
        k_tile_count<1><<<c->n_tiles, kThreads, 0, s>>>(
            nullptr, c->occ_bits, c->n_cells, c->n_words, c->cap, c->item_pref, c->tile_count,
            c->tile_offset, c->done, c->n_tiles, c->d_n, c->d_total, c->d_status, c->grid.g,
            c->bdiv, nullptr);
        DIVAS_LAUNCHED(c, "k_tile_count");
    }
    return DIVAS_OK;
}

// the full compaction: counts, then (when the active arrays exist) the list;
// seg_zero / seg_zero2 (nullable) are seg bitfields to clear on the way
// cull (nullable): a view batch culled per brick (the one-call step of a
// brick-ordered context).  The culling kernels run on the context's helper
// stream, concurrently with the compaction: the pyramids from the start (they
// read the masks only), the brick test once the occupancy bits are complete;
// s waits for them after the emit.
divas_status build_active(divas_ctx* c, const uint8_t* occ, const int32_t* coords, int64_t n_coords,
                          cudaStream_t s, uint32_t* seg_zero = nullptr,
                          uint32_t* seg_zero2 = nullptr, float* score_zero = nullptr,
                          const ViewBatch* cull_vb = nullptr, const CullBatch* cull_cb = nullptr) {
    const bool fork = cull_vb && c->active;
    if (fork) {
        DIVAS_CUDA(c, cudaEventRecord(c->fork[0], s));
        DIVAS_CUDA(c, cudaStreamWaitEvent(c->aux, c->fork[0], 0));
        const cudaError_t e = launch_pyramid(c, *cull_vb, *cull_cb, c->aux, false);
        if (e != cudaSuccess) return cuda_fail(c, e, "k_mask_pyramid");
    }
    divas_status st = build_counts(c, occ, coords, n_coords, s, score_zero, fork ? cull_vb : nullptr);
    if (st != DIVAS_OK || !c->active) return st;
    cudaError_t e = launch_dependent(c->brick ? k_tile_emit<true> : k_tile_emit<false>,
                                     emit_blocks(c->n_words, c->sm_count), s,
                                     (const uint32_t*)c->occ_bits, c->n_words, c->cap,
                                     c->brick ? c->bdiv : c->gdiv, (const uint32_t*)c->item_pref,
                                     (const uint32_t*)c->tile_offset, c->active, seg_zero,
                                     seg_zero2);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_tile_emit");
    DIVAS_LAUNCHED(c, "k_tile_emit");
    if (fork) DIVAS_CUDA(c, cudaStreamWaitEvent(s, c->fork[2], 0));
    return DIVAS_OK;
}

divas_status read_status(divas_ctx* c, cudaStream_t s) {
    int32_t st = 0;
    int32_t n = 0;
    DIVAS_CUDA(c, cudaMemcpyAsync(&st, c->d_status, 4, cudaMemcpyDeviceToHost, s));
    DIVAS_CUDA(c, cudaMemcpyAsync(&n, c->d_n, 4, cudaMemcpyDeviceToHost, s));
    DIVAS_CUDA(c, cudaStreamSynchronize(s));
    c->n_active = n;
    if (st) {
        DIVAS_CUDA(c, cudaMemsetAsync(c->d_status, 0, 4, s));
        if (st & kStatusBadCoord)
            return fail(c, DIVAS_E_INVALID, "a sparse coordinate lies outside the grid (skipped)");
        if (st & kStatusCapacity)
            return fail(c, DIVAS_E_CAPACITY, "occupied set exceeds the context capacity (truncated)");
    }
    return DIVAS_OK;
}

void free_all(divas_ctx* c) {
    if (c->sat) cudaFree(c->sat);
    if (c->wt) cudaFree(c->wt);
    if (c->pyr) cudaFree(c->pyr);
    if (c->brick_keep) cudaFree(c->brick_keep);
    if (c->cull_views) cudaFree(c->cull_views);
    if (c->fold_views) cudaFree(c->fold_views);
    for (cudaEvent_t& ev : c->fork)
        if (ev) cudaEventDestroy(ev);
    if (c->aux) cudaStreamDestroy(c->aux);
    void* ptrs[] = {c->occ_bits, c->item_pref, c->tile_count, c->tile_offset, c->done,
                    c->seg_bits, c->active,     c->W,          c->Z,           c->bits,
                    c->d_n,      c->d_status,   c->d_total,    c->d_nseg};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

extern "C" {

void divas_default_params(divas_params* out) {
    if (!out) return;
    out->tau_mask = 0.5f;
    out->gamma = 1.0f;
    out->alpha1 = 0.5f;
    out->tau_cons = 0.5f;
    out->eps = 1e-12f;
    out->z_near = 1e-6f;
    out->flags = 0;
}

divas_status divas_fuse_init(divas_ctx** out, const divas_grid* grid, const uint8_t* occ_dense,
                             const int32_t* coords, int64_t n_coords, const divas_params* params,
                             void* stream) {
    if (!out) return fail(nullptr, DIVAS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!grid || !params) return fail(nullptr, DIVAS_E_INVALID, "grid or params is NULL");
    if (grid->g < 1 || grid->g > 1024) return fail(nullptr, DIVAS_E_INVALID, "g must be in 1..1024");
    if (const char* why = grid_problem(grid, 1024)) return fail(nullptr, DIVAS_E_INVALID, why);
    if (grid->kind == 0) {
        if (!occ_dense || coords) return fail(nullptr, DIVAS_E_INVALID, "dense kind needs occ_dense only");
    } else if (grid->kind == 1) {
        if (occ_dense || n_coords < 0 || (n_coords > 0 && !coords))
            return fail(nullptr, DIVAS_E_INVALID, "sparse kind needs coords only");
    } else {
        return fail(nullptr, DIVAS_E_INVALID, "kind must be 0 (dense) or 1 (sparse)");
    }
    if (const char* why = params_problem(params)) return fail(nullptr, DIVAS_E_INVALID, why);
    if ((params->flags & DIVAS_ORDER_BRICKS) && grid->g % 8 != 0)
        return fail(nullptr, DIVAS_E_INVALID, "brick order needs g a multiple of 8");

    divas_ctx* c = new (std::nothrow) divas_ctx();
    if (!c) return fail(nullptr, DIVAS_E_OOM, "host allocation failed");
    c->grid = *grid;
    c->params = *params;
    c->G.origin[0] = grid->origin[0];
    c->G.origin[1] = grid->origin[1];
    c->G.origin[2] = grid->origin[2];
    c->G.h = grid->h;
    c->G.g = grid->g;
    c->G.contracted = grid->contracted ? 1 : 0;
    {
        int ex = 0;
        const double fr = frexp((double)grid->h, &ex);
        c->G.inv_h = fr == 0.5 ? (float)ldexp(1.0, 1 - ex) : 0.f;
        c->G.pad = 0;
    }
    c->F.gamma = params->gamma;
    c->F.alpha1 = params->alpha1;
    c->F.tau_m = params->tau_mask;
    c->F.logit_tau = logit_threshold(params->tau_mask);
    c->F.z_near = params->z_near;
    c->F.eps = params->eps;
    c->F.tau_cons = params->tau_cons;
    c->F.pad = 0;
    set_tolerances(c->G, c->F.gamma);
    c->gdiv = make_fast_div((uint32_t)grid->g);
    c->brick = (params->flags & DIVAS_ORDER_BRICKS) != 0;
    c->bdiv = make_fast_div((uint32_t)std::max(1, grid->g / 8));
    c->n_cells = (int64_t)grid->g * grid->g * grid->g;
    c->n_words = (c->n_cells + 31) / 32;
    c->n_tiles = (int32_t)((c->n_words + kTileSpan - 1) / kTileSpan);
    cudaStream_t s = S(stream);
    int dev = 0;
    divas_status st = DIVAS_OK;
    auto bail = [&](divas_status e) {
        g_init_error = c->err;
        free_all(c);
        delete c;
        return e;
    };
#define INIT_CUDA(call)                                                 \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, #call));    \
    } while (0)
    INIT_CUDA(cudaGetDevice(&dev));
    INIT_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
    INIT_CUDA(cudaMalloc(&c->occ_bits, c->n_words * 4));
    INIT_CUDA(cudaMalloc(&c->item_pref, (size_t)c->n_tiles * kTileItems * 4));
    INIT_CUDA(cudaMalloc(&c->tile_count, (size_t)c->n_tiles * 4));
    INIT_CUDA(cudaMalloc(&c->tile_offset, (size_t)c->n_tiles * 4));
    INIT_CUDA(cudaMalloc(&c->done, 4));
    INIT_CUDA(cudaMemsetAsync(c->done, 0, 4, s));
    INIT_CUDA(cudaMalloc(&c->seg_bits, c->n_words * 4));
    INIT_CUDA(cudaMalloc(&c->d_n, 4));
    INIT_CUDA(cudaMalloc(&c->d_status, 4));
    INIT_CUDA(cudaMalloc(&c->d_total, 8));
    INIT_CUDA(cudaMalloc(&c->d_nseg, 8));
    if (c->brick) {  // mask pyramids of up to 32 views of up to 2048 x 2048 pixels
        c->pyr_cap = (int64_t)kMaxViews * pyramid_floats(2048, 2048);
        INIT_CUDA(cudaMalloc(&c->pyr, c->pyr_cap * 4));
        INIT_CUDA(cudaMalloc(&c->brick_keep, (c->n_words / 16) * 4));
        INIT_CUDA(cudaMalloc(&c->cull_views, kMaxViews * sizeof(CullView)));
        INIT_CUDA(cudaMalloc(&c->fold_views, kMaxViews * sizeof(ViewC)));
        INIT_CUDA(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
        for (cudaEvent_t& ev : c->fork)
            INIT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    INIT_CUDA(cudaMemsetAsync(c->d_status, 0, 4, s));
    INIT_CUDA(cudaMemsetAsync(c->seg_bits, 0, c->n_words * 4, s));
    c->cap = INT32_MAX;  // first pass only counts
    st = build_active(c, occ_dense, coords, n_coords, s);
    if (st != DIVAS_OK) return bail(st);
    int64_t total = 0;
    INIT_CUDA(cudaMemcpyAsync(&total, c->d_total, 8, cudaMemcpyDeviceToHost, s));
    int32_t dst = 0;
    INIT_CUDA(cudaMemcpyAsync(&dst, c->d_status, 4, cudaMemcpyDeviceToHost, s));
    INIT_CUDA(cudaStreamSynchronize(s));
    if (dst & kStatusBadCoord) {
        c->err = "a sparse coordinate lies outside the grid";
        return bail(DIVAS_E_INVALID);
    }
    if (total > INT32_MAX - 1) {
        c->err = "occupied set too large";
        return bail(DIVAS_E_INVALID);
    }
    c->n_active = total;
    c->cap = total > 0 ? total : 1;
    INIT_CUDA(cudaMalloc(&c->active, c->cap * 4));
    INIT_CUDA(cudaMalloc(&c->W, c->cap * 4));
    INIT_CUDA(cudaMalloc(&c->Z, c->cap * 4));
    INIT_CUDA(cudaMalloc(&c->bits, c->cap * 4));
    st = build_active(c, occ_dense, coords, n_coords, s);
    if (st != DIVAS_OK) return bail(st);
    INIT_CUDA(cudaMemsetAsync(c->W, 0, c->cap * 4, s));
    INIT_CUDA(cudaMemsetAsync(c->Z, 0, c->cap * 4, s));
    INIT_CUDA(cudaMemsetAsync(c->bits, 0, c->cap * 4, s));
#undef INIT_CUDA
    *out = c;
    return DIVAS_OK;
}

divas_status divas_fuse_set_occupancy(divas_ctx* c, const uint8_t* occ_dense, const int32_t* coords,
                                      int64_t n_coords, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (c->grid.kind == 0 && (!occ_dense || coords))
        return fail(c, DIVAS_E_INVALID, "dense context needs occ_dense only");
    if (c->grid.kind == 1 && (occ_dense || n_coords < 0 || (n_coords > 0 && !coords)))
        return fail(c, DIVAS_E_INVALID, "sparse context needs coords only");
    cudaStream_t s = S(stream);
    // the seg bitfield is cleared on the way: it never holds a bit of a voxel
    // outside the current occupied set
    divas_status st = build_active(c, occ_dense, coords, n_coords, s, c->seg_bits);
    if (st != DIVAS_OK) return st;
    c->n_views = 0;
    c->n_active = c->cap;  // upper bound until the next synchronising call
    return DIVAS_OK;
}

// record stage event k (when given) on s; inside a stream capture it becomes
// an event-record node, so that graph replays time the stages
static divas_status record_stage(divas_ctx* c, void* const* events, int k, cudaStream_t s) {
    if (!events || !events[k]) return DIVAS_OK;
    cudaEvent_t ev = static_cast<cudaEvent_t>(events[k]);
    DIVAS_CUDA(c, capturing(s) ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                               : cudaEventRecord(ev, s));
    return DIVAS_OK;
}

// labels of n > 0 points
static divas_status launch_label(divas_ctx* c, const float* xyz, int64_t n, uint8_t* labels_out,
                                 cudaStream_t s) {
    const int blocks = grid_for((n + 3) / 4, c->sm_count, 64);
    const cudaError_t e =
        !c->G.contracted && c->G.inv_h != 0.f
            ? launch_dependent(k_label<true>, blocks, s, xyz, n, c->G,
                               (const uint32_t*)c->seg_bits, labels_out)
            : launch_dependent(k_label<false>, blocks, s, xyz, n, c->G,
                               (const uint32_t*)c->seg_bits, labels_out);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_label");
    DIVAS_LAUNCHED(c, "k_label");
    return DIVAS_OK;
}

// validate views and build their constants (view bits continue the context's count)
static divas_status make_batch(divas_ctx* c, const divas_view* views, int32_t n_views,
                               int32_t first_view, ViewBatch& vb) {
    if (!views || n_views < 1 || n_views > kMaxViews)
        return fail(c, DIVAS_E_INVALID, "n_views must be in 1..32 and views non-NULL");
    memset(&vb, 0, sizeof(vb));
    vb.n = n_views;
    for (int32_t k = 0; k < n_views; ++k) {
        divas_status st = check_camera(c, &views[k].cam);
        if (st != DIVAS_OK) return st;
        if (!views[k].depth || !views[k].mask) return fail(c, DIVAS_E_INVALID, "depth or mask is NULL");
        if (views[k].mask_type < 0 || views[k].mask_type > 2)
            return fail(c, DIVAS_E_INVALID, "bad mask_type");
        vb.v[k] = make_view(views[k].cam, c->G, views[k].depth, views[k].mask,
                            views[k].mask_type, first_view + k);
    }
    return DIVAS_OK;
}

static divas_status launch_fuse(divas_ctx* c, ViewBatch& vb, cudaStream_t s) {
    const int blocks = grid_for(c->cap, c->sm_count);
    const bool acc = c->n_views > 0;
    const int chunks = (vb.n + kViewChunk - 1) / kViewChunk;
    cudaError_t e;
    if (c->G.contracted)
        e = acc ? launch_fuse_chunks<true, true>(chunks, blocks, s, c->active, c->d_n, c->G, c->F,
                                                 vb, c->W, c->Z, c->bits)
                : launch_fuse_chunks<false, true>(chunks, blocks, s, c->active, c->d_n, c->G,
                                                  c->F, vb, c->W, c->Z, c->bits);
    else
        e = acc ? launch_fuse_chunks<true, false>(chunks, blocks, s, c->active, c->d_n, c->G,
                                                  c->F, vb, c->W, c->Z, c->bits)
                : launch_fuse_chunks<false, false>(chunks, blocks, s, c->active, c->d_n, c->G,
                                                   c->F, vb, c->W, c->Z, c->bits);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_fuse");
    DIVAS_LAUNCHED(c, "k_fuse");
    c->n_views += vb.n;
    return DIVAS_OK;
}

divas_status divas_fuse_add_view(divas_ctx* c, const divas_camera* cam, const float* depth,
                                 const void* mask, int32_t mask_type, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    divas_status st = check_camera(c, cam);
    if (st != DIVAS_OK) return st;
    if (!depth || !mask) return fail(c, DIVAS_E_INVALID, "depth or mask is NULL");
    if (mask_type < 0 || mask_type > 2) return fail(c, DIVAS_E_INVALID, "bad mask_type");
    ViewBatch vb;
    memset(&vb, 0, sizeof(vb));
    vb.n = 1;
    vb.v[0] = make_view(*cam, c->G, depth, mask, mask_type, c->n_views);
    return launch_fuse(c, vb, S(stream));
}

divas_status divas_fuse_add_views(divas_ctx* c, const divas_view* views, int32_t n_views,
                                  void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    ViewBatch vb;
    divas_status st = make_batch(c, views, n_views, c->n_views, vb);
    if (st != DIVAS_OK) return st;
    return launch_fuse(c, vb, S(stream));
}

}  // extern "C"

namespace {

// zero-fill what the scatter below ORs or writes into
// the caller's outputs start at zero (the context's own seg bitfield needs no
// clearing: it never holds a bit of an unoccupied voxel)
divas_status finalize_zero(divas_ctx* c, float* score_out, uint32_t* seg_bits_out, cudaStream_t s) {
    if (score_out && c->grid.kind == 0)
        DIVAS_CUDA(c, cudaMemsetAsync(score_out, 0, c->n_cells * 4, s));
    if (seg_bits_out) DIVAS_CUDA(c, cudaMemsetAsync(seg_bits_out, 0, c->n_words * 4, s));
    return DIVAS_OK;
}

divas_status finalize_scatter(divas_ctx* c, float* score_out, uint32_t* seg_bits_out,
                              uint32_t* vmask_out, unsigned long long* nseg, cudaStream_t s) {
    k_finalize<<<grid_for(c->cap, c->sm_count, 16), kThreads, 0, s>>>(
        c->active, c->d_n, c->grid.g, c->grid.kind == 0 ? 1 : 0, c->W, c->Z, c->bits, c->F.eps,
        c->F.tau_cons, score_out, c->seg_bits, seg_bits_out, vmask_out, nseg);
    DIVAS_LAUNCHED(c, "k_finalize");
    return DIVAS_OK;
}

divas_status finalize_count(divas_ctx* c, int64_t* n_seg_host, cudaStream_t s) {
    unsigned long long v = 0;
    DIVAS_CUDA(c, cudaMemcpyAsync(&v, c->d_nseg, 8, cudaMemcpyDeviceToHost, s));
    divas_status st = read_status(c, s);  // synchronises
    *n_seg_host = (int64_t)v;
    return st;
}

}  // namespace

extern "C" {

divas_status divas_fuse_finalize(divas_ctx* c, float* score_out, uint32_t* seg_bits_out,
                                 uint32_t* vmask_out, int64_t* n_seg_host, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    cudaStream_t s = S(stream);
    unsigned long long* nseg = n_seg_host ? c->d_nseg : nullptr;
    if (nseg) DIVAS_CUDA(c, cudaMemsetAsync(c->d_nseg, 0, 8, s));
    divas_status st = finalize_zero(c, score_out, seg_bits_out, s);
    if (st != DIVAS_OK) return st;
    st = finalize_scatter(c, score_out, seg_bits_out, vmask_out, nseg, s);
    if (st != DIVAS_OK) return st;
    if (n_seg_host) return finalize_count(c, n_seg_host, s);
    return DIVAS_OK;
}

divas_status divas_fuse_step(divas_ctx* c, const uint8_t* occ_dense, const int32_t* coords,
                             int64_t n_coords, const divas_view* views, int32_t n_views,
                             float* score_out, uint32_t* seg_bits_out, const float* xyz, int64_t n_pts,
                             uint8_t* labels_out, void* stream) {
    return divas_fuse_step_profiled(c, occ_dense, coords, n_coords, views, n_views, score_out,
                                    seg_bits_out, xyz, n_pts, labels_out, nullptr, stream);
}

divas_status divas_fuse_step_profiled(divas_ctx* c, const uint8_t* occ_dense,
                                      const int32_t* coords, int64_t n_coords,
                                      const divas_view* views, int32_t n_views, float* score_out,
                                      uint32_t* seg_bits_out, const float* xyz, int64_t n_pts,
                                      uint8_t* labels_out, void* const* stage_events,
                                      void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (c->grid.kind == 0 && (!occ_dense || coords))
        return fail(c, DIVAS_E_INVALID, "dense context needs occ_dense only");
    if (c->grid.kind == 1 && (occ_dense || n_coords < 0 || (n_coords > 0 && !coords)))
        return fail(c, DIVAS_E_INVALID, "sparse context needs coords only");
    if (n_pts < 0 || (n_pts > 0 && (!xyz || !labels_out)))
        return fail(c, DIVAS_E_INVALID, "bad point arguments");
    ViewBatch vb;
    divas_status st = make_batch(c, views, n_views, 0, vb);
    if (st != DIVAS_OK) return st;
    cudaStream_t s = S(stream);
    st = record_stage(c, stage_events, 0, s);
    if (st != DIVAS_OK) return st;
    // occupancy gate + active list; the seg bitfields are cleared on the way, and
    // a brick-ordered dense context's count kernel zeroes the score grid (the
    // fusion then writes the occupied cells' scores)
    const bool dense = c->grid.kind == 0;
    float* score_zero = dense && c->brick && score_out &&
                                (reinterpret_cast<uintptr_t>(score_out) & 15) == 0
                            ? score_out
                            : nullptr;
    if (dense && c->brick && score_out && !score_zero)
        DIVAS_CUDA(c, cudaMemsetAsync(score_out, 0, c->n_cells * 4, s));
    CullBatch cb;
    const bool cull = culling(c, vb, cb);
    st = build_active(c, occ_dense, coords, n_coords, s, c->seg_bits, seg_bits_out, score_zero,
                      cull ? &vb : nullptr, cull ? &cb : nullptr);
    if (st != DIVAS_OK) return st;
    st = record_stage(c, stage_events, 1, s);
    if (st != DIVAS_OK) return st;
    c->n_views = 0;
    c->n_active = c->cap;  // upper bound until the next synchronising call
    const bool zero = score_out && dense && !c->brick;
    // fusion of every view + finalize epilogue (both seg bitfields were
    // cleared) + the zeros of a dense score grid's unoccupied cells
    cudaError_t e = launch_fuse_fin(c, false, vb, s, score_out, false, seg_bits_out, false, zero,
                                    dense && c->brick, cull);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_fuse_fin");
    c->n_views = vb.n;
    st = record_stage(c, stage_events, 2, s);
    if (st != DIVAS_OK) return st;
    if (n_pts > 0) {
        st = launch_label(c, xyz, n_pts, labels_out, s);
        if (st != DIVAS_OK) return st;
    }
    return record_stage(c, stage_events, 3, s);
}

divas_status divas_fuse_update(divas_ctx* c, const divas_view* views, int32_t n_views,
                               float* score_out, uint32_t* seg_bits_out, uint32_t flags,
                               void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (flags & ~(uint32_t)DIVAS_KEEP_ZEROS) return fail(c, DIVAS_E_INVALID, "unknown flags");
    ViewBatch vb;
    divas_status st = make_batch(c, views, n_views, c->n_views, vb);
    if (st != DIVAS_OK) return st;
    cudaStream_t s = S(stream);
    const bool keep = (flags & DIVAS_KEEP_ZEROS) != 0;
    bool zero = !keep && score_out && c->grid.kind == 0;
    bool zeroed = false;
    if (zero && c->brick) {  // the bitfield is brick-major: zero the whole grid first
        DIVAS_CUDA(c, cudaMemsetAsync(score_out, 0, c->n_cells * 4, s));
        zero = false;
        zeroed = true;
    }
    if (!keep && seg_bits_out) DIVAS_CUDA(c, cudaMemsetAsync(seg_bits_out, 0, c->n_words * 4, s));
    // the context's seg bitfield holds this occupied set's previous seg (or
    // zeros): set and clear in place; seg_bits_out likewise when kept
    cudaError_t e = launch_fuse_fin(c, c->n_views > 0, vb, s, score_out, true, seg_bits_out, keep,
                                    zero, zeroed);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_fuse_fin");
    c->n_views += vb.n;
    return DIVAS_OK;
}

divas_status divas_label_points(divas_ctx* c, const float* xyz, int64_t n, uint8_t* labels_out,
                                void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (n < 0 || (n > 0 && (!xyz || !labels_out)))
        return fail(c, DIVAS_E_INVALID, "bad point arguments");
    if (n == 0) return DIVAS_OK;
    return launch_label(c, xyz, n, labels_out, S(stream));
}

divas_status divas_fuse_reset(divas_ctx* c, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    cudaStream_t s = S(stream);
    DIVAS_CUDA(c, cudaMemsetAsync(c->W, 0, c->cap * 4, s));
    DIVAS_CUDA(c, cudaMemsetAsync(c->Z, 0, c->cap * 4, s));
    DIVAS_CUDA(c, cudaMemsetAsync(c->bits, 0, c->cap * 4, s));
    c->n_views = 0;
    return DIVAS_OK;
}

divas_status divas_fuse_sync(divas_ctx* c, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    return read_status(c, S(stream));
}

int64_t divas_fuse_n_active(const divas_ctx* c) { return c ? c->n_active : -1; }

int32_t divas_fuse_n_views(const divas_ctx* c) { return c ? c->n_views : -1; }

divas_status divas_fuse_active_coords(divas_ctx* c, int32_t* coords_out, void* stream) {
    if (!c || !coords_out) return fail(c, DIVAS_E_INVALID, "NULL argument");
    k_active_coords<<<grid_for(c->cap, c->sm_count), kThreads, 0, S(stream)>>>(c->active, c->d_n,
                                                                             c->grid.g, coords_out);
    DIVAS_LAUNCHED(c, "k_active_coords");
    return DIVAS_OK;
}

divas_status divas_fuse_export_state(divas_ctx* c, float* W_out, float* Z_out, uint32_t* bits_out,
                                     void* stream) {
    if (!c || !W_out || !Z_out || !bits_out) return fail(c, DIVAS_E_INVALID, "NULL argument");
    cudaStream_t s = S(stream);
    DIVAS_CUDA(c, cudaMemcpyAsync(W_out, c->W, c->cap * 4, cudaMemcpyDeviceToDevice, s));
    DIVAS_CUDA(c, cudaMemcpyAsync(Z_out, c->Z, c->cap * 4, cudaMemcpyDeviceToDevice, s));
    DIVAS_CUDA(c, cudaMemcpyAsync(bits_out, c->bits, c->cap * 4, cudaMemcpyDeviceToDevice, s));
    return DIVAS_OK;
}

divas_status divas_fuse_import_state(divas_ctx* c, const float* W_in, const float* Z_in,
                                     const uint32_t* bits_in, int32_t n_views, void* stream) {
    if (!c || !W_in || !Z_in || !bits_in || n_views < 0)
        return fail(c, DIVAS_E_INVALID, "bad argument");
    cudaStream_t s = S(stream);
    DIVAS_CUDA(c, cudaMemcpyAsync(c->W, W_in, c->cap * 4, cudaMemcpyDeviceToDevice, s));
    DIVAS_CUDA(c, cudaMemcpyAsync(c->Z, Z_in, c->cap * 4, cudaMemcpyDeviceToDevice, s));
    DIVAS_CUDA(c, cudaMemcpyAsync(c->bits, bits_in, c->cap * 4, cudaMemcpyDeviceToDevice, s));
    c->n_views = n_views;
    return DIVAS_OK;
}

divas_status divas_fuse_backward(divas_ctx* c, const divas_view* views, int32_t n_views,
                                 const float* grad_score, float* const* grad_mask,
                                 float* const* grad_depth, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (!views || n_views < 1 || n_views > kMaxViews || !grad_score)
        return fail(c, DIVAS_E_INVALID, "bad backward arguments");
    ViewBatch vb;
    memset(&vb, 0, sizeof(vb));
    BackPtrs bp;
    memset(&bp, 0, sizeof(bp));
    vb.n = n_views;
    for (int32_t k = 0; k < n_views; ++k) {
        divas_status st = check_camera(c, &views[k].cam);
        if (st != DIVAS_OK) return st;
        if (!views[k].depth || !views[k].mask) return fail(c, DIVAS_E_INVALID, "depth or mask is NULL");
        if (views[k].mask_type < 0 || views[k].mask_type > 2)
            return fail(c, DIVAS_E_INVALID, "bad mask_type");
        vb.v[k] = make_view(views[k].cam, c->G, views[k].depth, views[k].mask,
                            views[k].mask_type, k);
        bp.gm[k] = grad_mask ? grad_mask[k] : nullptr;
        bp.gd[k] = grad_depth ? grad_depth[k] : nullptr;
    }
    const int blocks = grid_for(c->cap, c->sm_count);
    const int32_t dense = c->grid.kind == 0 ? 1 : 0;
    const int chunks = (n_views + kViewChunk - 1) / kViewChunk;
    cudaError_t e =
        c->G.contracted
            ? launch_backward_chunks<true>(chunks, blocks, S(stream), c->active, c->d_n, c->G,
                                           c->F, vb, bp, c->W, c->Z, grad_score, dense)
            : launch_backward_chunks<false>(chunks, blocks, S(stream), c->active, c->d_n, c->G,
                                            c->F, vb, bp, c->W, c->Z, grad_score, dense);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_backward");
    DIVAS_LAUNCHED(c, "k_backward");
    return DIVAS_OK;
}

divas_status divas_debug_project(divas_ctx* c, const divas_camera* cam, int32_t* pix_out,
                                 void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    divas_status st = check_camera(c, cam);
    if (st != DIVAS_OK) return st;
    if (!pix_out) return fail(c, DIVAS_E_INVALID, "pix_out is NULL");
    ViewC v = make_view(*cam, c->G, nullptr, nullptr, 0, 0);
    const int blocks = grid_for(c->cap, c->sm_count);
    if (c->G.contracted)
        k_debug_project<true><<<blocks, kThreads, 0, S(stream)>>>(c->active, c->d_n, c->G, c->F,
                                                                  v, pix_out);
    else
        k_debug_project<false><<<blocks, kThreads, 0, S(stream)>>>(c->active, c->d_n, c->G, c->F,
                                                                   v, pix_out);
    DIVAS_LAUNCHED(c, "k_debug_project");
    return DIVAS_OK;
}

divas_status divas_debug_rcp(const float* x, int64_t n, float* out_nr, float* out_ieee,
                             void* stream) {
    if (n < 0 || (n > 0 && (!x || !out_nr || !out_ieee))) return DIVAS_E_INVALID;
    if (n == 0) return DIVAS_OK;
    k_debug_rcp<<<(unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 4096), kThreads, 0,
                  S(stream)>>>(x, n, out_nr, out_ieee);
    return cudaGetLastError() == cudaSuccess ? DIVAS_OK : DIVAS_E_CUDA;
}

void divas_fuse_destroy(divas_ctx* c) {
    if (!c) return;
    free_all(c);
    (void)cudaGetLastError();  // teardown errors are not reported; do not leave them pending
    delete c;
}

const char* divas_last_error(const divas_ctx* c) {
    return c ? c->err.c_str() : g_init_error.c_str();
}

}  // extern "C"

// ===========================================================================
// Batched sessions: many contexts of uneven sizes and view counts in one
// persistent launch.  Work items are (session, tile of its active list);
// CTAs take items from a global counter (dynamic scheduling), stage the
// session's views in shared memory and fold them into kVPT voxels per thread.
// The per-vote arithmetic and the view order are those of the single-context
// kernels, so a session's result is bitwise the same alone or in a batch.
// ===========================================================================
namespace {

struct SessionDesc {
    const uint32_t* active;
    const int32_t* d_n;
    const float* W_in;
    const float* Z_in;
    const uint32_t* bits_in;
    float* W_out;
    float* Z_out;
    uint32_t* bits_out;
    GridC G;
    FuseC F;
    int32_t view_off, n_views, accumulate, dense;
    // brick-ordered session fused with culling: per brick, the views it may vote
    // in (null: every view)
    const uint32_t* brick_keep;
    // finalize / labels (filled at finalize time)
    float* score_out;
    uint32_t* seg_bits;
    const float* xyz;
    uint8_t* labels;
    int64_t n_pts;
};

// largest s with prefix[s] <= it (prefix[0] = 0, prefix[n] = total > it)
__device__ __forceinline__ int32_t find_session(const uint32_t* prefix, int32_t n, uint32_t it) {
    int32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= it) lo = mid; else hi = mid;
    }
    return lo;
}

// one CTA-wide work item: returns false when the work is exhausted
__device__ __forceinline__ bool next_item(int32_t* counter, const uint32_t* prefix, int32_t n,
                                          uint32_t& it, int32_t& sess) {
    __shared__ uint32_t s_it;
    __shared__ int32_t s_sess;
    __syncthreads();  // the previous item is done with shared state
    if (threadIdx.x == 0) {
        const uint32_t i = (uint32_t)atomicAdd(counter, 1);
        s_it = i;
        s_sess = i < __ldg(prefix + n) ? find_session(prefix, n, i) : -1;
    }
    __syncthreads();
    it = s_it;
    sess = s_sess;
    return sess >= 0;
}

template <bool kContracted, int kVPT>
__device__ __forceinline__ void batch_fuse_item(const SessionDesc& D, const ViewC* sv,
                                                int32_t a0, int32_t a1) {
    for (int32_t base = a0; base < a1; base += (int32_t)blockDim.x * kVPT) {
        VoxelGeom vg[kVPT];
        bool live[kVPT];
        float W[kVPT], Z[kVPT];
        uint32_t bits[kVPT];
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            const int32_t a = base + j * (int32_t)blockDim.x + (int32_t)threadIdx.x;
            live[j] = a < a1;
            const int32_t as = live[j] ? a : a0;
            vg[j] = voxel_geom<kContracted>(__ldg(D.active + as), D.G, D.F.gamma);
            W[j] = Z[j] = 0.f;
            bits[j] = 0u;
            if (D.accumulate && live[j]) {
                W[j] = D.W_in[a];
                Z[j] = D.Z_in[a];
                bits[j] = D.bits_in[a];
            }
        }
        fold_views_multi<kContracted, kVPT>(sv, D.n_views, vg, live, D.F, W, Z, bits);
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            const int32_t a = base + j * (int32_t)blockDim.x + (int32_t)threadIdx.x;
            if (live[j]) {
                D.W_out[a] = W[j];
                D.Z_out[a] = Z[j];
                D.bits_out[a] = bits[j];
            }
        }
    }
}

// a culled session's item: per group of 32 voxels the views some brick of
// theirs may vote in (the session's brick masks), folded in view order with
// the arithmetic of fold_views_multi (bitwise the full fold)
template <bool kContracted>
__device__ __forceinline__ void batch_fuse_item_cull(const SessionDesc& D, const ViewC* sv,
                                                     int32_t a0, int32_t a1) {
    const uint32_t nb = (uint32_t)D.G.g >> 3;
    for (int32_t base = a0; base < a1; base += (int32_t)blockDim.x) {
        const int32_t a = base + (int32_t)threadIdx.x;
        const bool live = a < a1;
        const uint32_t pk = __ldg(D.active + (live ? a : a0));
        // (no brick masks: every view)
        const uint32_t mine =
            !live ? 0u
            : D.brick_keep
                ? __ldg(D.brick_keep +
                        (((pk >> 23) * nb + ((pk >> 13) & 127u)) * nb + ((pk & 1023u) >> 3)))
                : 0xffffffffu;
        // only the session's views, whatever the masks hold
        const uint32_t keep = __reduce_or_sync(0xffffffffu, mine) &
                              (D.n_views >= 32 ? 0xffffffffu : (1u << D.n_views) - 1u);
        const VoxelGeom vg = voxel_geom<kContracted>(pk, D.G, D.F.gamma);
        if (!live) continue;
        float W = 0.f, Z = 0.f;
        uint32_t bits = 0u;
        if (D.accumulate) {
            W = D.W_in[a];
            Z = D.Z_in[a];
            bits = D.bits_in[a];
        }
        if (vg.ok) fold_views_kept<kContracted, -1>(sv, keep, vg, D.F, W, Z, bits);
        D.W_out[a] = W;
        D.Z_out[a] = Z;
        D.bits_out[a] = bits;
    }
}

// kCull: the work items are the culled sessions' (one voxel per thread), else
// the other sessions' (kVPT voxels per thread)
template <int kVPT, bool kCull = false>
__global__ void __launch_bounds__(kThreads) k_batch_fuse(const SessionDesc* __restrict__ S, int32_t n_sessions,
                             const uint32_t* __restrict__ prefix, const ViewC* __restrict__ views,
                             int32_t tile, int32_t* __restrict__ counter) {
    __shared__ __align__(16) ViewC sv[kMaxViews];  // read as 16-byte words by the culled fold
    uint32_t it;
    int32_t s;
    while (next_item(counter, prefix, n_sessions, it, s)) {
        const SessionDesc& D = S[s];
        const int32_t nv = D.n_views;
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(views + D.view_off);
            uint32_t* dst = reinterpret_cast<uint32_t*>(sv);
            const int32_t words = nv * (int32_t)(sizeof(ViewC) / 4);
            for (int32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
        }
        __syncthreads();
        const int32_t n = *D.d_n;
        const int32_t a0 = (int32_t)(it - __ldg(prefix + s)) * tile;
        const int32_t a1 = min(a0 + tile, n);
        if (a0 < a1) {
            if constexpr (kCull) {
                if (D.G.contracted)
                    batch_fuse_item_cull<true>(D, sv, a0, a1);
                else
                    batch_fuse_item_cull<false>(D, sv, a0, a1);
            } else {
                if (D.G.contracted)
                    batch_fuse_item<true, kVPT>(D, sv, a0, a1);
                else
                    batch_fuse_item<false, kVPT>(D, sv, a0, a1);
            }
        }
    }
}

// normalise + threshold for all sessions (score grids and seg bits zeroed before)
__global__ void __launch_bounds__(kThreads) k_batch_finalize(const SessionDesc* __restrict__ S,
                                                             int32_t n_sessions,
                                                             const uint32_t* __restrict__ prefix,
                                                             int32_t tile,
                                                             int32_t* __restrict__ counter) {
    uint32_t it;
    int32_t s;
    const int lane = threadIdx.x & 31;
    while (next_item(counter, prefix, n_sessions, it, s)) {
        const SessionDesc& D = S[s];
        const int32_t n = *D.d_n;
        const int32_t a0 = (int32_t)(it - __ldg(prefix + s)) * tile;
        const int32_t a1 = min(a0 + tile, n);
        for (int32_t base = a0 + (int32_t)(threadIdx.x & ~31u); base < a1;
             base += (int32_t)blockDim.x) {
            const int32_t a = base + lane;
            const bool live = a < a1;
            bool seg = false;
            int64_t lin = 0;
            if (live) {
                const float w = D.W_out[a], z = D.Z_out[a];
                const float p = z > D.F.eps ? __fdiv_rn(w, z) : 0.f;
                seg = p >= D.F.tau_cons;
                lin = packed_lin(__ldg(D.active + a), D.G.g);
                if (D.score_out) D.score_out[D.dense ? lin : (int64_t)a] = p;
            }
            seg_epilogue(live, seg, lin, D.seg_bits, true, nullptr, false);
        }
    }
}

// Pass 1 labels for all sessions (items over points)
__global__ void __launch_bounds__(kThreads) k_batch_label(const SessionDesc* __restrict__ S,
                                                          int32_t n_sessions,
                                                          const uint32_t* __restrict__ prefix,
                                                          int32_t tile,
                                                          int32_t* __restrict__ counter) {
    uint32_t it;
    int32_t s;
    while (next_item(counter, prefix, n_sessions, it, s)) {
        const SessionDesc& D = S[s];
        const int64_t p0 = (int64_t)(it - __ldg(prefix + s)) * tile;
        const int64_t p1 = min(p0 + tile, D.n_pts);
        for (int64_t a = p0 + threadIdx.x; a < p1; a += blockDim.x)
            D.labels[a] = label_one(D.xyz, a, D.G, D.seg_bits);
    }
}

}  // namespace

struct divas_batch {
    int32_t max_sessions = 0, max_views = 0;
    int32_t sm_count = 148;
    // double-buffered pinned staging: [sessions | views | 3 prefix arrays]
    unsigned char* h_stage[2] = {nullptr, nullptr};
    cudaEvent_t stage_done[2] = {nullptr, nullptr};
    int32_t cur = 0;
    size_t stage_bytes = 0, off_views = 0, off_prefix = 0;
    unsigned char* d_stage = nullptr;
    int32_t* d_counter = nullptr;
    // queue
    std::vector<divas_ctx*> ctxs;
    std::vector<int32_t> nq;
    int32_t views_used = 0;
    bool fused = false;
    // dry-run outputs
    float* dW = nullptr;
    float* dZ = nullptr;
    uint32_t* dbits = nullptr;
    int64_t dcap = 0;
    std::string err;
};

namespace {

divas_status bfail(divas_batch* b, divas_status st, const std::string& m) {
    if (b) b->err = m;
    return st;
}

SessionDesc* stage_sessions(divas_batch* b) {
    return reinterpret_cast<SessionDesc*>(b->h_stage[b->cur]);
}
ViewC* stage_views(divas_batch* b) {
    return reinterpret_cast<ViewC*>(b->h_stage[b->cur] + b->off_views);
}
uint32_t* stage_prefix(divas_batch* b, int which) {
    return reinterpret_cast<uint32_t*>(b->h_stage[b->cur] + b->off_prefix) +
           (size_t)which * (b->max_sessions + 1);
}

}  // namespace

extern "C" {

divas_status divas_batch_create(divas_batch** out, int32_t max_sessions, int32_t max_views) {
    if (!out || max_sessions < 1 || max_views < 1 || max_sessions > (1 << 20) ||
        max_views > (1 << 20))
        return fail(nullptr, DIVAS_E_INVALID, "bad batch limits");
    *out = nullptr;
    divas_batch* b = new (std::nothrow) divas_batch();
    if (!b) return fail(nullptr, DIVAS_E_OOM, "host allocation failed");
    b->max_sessions = max_sessions;
    b->max_views = max_views;
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    b->off_views = align(sizeof(SessionDesc) * max_sessions);
    b->off_prefix = b->off_views + align(sizeof(ViewC) * max_views);
    b->stage_bytes = b->off_prefix + align(sizeof(uint32_t) * 4 * (max_sessions + 1));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_stage[k]), b->stage_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->stage_done[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_stage, b->stage_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 16);
    if (e != cudaSuccess) {
        divas_batch_destroy(b);
        return cuda_fail(nullptr, e, "divas_batch_create");
    }
    b->ctxs.reserve(max_sessions);
    b->nq.reserve(max_sessions);
    *out = b;
    return DIVAS_OK;
}

divas_status divas_batch_queue(divas_batch* b, divas_ctx* c, const divas_view* views,
                               int32_t n_views) {
    if (!b || !c) return bfail(b, DIVAS_E_INVALID, "NULL batch or context");
    if (b->fused) return bfail(b, DIVAS_E_STATE, "finalize or clear the fused batch first");
    if (!views || n_views < 1 || n_views > kMaxViews)
        return bfail(b, DIVAS_E_INVALID, "n_views must be in 1..32");
    if ((int32_t)b->ctxs.size() >= b->max_sessions) return bfail(b, DIVAS_E_CAPACITY, "batch full");
    if (b->views_used + n_views > b->max_views) return bfail(b, DIVAS_E_CAPACITY, "too many views");
    for (divas_ctx* q : b->ctxs)
        if (q == c) return bfail(b, DIVAS_E_INVALID, "a context may appear once per batch");
    if (b->ctxs.empty()) {  // first entry: the staging buffer must be free again
        cudaError_t e = cudaEventSynchronize(b->stage_done[b->cur]);
        if (e != cudaSuccess) return bfail(b, DIVAS_E_CUDA, cudaGetErrorString(e));
    }
    ViewC* hv = stage_views(b) + b->views_used;
    for (int32_t k = 0; k < n_views; ++k) {
        divas_status st = check_camera(c, &views[k].cam);
        if (st != DIVAS_OK) return bfail(b, st, c->err);
        if (!views[k].depth || !views[k].mask || views[k].mask_type < 0 || views[k].mask_type > 2)
            return bfail(b, DIVAS_E_INVALID, "bad view");
        hv[k] = make_view(views[k].cam, c->G, views[k].depth, views[k].mask, views[k].mask_type,
                          c->n_views + k);
    }
    SessionDesc& D = stage_sessions(b)[b->ctxs.size()];
    memset(&D, 0, sizeof(D));
    D.active = c->active;
    D.d_n = c->d_n;
    D.W_in = D.W_out = c->W;
    D.Z_in = D.Z_out = c->Z;
    D.bits_in = D.bits_out = c->bits;
    D.G = c->G;
    D.F = c->F;
    D.view_off = b->views_used;
    D.n_views = n_views;
    D.accumulate = c->n_views > 0 ? 1 : 0;
    D.dense = c->grid.kind == 0 ? 1 : 0;
    D.seg_bits = c->seg_bits;
    b->ctxs.push_back(c);
    b->nq.push_back(n_views);
    b->views_used += n_views;
    return DIVAS_OK;
}

divas_status divas_batch_fuse(divas_batch* b, const divas_schedule* sched, int32_t dry_run,
                              void* stream) {
    if (!b || !sched) return bfail(b, DIVAS_E_INVALID, "NULL argument");
    if (b->fused) return bfail(b, DIVAS_E_STATE, "batch already fused");
    const int32_t ns = (int32_t)b->ctxs.size();
    if (ns == 0) return DIVAS_OK;
    const int vpt = sched->voxels_per_thread;
    if (!(sched->threads == 64 || sched->threads == 128 || sched->threads == 256) ||
        !(vpt == 1 || vpt == 2 || vpt == 4) || sched->ctas_per_sm < 1 || sched->ctas_per_sm > 32 ||
        sched->tile < sched->threads * vpt || sched->tile % (sched->threads * vpt) != 0)
        return bfail(b, DIVAS_E_INVALID, "bad schedule");
    cudaStream_t s = S(stream);
    SessionDesc* hs = stage_sessions(b);
    // brick-ordered sessions: their views' mask pyramids and bricks' kept views,
    // read by the culled fusion below
    const ViewC* hv = stage_views(b);
    // (an earlier copy of this staging buffer may still be pending on the stream
    // when the batch is fused again, e.g. repeated dry runs: each field is
    // written once, with its final value)
    for (int32_t k = 0; k < ns; ++k) {
        const divas_ctx* c = b->ctxs[k];
        const uint32_t* keep = nullptr;
        if (c->brick && hs[k].n_views >= 1 && hs[k].n_views <= kMaxViews) {
            ViewBatch vb;
            memset(&vb, 0, sizeof(vb));
            vb.n = hs[k].n_views;
            for (int32_t v = 0; v < vb.n; ++v) vb.v[v] = hv[hs[k].view_off + v];
            CullBatch cb;
            if (culling(c, vb, cb)) {
                cudaError_t ce = launch_pyramid(c, vb, cb, s);
                if (ce == cudaSuccess) ce = launch_brick_views(c, vb, s);
                if (ce != cudaSuccess) return bfail(b, DIVAS_E_CUDA, cudaGetErrorString(ce));
                keep = c->brick_keep;
            }
        }
        hs[k].brick_keep = keep;
    }
    // tile prefixes over capacities (the device count bounds the real work): the
    // culled sessions' items in prefix 3, the others' in prefix 0
    uint32_t* pf = stage_prefix(b, 0);
    uint32_t* pc = stage_prefix(b, 3);
    pf[0] = pc[0] = 0;
    int64_t total_cap = 0;
    for (int32_t k = 0; k < ns; ++k) {
        const int64_t cap = b->ctxs[k]->cap;
        const uint32_t tiles = (uint32_t)((cap + sched->tile - 1) / sched->tile);
        pf[k + 1] = pf[k] + (hs[k].brick_keep ? 0u : tiles);
        pc[k + 1] = pc[k] + (hs[k].brick_keep ? tiles : 0u);
        total_cap += cap;
    }
    if (dry_run) {  // outputs go to scratch: the contexts are left untouched
        if (total_cap > b->dcap) {
            if (b->dW) cudaFree(b->dW);
            if (b->dZ) cudaFree(b->dZ);
            if (b->dbits) cudaFree(b->dbits);
            b->dW = b->dZ = nullptr;
            b->dbits = nullptr;
            b->dcap = 0;
            cudaError_t e = cudaMalloc(&b->dW, total_cap * 4);
            if (e == cudaSuccess) e = cudaMalloc(&b->dZ, total_cap * 4);
            if (e == cudaSuccess) e = cudaMalloc(&b->dbits, total_cap * 4);
            if (e != cudaSuccess) return bfail(b, DIVAS_E_OOM, cudaGetErrorString(e));
            b->dcap = total_cap;
        }
        int64_t off = 0;
        for (int32_t k = 0; k < ns; ++k) {
            hs[k].W_out = b->dW + off;
            hs[k].Z_out = b->dZ + off;
            hs[k].bits_out = b->dbits + off;
            off += b->ctxs[k]->cap;
        }
    } else {
        for (int32_t k = 0; k < ns; ++k) {
            hs[k].W_out = b->ctxs[k]->W;
            hs[k].Z_out = b->ctxs[k]->Z;
            hs[k].bits_out = b->ctxs[k]->bits;
        }
    }
    // (under stream capture the copy node keeps reading this staging buffer on
    // every replay: the batch must not be reused while such a graph is alive)
    cudaError_t e = cudaMemcpyAsync(b->d_stage, b->h_stage[b->cur], b->stage_bytes,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !capturing(s)) e = cudaEventRecord(b->stage_done[b->cur], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, 16, s);
    if (e != cudaSuccess) return bfail(b, DIVAS_E_CUDA, cudaGetErrorString(e));
    const SessionDesc* dS = reinterpret_cast<const SessionDesc*>(b->d_stage);
    const ViewC* dV = reinterpret_cast<const ViewC*>(b->d_stage + b->off_views);
    const uint32_t* dP = reinterpret_cast<const uint32_t*>(b->d_stage + b->off_prefix);
    const uint32_t* dPc = dP + (size_t)3 * (b->max_sessions + 1);
    if (pf[ns] > 0) {
        const int grid = std::max(1, std::min<int>(b->sm_count * sched->ctas_per_sm, (int)pf[ns]));
        switch (vpt) {
            case 1: k_batch_fuse<1><<<grid, sched->threads, 0, s>>>(dS, ns, dP, dV, sched->tile, b->d_counter); break;
            case 2: k_batch_fuse<2><<<grid, sched->threads, 0, s>>>(dS, ns, dP, dV, sched->tile, b->d_counter); break;
            default: k_batch_fuse<4><<<grid, sched->threads, 0, s>>>(dS, ns, dP, dV, sched->tile, b->d_counter); break;
        }
    }
    if (pc[ns] > 0) {
        const int grid = std::max(1, std::min<int>(b->sm_count * sched->ctas_per_sm, (int)pc[ns]));
        k_batch_fuse<1, true><<<grid, sched->threads, 0, s>>>(dS, ns, dPc, dV, sched->tile,
                                                             b->d_counter + 3);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, DIVAS_E_CUDA, std::string("k_batch_fuse: ") + cudaGetErrorString(e));
    if (!dry_run) {
        for (int32_t k = 0; k < ns; ++k) b->ctxs[k]->n_views += b->nq[k];
        b->fused = true;
    }
    return DIVAS_OK;
}

divas_status divas_batch_finalize(divas_batch* b, float* const* score_out, const float* const* xyz,
                                  const int64_t* n_pts, uint8_t* const* labels_out, uint32_t flags,
                                  void* stream) {
    if (!b) return bfail(b, DIVAS_E_INVALID, "NULL batch");
    if (flags & ~(uint32_t)DIVAS_KEEP_ZEROS) return bfail(b, DIVAS_E_INVALID, "unknown flags");
    const bool keep = (flags & DIVAS_KEEP_ZEROS) != 0;
    const int32_t ns = (int32_t)b->ctxs.size();
    if (ns == 0) return DIVAS_OK;
    if (!b->fused) return bfail(b, DIVAS_E_STATE, "fuse the batch first (dry runs do not count)");
    cudaStream_t s = S(stream);
    SessionDesc* hs = stage_sessions(b);
    uint32_t* pf = stage_prefix(b, 1);
    uint32_t* pl = stage_prefix(b, 2);
    const int32_t tile = 4096;
    pf[0] = pl[0] = 0;
    bool any_pts = false;
    for (int32_t k = 0; k < ns; ++k) {
        divas_ctx* c = b->ctxs[k];
        hs[k].score_out = score_out ? score_out[k] : nullptr;
        hs[k].xyz = xyz ? xyz[k] : nullptr;
        hs[k].labels = labels_out ? labels_out[k] : nullptr;
        hs[k].n_pts = (xyz && n_pts && labels_out && xyz[k] && labels_out[k]) ? n_pts[k] : 0;
        if (hs[k].n_pts < 0) return bfail(b, DIVAS_E_INVALID, "negative point count");
        any_pts |= hs[k].n_pts > 0;
        pf[k + 1] = pf[k] + (uint32_t)((c->cap + tile - 1) / tile);
        pl[k + 1] = pl[k] + (uint32_t)((hs[k].n_pts + tile - 1) / tile);
        // the session's seg bitfield is set and cleared in place (it never
        // holds a bit of an unoccupied voxel); a dense score grid is zeroed
        // unless the caller keeps its zeros
        if (hs[k].score_out && c->grid.kind == 0 && !keep) {
            const cudaError_t e = cudaMemsetAsync(hs[k].score_out, 0, c->n_cells * 4, s);
            if (e != cudaSuccess) return bfail(b, DIVAS_E_CUDA, cudaGetErrorString(e));
        }
    }
    // the staging buffer is the one of the fuse call; the copy orders after it on the stream
    cudaError_t e = cudaMemcpyAsync(b->d_stage, b->h_stage[b->cur], b->stage_bytes,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !capturing(s)) e = cudaEventRecord(b->stage_done[b->cur], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, 16, s);
    if (e != cudaSuccess) return bfail(b, DIVAS_E_CUDA, cudaGetErrorString(e));
    const SessionDesc* dS = reinterpret_cast<const SessionDesc*>(b->d_stage);
    const uint32_t* dPf = reinterpret_cast<const uint32_t*>(b->d_stage + b->off_prefix) +
                          (size_t)(b->max_sessions + 1);
    const uint32_t* dPl = dPf + (size_t)(b->max_sessions + 1);
    int grid = std::max(1, std::min<int>(b->sm_count * 8, (int)pf[ns]));
    k_batch_finalize<<<grid, kThreads, 0, s>>>(dS, ns, dPf, tile, b->d_counter + 1);
    e = cudaGetLastError();
    if (e == cudaSuccess && any_pts) {
        grid = std::max(1, std::min<int>(b->sm_count * 8, (int)pl[ns]));
        k_batch_label<<<grid, kThreads, 0, s>>>(dS, ns, dPl, tile, b->d_counter + 2);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bfail(b, DIVAS_E_CUDA, cudaGetErrorString(e));
    return divas_batch_clear(b);
}

divas_status divas_batch_clear(divas_batch* b) {
    if (!b) return DIVAS_E_INVALID;
    b->ctxs.clear();
    b->nq.clear();
    b->views_used = 0;
    b->fused = false;
    b->cur ^= 1;  // the next batch stages into the other buffer
    return DIVAS_OK;
}

int32_t divas_batch_size(const divas_batch* b) { return b ? (int32_t)b->ctxs.size() : -1; }

const char* divas_batch_last_error(const divas_batch* b) { return b ? b->err.c_str() : ""; }

void divas_batch_destroy(divas_batch* b) {
    if (!b) return;
    for (int k = 0; k < 2; ++k) {
        if (b->stage_done[k]) {
            cudaEventSynchronize(b->stage_done[k]);
            cudaEventDestroy(b->stage_done[k]);
        }
        if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
    }
    if (b->d_stage) cudaFree(b->d_stage);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->dW) cudaFree(b->dW);
    if (b->dZ) cudaFree(b->dZ);
    if (b->dbits) cudaFree(b->dbits);
    (void)cudaGetLastError();  // teardown errors are not reported; do not leave them pending
    delete b;
}

}  // extern "C"

// depth-tuple mode (thick gates on the depth tuple + thin footprint path)
#include "tuple_mode.cuh"
#include "weighting.cuh"
#include "occupancy.cuh"
#include "surfels.cuh"
// the NeRF variant of the depth-tuple mode
#include "nerf_mode.cuh"

// ===========================================================================
// Allocation-free one-shot fusion (no counterpart in the paper)
//
// Some callers must not allocate device memory while they run: a plug-in
// invoked once per frame inside a host application that owns all GPU memory
// (where cudaMalloc would synchronise the device and stall the frame), or code
// running under a strict no-allocation policy between frames.  For them,
// divas_fuse_dense_noalloc runs the whole dense pipeline -- occupancy gate and
// active list, fusion of the views, normalisation and consensus -- with its
// scratch in one file-scope device array instead of context memory.
//
// The array holds grids of up to 64^3 cells and is reserved on every GPU that
// loads this library until the process exits (about 4.3 MB).  All calls share
// it and it keeps the previous call's contents, so every part that must start
// at zero is cleared by the call itself; calls that overlap on the GPU (two
// streams, or two host threads) race on it.  The first call on a device looks
// up the array's device address with cudaGetSymbolAddress, once per device and
// with that device current; make that first call before any stream capture.
// ===========================================================================
namespace {

constexpr int64_t kNoAllocMaxCells = 1 << 18;  // 64^3
constexpr int64_t kNoAllocWords = kNoAllocMaxCells / 32;
constexpr int64_t kNoAllocTiles = (kNoAllocWords + kTileSpan - 1) / kTileSpan;

constexpr int64_t na_align(int64_t x) { return (x + 255) / 256 * 256; }
constexpr int64_t kNaOccBits = 0;
constexpr int64_t kNaSeg = kNaOccBits + na_align(kNoAllocWords * 4);
constexpr int64_t kNaItemPref = kNaSeg + na_align(kNoAllocWords * 4);
constexpr int64_t kNaTileCount = kNaItemPref + na_align(kNoAllocTiles * kTileItems * 4);
constexpr int64_t kNaTileOffset = kNaTileCount + na_align(kNoAllocTiles * 4);
constexpr int64_t kNaDone = kNaTileOffset + na_align(kNoAllocTiles * 4);
constexpr int64_t kNaActive = kNaDone + 256;
constexpr int64_t kNaW = kNaActive + na_align(kNoAllocMaxCells * 4);
constexpr int64_t kNaZ = kNaW + na_align(kNoAllocMaxCells * 4);
constexpr int64_t kNaBits = kNaZ + na_align(kNoAllocMaxCells * 4);
constexpr int64_t kNaN = kNaBits + na_align(kNoAllocMaxCells * 4);
constexpr int64_t kNaStatus = kNaN + 256;
constexpr int64_t kNaTotal = kNaStatus + 256;
constexpr int64_t kNoAllocBytes = kNaTotal + 256;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_dev_ptr[256] = {nullptr};
thread_local std::string g_noalloc_error;  // per host thread, like the init error

divas_status noalloc_fail(divas_status st, const std::string& msg) {
    g_noalloc_error = msg;
    return st;
}

}  // namespace

extern "C" divas_status divas_fuse_dense_noalloc(const divas_grid* grid, const uint8_t* occ_dense,
                                                 const divas_view* views, int32_t n_views,
                                                 const divas_params* params, float* score_out,
                                                 uint32_t* seg_bits_out, void* stream) {
    if (!grid || !params || !occ_dense || !views)
        return noalloc_fail(DIVAS_E_INVALID, "NULL argument");
    if (grid->kind != 0 || grid->contracted)
        return noalloc_fail(DIVAS_E_INVALID, "only plain dense grids (kind 0, not contracted)");
    // the side is bounded before any product of it is formed
    if (grid->g < 1 || grid->g > 64)
        return noalloc_fail(DIVAS_E_INVALID,
                            "grid too large for the allocation-free path (at most 64^3 cells)");
    if (const char* why = grid_problem(grid, 64)) return noalloc_fail(DIVAS_E_INVALID, why);
    if (n_views < 1 || n_views > kMaxViews)
        return noalloc_fail(DIVAS_E_INVALID, "n_views must be in 1..32");
    if (const char* why = params_problem(params)) return noalloc_fail(DIVAS_E_INVALID, why);
    if (params->flags & DIVAS_ORDER_BRICKS)
        return noalloc_fail(DIVAS_E_INVALID, "brick order needs a sparse prior");
    for (int32_t k = 0; k < n_views; ++k) {
        if (const char* why = camera_problem(&views[k].cam))
            return noalloc_fail(DIVAS_E_INVALID, why);
        if (!views[k].depth || !views[k].mask || views[k].mask_type < 0 || views[k].mask_type > 2)
            return noalloc_fail(DIVAS_E_INVALID, "bad view");
    }
    cudaStream_t s = S(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256)
        return noalloc_fail(DIVAS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_dev_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return noalloc_fail(DIVAS_E_CUDA,
                                    std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_dev_ptr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_noalloc_dev_ptr[dev]);
    }
    uint32_t* occ_bits = reinterpret_cast<uint32_t*>(base + kNaOccBits);
    uint32_t* seg_bits = reinterpret_cast<uint32_t*>(base + kNaSeg);
    uint32_t* item_pref = reinterpret_cast<uint32_t*>(base + kNaItemPref);
    uint32_t* tile_count = reinterpret_cast<uint32_t*>(base + kNaTileCount);
    uint32_t* tile_offset = reinterpret_cast<uint32_t*>(base + kNaTileOffset);
    uint32_t* done = reinterpret_cast<uint32_t*>(base + kNaDone);
    uint32_t* active = reinterpret_cast<uint32_t*>(base + kNaActive);
    float* W = reinterpret_cast<float*>(base + kNaW);
    float* Z = reinterpret_cast<float*>(base + kNaZ);
    uint32_t* bits = reinterpret_cast<uint32_t*>(base + kNaBits);
    int32_t* d_n = reinterpret_cast<int32_t*>(base + kNaN);
    int32_t* d_status = reinterpret_cast<int32_t*>(base + kNaStatus);
    int64_t* d_total = reinterpret_cast<int64_t*>(base + kNaTotal);

    GridC G;
    for (int q = 0; q < 3; ++q) G.origin[q] = grid->origin[q];
    G.h = grid->h;
    G.g = grid->g;
    G.contracted = 0;
    {
        int ex = 0;
        const double fr = frexp((double)grid->h, &ex);
        G.inv_h = fr == 0.5 ? (float)ldexp(1.0, 1 - ex) : 0.f;
        G.pad = 0;
    }
    FuseC F;
    F.gamma = params->gamma;
    F.alpha1 = params->alpha1;
    F.tau_m = params->tau_mask;
    F.logit_tau = logit_threshold(params->tau_mask);
    F.z_near = params->z_near;
    F.eps = params->eps;
    F.tau_cons = params->tau_cons;
    F.pad = 0;
    set_tolerances(G, F.gamma);
    FastDiv gdiv;
    {
        const uint32_t d = (uint32_t)grid->g;
        int32_t l = 0;
        while ((1ull << l) < d) ++l;
        gdiv.d = d;
        gdiv.l = l;
        gdiv.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
        gdiv.pad = 0;
    }
    ViewBatch vb;
    memset(&vb, 0, sizeof(vb));
    vb.n = n_views;
    for (int32_t k = 0; k < n_views; ++k)
        vb.v[k] = make_view(views[k].cam, G, views[k].depth, views[k].mask, views[k].mask_type, k);
    const int64_t n_cells = (int64_t)grid->g * grid->g * grid->g;
    const int64_t n_words = (n_cells + 31) / 32;
    const int32_t n_tiles = (int32_t)((n_words + kTileSpan - 1) / kTileSpan);
    const int64_t cap = kNoAllocMaxCells;
    int sm_count = 148;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
#define NA_CHECK(what)                                                                \
    do {                                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess)                                                        \
            return noalloc_fail(DIVAS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    // state that must start at zero on every call
    e = cudaMemsetAsync(d_status, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(done, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(seg_bits, 0, n_words * 4, s);
    if (e == cudaSuccess && score_out) e = cudaMemsetAsync(score_out, 0, n_cells * 4, s);
    if (e == cudaSuccess && seg_bits_out) e = cudaMemsetAsync(seg_bits_out, 0, n_words * 4, s);
    if (e != cudaSuccess)
        return noalloc_fail(DIVAS_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_tile_count<0><<<n_tiles, kThreads, 0, s>>>(occ_dense, occ_bits, n_cells, n_words, cap,
                                                     item_pref, tile_count, tile_offset, done,
                                                     n_tiles, d_n, d_total, d_status, grid->g,
                                                     gdiv, nullptr);
    NA_CHECK("k_tile_count");
    k_tile_emit<false><<<emit_blocks(n_words, sm_count), kThreads, 0, s>>>(
        occ_bits, n_words, cap, gdiv, item_pref, tile_offset, active, nullptr, nullptr);
    NA_CHECK("k_tile_emit");
    const int blocks = grid_for(n_cells, sm_count);
    e = launch_fuse_chunks<false, false>((n_views + kViewChunk - 1) / kViewChunk, blocks, s,
                                         active, d_n, G, F, vb, W, Z, bits);
    if (e != cudaSuccess)
        return noalloc_fail(DIVAS_E_CUDA, std::string("k_fuse: ") + cudaGetErrorString(e));
    k_finalize<<<grid_for(n_cells, sm_count, 16), kThreads, 0, s>>>(
        active, d_n, grid->g, 1, W, Z, bits, F.eps, F.tau_cons, score_out, seg_bits, seg_bits_out,
        nullptr, nullptr);
    NA_CHECK("k_finalize");
#undef NA_CHECK
    return DIVAS_OK;
}

extern "C" const char* divas_noalloc_last_error(void) { return g_noalloc_error.c_str(); }
