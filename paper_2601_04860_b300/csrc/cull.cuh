// cull.cuh -- warp-level view culling for brick-ordered active lists.
//
// With the active list in brick-major order the 32 voxels of a warp lie in one
// or a few neighbouring 8^3 bricks, so their projections into a view cover a
// small screen rectangle.  A view can vote for none of them when every pixel
// of that rectangle fails the mask gate (raw < threshold): the fusion then
// skips the view for the whole warp -- projection, raster loads and gates --
// and, since a skipped view would have added nothing to any of the warp's
// voxels, every result is bitwise the one without culling.
//
// The rectangle: the warp's voxel centres (in the coordinates the projection
// rows take: uncontracted world positions on contracted grids, lattice
// coordinates n = 2 idx + 1 on plain grids) span an axis-aligned box; with
// the whole box in front of the camera, u = (K_u . x + T_u) / (R_z . x + t_z)
// is linear-fractional with a positive denominator there, so its extremes
// over the box are at the box's 8 corners (likewise v).  The corners are
// projected in FP32.  A projection's FP32 error (three-FMA rows, a reciprocal
// within an ulp, a product) is below 2^-22 ((S_u + |u| S_z) / p_z + |u|),
// with S_u = sum_j |K_uj x_j| + |T_u| <= sum_j |K_uj| max_j |x_j| + |T_u| over
// the box (likewise S_z; the sums per view from the host, rounded up).  The
// rectangle is widened by
// 2 pixels plus 2^-18 ((S_u + |u| S_z) / p_z,min + |u|) -- 16 times both
// the corners' and the voxels' error bounds -- and a box whose nearest corner
// is within 2^-18 S_z of the camera plane keeps the view.
//
// The mask test: a max pyramid of the raw mask values (levels 3..6: texels of
// 8..64 pixels), built per batch of views; a rectangle of span s pixels is
// covered by at most 5 x 5 texels of level max(3, ceil(log2 s) - 2); spans
// above 256 pixels keep the view.  The maximum below the gate threshold (NaN
// pixels never pass the gate and never raise the maximum) culls the view.
#pragma once

#include <cstdint>

#include "fuse_math.cuh"

namespace divas {

constexpr int kPyrL0 = 3;       // finest pyramid level (8-pixel texels)
constexpr int kPyrLevels = 4;   // levels 3..6
constexpr int kPyrTile = 64;    // pixels per side of a level-6 texel (one CTA)
constexpr int kCullTexels = 5;  // pyramid texels per side that one brick test reads

// per view: the gate threshold, the raster size and the pyramid's layout
struct CullC {
    float thr;        // the mask gate passes iff raw >= thr
    float su, sv, sz; // sum_j |row_j| of the u, v and depth rows (rounded up)
    float cu, cv, cz; // |constant| of each row
    int32_t W, H;
    int32_t off[kPyrLevels];  // offset of level kPyrL0 + l in the pyramid buffer (floats)
    int32_t lw[kPyrLevels];   // texels per row / column of that level
    int32_t lh[kPyrLevels];
};

struct CullBatch {
    float* pyr;
    int32_t n;
    int32_t pad;
    CullC v[kMaxViews];
};

// order-preserving map of floats to signed ints (an involution)
__device__ __forceinline__ int32_t ordered_key(float x) {
    const int32_t b = __float_as_int(x);
    return b ^ ((b >> 31) & 0x7fffffff);
}

__device__ __forceinline__ float from_ordered_key(int32_t k) {
    return __int_as_float(k ^ ((k >> 31) & 0x7fffffff));
}

// per-view constants the brick test reads with a lane-varying view index,
// written to global memory by the pyramid kernel (one CTA per view)
struct CullView {
    float r[12];  // rows u (0..2), v (3..5), z (6..8) and constants (9..11)
    CullC c;
};

// Max pyramid, levels 3..6, of one 64 x 64 pixel tile of one view per CTA
// (grid: tiles x, tiles y, views; 256 threads).  Thread t reads column
// t & 63 of rows 16 (t >> 6) .. + 15 (coalesced along rows), takes the max of
// each 8 rows, then of 8 neighbouring columns (lanes); the higher levels
// reduce in shared memory.  Pixels outside the raster count as -inf.
//
// It reads the masks only, so it runs while its predecessor on the stream
// finishes; it waits for that kernel before it ends, so that a kernel waiting
// for this one has also waited for the one before.
__global__ void __launch_bounds__(256) k_mask_pyramid(const __grid_constant__ ViewBatch VB,
                                                      const __grid_constant__ CullBatch CB,
                                                      CullView* __restrict__ views_out,
                                                      ViewC* __restrict__ fold_out) {
    __shared__ float l3[8][8];
    allow_dependents();
    const int v = blockIdx.z;
    const ViewC& V = VB.v[v];
    const CullC& C = CB.v[v];
    const int t = threadIdx.x, lane = t & 31;
    if (blockIdx.x == 0 && blockIdx.y == 0 && t == 0) {
        CullView cv;
#pragma unroll
        for (int k = 0; k < 9; ++k) cv.r[k] = V.A[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) cv.r[9 + k] = V.C[k];
        cv.c = C;
        views_out[v] = cv;
        fold_out[v] = V;
    }
    const int x = blockIdx.x * kPyrTile + (t & 63);
    const int yb = blockIdx.y * kPyrTile + 16 * (t >> 6);
    // all 16 loads first, unconditional at clamped coordinates (the mask type
    // is uniform), then the maxima over the pixels inside the raster
    const int W = V.W, H = V.H;
    const int xc = min(x, W - 1);
    const bool xin = x < W;
    float val[16];
    if (V.mask_type == kMaskF16) {
        const unsigned short* mp = reinterpret_cast<const unsigned short*>(V.mask) + xc;
        unsigned short u[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) u[r] = __ldg(mp + min(yb + r, H - 1) * W);
#pragma unroll
        for (int r = 0; r < 16; ++r) val[r] = __half2float(__ushort_as_half(u[r]));
    } else {
        const float* mp = reinterpret_cast<const float*>(V.mask) + xc;
#pragma unroll
        for (int r = 0; r < 16; ++r) val[r] = __ldg(mp + min(yb + r, H - 1) * W);
    }
    float m[2] = {-INFINITY, -INFINITY};
#pragma unroll
    for (int r = 0; r < 16; ++r)
        if (xin && yb + r < H) m[r >> 3] = fmaxf(m[r >> 3], val[r]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float a = m[h];
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 1));
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 2));
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 4));
        if ((lane & 7) == 0) l3[2 * (t >> 6) + h][(t & 63) >> 3] = a;
    }
    __syncthreads();
    float* pyr = CB.pyr;
    // level 3: 8 x 8 texels of this tile
    if (t < 64) {
        const int tx = blockIdx.x * 8 + (t & 7), ty = blockIdx.y * 8 + (t >> 3);
        if (tx < C.lw[0] && ty < C.lh[0]) pyr[C.off[0] + ty * C.lw[0] + tx] = l3[t >> 3][t & 7];
    }
    // levels 4, 5, 6: 4 x 4, 2 x 2, 1 x 1 texels
    if (t < 16) {
        const int i = t & 3, j = t >> 2;
        const float a = fmaxf(fmaxf(l3[2 * j][2 * i], l3[2 * j][2 * i + 1]),
                              fmaxf(l3[2 * j + 1][2 * i], l3[2 * j + 1][2 * i + 1]));
        const int tx = blockIdx.x * 4 + i, ty = blockIdx.y * 4 + j;
        if (tx < C.lw[1] && ty < C.lh[1]) pyr[C.off[1] + ty * C.lw[1] + tx] = a;
        // 2 x 2 from the 4 x 4 held by lanes 0..15 (lane = 4 j + i)
        float b = fmaxf(a, __shfl_xor_sync(0x0000ffffu, a, 1));
        b = fmaxf(b, __shfl_xor_sync(0x0000ffffu, b, 4));
        if ((i & 1) == 0 && (j & 1) == 0) {
            const int ux = blockIdx.x * 2 + (i >> 1), uy = blockIdx.y * 2 + (j >> 1);
            if (ux < C.lw[2] && uy < C.lh[2]) pyr[C.off[2] + uy * C.lw[2] + ux] = b;
        }
        float c = fmaxf(b, __shfl_xor_sync(0x0000ffffu, b, 2));
        c = fmaxf(c, __shfl_xor_sync(0x0000ffffu, c, 8));
        if (t == 0) pyr[C.off[3] + blockIdx.y * C.lw[3] + blockIdx.x] = c;
    }
    wait_for_producer();
}

// Whether view V can see a voxel centre of the box [lo, hi] (projection
// coordinates) in a pixel that passes its mask gate: false only when every
// centre of the box is certain to project outside the raster or onto pixels
// whose pyramid maximum is below the gate threshold.  One lane, eight corners.
__device__ __forceinline__ bool box_may_vote(const CullView& cv, const float* pyr,
                                             const float* lo, const float* hi) {
    const float* r = cv.r;
    const CullC& C = cv.c;
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    float zmin = INFINITY, xm = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) xm = fmaxf(xm, fmaxf(fabsf(lo[a]), fabsf(hi[a])));
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const float x0 = (corner & 1) ? hi[0] : lo[0];
        const float x1 = (corner & 2) ? hi[1] : lo[1];
        const float x2 = (corner & 4) ? hi[2] : lo[2];
        const float pz = __fmaf_rn(r[6], x0, __fmaf_rn(r[7], x1, __fmaf_rn(r[8], x2, r[11])));
        const float pu = __fmaf_rn(r[0], x0, __fmaf_rn(r[1], x1, __fmaf_rn(r[2], x2, r[9])));
        const float pv = __fmaf_rn(r[3], x0, __fmaf_rn(r[4], x1, __fmaf_rn(r[5], x2, r[10])));
        zmin = fminf(zmin, pz);
        const float inv = rcp_nr(pz);
        const float u = __fmul_rn(pu, inv), w = __fmul_rn(pv, inv);
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        vmin = fminf(vmin, w);
        vmax = fmaxf(vmax, w);
    }
    // S of each row over the box: sum_j |row_j| max_j |x_j| + |constant|
    const float sz = __fmaf_ru(C.sz, xm, C.cz);
    if (!(zmin > 0x1p-18f * sz)) return true;  // the box reaches too close to the camera plane
    const float su = __fmaf_ru(C.su, xm, C.cu), sv = __fmaf_ru(C.sv, xm, C.cv);
    const float au = fmaxf(fabsf(umin), fabsf(umax));
    const float av = fmaxf(fabsf(vmin), fabsf(vmax));
    // 1 / zmin within an ulp, taken up by one ulp more
    const float iz = __fmul_ru(rcp_nr(zmin), 1.f + 0x1p-22f);
    const float mu = __fmaf_ru(0x1p-18f, __fmaf_ru(__fmaf_ru(au, sz, su), iz, au), 2.f);
    const float mv = __fmaf_ru(0x1p-18f, __fmaf_ru(__fmaf_ru(av, sz, sv), iz, av), 2.f);
    const float fu0 = umin - mu, fu1 = umax + mu, fv0 = vmin - mv, fv1 = vmax + mv;
    if (!(fu0 <= fu1 && fv0 <= fv1)) return true;  // NaN: no bound
    if (fu1 < 0.f || fv1 < 0.f || fu0 >= (float)C.W || fv0 >= (float)C.H) return false;
    const int32_t iu0 = (int32_t)floorf(fmaxf(fu0, 0.f));
    const int32_t iu1 = (int32_t)floorf(fminf(fu1, (float)(C.W - 1)));
    const int32_t iv0 = (int32_t)floorf(fmaxf(fv0, 0.f));
    const int32_t iv1 = (int32_t)floorf(fminf(fv1, (float)(C.H - 1)));
    const int32_t span = max(iu1 - iu0, iv1 - iv0) + 1;
    // level: texels of at least span / 4 pixels, so the rectangle meets at most
    // kCullTexels of them per side
    const int32_t L = max(kPyrL0, (32 - __clz(span - 1)) - 2);
    if (L >= kPyrL0 + kPyrLevels) return true;  // too wide for the pyramid
    // the texels of the rectangle; indices past it are clamped to it (repeated
    // texels do not change the maximum), so that all loads are issued before
    // the first is used
    const float* lev = pyr + C.off[L - kPyrL0];
    const int32_t lw = C.lw[L - kPyrL0];
    const int32_t tx0 = iu0 >> L, tx1 = iu1 >> L, ty0 = iv0 >> L, ty1 = iv1 >> L;
    int32_t xs[kCullTexels], ys[kCullTexels];
#pragma unroll
    for (int a = 0; a < kCullTexels; ++a) {
        xs[a] = min(tx0 + a, tx1);
        ys[a] = min(ty0 + a, ty1);
    }
    float t[kCullTexels * kCullTexels];
#pragma unroll
    for (int a = 0; a < kCullTexels; ++a)
#pragma unroll
        for (int b = 0; b < kCullTexels; ++b) t[kCullTexels * a + b] = __ldg(lev + ys[a] * lw + xs[b]);
    float mx = -INFINITY;
#pragma unroll
    for (int a = 0; a < kCullTexels * kCullTexels; ++a) mx = fmaxf(mx, t[a]);
    return mx >= C.thr;
}

// The voxel centres of brick (bi, bj, bk) (8^3 cells) as a box in projection
// coordinates: lattice coordinates n = 2 idx + 1 on plain grids (exact); on
// contracted grids, the contracted box of centres mapped by x = c s(|c|) with
// s(rho) = 1 for rho <= 1 and 1 / (rho (2 - rho)) above (increasing in rho),
// so x lies in the interval product of c's box and [s(rho_min), s(rho_max)].
// FP32 with directed rounding (each bound rounded outwards), then widened by
// 2^-18 of its magnitude to hold the FP32 centres of the voxels.  False when
// the box reaches |c| >= 2 (no bound on the world positions).
__device__ __forceinline__ bool brick_box(uint32_t bi, uint32_t bj, uint32_t bk, const GridC& G,
                                          float* lo, float* hi) {
    const uint32_t b3[3] = {bi, bj, bk};
    if (!G.contracted) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = (float)(16 * b3[a] + 1);
            hi[a] = (float)(16 * b3[a] + 15);
        }
        return true;
    }
    float clo[3], chi[3], r2min = 0.f, r2max = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        clo[a] = __fmaf_rd((float)(8 * b3[a]) + 0.5f, G.h, G.origin[a]);
        chi[a] = __fmaf_ru((float)(8 * b3[a]) + 7.5f, G.h, G.origin[a]);
        const float near = clo[a] > 0.f ? clo[a] : (chi[a] < 0.f ? -chi[a] : 0.f);
        const float far = fmaxf(fabsf(clo[a]), fabsf(chi[a]));
        r2min = __fmaf_rd(near, near, r2min);
        r2max = __fmaf_ru(far, far, r2max);
    }
    const float rmin = __fsqrt_rd(r2min), rmax = __fsqrt_ru(r2max);
    if (!(rmax < 2.f)) return false;
    // s(rmin) rounded down, s(rmax) rounded up
    const float smin = rmin <= 1.f ? 1.f : __frcp_rd(__fmul_ru(rmin, __fsub_ru(2.f, rmin)));
    const float smax = rmax <= 1.f ? 1.f : __frcp_ru(__fmul_rd(rmax, __fsub_rd(2.f, rmax)));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float l = fminf(fminf(__fmul_rd(clo[a], smin), __fmul_rd(clo[a], smax)),
                              fminf(__fmul_rd(chi[a], smin), __fmul_rd(chi[a], smax)));
        const float h = fmaxf(fmaxf(__fmul_ru(clo[a], smin), __fmul_ru(clo[a], smax)),
                              fmaxf(__fmul_ru(chi[a], smin), __fmul_ru(chi[a], smax)));
        const float slack = __fmaf_ru(0x1p-18f, fmaxf(fabsf(l), fabsf(h)), 0x1p-100f);
        lo[a] = __fsub_rd(l, slack);
        hi[a] = __fadd_ru(h, slack);
    }
    return true;
}

// Per brick, the views (bit v) that some voxel of the brick may vote in; bricks
// without an occupied cell (brick-major occupancy words all zero) get 0.  A
// warp takes P = min(8, 32 / n) bricks at a time, lane l testing view l % n of
// brick l / n.  Reads the compaction's bitfield, the pyramids and the views'
// constants: launched after the pyramid kernel (as its programmatic dependent,
// or in plain stream order on a branch that has waited for the bitfield), it
// waits for its predecessor before any read.
__global__ void __launch_bounds__(256) k_brick_views(const CullView* __restrict__ sv, int32_t n,
                                                     const float* __restrict__ pyr, GridC G,
                                                     FastDiv bdiv,
                                                     const uint32_t* __restrict__ occ_bits,
                                                     int64_t n_bricks,
                                                     uint32_t* __restrict__ brick_keep) {
    wait_for_producer();  // the views' constants and the pyramids
    allow_dependents();
    const int lane = threadIdx.x & 31;
    const int P = min(8, 32 / n);
    const int slot = lane / n, view = lane - slot * n;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * P; b0 < n_bricks;
         b0 += n_warps * P) {
        // occupancy of the P bricks: lane l reads word l & 15 of brick 2 k + (l >> 4)
        uint32_t occupied = 0u;  // bit p: brick b0 + p holds an occupied cell
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t b = b0 + 2 * k + (lane >> 4);
            const uint32_t wv = (2 * k + (lane >> 4) < P && b < n_bricks)
                                    ? __ldg(occ_bits + b * 16 + (lane & 15)) : 0u;
            const uint32_t m = __ballot_sync(0xffffffffu, wv != 0u);
            occupied |= ((m & 0xffffu) ? 1u : 0u) << (2 * k);
            occupied |= ((m >> 16) ? 1u : 0u) << (2 * k + 1);
        }
        const int64_t b = b0 + slot;
        bool vote = false;
        if (slot < P && b < n_bricks && ((occupied >> slot) & 1u)) {
            const uint32_t r = fast_div((uint32_t)b, bdiv), bk = fast_div(r, bdiv);
            const uint32_t bi = (uint32_t)b - r * bdiv.d, bj = r - bk * bdiv.d;
            float lo[3], hi[3];
            vote = !brick_box(bi, bj, bk, G, lo, hi) || box_may_vote(sv[view], pyr, lo, hi);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, vote);
        if (view == 0 && slot < P && b < n_bricks)
            brick_keep[b] = n == 32 ? m : (m >> (slot * n)) & ((1u << n) - 1u);
    }
}

// A view's constants from a shared-memory copy of the batch (16-byte aligned):
// seven 16-byte loads with a warp-uniform address.
__device__ __forceinline__ ViewC view_from_shared(const ViewC* sv, int32_t v) {
    const uint4* p = reinterpret_cast<const uint4*>(sv + v);
    union {
        uint4 w[sizeof(ViewC) / 16];
        ViewC V;
    } u;
#pragma unroll
    for (int k = 0; k < (int)(sizeof(ViewC) / 16); ++k) u.w[k] = p[k];
    return u.V;
}

// Fold the views of `keep` (ascending view order, four at a time: the same
// per-view arithmetic and order as fold_views over all views, which it matches
// bitwise when the skipped views vote nowhere).  The view index is
// warp-uniform; the views' constants come from the CTA's shared-memory copy
// of the batch.
template <bool kContracted, int kMT>
__device__ __forceinline__ void fold_views_kept(const ViewC* sv, uint32_t keep,
                                                const VoxelGeom& vg, const FuseC& F, float& W,
                                                float& Z, uint32_t& bits) {
    static_assert(sizeof(ViewC) % 16 == 0, "views copy as 16-byte words");
    uint32_t rem = keep;
    while (rem) {
        int32_t vi[kViewChunk];
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q) {
            vi[q] = rem ? __ffs(rem) - 1 : -1;
            rem &= rem - 1u;
        }
        int32_t pix[kViewChunk];
        float pzh[kViewChunk], pzl[kViewChunk], D[kViewChunk], raw[kViewChunk];
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q) {
            pix[q] = -1;
            pzh[q] = pzl[q] = 0.f;
            if (vi[q] >= 0) {
                const ViewC V = view_from_shared(sv, vi[q]);
                pix[q] = project<kContracted>(V, vg, F.z_near, pzh[q], pzl[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q)
            if (vi[q] >= 0) {
                const ViewC V = view_from_shared(sv, vi[q]);
                load_raster<kMT>(V, pix[q], D[q], raw[q]);
            }
        uint32_t acc = 0u;
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q) {
            if (vi[q] < 0) break;
            const ViewC V = view_from_shared(sv, vi[q]);
            if (pre_gates<kContracted, kMT>(V, vg, F, pix[q], pzh[q], D[q], raw[q])) acc |= 1u << q;
        }
        if (acc) {
#pragma unroll
            for (int q = 0; q < kViewChunk; ++q) {
                if (acc & (1u << q)) {
                    const ViewC V = view_from_shared(sv, vi[q]);
                    const float e = depth_error<kContracted>(V, vg, pzh[q], pzl[q], D[q]);
                    if (!(fabsf(e) <= vg.Delta)) continue;
                    float m, w;
                    weight<kMT>(V, vg, F, raw[q], e, m, w);
                    W = __fmaf_rn(m, w, W);
                    Z = __fadd_rn(Z, w);
                    bits |= V.bit;
                }
            }
        }
    }
}

}  // namespace divas
