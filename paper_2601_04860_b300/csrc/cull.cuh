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
// covered by at most 3 x 3 texels of level max(3, ceil(log2 s) - 1); spans
// above 128 pixels keep the view.  The maximum below the gate threshold (NaN
// pixels never pass the gate and never raise the maximum) culls the view.
#pragma once

#include <cstdint>

#include "fuse_math.cuh"

namespace divas {

constexpr int kPyrL0 = 3;       // finest pyramid level (8-pixel texels)
constexpr int kPyrLevels = 4;   // levels 3..6
constexpr int kPyrTile = 64;    // pixels per side of a level-6 texel (one CTA)

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
                                                      const __grid_constant__ CullBatch CB) {
    __shared__ float l3[8][8];
    allow_dependents();
    const int v = blockIdx.z;
    const ViewC& V = VB.v[v];
    const CullC& C = CB.v[v];
    const int t = threadIdx.x, lane = t & 31;
    const int x = blockIdx.x * kPyrTile + (t & 63);
    const int yb = blockIdx.y * kPyrTile + 16 * (t >> 6);
    // all 16 loads first (the mask type is uniform), then the maxima
    float val[16];
    if (V.mask_type == kMaskF16) {
        const unsigned short* mp = reinterpret_cast<const unsigned short*>(V.mask);
#pragma unroll
        for (int r = 0; r < 16; ++r)
            val[r] = x < V.W && yb + r < V.H
                         ? __half2float(__ushort_as_half(__ldg(mp + (yb + r) * V.W + x)))
                         : -INFINITY;
    } else {
        const float* mp = reinterpret_cast<const float*>(V.mask);
#pragma unroll
        for (int r = 0; r < 16; ++r)
            val[r] = x < V.W && yb + r < V.H ? __ldg(mp + (yb + r) * V.W + x) : -INFINITY;
    }
    float m[2] = {-INFINITY, -INFINITY};
#pragma unroll
    for (int r = 0; r < 16; ++r) m[r >> 3] = fmaxf(m[r >> 3], val[r]);
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

// per-view constants the cull reads with a lane-varying view index, staged in
// shared memory once per CTA
struct CullView {
    float r[12];  // rows u (0..2), v (3..5), z (6..8) and constants (9..11)
    CullC c;
};

// Stage the batch's cull constants (all threads of the CTA; ends with a
// barrier).
__device__ __forceinline__ void stage_cull_views(const ViewBatch& VB, const CullBatch& CB,
                                                 CullView* sv) {
    for (int v = threadIdx.x; v < VB.n; v += blockDim.x) {
        const ViewC& V = VB.v[v];
#pragma unroll
        for (int k = 0; k < 9; ++k) sv[v].r[k] = V.A[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) sv[v].r[9 + k] = V.C[k];
        sv[v].c = CB.v[v];
    }
    __syncthreads();
}

// Views [0, n) that some lane of the warp may vote in, as a bitmask (bit v).
// live: this lane holds a voxel with a position (the rest are ignored); p: the
// lane's projection coordinates.  Warp-uniform: every lane calls it.
__device__ __forceinline__ uint32_t cull_views(const CullView* sv, const float* pyr, int32_t n,
                                               bool live, const float* p) {
    const int lane = threadIdx.x & 31;
    int32_t kmin[3], kmax[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int32_t k = ordered_key(p[a]);
        kmin[a] = __reduce_min_sync(0xffffffffu, live ? k : INT32_MAX);
        kmax[a] = __reduce_max_sync(0xffffffffu, live ? k : INT32_MIN);
    }
    if (kmin[0] == INT32_MAX) return 0u;  // no voxel to vote for
    float lo[3], hi[3], xm = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = from_ordered_key(kmin[a]);
        hi[a] = from_ordered_key(kmax[a]);
        xm = fmaxf(xm, fmaxf(fabsf(lo[a]), fabsf(hi[a])));
    }
    const int half = lane & 1;
    uint32_t keep_all = 0u;
    for (int32_t v0 = 0; v0 < n; v0 += 16) {
        const int32_t q = v0 + (lane >> 1);
        const bool has = q < n;
        float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
        float zmin = INFINITY;
        if (has) {
            const float* r = sv[q].r;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int corner = 4 * half + cc;
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
        }
        // the partner lane holds the other four corners
        umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, 1));
        umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, 1));
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, 1));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 1));
        zmin = fminf(zmin, __shfl_xor_sync(0xffffffffu, zmin, 1));
        bool keep = false;
        float mx = -INFINITY;
        int32_t L = 0, tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        if (has) {
            const CullC& C = sv[q].c;
            // S of each row over the box: sum_j |row_j| max_j |x_j| + |constant|
            const float sz = __fmaf_ru(C.sz, xm, C.cz);
            if (!(zmin > 0x1p-18f * sz)) {
                keep = true;  // the box reaches too close to (or behind) the camera plane
            } else {
                const float su = __fmaf_ru(C.su, xm, C.cu), sv_ = __fmaf_ru(C.sv, xm, C.cv);
                const float au = fmaxf(fabsf(umin), fabsf(umax));
                const float av = fmaxf(fabsf(vmin), fabsf(vmax));
                // 1 / zmin within an ulp, taken up by one ulp more
                const float iz = __fmul_ru(rcp_nr(zmin), 1.f + 0x1p-22f);
                const float mu = __fmaf_ru(0x1p-18f, __fmaf_ru(__fmaf_ru(au, sz, su), iz, au), 2.f);
                const float mv = __fmaf_ru(0x1p-18f, __fmaf_ru(__fmaf_ru(av, sz, sv_), iz, av), 2.f);
                const float fu0 = umin - mu, fu1 = umax + mu, fv0 = vmin - mv, fv1 = vmax + mv;
                if (!(fu0 <= fu1 && fv0 <= fv1)) {
                    keep = true;  // NaN: no bound
                } else if (fu1 < 0.f || fv1 < 0.f || fu0 >= (float)C.W || fv0 >= (float)C.H) {
                    keep = false;  // every centre projects outside the raster
                } else {
                    const int32_t iu0 = (int32_t)floorf(fmaxf(fu0, 0.f));
                    const int32_t iu1 = (int32_t)floorf(fminf(fu1, (float)(C.W - 1)));
                    const int32_t iv0 = (int32_t)floorf(fmaxf(fv0, 0.f));
                    const int32_t iv1 = (int32_t)floorf(fminf(fv1, (float)(C.H - 1)));
                    const int32_t span = max(iu1 - iu0, iv1 - iv0) + 1;
                    L = max(kPyrL0, (32 - __clz(span - 1)) - 1);
                    if (L >= kPyrL0 + kPyrLevels) {
                        keep = true;  // too wide for the pyramid
                    } else {
                        tx0 = iu0 >> L;
                        tx1 = iu1 >> L;
                        ty0 = iv0 >> L;
                        ty1 = iv1 >> L;
                    }
                }
            }
        }
        // the pair splits the (at most 3 x 3) texels: rows ty0, ty0 + 1 on the
        // even lane, row ty0 + 2 on the odd one
        if (tx1 >= tx0) {
            const CullC& C = sv[q].c;
            const float* lev = pyr + C.off[L - kPyrL0];
            const int32_t lw = C.lw[L - kPyrL0];
            const int32_t ya = half ? ty0 + 2 : ty0, yb = half ? ty0 + 2 : min(ty0 + 1, ty1);
            for (int32_t y = ya; y <= min(yb, ty1); ++y)
                for (int32_t xx = tx0; xx <= tx1; ++xx) mx = fmaxf(mx, __ldg(lev + y * lw + xx));
        }
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        if (has && tx1 >= tx0) keep = mx >= sv[q].c.thr;
        // view q's verdict sits on lanes 2 (q - v0) and 2 (q - v0) + 1
        uint32_t b = __ballot_sync(0xffffffffu, keep && half == 0) & 0x55555555u;
        b = (b | (b >> 1)) & 0x33333333u;
        b = (b | (b >> 2)) & 0x0f0f0f0fu;
        b = (b | (b >> 4)) & 0x00ff00ffu;
        b = (b | (b >> 8)) & 0x0000ffffu;
        keep_all |= b << v0;
    }
    return keep_all;
}

// Fold the views of `keep` (ascending view order, four at a time: the same
// per-view arithmetic and order as fold_views over all views, which it matches
// bitwise when the skipped views vote nowhere).  The view index is warp-uniform.
template <bool kContracted, int kMT>
__device__ __forceinline__ void fold_views_kept(const ViewBatch& VB, uint32_t keep,
                                                const VoxelGeom& vg, const FuseC& F, float& W,
                                                float& Z, uint32_t& bits) {
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
            if (vi[q] >= 0) pix[q] = project<kContracted>(VB.v[vi[q]], vg, F.z_near, pzh[q], pzl[q]);
        }
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q)
            if (vi[q] >= 0) load_raster<kMT>(VB.v[vi[q]], pix[q], D[q], raw[q]);
        float e[kViewChunk];
        uint32_t acc = 0u;
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q) {
            if (vi[q] < 0) break;
            const ViewC& V = VB.v[vi[q]];
            const bool pass =
                kContracted ? pre_gates<true, kMT>(V, vg, F, pix[q], pzh[q], D[q], raw[q])
                            : gates<false, kMT>(V, vg, F, pix[q], pzh[q], pzl[q], D[q], raw[q], e[q]);
            if (pass) acc |= 1u << q;
        }
        if (acc) {
#pragma unroll
            for (int q = 0; q < kViewChunk; ++q) {
                if (acc & (1u << q)) {
                    const ViewC& V = VB.v[vi[q]];
                    if constexpr (kContracted) {
                        e[q] = depth_error<true>(V, vg, pzh[q], pzl[q], D[q]);
                        if (!(fabsf(e[q]) <= vg.Delta)) continue;
                    }
                    float m, w;
                    weight<kMT>(V, vg, F, raw[q], e[q], m, w);
                    W = __fmaf_rn(m, w, W);
                    Z = __fadd_rn(Z, w);
                    bits |= V.bit;
                }
            }
        }
    }
}

}  // namespace divas
