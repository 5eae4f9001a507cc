// tuple_mode.cuh -- depth-tuple mode of the fusion (Sec. 3.5 "Planar-to-ray
// depth correction" .. "Thin-structure path"; Algorithms "Thick-Structure
// Segmentation for 2DGS" and "Thin-Structure Segmentation for 2DGS",
// Appendix B.5), included by divas_fuse.cu after the context definition.
//
// Per view the caller hands over the depth tuple (d_min, d_med, d_max planar
// FP32, the splat count n_samp as uint16) with the mask and the camera-target
// distance d_cam.  Per view the library builds two integral images of n_samp
// (uint32 and uint64, modular: a four-corner query is exact for footprints of
// fewer than 2^16 pixels), then one thread per active voxel evaluates, view by
// view in index order:
//
//   - the centre and its 8 corners (plain grids: lattice points n and n +- 1,
//     projected with the same exact depth row and intrinsics-folded pixel
//     rows as the centre); the footprint box of the corners' pixels;
//   - footprint statistics from the integral images (mean, and the layered
//     test n > mean + sigma decided exactly in 128-bit integers);
//   - the thick path: trust / see-through / front, the asymmetric depth gate
//     with the tightened tolerance gamma h_v / (1 + beta E), the spatial gate
//     and the depth-band weight.  Every ray-space quantity is its planar
//     counterpart times 1 / cos(theta) = |p| / p_z (the ray through the
//     voxel's own projection), so the spatial gate is (|p| / p_z) |x_d -
//     clip(x_d, d_min, d_ref)| <= h_v pi_dg and the weight's offset is
//     (s - d_min) - (d_max - d_min) / 2 in planar depths, both formed from
//     exact differences;
//   - the behind-surface gate and, when the thick path did not vote, the thin
//     path: a loop over the footprint's pixels with the per-pixel tightened
//     asymmetric gate, the two counters, the peak mask and the nearest
//     unprojected mask-positive pixel.
//
// The occupied set is binary here: every active voxel has density 1, so
// rho_thin <= 1 keeps the thin path on and rho_thin > 1 turns it off.
#pragma once

namespace {

constexpr int kMaxTupleViews = 16;  // per launch (the batch fits the 4 KB parameter space)

struct TViewC {
    ViewC base;                      // projection constants; base.depth = d_min, base.mask
    const float* d_med;
    const float* d_max;
    const uint16_t* n_samp;
    const uint32_t* sat1;            // (H + 1) x (W + 1) integral image of n_samp (mod 2^32),
    const unsigned long long* sat2;  // same of n_samp^2 (mod 2^64); NULL: sums taken directly
    float cd[9];                     // camera-row offsets of the corners, per grid axis q:
                                     // (cd[q], cd[3 + q], cd[6 + q]) (contracted: x 0.5 h_v)
    float st_thr;                    // gamma_st * d_cam (see-through threshold on d_med)
    float inv_fx, inv_fy;            // 1 / fx, 1 / fy (unprojection)
    const float* tile_max;           // largest mask key of each kMaskTile^2 pixel tile
    const float* tile_dil;           // the same over each tile's 3 x 3 tile neighbourhood;
                                     // NULL: footprints may reach beyond it (no pre-check)
    int32_t tiles_w;                 // tiles per row
    float key_thr;                   // no thin vote unless some key in the footprint reaches it
    float R[9], t[3];                // the camera as given (world -> camera, row-major): the
                                     // exact re-evaluation of decisions near a gate
};

struct TViewBatch {
    int32_t n;
    int32_t pad;
    TViewC v[kMaxTupleViews];
};
// (beyond the classic 4 KB: kernel parameters up to 32 KB, CUDA 12.1 and later)
static_assert(sizeof(TViewBatch) <= 4600, "a tuple view batch and the other arguments");

struct TupleC {
    float beta, tau_thin, rho_cover, rho_occ, n_abs, dist_gate, behind_margin, k_dg;
    int32_t thin_on;
    int32_t pad;
};

// camera depth (hi + lo), camera rows (plain grids: r0 = u p_z, r1 = v p_z
// with the intrinsics folded in; contracted: r0 = p_x, r1 = p_y) and pixel
// coordinates of a lattice point (plain: n = 2 idx + 1) or a world point
// (contracted: hi + lo); false when it is not in front of the camera
template <bool kContracted>
__device__ __forceinline__ bool project_uv(const ViewC& V, const float* nh, const float* nl,
                                           float z_near, float& pzh, float& pzl, float& r0,
                                           float& r1, float& u, float& v) {
    float pz;
    if (!kContracted) {
        lattice_row(V.A + 6, V.B, V.C[2], V.E, nh, pzh, pzl);
        pz = __fadd_rn(pzh, pzl);
        const bool front = pz > z_near && pz <= FLT_MAX;
        const float inv = rcp_nr(front ? pz : 1.f);
        r0 = __fmaf_rn(V.A[0], nh[0], __fmaf_rn(V.A[1], nh[1], __fmaf_rn(V.A[2], nh[2], V.C[0])));
        r1 = __fmaf_rn(V.A[3], nh[0], __fmaf_rn(V.A[4], nh[1], __fmaf_rn(V.A[5], nh[2], V.C[1])));
        u = __fmul_rn(r0, inv);
        v = __fmul_rn(r1, inv);
        return front;
    }
    dot3c(V.A[6], V.A[7], V.A[8], nh, nl, V.C[2], pzh, pzl);
    pz = pzh;
    r0 = __fmaf_rn(V.A[0], nh[0], __fmaf_rn(V.A[1], nh[1], __fmaf_rn(
        V.A[2], nh[2], __fmaf_rn(V.A[0], nl[0], __fmaf_rn(V.A[1], nl[1], __fmaf_rn(
        V.A[2], nl[2], V.C[0]))))));
    r1 = __fmaf_rn(V.A[3], nh[0], __fmaf_rn(V.A[4], nh[1], __fmaf_rn(
        V.A[5], nh[2], __fmaf_rn(V.A[3], nl[0], __fmaf_rn(V.A[4], nl[1], __fmaf_rn(
        V.A[5], nl[2], V.C[1]))))));
    const bool front = pz > z_near && pz <= FLT_MAX;
    const float inv = rcp_nr(front ? pz : 1.f);
    u = __fmaf_rn(V.K[0], __fmul_rn(r0, inv), V.K[2]);
    v = __fmaf_rn(V.K[1], __fmul_rn(r1, inv), V.K[3]);
    return front;
}

__device__ __forceinline__ float centre_depth(const TViewC& T, int x, int y) {
    x = min(max(x, 0), T.base.W - 1);
    y = min(max(y, 0), T.base.H - 1);
    const int32_t q = y * T.base.W + x;
    return __fmul_rn(0.5f, __fadd_rn(__ldg(T.base.depth + q), __ldg(T.d_max + q)));
}

// depth-gradient factor at pixel (x, y) (App. D)
__device__ __forceinline__ float pi_dg(const TViewC& T, int x, int y, float k) {
    if (k == 0.f) return 1.f;
    const float a = centre_depth(T, x + 1, y), b = centre_depth(T, x - 1, y);
    const float c = centre_depth(T, x, y + 1), d = centre_depth(T, x, y - 1);
    if (!(fabsf(a) <= FLT_MAX && fabsf(b) <= FLT_MAX && fabsf(c) <= FLT_MAX && fabsf(d) <= FLT_MAX))
        return 0.f;
    const float gx = __fsub_rn(a, b), gy = __fsub_rn(c, d);
    return expf(-__fmul_rn(k, __fmaf_rn(gx, gx, __fmul_rn(gy, gy))));
}

// n > mean + sigma for a pixel of the footprint: with d = n A - S1 and
// Q = A S2 - S1^2 (both exact integers), d > 0 and d^2 > Q
__device__ __forceinline__ bool layered_q(uint32_t n, uint32_t A, unsigned long long S1,
                                          unsigned __int128 Q) {
    const long long d = (long long)n * (long long)A - (long long)S1;
    return d > 0 && (unsigned __int128)d * (unsigned __int128)d > Q;
}

// ---------------------------------------------------------------------------
// Exact re-evaluation of distance decisions near their gates.  The FP32
// distances of the kernels carry rounding of order 2^-24 of the coordinates'
// magnitudes; when one lies within a bound of that size of its gate, the
// decision is taken again in FP64, in world coordinates, with the same
// operations as the FP64 definition (pixel centre unprojected at its depth,
// x = R^T (p_c - t); camera point p = R x + t), so that the result agrees with
// it wherever the distance is farther than 1e-6 of the gate from it.
// ---------------------------------------------------------------------------
// world centre of a voxel in FP64: plain grids o + n h / 2 (n = 2 idx + 1, so
// (idx + 1/2) h exactly as one rounding), contracted grids hi + lo
__device__ __forceinline__ void centre64(const VoxelGeom& vg, const GridC& G, double* x) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
        x[q] = G.contracted ? __dadd_rn((double)vg.xh[q], (double)vg.xl[q])
                            : __dadd_rn((double)G.origin[q],
                                        __dmul_rn(__dmul_rn((double)vg.xh[q], 0.5), (double)G.h));
}

// an FP32 distance d is re-decided when |d - gate| is within this bound: 32
// units of 2^-24 of the magnitudes it is formed from (world centre, camera
// translation, camera depth times the largest pixel-ray slope), many times the
// few roundings of those magnitudes the FP32 distance carries
__device__ __forceinline__ float recheck_band(const TViewC& T, const VoxelGeom& vg,
                                              const GridC& G, float pz) {
    const ViewC& V = T.base;
    const float slope = __fadd_rn(2.f, __fadd_rn(__fdiv_rn(fabsf(V.K[2]) + (float)V.W, fabsf(V.K[0])),
                                                 __fdiv_rn(fabsf(V.K[3]) + (float)V.H, fabsf(V.K[1]))));
    float mag = 1.f + fabsf(T.t[0]) + fabsf(T.t[1]) + fabsf(T.t[2]) + fabsf(pz) * slope;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        mag += G.contracted ? fabsf(vg.xh[q]) : fabsf(G.origin[q]) + fabsf(vg.xh[q]) * G.h;
    return __fmul_rn(0x1p-19f, mag);
}

// squared world distance from the voxel centre x to pixel (px, py) unprojected
// at planar depth d: R^T (p_c - t) - x, p_c = ((px + 1/2 - cx) / fx d,
// (py + 1/2 - cy) / fy d, d)
__device__ __forceinline__ double unproject_d2(const TViewC& T, int px, int py, float d,
                                               const double* x) {
    const ViewC& V = T.base;
    const double dd = (double)d;
    const double pc[3] = {
        __dmul_rn(__ddiv_rn(__dsub_rn(__dadd_rn((double)px, 0.5), (double)V.K[2]), (double)V.K[0]), dd),
        __dmul_rn(__ddiv_rn(__dsub_rn(__dadd_rn((double)py, 0.5), (double)V.K[3]), (double)V.K[1]), dd),
        dd};
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double w = __dadd_rn(__dadd_rn(__dmul_rn((double)T.R[r], __dsub_rn(pc[0], (double)T.t[0])),
                                             __dmul_rn((double)T.R[3 + r], __dsub_rn(pc[1], (double)T.t[1]))),
                                   __dmul_rn((double)T.R[6 + r], __dsub_rn(pc[2], (double)T.t[2])));
        const double e = __dsub_rn(w, x[r]);
        s = __dadd_rn(s, __dmul_rn(e, e));
    }
    return s;
}

// The same test as a threshold on n: with r = floor(sqrt(Q)), d^2 > Q and
// d > 0 exactly when d >= r + 1, i.e. n >= n* = ceil((S1 + r + 1) / A).
// Taken when Q < 2^48 (r < 2^24: the float estimates below are within a few
// units and the corrections are exact integer tests); false otherwise, and the
// caller uses layered_q.
__device__ __forceinline__ bool layered_threshold(uint32_t A, unsigned long long S1,
                                                  unsigned __int128 Q, uint32_t& n_star) {
    if (Q >= ((unsigned __int128)1 << 48) || S1 >= (1ull << 40)) return false;
    const unsigned long long q = (unsigned long long)Q;
    unsigned long long r = (unsigned long long)__fsqrt_rn((float)q);
    while (r * r > q) --r;
    while ((r + 1) * (r + 1) <= q) ++r;
    const unsigned long long need = S1 + r + 1;  // n A >= need
    unsigned long long n = (unsigned long long)ceilf(__fdiv_rn((float)need, (float)A));
    while (n * A < need) ++n;
    while (n > 0 && (n - 1) * A >= need) --n;
    n_star = n > 65536ull ? 65536u : (uint32_t)n;  // n_samp < 65536: never layered
    return true;
}

// mask bits at pixel q (binary16 or FP32 / logit bits), loaded ahead of use
template <int kMT = -1>
__device__ __forceinline__ uint32_t mask_bits(const ViewC& V, int32_t q) {
    return mask_type_of<kMT>(V) == kMaskF16
               ? (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(V.mask) + q)
               : __ldg(reinterpret_cast<const uint32_t*>(V.mask) + q);
}

// probability and "mask positive" (m > 1/2; logit l > 0) of loaded mask bits
template <int kMT = -1>
__device__ __forceinline__ float mask_from_bits(const ViewC& V, uint32_t raw, bool& half) {
    if (mask_type_of<kMT>(V) == kMaskF16) {
        const float m = __half2float(__ushort_as_half((unsigned short)raw));
        half = m > 0.5f;
        return m;
    }
    const float x = __uint_as_float(raw);
    if (mask_type_of<kMT>(V) == kMaskLogit) {
        half = x > 0.f;
        return __frcp_rn(__fadd_rn(1.f, expf(-x)));
    }
    half = x > 0.5f;
    return x;
}

constexpr int kMaskTile = 8;  // tile edge of the per-view mask-key maxima

// whether some pixel of [i0, i1] x [j0, j1] may carry a mask key >= key_thr
// (its tile's maximum reaches it); false means no thin vote is possible there
__device__ __forceinline__ bool box_may_vote(const TViewC& T, int i0, int i1, int j0, int j1) {
    for (int ty = j0 / kMaskTile; ty <= j1 / kMaskTile; ++ty)
        for (int tx = i0 / kMaskTile; tx <= i1 / kMaskTile; ++tx)
            if (__ldg(T.tile_max + ty * T.tiles_w + tx) >= T.key_thr) return true;
    return false;
}

constexpr int kThinGroup = 4;  // footprint pixels whose loads are in flight together

// The pixel-coordinate box of a voxel's 8 corners, each the centre's camera
// rows plus or minus the three axis offsets (plain grids: lattice steps of
// the folded pixel rows and of the depth; contracted grids: the rotation's
// columns times h_v / 2); false when a corner is not in front of z_near.
template <bool kContracted>
__device__ __forceinline__ bool corner_box(const TViewC& T, float hv, float z_near, float pzh,
                                           float pzl, float r0, float r1, float& umin, float& umax,
                                           float& vmin, float& vmax) {
    const ViewC& V = T.base;
    umin = FLT_MAX; umax = -FLT_MAX; vmin = FLT_MAX; vmax = -FLT_MAX;
    bool corners = true;
    const float pz = kContracted ? pzh : __fadd_rn(pzh, pzl);
    const float sc = kContracted ? __fmul_rn(0.5f, hv) : 1.f;
    float d0[3], d1[3], d2[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        d0[q] = __fmul_rn(T.cd[q], sc);
        d1[q] = __fmul_rn(T.cd[3 + q], sc);
        d2[q] = __fmul_rn(T.cd[6 + q], sc);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float c0 = r0, c1 = r1, c2 = pz;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const bool up = (c >> q) & 1;
            c0 = up ? __fadd_rn(c0, d0[q]) : __fsub_rn(c0, d0[q]);
            c1 = up ? __fadd_rn(c1, d1[q]) : __fsub_rn(c1, d1[q]);
            c2 = up ? __fadd_rn(c2, d2[q]) : __fsub_rn(c2, d2[q]);
        }
        corners = corners && c2 > z_near && c2 <= FLT_MAX;
        const float inv = rcp_nr(c2 > z_near && c2 <= FLT_MAX ? c2 : 1.f);
        float cu, cv;
        if (kContracted) {
            cu = __fmaf_rn(V.K[0], __fmul_rn(c0, inv), V.K[2]);
            cv = __fmaf_rn(V.K[1], __fmul_rn(c1, inv), V.K[3]);
        } else {
            cu = __fmul_rn(c0, inv);
            cv = __fmul_rn(c1, inv);
        }
        umin = fminf(umin, cu); umax = fmaxf(umax, cu);
        vmin = fminf(vmin, cv); vmax = fmaxf(vmax, cv);
    }
    return corners;
}

// Whether view T can add a vote to the voxel (a thick or a thin candidate):
// the centre pixel's d_min, d_med and mask decide (most voxels are behind the
// visible surface and stop there); a thick candidate also needs a finite
// d_max, a thin-only candidate a mask key >= key_thr within one tile of its
// centre's tile (when every footprint of the view stays there).
template <bool kContracted, int kMT = -1>
__device__ __forceinline__ bool tuple_candidate(const TViewC& T, const VoxelGeom& vg, const FuseC& F,
                                                const TupleC& TP) {
    const ViewC& V = T.base;
    float pzh, pzl, r0, r1, u, v;
    if (!project_uv<kContracted>(V, vg.xh, vg.xl, F.z_near, pzh, pzl, r0, r1, u, v)) return false;
    const int32_t pix = pixel_index(V, true, u, v);
    if (pix < 0) return false;
    const float dmin = __ldg(V.depth + pix), dmed = __ldg(T.d_med + pix);
    const uint32_t mraw = mask_bits<kMT>(V, pix);
    bool half;
    const float m = mask_from_bits<kMT>(V, mraw, half);
    const int32_t mt = mask_type_of<kMT>(V);
    const float raw_gate = mt == kMaskLogit ? __uint_as_float(mraw) : m;
    const bool pass = raw_gate >= (mt == kMaskLogit ? F.logit_tau : F.tau_m);
    const bool trusted = dmin <= dmed;
    if (pass && trusted && dmin > 0.f && dmin <= FLT_MAX && dmed > 0.f && dmed <= FLT_MAX) {
        const float dmax = __ldg(T.d_max + pix);
        if (dmax > 0.f && dmax <= FLT_MAX) return true;  // thick candidate
    }
    const bool seethru = dmed > T.st_thr;
    const float dsurf = (trusted && seethru) ? dmin : dmed;
    const float e_surf = __fadd_rn(__fsub_rn(pzh, dsurf), pzl);
    if (!TP.thin_on || e_surf > __fmul_rn(TP.behind_margin, vg.hv)) return false;
    if (T.tile_dil)
        return __ldg(T.tile_dil + (pix / V.W / kMaskTile) * T.tiles_w + (pix % V.W) / kMaskTile) >=
               T.key_thr;
    return true;
}

// One footprint pixel of the thin path: valid (the asymmetric, tightened
// depth gate against its reference depth dq, d_med not below eps) and the
// reference depth (d_min for a trusted front pixel, else d_med)
__device__ __forceinline__ bool thin_pixel_valid(float qmed, float qmin, uint32_t nq, float mean,
                                                 bool thr, uint32_t n_star, uint32_t A,
                                                 unsigned long long S1, unsigned __int128 Q,
                                                 const TViewC& T, const TupleC& TP, const FuseC& F,
                                                 float pzh, float pzl, float t_full, float& dq) {
    const float Eq = fmaxf(__fsub_rn((float)nq, mean), 0.f);
    const float den = __fmaf_rn(TP.beta, Eq, 1.f);
    const bool lay = thr ? nq >= n_star : layered_q(nq, A, S1, Q);
    const bool fq = (lay || qmed > T.st_thr) && qmin <= qmed;
    dq = fq ? qmin : qmed;
    const float e = __fadd_rn(__fsub_rn(pzh, dq), pzl);
    const float lhs = fq ? e : fabsf(e);
    // lhs <= t_full / den, as lhs den <= t_full (den >= 1)
    return !(qmed < F.eps) && __fmul_rn(lhs, den) <= t_full;
}

// "mask positive" (m > 1/2; logits l > 0) and the key of loaded mask bits
template <int kMT>
__device__ __forceinline__ bool thin_mask_key(const ViewC& V, uint32_t raw, float& key) {
    if (mask_type_of<kMT>(V) == kMaskF16) {
        key = __half2float(__ushort_as_half((unsigned short)raw));
        return key > 0.5f;
    }
    key = __uint_as_float(raw);
    return mask_type_of<kMT>(V) == kMaskLogit ? key > 0.f : key > 0.5f;
}

// The thin path's nearest squared distance in FP64 (unproject_d2 over the
// valid mask-positive pixels of the box, the same per-pixel decisions as the
// FP32 loop): the exact re-evaluation of a distance gate decision.
template <int kMT>
__device__ __noinline__ double thin_d2_exact(const TViewC& T, const FuseC& F, const TupleC& TP,
                                             const double* x, int i0, int i1, int j0, int j1,
                                             float mean, bool thr, uint32_t n_star, uint32_t A,
                                             unsigned long long S1, unsigned __int128 Q, float pzh,
                                             float pzl, float t_full) {
    const ViewC& V = T.base;
    double best = INFINITY;
    for (int yy = j0; yy <= j1; ++yy)
        for (int xx = i0; xx <= i1; ++xx) {
            const int32_t q = yy * V.W + xx;
            float dq, key;
            const bool valid = thin_pixel_valid(__ldg(T.d_med + q), __ldg(V.depth + q),
                                                __ldg(T.n_samp + q), mean, thr, n_star, A, S1, Q,
                                                T, TP, F, pzh, pzl, t_full, dq);
            if (valid && thin_mask_key<kMT>(V, mask_bits<kMT>(V, q), key))
                best = fmin(best, unproject_d2(T, xx, yy, dq, x));
        }
    return best;
}

// One view of one voxel, in full: the centre pixel's candidates, the
// footprint box from the centre's camera rows plus the corners' offsets, its
// statistics from the integral images or, for views whose footprints are
// known to be small, summed directly, the thick gates and weight, and the thin
// path over the footprint's pixels (evaluated without branches, kThinGroup at
// a time with their loads issued together).  Adds the view's vote, if any.
// The vote is returned, not added: kind 1 thick (x = m, y = w: W += m w,
// Z += w), kind 2 thin (x = t: W += t, Z += 1), kind 0 none.
template <bool kContracted, int kMT = -1>
__device__ __forceinline__ void tuple_view(const TViewC& T, const VoxelGeom& vg, const GridC& G,
                                           const FuseC& F, const TupleC& TP, int& kind, float& x,
                                           float& y) {
    kind = 0;
    const ViewC& V = T.base;
    const float hv = vg.hv;                       // world edge h_v
    const float t_full = __fmul_rn(F.gamma, hv);  // the untightened depth tolerance
    float pzh, pzl, r0, r1, u, v;
    if (!project_uv<kContracted>(V, vg.xh, vg.xl, F.z_near, pzh, pzl, r0, r1, u, v)) return;
    const int32_t pix = pixel_index(V, true, u, v);
    if (pix < 0) return;
    // the centre pixel: d_min, d_med and the mask decide the candidates
    const float dmin = __ldg(V.depth + pix), dmed = __ldg(T.d_med + pix);
    const uint32_t mraw = mask_bits<kMT>(V, pix);
    bool half;
    const float m = mask_from_bits<kMT>(V, mraw, half);
    const int32_t mt = mask_type_of<kMT>(V);
    const float raw_gate = mt == kMaskLogit ? __uint_as_float(mraw) : m;
    const bool pass = raw_gate >= (mt == kMaskLogit ? F.logit_tau : F.tau_m);
    const bool trusted = dmin <= dmed;
    const bool seethru = dmed > T.st_thr;
    // behind-surface gate (it only blocks the thin path)
    const float dsurf = (trusted && seethru) ? dmin : dmed;
    const float e_surf = __fadd_rn(__fsub_rn(pzh, dsurf), pzl);
    const bool thin_cand = TP.thin_on && !(e_surf > __fmul_rn(TP.behind_margin, hv));
    bool thick_cand = pass && trusted && dmin > 0.f && dmin <= FLT_MAX && dmed > 0.f &&
                      dmed <= FLT_MAX;
    if (!thick_cand && !thin_cand) return;  // neither path can vote
    float dmax = 0.f;
    uint32_t nc = 0u;
    if (thick_cand) {
        dmax = __ldg(T.d_max + pix);
        nc = __ldg(T.n_samp + pix);
        thick_cand = dmax > 0.f && dmax <= FLT_MAX;
    }
    if (!thick_cand && !thin_cand) return;
    // footprint: the pixel box of the 8 corners
    float umin, umax, vmin, vmax;
    if (!corner_box<kContracted>(T, hv, F.z_near, pzh, pzl, r0, r1, umin, umax, vmin, vmax)) return;
    const float Wf = (float)V.W, Hf = (float)V.H;
    // pixel box, clamped to the image before the integer conversions
    const int i0 = (int)fminf(fmaxf(floorf(umin), 0.f), Wf);
    const int i1 = (int)fmaxf(fminf(floorf(umax), Wf - 1.f), -1.f);
    const int j0 = (int)fminf(fmaxf(floorf(vmin), 0.f), Hf);
    const int j1 = (int)fmaxf(fminf(floorf(vmax), Hf - 1.f), -1.f);
    if (!(i0 <= i1 && j0 <= j1)) return;  // (cannot happen: the centre is in frame)
    const uint32_t A = (uint32_t)(i1 - i0 + 1) * (uint32_t)(j1 - j0 + 1);  // <= W H < 2^31
    // the thin path's pixel floor n_min; n_depth <= A, so a footprint
    // of fewer pixels cannot vote
    const float cu0 = fmaxf(umin, 0.f), cu1 = fminf(umax, Wf);
    const float cv0 = fmaxf(vmin, 0.f), cv1 = fminf(vmax, Hf);
    const float AB = __fmul_rn(__fsub_rn(cu1, cu0), __fsub_rn(cv1, cv0));
    const float n_min = fmaxf(TP.n_abs, ceilf(__fmul_rn(TP.rho_occ, AB)));
    const bool thin_reach = thin_cand && !((float)A < n_min) && box_may_vote(T, i0, i1, j0, j1);
    if (!thick_cand && !thin_reach) return;
    // footprint statistics S1 = sum n, S2 = sum n^2 (exact)
    unsigned long long S1 = 0ull, S2 = 0ull;
    if (T.sat1) {
        const int32_t sw = V.W + 1;
        S1 = (uint32_t)(__ldg(T.sat1 + (j1 + 1) * sw + i1 + 1) - __ldg(T.sat1 + j0 * sw + i1 + 1) -
                        __ldg(T.sat1 + (j1 + 1) * sw + i0) + __ldg(T.sat1 + j0 * sw + i0));
        S2 = __ldg(T.sat2 + (j1 + 1) * sw + i1 + 1) - __ldg(T.sat2 + j0 * sw + i1 + 1) -
             __ldg(T.sat2 + (j1 + 1) * sw + i0) + __ldg(T.sat2 + j0 * sw + i0);
    } else {
        for (int yy = j0; yy <= j1; ++yy) {
            const uint16_t* row = T.n_samp + yy * V.W;
#pragma unroll 4
            for (int xx = i0; xx <= i1; ++xx) {
                const unsigned long long x = __ldg(row + xx);
                S1 += x;
                S2 += x * x;
            }
        }
    }
    // A S2 - S1^2 = A^2 sigma^2 >= 0 (Cauchy-Schwarz on exact sums)
    const unsigned __int128 Q = (unsigned __int128)A * S2 - (unsigned __int128)S1 * S1;
    uint32_t n_star = 0u;
    const bool thr = layered_threshold(A, S1, Q, n_star);
    const float mean = __fdiv_rn((float)S1, (float)A);
    if (thick_cand) {
        const bool lay = thr ? nc >= n_star : layered_q(nc, A, S1, Q);
        const bool front = lay || seethru;  // trusted here
        const float dref = front ? dmin : dmed;
        const float du = __fdiv_rn(__fsub_rn(u, V.K[2]), V.K[0]);
        const float dv = __fdiv_rn(__fsub_rn(v, V.K[3]), V.K[1]);
        const float ray = __fsqrt_rn(__fadd_rn(1.f, __fmaf_rn(du, du, __fmul_rn(dv, dv))));
        // x_d - d_min and x_d - d_ref from exact differences
        const float e_min = __fadd_rn(__fsub_rn(pzh, dmin), pzl);
        const float e_ref = __fadd_rn(__fsub_rn(pzh, dref), pzl);
        // s = clip(x_d, d_min, d_ref): its offset from d_min and its distance to x_d
        float s_off, dist;
        if (e_min < 0.f) { s_off = 0.f; dist = -e_min; }
        else if (e_ref > 0.f) { s_off = __fsub_rn(dref, dmin); dist = e_ref; }
        else { s_off = e_min; dist = 0.f; }
        const float tau_sp = __fmul_rn(hv, pi_dg(T, pix % V.W, pix / V.W, TP.k_dg));
        const float E = fmaxf(__fsub_rn((float)nc, mean), 0.f);
        const float tdep = __fdiv_rn(t_full, __fmaf_rn(TP.beta, E, 1.f));
        const float e_med = __fadd_rn(__fsub_rn(pzh, dmed), pzl);
        const bool vd = front ? (e_min <= tdep) : (fabsf(e_med) <= tdep);
        if (__fmul_rn(ray, dist) <= tau_sp && vd) {
            const float hw_p = __fmul_rn(0.5f, __fsub_rn(dmax, dmin));
            const float hw_r = fmaxf(__fmul_rn(hw_p, ray), F.eps);
            const float r = __fdiv_rn(__fmul_rn(ray, __fsub_rn(s_off, hw_p)), hw_r);
            const float w = expf(-__fmul_rn(F.alpha1, __fmul_rn(r, r)));
            kind = 1;
            x = m;
            y = w;
            return;  // the thin path runs only where the thick path did not vote
        }
    }
    if (!thin_reach) return;
    // thin path over the footprint's pixels (row-major).  Distances
    // are taken in camera coordinates (rotations keep them): the
    // voxel centre p = (p_x, p_y, p_z), a pixel (x, y) unprojected
    // at depth d to (((x + 1/2) - cx) d / fx, ((y + 1/2) - cy) d / fy, d).
    const float px = __fmul_rn(__fmul_rn(__fsub_rn(u, V.K[2]), T.inv_fx), __fadd_rn(pzh, pzl));
    const float py = __fmul_rn(__fmul_rn(__fsub_rn(v, V.K[3]), T.inv_fy), __fadd_rn(pzh, pzl));
    const bool logit = mask_type_of<kMT>(V) == kMaskLogit;
    int n_depth = 0, n_md = 0;
    float mkey = -FLT_MAX;  // the peak mask of the valid mask-positive pixels, as its key
    float d2 = FLT_MAX;
    int xx = i0, yy = j0;
    for (uint32_t p0 = 0; p0 < A; p0 += kThinGroup) {
        // n_depth can no longer reach n_min: no vote
        if ((float)((uint32_t)n_depth + (A - p0)) < n_min) break;
        int gx[kThinGroup], gy[kThinGroup];
        float gmed[kThinGroup], gmin[kThinGroup];
        uint32_t gn[kThinGroup], gm[kThinGroup];
#pragma unroll
        for (int k = 0; k < kThinGroup; ++k) {
            gx[k] = xx;
            gy[k] = yy;
            if (++xx > i1) {
                xx = i0;
                ++yy;
            }
            gmed[k] = -1.f;  // past the footprint: skipped like d_med < eps
            gmin[k] = 0.f;
            gn[k] = 0u;
            gm[k] = 0u;
            if (p0 + k < A) {
                const int32_t q = gy[k] * V.W + gx[k];
                gmed[k] = __ldg(T.d_med + q);
                gmin[k] = __ldg(V.depth + q);
                gn[k] = __ldg(T.n_samp + q);
                gm[k] = mask_bits<kMT>(V, q);
            }
        }
#pragma unroll
        for (int k = 0; k < kThinGroup; ++k) {
            float dq, key;
            const bool valid = thin_pixel_valid(gmed[k], gmin[k], gn[k], mean, thr, n_star, A, S1,
                                                Q, T, TP, F, pzh, pzl, t_full, dq);
            const bool hq = thin_mask_key<kMT>(V, gm[k], key);
            const float ax = __fmul_rn(__fsub_rn((float)gx[k] + 0.5f, V.K[2]), T.inv_fx);
            const float ay = __fmul_rn(__fsub_rn((float)gy[k] + 0.5f, V.K[3]), T.inv_fy);
            const float dx = __fsub_rn(__fmul_rn(ax, dq), px);
            const float dy = __fsub_rn(__fmul_rn(ay, dq), py);
            const float dz = __fsub_rn(__fsub_rn(dq, pzh), pzl);
            const float dd = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
            const bool md = valid && hq;
            n_depth += valid ? 1 : 0;
            n_md += md ? 1 : 0;
            mkey = md ? fmaxf(mkey, key) : mkey;
            d2 = md ? fminf(d2, dd) : d2;
        }
    }
    if (n_md > 0 && (float)n_depth >= n_min &&
        (float)n_md >= __fmul_rn(TP.rho_cover, (float)n_depth)) {
        const float gate = __fmul_rn(TP.dist_gate, hv);
        // the probability of the peak key (the sigmoid is increasing)
        const float m_max = logit ? __frcp_rn(__fadd_rn(1.f, expf(-mkey))) : mkey;
        if (m_max >= TP.tau_thin) {
            bool inside = d2 <= __fmul_rn(gate, gate);
            if (fabsf(__fsub_rn(__fsqrt_rn(d2), gate)) <=
                recheck_band(T, vg, G, __fadd_rn(pzh, pzl))) {
                double xw[3];
                centre64(vg, G, xw);
                const double g64 = __dmul_rn((double)TP.dist_gate, (double)hv);
                inside = thin_d2_exact<kMT>(T, F, TP, xw, i0, i1, j0, j1, mean, thr, n_star, A, S1,
                                            Q, pzh, pzl, t_full) <= __dmul_rn(g64, g64);
            }
            if (inside) {
                kind = 2;
                x = m_max;
            }
        }
    }
}

// Pass 1 of a tuple launch, one thread per active voxel: the candidate views
// (a bit each) from the centre pixels alone; voxels with any are appended to
// the heavy list (warp-aggregated), the others are done (no view votes).
// Zeroes the accumulators first when the context holds no views yet.  The
// view loop is unrolled to kN (>= the batch's views) so that the views'
// constants are addressed at compile time.
template <bool kContracted, int kN, int kMT = -1>
__global__ void __launch_bounds__(kThreads) k_tuple_scan(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, GridC G, FuseC F,
    const __grid_constant__ TViewBatch TB, TupleC TP, int32_t accumulate, float* __restrict__ W,
    float* __restrict__ Z, uint32_t* __restrict__ bits, uint2* __restrict__ heavy,
    int32_t* __restrict__ n_heavy) {
    const int32_t n = *d_n;
    const int lane = threadIdx.x & 31;
    const int32_t stride = gridDim.x * blockDim.x;
    // warp-uniform loop: every lane reaches the ballot
    for (int32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < n; base += stride) {
        const int32_t a = base + lane;
        uint32_t cand = 0u;
        if (a < n) {
            if (!accumulate) {
                W[a] = 0.f;
                Z[a] = 0.f;
                bits[a] = 0u;
            }
            const VoxelGeom vg = voxel_geom<kContracted>(__ldg(active + a), G, F.gamma);
            if (vg.ok) {
#pragma unroll
                for (int i = 0; i < kN; ++i)
                    if (i < TB.n && tuple_candidate<kContracted, kMT>(TB.v[i], vg, F, TP)) cand |= 1u << i;
            }
        }
        const unsigned hb = __ballot_sync(0xffffffffu, cand != 0u);
        if (hb) {
            const int lead = __ffs(hb) - 1;
            int32_t slot = 0;
            if (lane == lead) slot = atomicAdd(n_heavy, __popc(hb));
            slot = __shfl_sync(0xffffffffu, slot, lead);
            if (cand) heavy[slot + __popc(hb & ((1u << lane) - 1u))] = make_uint2((uint32_t)a, cand);
        }
    }
}

// Pass 2: two heavy voxels per warp, a half-warp each; lane i of a half
// computes view i's vote (views run in parallel), then the half's first lane
// adds the votes in view order (every voxel still sums its votes in view
// order, with the same FMA and additions).
template <bool kContracted, int kMT = -1>
__global__ void __launch_bounds__(kThreads, 4) k_tuple_heavy(
    const uint32_t* __restrict__ active, const uint2* __restrict__ heavy,
    const int32_t* __restrict__ n_heavy, GridC G, FuseC F, const __grid_constant__ TViewBatch TB,
    TupleC TP, float* __restrict__ W, float* __restrict__ Z, uint32_t* __restrict__ bits) {
    static_assert(kMaxTupleViews <= 16, "a half-warp holds one voxel's views");
    // the views in shared memory, an odd number of 8-byte words apart (the
    // pointers stay aligned), so that the lanes of a half-warp (one view
    // each) read different banks
    static_assert(sizeof(TViewC) % 8 == 0 && alignof(TViewC) == 8, "view constants copy as 8-byte words");
    constexpr int kIn = (int)(sizeof(TViewC) / 8);
    constexpr int kWords = kIn | 1;
    __shared__ uint2 sv[kMaxTupleViews * kWords];
    {
        const uint2* src = reinterpret_cast<const uint2*>(&TB.v[0]);
        for (int w = threadIdx.x; w < TB.n * kIn; w += blockDim.x)
            sv[(w / kIn) * kWords + (w % kIn)] = src[w];
        __syncthreads();
    }
    const int32_t n = *n_heavy;
    const int l = threadIdx.x & 15;
    const int32_t halves = (gridDim.x * blockDim.x) >> 4;
    // half-warp-uniform loop: both halves of a warp reach the shuffles
    for (int32_t s0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 4; s0 - ((threadIdx.x >> 4) & 1) < n;
         s0 += halves) {
        const bool live = s0 < n;
        uint2 h = make_uint2(0u, 0u);
        if (live) h = heavy[s0];
        int kind = 0;
        float x = 0.f, y = 0.f;
        if (live && ((h.y >> l) & 1u)) {
            const VoxelGeom vg = voxel_geom<kContracted>(__ldg(active + h.x), G, F.gamma);
            tuple_view<kContracted, kMT>(*reinterpret_cast<const TViewC*>(sv + l * kWords), vg, G, F,
                                         TP, kind, x, y);
        }
        float Ws = 0.f, Zs = 0.f;
        uint32_t b = 0u;
        if (live && l == 0) {
            Ws = W[h.x];
            Zs = Z[h.x];
            b = bits[h.x];
        }
        for (int i = 0; i < TB.n; ++i) {
            const int ki = __shfl_sync(0xffffffffu, kind, i, 16);
            const float xi = __shfl_sync(0xffffffffu, x, i, 16);
            const float yi = __shfl_sync(0xffffffffu, y, i, 16);
            if (ki == 1) {
                Ws = __fmaf_rn(xi, yi, Ws);
                Zs = __fadd_rn(Zs, yi);
                b |= TB.v[i].base.bit;
            } else if (ki == 2) {
                Ws = __fadd_rn(Ws, xi);
                Zs = __fadd_rn(Zs, 1.f);
                b |= TB.v[i].base.bit;
            }
        }
        if (live && l == 0) {
            W[h.x] = Ws;
            Z[h.x] = Zs;
            bits[h.x] = b;
        }
    }
}

// per view, the largest mask key (binary16 value, FP32 probability or logit)
// of each kMaskTile x kMaskTile pixel tile (edge tiles clipped; NaN keys are
// ignored: they never count as mask-positive), and its maximum over the 3 x 3
// tile neighbourhood.  A block covers 16 x 16 tiles plus a one-tile halo
// (blockIdx.z = view).
struct TileJob {
    const void* mask;
    float* out;   // tile maxima
    float* dil;   // neighbourhood maxima
    int32_t W, H, mask_type, tiles_w;
    int32_t vec;  // rows start on 16-byte boundaries: tile rows load as 16-byte words
    int32_t pad;
};

struct TileJobs {
    int32_t n;
    int32_t pad;
    TileJob j[kMaxViews];
};

constexpr int kTileBlock = 16;

__device__ __forceinline__ float mask_key(const void* mask, int32_t mask_type, int32_t q) {
    return mask_type == kMaskF16
               ? __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(mask) + q)))
               : __ldg(reinterpret_cast<const float*>(mask) + q);
}

__global__ void __launch_bounds__(kTileBlock * kTileBlock, 4) k_mask_tiles(const __grid_constant__ TileJobs J) {
    const TileJob& jb = J.j[blockIdx.z];
    const int32_t tw = jb.tiles_w, th = (jb.H + kMaskTile - 1) / kMaskTile;
    const int32_t bx = blockIdx.x * kTileBlock, by = blockIdx.y * kTileBlock;
    if (bx >= tw || by >= th) return;  // past this view's tiles (whole block)
    constexpr int kS = kTileBlock + 2;
    __shared__ float tm[kS][kS];
    for (int k = threadIdx.x; k < kS * kS; k += blockDim.x) {
        const int32_t tx = bx - 1 + k % kS, ty = by - 1 + k / kS;
        float mx = -FLT_MAX;
        if (tx >= 0 && tx < tw && ty >= 0 && ty < th) {
            const int32_t x0 = tx * kMaskTile, y0 = ty * kMaskTile;
            const bool full = x0 + kMaskTile <= jb.W && y0 + kMaskTile <= jb.H;
            if (full && jb.vec) {  // rows of the tile as 16-byte loads (aligned rows)
                if (jb.mask_type == kMaskF16) {
#pragma unroll
                    for (int r = 0; r < kMaskTile; ++r) {
                        const uint4 w = __ldg(reinterpret_cast<const uint4*>(
                            reinterpret_cast<const unsigned short*>(jb.mask) + (y0 + r) * jb.W + x0));
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t wk = k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
                            mx = fmaxf(mx, fmaxf(__half2float(__ushort_as_half((unsigned short)(wk & 0xffffu))),
                                                 __half2float(__ushort_as_half((unsigned short)(wk >> 16)))));
                        }
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < kMaskTile; ++r)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float4 f = __ldg(reinterpret_cast<const float4*>(
                                reinterpret_cast<const float*>(jb.mask) + (y0 + r) * jb.W + x0 + 4 * h));
                            mx = fmaxf(mx, fmaxf(fmaxf(f.x, f.y), fmaxf(f.z, f.w)));
                        }
                }
            } else if (full) {
#pragma unroll
                for (int r = 0; r < kMaskTile; ++r)
#pragma unroll
                    for (int c = 0; c < kMaskTile; ++c)
                        mx = fmaxf(mx, mask_key(jb.mask, jb.mask_type, (y0 + r) * jb.W + x0 + c));
            } else {
                for (int32_t y = y0; y < min(y0 + kMaskTile, jb.H); ++y)
                    for (int32_t x = x0; x < min(x0 + kMaskTile, jb.W); ++x)
                        mx = fmaxf(mx, mask_key(jb.mask, jb.mask_type, y * jb.W + x));
            }
        }
        tm[k / kS][k % kS] = mx;
    }
    __syncthreads();
    const int lx = threadIdx.x % kTileBlock, ly = threadIdx.x / kTileBlock;  // 256 threads: 16 x 16
    const int32_t tx = bx + lx, ty = by + ly;
    if (tx < tw && ty < th) {
        float d = -FLT_MAX;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) d = fmaxf(d, tm[ly + dy][lx + dx]);
        jb.out[ty * tw + tx] = tm[ly + 1][lx + 1];
        jb.dil[ty * tw + tx] = d;
    }
}

// integral images of the views' n_samp, all views of a call in two launches:
// (H + 1) x (W + 1) per view with a zero first row and column, uint32 sums of
// n and uint64 sums of n^2 (both modular).  The rows are cut into strips of
// kSatRows: the first launch sums each strip's columns, the second gives each
// strip its column offsets (the totals of the strips above) and scans its rows
// across the block, writing every entry once.
constexpr int kSatRows = 32;      // rows per strip
constexpr int kSatThreads = 256;
constexpr int kSatCPT = 4;        // consecutive columns per thread in a segment

struct SatJob {
    const uint16_t* n;
    uint32_t* s1;               // (H + 1) x (W + 1)
    unsigned long long* s2;
    uint32_t* t1;               // strip column totals, ceil(H / kSatRows) x W
    unsigned long long* t2;
    int32_t W, H;
};

struct SatJobs {
    int32_t n;
    int32_t pad;
    SatJob j[kMaxViews];
};

// blockIdx.x = strip, blockIdx.y = view
__global__ void __launch_bounds__(kSatThreads) k_sat_strip_totals(const __grid_constant__ SatJobs J) {
    const SatJob& jb = J.j[blockIdx.y];
    const int32_t W = jb.W, H = jb.H, k = blockIdx.x;
    if (k * kSatRows >= H) return;  // past this view's strips (whole block)
    const int32_t y0 = k * kSatRows, y1 = min(y0 + kSatRows, H);
    for (int32_t x = threadIdx.x; x < W; x += kSatThreads) {
        uint32_t a1 = 0u;
        unsigned long long a2 = 0ull;
#pragma unroll 8
        for (int32_t y = y0; y < y1; ++y) {
            const uint32_t v = __ldg(jb.n + y * W + x);
            a1 += v;
            a2 += (unsigned long long)v * v;
        }
        jb.t1[k * W + x] = a1;
        jb.t2[k * W + x] = a2;
    }
}

__global__ void __launch_bounds__(kSatThreads) k_sat_strip_fill(const __grid_constant__ SatJobs J) {
    const SatJob& jb = J.j[blockIdx.y];
    const int32_t W = jb.W, H = jb.H, sw = W + 1, k = blockIdx.x;
    if (k * kSatRows >= H) return;  // past this view's strips (whole block)
    const int32_t y0 = k * kSatRows, y1 = min(y0 + kSatRows, H);
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    __shared__ uint32_t c1[kSatRows];  // each row's running total over the column segments
    __shared__ unsigned long long c2[kSatRows];
    __shared__ uint32_t w1[kSatThreads / 32];
    __shared__ unsigned long long w2[kSatThreads / 32];
    if (tid < kSatRows) {
        c1[tid] = 0u;
        c2[tid] = 0ull;
    }
    if (k == 0)
        for (int32_t x = tid; x < sw; x += kSatThreads) {  // the zero first row
            jb.s1[x] = 0u;
            jb.s2[x] = 0ull;
        }
    for (int32_t y = y0 + tid; y < y1; y += kSatThreads) {  // the zero first column
        jb.s1[(y + 1) * sw] = 0u;
        jb.s2[(y + 1) * sw] = 0ull;
    }
    __syncthreads();
    for (int32_t seg = 0; seg < W; seg += kSatThreads * kSatCPT) {
        const int32_t xb = seg + tid * kSatCPT;
        uint32_t C1[kSatCPT];             // column sums of rows 0 .. y
        unsigned long long C2[kSatCPT];
#pragma unroll
        for (int j = 0; j < kSatCPT; ++j) {
            C1[j] = 0u;
            C2[j] = 0ull;
        }
        for (int32_t kk = 0; kk < k; ++kk) {  // the strips above
#pragma unroll
            for (int j = 0; j < kSatCPT; ++j)
                if (xb + j < W) {
                    C1[j] += jb.t1[kk * W + xb + j];
                    C2[j] += jb.t2[kk * W + xb + j];
                }
        }
        for (int32_t y = y0; y < y1; ++y) {
            uint32_t r1 = 0u, o1[kSatCPT];
            unsigned long long r2 = 0ull, o2[kSatCPT];
#pragma unroll
            for (int j = 0; j < kSatCPT; ++j) {
                const uint32_t v = xb + j < W ? (uint32_t)__ldg(jb.n + y * W + xb + j) : 0u;
                C1[j] += v;
                C2[j] += (unsigned long long)v * v;
                r1 += C1[j];
                r2 += C2[j];
                o1[j] = r1;
                o2[j] = r2;
            }
            // exclusive scan of the threads' totals across the block
            uint32_t i1 = r1;
            unsigned long long i2 = r2;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t a1 = __shfl_up_sync(0xffffffffu, i1, o);
                const unsigned long long a2 = __shfl_up_sync(0xffffffffu, i2, o);
                if (lane >= o) {
                    i1 += a1;
                    i2 += a2;
                }
            }
            if (lane == 31) {
                w1[wp] = i1;
                w2[wp] = i2;
            }
            __syncthreads();
            uint32_t e1 = i1 - r1 + c1[y - y0];
            unsigned long long e2 = i2 - r2 + c2[y - y0];
            for (int w = 0; w < wp; ++w) {
                e1 += w1[w];
                e2 += w2[w];
            }
#pragma unroll
            for (int j = 0; j < kSatCPT; ++j)
                if (xb + j < W) {
                    jb.s1[(y + 1) * sw + xb + j + 1] = e1 + o1[j];
                    jb.s2[(y + 1) * sw + xb + j + 1] = e2 + o2[j];
                }
            __syncthreads();  // every thread has read w1, w2 and the row's carry
            if (tid == kSatThreads - 1) {  // the segment's last column: the row's new carry
                c1[y - y0] = e1 + r1;
                c2[y - y0] = e2 + r2;
            }
        }
    }
}

}  // namespace

// Views whose footprints are known to hold at most this many pixels take
// their footprint sums directly from n_samp (no integral images).
constexpr int64_t kDirectSums = 256;

// Bounds on any in-frame voxel's footprint box in a camera, for a plain grid:
// the half-extents (pixels) of the box around the centre's projection, and
// its pixel count (false, no bound: contracted grids, or the grid reaches the
// camera plane).  A corner q = p + delta of a voxel centred at camera point p
// (|delta| <= r = (sqrt 3 / 2) h) moves u by at most fx r (1 + |p_x| / p_z) /
// (p_z - r); |p_x| / p_z <= max(cx, W - cx) / fx for a centre in frame, and
// p_z is at least the smallest camera depth over the grid's bounding box (the
// minimum of a linear function over its corners).  The half-extents carry a
// 0.1% + 0.05 pixel allowance for the kernel's FP32 corners.
static bool footprint_bound(const divas_camera& cam, const GridC& G, float z_near, float& half_u,
                            float& half_v, int64_t& pixels) {
    half_u = half_v = 0.f;
    pixels = INT64_MAX;
    if (G.contracted) return false;
    const double h = G.h, ext = (double)G.g * G.h;
    double zmin = 1e300;
    for (int c = 0; c < 8; ++c) {
        double z = cam.t[2];
        for (int j = 0; j < 3; ++j)
            z += (double)cam.R[6 + j] * ((double)G.origin[j] + (((c >> j) & 1) ? ext : 0.0));
        zmin = std::min(zmin, z);
    }
    const double r = 0.5 * std::sqrt(3.0) * h;
    if (!(zmin - r > std::max((double)z_near, 1e-30))) return false;
    const double tx = std::max((double)cam.cx, (double)cam.W - cam.cx) / cam.fx;
    const double ty = std::max((double)cam.cy, (double)cam.H - cam.cy) / cam.fy;
    const double du = cam.fx * r * (1.0 + tx) / (zmin - r);
    const double dv = cam.fy * r * (1.0 + ty) / (zmin - r);
    if (!(du < 1e8 && dv < 1e8)) return false;
    half_u = (float)(du * 1.001 + 0.05);
    half_v = (float)(dv * 1.001 + 0.05);
    const int64_t nu = (int64_t)std::floor(2.0 * half_u) + 2, nv = (int64_t)std::floor(2.0 * half_v) + 2;
    pixels = std::min<int64_t>(nu, cam.W) * std::min<int64_t>(nv, cam.H);
    return true;
}

// the mask key a thin vote needs somewhere in its footprint: m_max >=
// tau_thin.  binary16 / FP32 probabilities: the key is the probability.
// Logits: sigmoid_FP32(l) is within 5e-7 (relative) of sigmoid(l), so a logit
// below logit(tau (1 - 4e-6)) cannot give tau; tau >= 1 needs sigmoid_FP32(l)
// = 1, i.e. l > 16.
static float thin_key_threshold(int32_t mask_type, float tau_thin) {
    if (mask_type != kMaskLogit) return tau_thin;
    if (!(tau_thin < 1.f)) return 16.f;
    const double tp = (double)tau_thin * (1.0 - 4e-6);
    return (float)std::log(tp / (1.0 - tp));
}

// every view of the batch has a binary16 mask: the kernels take the mask type
// as a compile-time constant (no per-view or per-pixel branches on it)
static bool batch_all_f16(const TViewBatch& tb) {
    for (int32_t i = 0; i < tb.n; ++i)
        if (tb.v[i].base.mask_type != kMaskF16) return false;
    return true;
}

template <bool kC, int kMT>
static divas_status launch_tuple_scan(int nv, int blocks, cudaStream_t s, divas_ctx* c, const TViewBatch& tb,
                              const TupleC& T, int32_t acc, uint2* heavy, int32_t* n_heavy) {
#define DIVAS_TUPLE_SCAN(N)                                                                      \
    k_tuple_scan<kC, N, kMT><<<blocks, kThreads, 0, s>>>(c->active, c->d_n, c->G, c->F, tb, T, acc, \
                                                   c->W, c->Z, c->bits, heavy, n_heavy)
    if (nv <= 4) DIVAS_TUPLE_SCAN(4);
    else if (nv <= 8) DIVAS_TUPLE_SCAN(8);
    else DIVAS_TUPLE_SCAN(16);
#undef DIVAS_TUPLE_SCAN
    DIVAS_LAUNCHED(c, "k_tuple_scan");
    return DIVAS_OK;
}

static size_t tile_bytes_of(int32_t W, int32_t H) {  // both maps
    const size_t n = (size_t)((W + kMaskTile - 1) / kMaskTile) * ((H + kMaskTile - 1) / kMaskTile);
    return 2 * ((n * 4 + 255) / 256 * 256);
}

// scratch of one view's integral images and strip totals (256-byte aligned)
static size_t sat_bytes_of(int32_t W, int32_t H) {
    const size_t cells = (size_t)(W + 1) * (H + 1);
    const size_t tot = (size_t)((H + kSatRows - 1) / kSatRows) * W;
    const size_t b = (cells + tot) * 12;
    return (b + 255) / 256 * 256;
}

// The mask-key tile maxima of every view (k_mask_tiles, one launch), both
// maps of view k at cur + the sum of the earlier views' tile_bytes_of; cur
// is advanced past them.
static divas_status launch_tile_maps(divas_ctx* c, const divas_tuple_view* views, int32_t n_views,
                                     unsigned char*& cur, TileJobs& tj, cudaStream_t s) {
    memset(&tj, 0, sizeof(tj));
    tj.n = n_views;
    int32_t max_tw = 0, max_th = 0;
    for (int32_t k = 0; k < n_views; ++k) {
        const divas_tuple_view& v = views[k];
        TileJob& jb = tj.j[k];
        jb.mask = v.mask;
        jb.W = v.cam.W;
        jb.H = v.cam.H;
        jb.mask_type = v.mask_type;
        jb.tiles_w = (v.cam.W + kMaskTile - 1) / kMaskTile;
        const size_t row_bytes = (size_t)v.cam.W * (v.mask_type == kMaskF16 ? 2 : 4);
        jb.vec = (reinterpret_cast<uintptr_t>(v.mask) % 16 == 0 && row_bytes % 16 == 0) ? 1 : 0;
        const int32_t th = (v.cam.H + kMaskTile - 1) / kMaskTile;
        const size_t half = tile_bytes_of(v.cam.W, v.cam.H) / 2;
        jb.out = reinterpret_cast<float*>(cur);
        jb.dil = reinterpret_cast<float*>(cur + half);
        max_tw = std::max(max_tw, jb.tiles_w);
        max_th = std::max(max_th, th);
        cur += 2 * half;
    }
    k_mask_tiles<<<dim3((max_tw + kTileBlock - 1) / kTileBlock, (max_th + kTileBlock - 1) / kTileBlock,
                        n_views),
                   kTileBlock * kTileBlock, 0, s>>>(tj);
    DIVAS_LAUNCHED(c, "k_mask_tiles");
    return DIVAS_OK;
}

// ---------------------------------------------------------------------------
// C ABI of the tuple mode
// ---------------------------------------------------------------------------
extern "C" {

divas_tuple_params divas_default_tuple_params(void) {
    divas_tuple_params p;
    p.beta = 0.05f;
    p.gamma_st = 1.5f;
    p.tau_thin = 0.6f;
    p.rho_cover = 0.5f;
    p.rho_occ = 0.1f;
    p.n_abs = 25.f;
    p.dist_gate = 1.5f;
    p.behind_margin = 2.f;
    p.k_dg = 0.f;
    p.rho_thin = 1.f;
    return p;
}

divas_status divas_fuse_add_views_tuple(divas_ctx* c, const divas_tuple_view* views,
                                        int32_t n_views, const divas_tuple_params* tp,
                                        void* stream) {
    return divas_fuse_add_views_tuple_profiled(c, views, n_views, tp, nullptr, stream);
}

divas_status divas_fuse_add_views_tuple_profiled(divas_ctx* c, const divas_tuple_view* views,
                                                 int32_t n_views, const divas_tuple_params* tp,
                                                 void* const* stage_events, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (!views || !tp || n_views < 1 || n_views > kMaxViews)
        return fail(c, DIVAS_E_INVALID, "n_views must be in 1..32, views and tp non-NULL");
    if (!(tp->beta >= 0.f) || !(tp->rho_cover >= 0.f) || !(tp->rho_occ >= 0.f) ||
        !(tp->n_abs >= 0.f) || !(tp->dist_gate >= 0.f) || !(tp->behind_margin >= 0.f) ||
        !(tp->k_dg >= 0.f) || !(tp->tau_thin > 0.f) || !(tp->gamma_st == tp->gamma_st) ||
        !(tp->rho_thin == tp->rho_thin))
        return fail(c, DIVAS_E_INVALID, "tuple params out of range");
    // scratch: the heavy list and its count, the mask-tile maxima, the
    // integral images
    const size_t heavy_bytes = ((size_t)c->cap * 8 + 256 + 255) / 256 * 256;
    size_t need = heavy_bytes;
    bool direct[kMaxViews];
    float half_u[kMaxViews], half_v[kMaxViews];
    for (int32_t k = 0; k < n_views; ++k) {
        divas_status st = check_camera(c, &views[k].cam);
        if (st != DIVAS_OK) return st;
        const divas_tuple_view& v = views[k];
        if (!v.d_min || !v.d_med || !v.d_max || !v.n_samp || !v.mask)
            return fail(c, DIVAS_E_INVALID, "a tuple raster is NULL");
        if (v.mask_type < 0 || v.mask_type > 2) return fail(c, DIVAS_E_INVALID, "bad mask_type");
        if (!(v.d_cam == v.d_cam)) return fail(c, DIVAS_E_INVALID, "d_cam is NaN");
        if ((int64_t)(v.cam.W + 1) * (v.cam.H + 1) > INT32_MAX)
            return fail(c, DIVAS_E_INVALID, "(W + 1) (H + 1) must fit in int32");
        int64_t pixels = 0;
        footprint_bound(v.cam, c->G, c->F.z_near, half_u[k], half_v[k], pixels);
        direct[k] = pixels <= kDirectSums;
        need += tile_bytes_of(v.cam.W, v.cam.H);
        if (!direct[k]) need += sat_bytes_of(v.cam.W, v.cam.H);
    }
    cudaStream_t s = S(stream);
    if (need > c->sat_bytes) {  // integral-image scratch, grown on demand
        if (capturing(s))
            return fail(c, DIVAS_E_STATE, "tuple scratch must grow outside a stream capture");
        DIVAS_CUDA(c, cudaStreamSynchronize(s));
        if (c->sat) cudaFree(c->sat);
        c->sat = nullptr;
        c->sat_bytes = 0;
        DIVAS_CUDA(c, cudaMalloc(&c->sat, need));
        c->sat_bytes = need;
    }
    TupleC T;
    T.beta = tp->beta;
    T.tau_thin = tp->tau_thin;
    T.rho_cover = tp->rho_cover;
    T.rho_occ = tp->rho_occ;
    T.n_abs = tp->n_abs;
    T.dist_gate = tp->dist_gate;
    T.behind_margin = tp->behind_margin;
    T.k_dg = tp->k_dg;
    T.thin_on = tp->rho_thin <= 1.f ? 1 : 0;
    T.pad = 0;
    divas_status st = record_stage(c, stage_events, 0, s);
    if (st != DIVAS_OK) return st;
    unsigned char* cur = static_cast<unsigned char*>(c->sat);
    int32_t* n_heavy = reinterpret_cast<int32_t*>(cur);
    uint2* heavy = reinterpret_cast<uint2*>(cur + 256);
    cur += heavy_bytes;
    // the mask-key tile maxima of every view, in one launch
    TileJobs tj;
    st = launch_tile_maps(c, views, n_views, cur, tj, s);
    if (st != DIVAS_OK) return st;
    // integral images of the views that need them, in two launches
    SatJobs jobs;
    memset(&jobs, 0, sizeof(jobs));
    const uint32_t* sat1[kMaxViews] = {};
    const unsigned long long* sat2[kMaxViews] = {};
    int32_t max_strips = 0;
    for (int32_t k = 0; k < n_views; ++k) {
        if (direct[k]) continue;
        const divas_tuple_view& v = views[k];
        const size_t cells = (size_t)(v.cam.W + 1) * (v.cam.H + 1);
        const int32_t strips = (v.cam.H + kSatRows - 1) / kSatRows;
        const size_t tot = (size_t)strips * v.cam.W;
        SatJob& jb = jobs.j[jobs.n++];
        jb.n = v.n_samp;
        jb.s2 = reinterpret_cast<unsigned long long*>(cur);
        jb.t2 = reinterpret_cast<unsigned long long*>(cur + cells * 8);
        jb.s1 = reinterpret_cast<uint32_t*>(cur + (cells + tot) * 8);
        jb.t1 = reinterpret_cast<uint32_t*>(cur + (cells + tot) * 8 + cells * 4);
        jb.W = v.cam.W;
        jb.H = v.cam.H;
        sat1[k] = jb.s1;
        sat2[k] = jb.s2;
        cur += sat_bytes_of(v.cam.W, v.cam.H);
        max_strips = std::max(max_strips, strips);
    }
    if (jobs.n > 0) {
        k_sat_strip_totals<<<dim3(max_strips, jobs.n), kSatThreads, 0, s>>>(jobs);
        DIVAS_LAUNCHED(c, "k_sat_strip_totals");
        k_sat_strip_fill<<<dim3(max_strips, jobs.n), kSatThreads, 0, s>>>(jobs);
        DIVAS_LAUNCHED(c, "k_sat_strip_fill");
    }
    st = record_stage(c, stage_events, 1, s);
    if (st != DIVAS_OK) return st;
    for (int32_t k0 = 0; k0 < n_views; k0 += kMaxTupleViews) {
        const bool last = k0 + kMaxTupleViews >= n_views;
        TViewBatch tb;
        memset(&tb, 0, sizeof(tb));
        tb.n = std::min<int32_t>(kMaxTupleViews, n_views - k0);
        for (int32_t j = 0; j < tb.n; ++j) {
            const divas_tuple_view& v = views[k0 + j];
            TViewC& t = tb.v[j];
            t.base = make_view(v.cam, c->G, v.d_min, v.mask, v.mask_type, c->n_views + k0 + j,
                               false);
            t.d_med = v.d_med;
            t.d_max = v.d_max;
            t.n_samp = v.n_samp;
            t.sat1 = sat1[k0 + j];
            t.sat2 = sat2[k0 + j];
            // corner offsets per grid axis: plain grids the lattice step of
            // the camera rows (pixel rows with the intrinsics folded in, and
            // depth hi + lo), contracted grids the rotation's columns
            for (int q = 0; q < 3; ++q) {
                if (c->G.contracted) {
                    for (int r = 0; r < 3; ++r) t.cd[3 * r + q] = v.cam.R[3 * r + q];
                } else {
                    t.cd[q] = t.base.A[q];
                    t.cd[3 + q] = t.base.A[3 + q];
                    t.cd[6 + q] = (float)((double)t.base.A[6 + q] + (double)t.base.B[q]);
                }
            }
            t.st_thr = (float)((double)tp->gamma_st * (double)v.d_cam);
            t.inv_fx = (float)(1.0 / (double)v.cam.fx);
            t.inv_fy = (float)(1.0 / (double)v.cam.fy);
            t.tile_max = tj.j[k0 + j].out;
            // the one-load pre-check holds when every footprint stays within
            // kMaskTile pixels of its centre (then within one tile of its tile)
            const bool near = half_u[k0 + j] > 0.f && half_u[k0 + j] <= (float)kMaskTile &&
                              half_v[k0 + j] <= (float)kMaskTile;
            t.tile_dil = near ? tj.j[k0 + j].dil : nullptr;
            t.tiles_w = tj.j[k0 + j].tiles_w;
            t.key_thr = thin_key_threshold(v.mask_type, tp->tau_thin);
            memcpy(t.R, v.cam.R, sizeof(t.R));
            memcpy(t.t, v.cam.t, sizeof(t.t));
        }
        const int blocks = grid_for(c->cap, c->sm_count);
        const int32_t acc = c->n_views + k0 > 0 ? 1 : 0;
        DIVAS_CUDA(c, cudaMemsetAsync(n_heavy, 0, sizeof(int32_t), s));
        const int nv = tb.n;
        const bool f16 = batch_all_f16(tb);
        if (c->G.contracted)
            st = f16 ? launch_tuple_scan<true, kMaskF16>(nv, blocks, s, c, tb, T, acc, heavy, n_heavy)
                     : launch_tuple_scan<true, -1>(nv, blocks, s, c, tb, T, acc, heavy, n_heavy);
        else
            st = f16 ? launch_tuple_scan<false, kMaskF16>(nv, blocks, s, c, tb, T, acc, heavy, n_heavy)
                     : launch_tuple_scan<false, -1>(nv, blocks, s, c, tb, T, acc, heavy, n_heavy);
        if (st != DIVAS_OK) return st;
        if (last) {
            st = record_stage(c, stage_events, 2, s);
            if (st != DIVAS_OK) return st;
        }
#define DIVAS_TUPLE_HEAVY(KC, MT)                                                                  \
    k_tuple_heavy<KC, MT><<<blocks, kThreads, 0, s>>>(c->active, heavy, n_heavy, c->G, c->F, tb, T,  \
                                                      c->W, c->Z, c->bits)
        if (c->G.contracted) {
            if (f16) DIVAS_TUPLE_HEAVY(true, kMaskF16);
            else DIVAS_TUPLE_HEAVY(true, -1);
        } else {
            if (f16) DIVAS_TUPLE_HEAVY(false, kMaskF16);
            else DIVAS_TUPLE_HEAVY(false, -1);
        }
#undef DIVAS_TUPLE_HEAVY
        DIVAS_LAUNCHED(c, "k_tuple_heavy");
    }
    c->n_views += n_views;
    return record_stage(c, stage_events, 3, s);
}

divas_status divas_debug_integral_images(const uint16_t* n_samp, int32_t W, int32_t H,
                                         uint32_t* s1, uint64_t* s2, void* stream) {
    if (!n_samp || !s1 || !s2 || W < 1 || H < 1 || (int64_t)(W + 1) * (H + 1) > INT32_MAX)
        return DIVAS_E_INVALID;
    const int32_t strips = (H + kSatRows - 1) / kSatRows;
    void* tot = nullptr;
    if (cudaMalloc(&tot, (size_t)strips * W * 12) != cudaSuccess) {
        (void)cudaGetLastError();
        return DIVAS_E_CUDA;
    }
    SatJobs jobs;
    memset(&jobs, 0, sizeof(jobs));
    jobs.n = 1;
    jobs.j[0].n = n_samp;
    jobs.j[0].s1 = s1;
    jobs.j[0].s2 = reinterpret_cast<unsigned long long*>(s2);
    jobs.j[0].t2 = static_cast<unsigned long long*>(tot);
    jobs.j[0].t1 = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(tot) + (size_t)strips * W * 8);
    jobs.j[0].W = W;
    jobs.j[0].H = H;
    const cudaStream_t s = S(stream);
    k_sat_strip_totals<<<dim3(strips, 1), kSatThreads, 0, s>>>(jobs);
    k_sat_strip_fill<<<dim3(strips, 1), kSatThreads, 0, s>>>(jobs);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(tot);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? DIVAS_OK : DIVAS_E_CUDA;
}

}  // extern "C"
