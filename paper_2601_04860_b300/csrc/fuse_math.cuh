// fuse_math.cuh -- per-voxel, per-view arithmetic of the thick-path fusion.
//
// One (voxel, view) pair is evaluated exactly as Algorithms A.2 / B.5 state
// the thick path (Sec. 3.5): project the voxel centre, read depth and mask at
// the pixel, gate on the mask (m >= tau) and on depth consistency
// (|p_z - D| <= gamma h_v), and add the Gaussian depth weight
// w = exp(-alpha1 (e / Delta)^2) (Eq. gs-depthweight with the depth band
// [D - Delta, D + Delta]) to W and Z (Eq. vmask).  The evaluation is split in
// three steps -- project(), load_raster(), decide() -- so that the fusion
// kernel can issue the raster loads of several views back to back while
// every kernel (single view, many views, adjoint, projection hook) still runs
// the very same arithmetic.  The library is compiled with -fmad=false, so
// only the explicit __fmaf_rn below are fused and all kernels round alike.
//
// Precision.  Decisions (pixel index, gates) and weights must agree with a
// double-precision evaluation.  Plain FP32 would not do for the depth: p_z ~
// 2.5 carries ~2.4e-7 rounding while e = p_z - D is compared with Delta ~
// 8e-3, so e / Delta would be off by ~4e-5.  Two schemes are used:
//
//  * Plain grids (lattice projection).  Voxel centres are x = o + (h/2) n
//    with n = 2 idx + 1 an odd integer (|n| < 2^11), so camera coordinates
//    are p = T + M n with T = R o + t and M = (h/2) R, formed on the host in
//    double.  The depth row is split into a "hi" part rounded to a multiple
//    of a power of two 2^q -- chosen so that |T_z| + sum |M_z| (2g - 1) <
//    2^(q+24) -- and a small "lo" remainder.  Every partial sum of
//    T_hi + M_hi n is then a multiple of 2^q below 2^(q+24): the FMA chain
//    is exact in FP32, and the lo chain adds a term of
//    relative size 2^-36.  The pixel coordinates only decide which pixel is
//    read, so they take the intrinsics-folded rows u p_z = (fx M_x + cx M_z) n
//    + (fx T_x + cx T_z) (and likewise v) in one plain chain each and a
//    multiply by 1 / p_z: a few ulp of |Ku n| + |Tu|, i.e. about 1e-4 pixel
//    for the benchmark cameras, well inside the 1e-6-relative band within
//    which a pixel decision counts as a tie.
//
//  * Contracted grids.  Centres are uncontracted in hi + lo pairs; the three
//    rows are plain FMA chains over the hi and lo parts, which place the
//    pixel (inside the same tie band as above).  The depth gate first screens
//    the plain depth: a bound on its error (x_s = fl(x_hi + x_lo) within 2^-24
//    of |x_hi| + |x_lo| per coordinate, three roundings of partial sums below
//    S = sum |R_zj| (|x_hi,j| + |x_lo,j|) + |t_z|: at most 2^-21.9 S)
//    widened to 2^-19 S rejects |e| > Delta for certain.
//    Only pairs that pass every other gate and the screen (about 0.1% of
//    the voxel-views of an unbounded scene) form the depth as a compensated
//    dot product (error-free products via FMA and error-free sums: Ogita,
//    Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
//    2005) and decide on it, so decisions and weights are those of the
//    compensated depth everywhere.
//
// In both, e = (p_z,hi - D) + p_z,lo, where p_z,hi - D is exact by
// Sterbenz's lemma whenever the depth gate can pass.
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda_fp16.h>

namespace divas {

constexpr int kMaxViews = 32;

// Programmatic dependent launch: a kernel launched with the programmatic
// stream serialization attribute may start while its predecessor on the
// stream finishes; it waits in wait_for_producer (which returns at once for a
// kernel launched without the attribute) before it reads that kernel's
// results, and a producer that lets its dependents start early says so with
// allow_dependents.
__device__ __forceinline__ void wait_for_producer() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void allow_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

constexpr int kViewChunk = 4;  // views whose raster loads are issued together

// ---------------------------------------------------------------------------
// error-free transformations (round-to-nearest FP32, no contraction)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// hi + lo = a0 xh0 + a1 xh1 + a2 xh2 + c + (a . xl), relative error ~2^-44
__device__ __forceinline__ void dot3c(float a0, float a1, float a2, const float* xh,
                                      const float* xl, float c, float& hi, float& lo) {
    float p0, e0, p1, e1, p2, e2;
    two_prod(a0, xh[0], p0, e0);
    two_prod(a1, xh[1], p1, e1);
    two_prod(a2, xh[2], p2, e2);
    float s, t1, t2, t3;
    two_sum(c, p0, s, t1);
    two_sum(s, p1, s, t2);
    two_sum(s, p2, s, t3);
    float l = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, t1)), __fadd_rn(t2, t3));
    l = __fmaf_rn(a0, xl[0], __fmaf_rn(a1, xl[1], __fmaf_rn(a2, xl[2], l)));
    two_sum(s, l, hi, lo);
}

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
// One view, passed by value inside kernel parameters.
//   plain grid:      A = M_hi, B = M_lo (row-major 3x3), C = T_hi, E = T_lo
//   contracted grid: A = R, C = t (B, E unused)
// Per-view constants (112 bytes, so that a batch of 32 views stays within the
// classic 4 KB kernel-parameter space).  Plain grids: A = (Ku, Kv, M_z hi),
// B = M_z lo, C = (Tu, Tv, T_z hi), E = T_z lo; K = (M_z rounded to float,
// the depth screen's slack 2^-20 b_max rounded up, b_max = |T_z| + 2 g
// sum_j |M_zj|) -- K holds the intrinsics (fx, fy, cx, cy) only for the
// depth-tuple modes' unfolded views.  Contracted grids: A = (Ku,
// Kv, R_z) with Ku = fx R_x + cx R_z, Kv = fy R_y + cy R_z, C = (fx t_x + cx
// t_z, fy t_y + cy t_z, t_z); the depth screen's bound is
// B[0] n1 + E >= 2^-19 S with B[0] >= 2^-19 max_j |R_zj| and E = 2^-19 |t_z|
// (n1 = sum_j |x_hi,j| + |x_lo,j| per voxel); B[1], B[2] are unused.
struct ViewC {
    float A[9];
    float B[3];
    float C[3];
    float E;
    float K[4];
    int32_t W, H;    // raster size (W is the row pitch in elements)
    int32_t mask_type;
    uint32_t bit;    // 1 << view index, 0 from view 32 on
    const float* depth;
    const void* mask;
};
static_assert(sizeof(ViewC) == 112, "ViewC layout");

// pixel index of (u, v) -- finite, as they are in front of the camera -- or -1
// outside the half-open frame [0, W) x [0, H): floor(u) in [0, W) iff
// 0 <= u < W, so one unsigned compare per axis on the floor conversions that
// the index needs anyway (saturated conversions of huge values fall outside)
__device__ __forceinline__ int32_t pixel_index(const ViewC& V, bool front, float u, float v) {
    const int32_t iu = __float2int_rd(u), iv = __float2int_rd(v);
    const bool in = front && (uint32_t)iu < (uint32_t)V.W && (uint32_t)iv < (uint32_t)V.H;
    return in ? iv * V.W + iu : -1;
}

struct ViewBatch {
    int32_t n;
    int32_t pad;
    ViewC v[kMaxViews];
};
static_assert(sizeof(ViewBatch) <= 3900, "a view batch and the other kernel arguments fit 4 KB");

struct GridC {
    float origin[3];
    float h;
    int32_t g;
    int32_t contracted;
    float inv_h;  // 1/h when h is a power of two (exact), else 0
    int32_t pad;
    // plain grids: Delta = fl(gamma h), 1 / Delta (rounded to nearest) and
    // Delta (1 + 2^-20) rounded up, the same for every voxel
    float delta, inv_delta, delta_s;
    int32_t pad2;
};

struct FuseC {
    float gamma, alpha1, tau_m, logit_tau, z_near, eps, tau_cons;
    int32_t pad;
};

enum : int32_t { kMaskF32 = 0, kMaskF16 = 1, kMaskLogit = 2 };

// ---------------------------------------------------------------------------
// voxel centre and its depth tolerance Delta = gamma h_v
// ---------------------------------------------------------------------------
struct VoxelGeom {
    float xh[3], xl[3];  // plain grid: xh = n = 2 idx + 1, xl unused
    float Delta, invDelta;
    float hv;            // world edge h_v
    // contracted grids: x_s = fl(x_hi + x_lo), the centre the plain rows use,
    // and for the depth screen n1 = sum_j |x_hi,j| + |x_lo,j| (rounded up);
    // both kinds: Delta (1 + 2^-20) rounded up
    float xs[3];
    float n1, DeltaS;
    bool ok;  // false: contracted centre with |c| >= 2 (no world position)
};

// n / d for 32-bit n by a divisor fixed per context: multiply-high and shift
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994); exact for every 32-bit n.
struct FastDiv {
    uint32_t m, d;
    int32_t l;
    int32_t pad;
};

__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
    if (f.l == 0) return n;  // d = 1
    const uint32_t t = __umulhi(n, f.m);
    return (t + ((n - t) >> 1)) >> (f.l - 1);
}

// active-list entries are packed voxel coordinates i | j << 10 | k << 20
__device__ __forceinline__ void unpack(uint32_t pk, int32_t& i, int32_t& j, int32_t& k) {
    i = (int32_t)(pk & 1023u);
    j = (int32_t)((pk >> 10) & 1023u);
    k = (int32_t)(pk >> 20);
}

__device__ __forceinline__ int64_t packed_lin(uint32_t pk, int32_t g) {
    int32_t i, j, k;
    unpack(pk, i, j, k);
    return ((int64_t)k * g + j) * g + i;
}

// ---------------------------------------------------------------------------
// reciprocal of a normal, positive float: the hardware approximation (relative
// error below 2^-22) refined by one Newton-Raphson step r' = r + r (1 - x r),
// which squares the error; the result is within one ulp of 1/x.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_nr(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return __fmaf_rn(r, __fmaf_rn(-x, r, 1.f), r);
}

template <bool kContracted>
__device__ __forceinline__ VoxelGeom voxel_geom(uint32_t pk, const GridC& G, float gamma) {
    VoxelGeom vg;
    int32_t i, j, k;
    unpack(pk, i, j, k);
    vg.ok = true;
    if (!kContracted) {
        vg.xh[0] = (float)(2 * i + 1);
        vg.xh[1] = (float)(2 * j + 1);
        vg.xh[2] = (float)(2 * k + 1);
        vg.xl[0] = vg.xl[1] = vg.xl[2] = 0.f;
        vg.hv = G.h;
        vg.Delta = G.delta;  // fl(gamma h), from the host
        vg.invDelta = G.inv_delta;
        vg.DeltaS = G.delta_s;
        return vg;
    }
    const float idx[3] = {(float)i, (float)j, (float)k};
    float ch[3], cl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // c = origin + (idx + 1/2) h, exactly as hi + lo
        float p, pe, s, se;
        two_prod(__fadd_rn(idx[a], 0.5f), G.h, p, pe);
        two_sum(G.origin[a], p, s, se);
        ch[a] = s;
        cl[a] = __fadd_rn(se, pe);
    }
    float hv = G.h;
    // n2 = |c|^2 as hi + lo
    float s = 0.f, e = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float p, pe, t;
        two_prod(ch[a], ch[a], p, pe);
        two_sum(s, p, s, t);
        e = __fadd_rn(e, __fadd_rn(__fadd_rn(t, pe), __fmul_rn(2.f, __fmul_rn(ch[a], cl[a]))));
    }
    float n2h, n2l;
    two_sum(s, e, n2h, n2l);
    const bool outside = (n2h > 4.f) || (n2h == 4.f && n2l >= 0.f);
    const bool inner = (n2h < 1.f) || (n2h == 1.f && n2l <= 0.f);
#pragma unroll
    for (int a = 0; a < 3; ++a) { vg.xh[a] = ch[a]; vg.xl[a] = cl[a]; }
    if (outside) {
        vg.ok = false;
    } else if (!inner) {
        // rho = sqrt(n2) as hi + lo
        const float rh = __fsqrt_rn(n2h);
        const float rl = __fmul_rn(__fadd_rn(__fmaf_rn(-rh, rh, n2h), n2l), rcp_nr(__fmul_rn(2.f, rh)));
        // d = 2 - rho (2 - rh is exact for rh in [1, 2])
        float dh, dl;
        two_sum(__fsub_rn(2.f, rh), -rl, dh, dl);
        // den = rho d
        float qh, ql;
        two_prod(rh, dh, qh, ql);
        ql = __fadd_rn(ql, __fadd_rn(__fmul_rn(rh, dl), __fmul_rn(rl, dh)));
        two_sum(qh, ql, qh, ql);
        // sc = 1 / den (the lo part corrects the hi reciprocal's error)
        const float sh = rcp_nr(qh);
        const float res = __fsub_rn(__fmaf_rn(-sh, qh, 1.f), __fmul_rn(sh, ql));
        const float sl = __fmul_rn(sh, res);
        // x = c sc
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float xh, xe;
            two_prod(ch[a], sh, xh, xe);
            xe = __fadd_rn(xe, __fadd_rn(__fmul_rn(ch[a], sl), __fmul_rn(cl[a], sh)));
            two_sum(xh, xe, vg.xh[a], vg.xl[a]);
        }
        const float d = __fadd_rn(dh, dl);
        hv = __fmul_rn(G.h, rcp_nr(__fmul_rn(d, d)));  // largest stretch of the inverse contraction
    }
    vg.hv = hv;
    vg.Delta = __fmul_rn(gamma, hv);
    vg.invDelta = rcp_nr(vg.Delta);
    vg.n1 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vg.xs[a] = __fadd_rn(vg.xh[a], vg.xl[a]);
        vg.n1 = __fadd_ru(vg.n1, __fadd_ru(fabsf(vg.xh[a]), fabsf(vg.xl[a])));
    }
    vg.DeltaS = __fmul_ru(vg.Delta, 1.f + 0x1p-20f);
    return vg;
}

// ---------------------------------------------------------------------------
// step 1: projection -> pixel index (or -1) and camera depth p_z = hi + lo
// (branch-free: every quantity is computed, validity is a predicate)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void lattice_row(const float* Mh, const float* Ml, float Th, float Tl,
                                            const float* n, float& hi, float& lo) {
    hi = __fmaf_rn(Mh[0], n[0], __fmaf_rn(Mh[1], n[1], __fmaf_rn(Mh[2], n[2], Th)));  // exact
    lo = __fmaf_rn(Ml[0], n[0], __fmaf_rn(Ml[1], n[1], __fmaf_rn(Ml[2], n[2], Tl)));
}

template <bool kContracted>
__device__ __forceinline__ int32_t project(const ViewC& V, const VoxelGeom& vg, float z_near,
                                           float& pzh, float& pzl) {
    float pz, u, v;
    if (!kContracted) {
        // the depth in a plain FMA chain over the rounded row (within 2^-21.6
        // b_max of the exact lattice depth; made exact by depth_error where the
        // screen lets it pass), returned as (plain, 0); the pixel rows
        // u p_z = Ku n + Tu and v p_z = Kv n + Tv likewise (a few ulp of
        // |Ku n| + |Tu|: about 1e-4 pixel on the benchmark cameras)
        pz = __fmaf_rn(V.K[0], vg.xh[0], __fmaf_rn(V.K[1], vg.xh[1], __fmaf_rn(V.K[2], vg.xh[2], V.C[2])));
        pzh = pz;
        pzl = 0.f;
        const float pu = __fmaf_rn(V.A[0], vg.xh[0],
                                   __fmaf_rn(V.A[1], vg.xh[1], __fmaf_rn(V.A[2], vg.xh[2], V.C[0])));
        const float pv = __fmaf_rn(V.A[3], vg.xh[0],
                                   __fmaf_rn(V.A[4], vg.xh[1], __fmaf_rn(V.A[5], vg.xh[2], V.C[1])));
        const bool front = pz > z_near && pz <= FLT_MAX;
        const float inv = rcp_nr(front ? pz : 1.f);
        u = __fmul_rn(pu, inv);
        v = __fmul_rn(pv, inv);
        return pixel_index(V, front, u, v);
    }
    // the three rows in plain FMA chains over the rounded centre x_s: the
    // depth row R_z x + t_z and the intrinsics-folded pixel rows
    // u p_z = (fx R_x + cx R_z) x + (fx t_x + cx t_z) (and likewise v), each
    // within 4 ulp of sum_j |row_j x_j| + |const| (about 1e-4 pixel at |x| = 256
    // for the benchmark cameras); the depth is returned as (plain, 0) and made
    // exact by depth_error only where the screen lets it pass
    pz = __fmaf_rn(V.A[6], vg.xs[0], __fmaf_rn(V.A[7], vg.xs[1], __fmaf_rn(V.A[8], vg.xs[2], V.C[2])));
    pzh = pz;
    pzl = 0.f;
    const float pu = __fmaf_rn(V.A[0], vg.xs[0], __fmaf_rn(V.A[1], vg.xs[1], __fmaf_rn(V.A[2], vg.xs[2], V.C[0])));
    const float pv = __fmaf_rn(V.A[3], vg.xs[0], __fmaf_rn(V.A[4], vg.xs[1], __fmaf_rn(V.A[5], vg.xs[2], V.C[1])));
    const bool front = pz > z_near && pz <= FLT_MAX;
    const float inv = rcp_nr(front ? pz : 1.f);
    u = __fmul_rn(pu, inv);
    v = __fmul_rn(pv, inv);
    return pixel_index(V, front, u, v);
}

// ---------------------------------------------------------------------------
// step 2: raster reads (depth and the mask's raw value, widened to float);
// an invalid pixel reads pixel 0 (always in bounds) and is discarded later
// ---------------------------------------------------------------------------
// the view's mask type: kMT when it is fixed at compile time (kMT >= 0)
template <int kMT>
__device__ __forceinline__ int32_t mask_type_of(const ViewC& V) {
    return kMT >= 0 ? kMT : V.mask_type;
}

template <int kMT = -1>
__device__ __forceinline__ void load_raster(const ViewC& V, int32_t pix, float& D, float& raw) {
    const int32_t p = pix >= 0 ? pix : 0;
    D = __ldg(V.depth + p);
    if (mask_type_of<kMT>(V) == kMaskF16)
        raw = __half2float(
            __ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(V.mask) + p)));
    else
        raw = __ldg(reinterpret_cast<const float*>(V.mask) + p);
}

// ---------------------------------------------------------------------------
// step 3: gates (predicates) and, for an accepted vote, the weight
// ---------------------------------------------------------------------------
// False only where |e| > Delta for certain.  Contracted grids: the plain depth
// pz differs from the exact one by at most 2^-21.9 S; fl(pz - D) adds 2^-24
// of itself; the exact e = fl(fl(p_z,hi - D) + p_z,lo) is within 2^-23 of
// its own size of p_z - D.  So |e| <= Delta implies
// |fl(pz - D)| <= Delta (1 + 2^-22) + 2^-21.2 S, which the threshold
// Delta (1 + 2^-20) + 2^-19 S, summed rounding up, exceeds.  Plain grids:
// the plain depth is within 5.2 2^-24 b_max of the exact pair (rounded row,
// T_z's lo part left out, three FMAs), so |e| <= Delta implies
// |fl(pz - D)| <= Delta (1 + 2^-21.9) + 5.3 2^-24 b_max, below the
// threshold Delta (1 + 2^-20) + 2^-20 b_max summed rounding up.
template <bool kContracted>
__device__ __forceinline__ bool depth_screen(const ViewC& V, const VoxelGeom& vg, float pzh,
                                             float D) {
    const float thr = kContracted ? __fadd_ru(vg.DeltaS, __fmaf_ru(V.B[0], vg.n1, V.E))
                                  : __fadd_ru(vg.DeltaS, V.K[3]);
    return fabsf(__fsub_rn(pzh, D)) <= thr;
}

// e = p_z - D from the exact depth: plain grids the lattice row as hi + lo
// (the hi chain is exact), contracted grids the compensated dot product
template <bool kContracted>
__device__ __forceinline__ float depth_error(const ViewC& V, const VoxelGeom& vg, float pzh,
                                             float pzl, float D) {
    if (kContracted)
        dot3c(V.A[6], V.A[7], V.A[8], vg.xh, vg.xl, V.C[2], pzh, pzl);
    else
        lattice_row(V.A + 6, V.B, V.C[2], V.E, vg.xh, pzh, pzl);
    return __fadd_rn(__fsub_rn(pzh, D), pzl);
}

// the gates before the depth gate: a pixel in frame, a surface there (+inf,
// NaN or <= 0 depth: none), the mask gate and the depth screen
template <bool kContracted, int kMT = -1>
__device__ __forceinline__ bool pre_gates(const ViewC& V, const VoxelGeom& vg, const FuseC& F,
                                          int32_t pix, float pzh, float D, float raw) {
    const float thr = mask_type_of<kMT>(V) == kMaskLogit ? F.logit_tau : F.tau_m;
    return pix >= 0 && D > 0.f && D <= FLT_MAX && raw >= thr &&
           depth_screen<kContracted>(V, vg, pzh, D);
}

template <bool kContracted, int kMT = -1>
__device__ __forceinline__ bool gates(const ViewC& V, const VoxelGeom& vg, const FuseC& F,
                                      int32_t pix, float pzh, float pzl, float D, float raw,
                                      float& e) {
    if (!pre_gates<kContracted, kMT>(V, vg, F, pix, pzh, D, raw)) return false;
    e = depth_error<kContracted>(V, vg, pzh, pzl, D);
    return fabsf(e) <= vg.Delta;
}

template <int kMT = -1>
__device__ __forceinline__ void weight(const ViewC& V, const VoxelGeom& vg, const FuseC& F,
                                       float raw, float e, float& m, float& w) {
    m = mask_type_of<kMT>(V) == kMaskLogit ? __frcp_rn(__fadd_rn(1.f, expf(-raw))) : raw;
    const float r = __fmul_rn(e, vg.invDelta);
    w = expf(-__fmul_rn(F.alpha1, __fmul_rn(r, r)));
}

// One accepted thick-path vote: everything the adjoint needs.
struct Vote {
    int32_t pix;
    float m, w, e;
};

template <bool kContracted>
__device__ __forceinline__ bool eval_vote(const ViewC& V, const VoxelGeom& vg, const FuseC& F,
                                          Vote& out) {
    float pzh, pzl, D, raw;
    const int32_t pix = project<kContracted>(V, vg, F.z_near, pzh, pzl);
    load_raster(V, pix, D, raw);
    if (!gates<kContracted>(V, vg, F, pix, pzh, pzl, D, raw, out.e)) return false;
    weight(V, vg, F, raw, out.e, out.m, out.w);
    out.pix = pix;
    return true;
}

// Fold views [0, VB.n) of a batch into (W, Z, bits), in view order, for
// VB.n <= 4 kChunks.  The view loop is unrolled at compile time so that every
// view constant is an immediate constant-bank operand (a runtime view index
// would turn each of them into a register-indexed constant load); the raster
// loads of kViewChunk views are issued before any of them is consumed, and
// only accepted votes (a few percent) branch into the weight computation.
// kF16Full: every view's mask is binary16 and VB.n == 4 kChunks, so the mask
// type and the view count are compile-time constants (no per-view branches
// on them); the arithmetic is the same.
template <bool kContracted, int kChunks, bool kF16Full = false>
__device__ __forceinline__ void fold_views(const ViewBatch& VB, const VoxelGeom& vg,
                                           const FuseC& F, float& W, float& Z, uint32_t& bits) {
    constexpr int kMT = kF16Full ? kMaskF16 : -1;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
        int32_t pix[kViewChunk];
        float pzh[kViewChunk], pzl[kViewChunk], D[kViewChunk], raw[kViewChunk];
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q) {
            pix[q] = -1;
            if (kF16Full || c * kViewChunk + q < VB.n)
                pix[q] = project<kContracted>(VB.v[c * kViewChunk + q], vg, F.z_near, pzh[q], pzl[q]);
        }
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q)
            if (kF16Full || c * kViewChunk + q < VB.n)
                load_raster<kMT>(VB.v[c * kViewChunk + q], pix[q], D[q], raw[q]);
        // the chunk's gates up to the depth screen as predicates, then one
        // branch into the (rare) candidates, whose exact depth decides and
        // weighs, added in view order
        uint32_t acc = 0u;
#pragma unroll
        for (int q = 0; q < kViewChunk; ++q) {
            if (!kF16Full && c * kViewChunk + q >= VB.n) break;
            const ViewC& V = VB.v[c * kViewChunk + q];
            if (pre_gates<kContracted, kMT>(V, vg, F, pix[q], pzh[q], D[q], raw[q])) acc |= 1u << q;
        }
        if (acc) {
#pragma unroll
            for (int q = 0; q < kViewChunk; ++q) {
                if (acc & (1u << q)) {
                    const ViewC& V = VB.v[c * kViewChunk + q];
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


// Fold the views sv[0, n) (a runtime count, e.g. a session's views staged in
// shared memory) into kVPT independent voxels at once: the same per-view
// arithmetic and the same view order as fold_views, so the results are
// bitwise identical.  kVPT voxels x (4 / kVPT) views of projections and raster
// loads are in flight together.
template <bool kContracted, int kVPT>
__device__ __forceinline__ void fold_views_multi(const ViewC* sv, int32_t n, const VoxelGeom* vg,
                                                 const bool* live, const FuseC& F, float* W,
                                                 float* Z, uint32_t* bits) {
    constexpr int kC = kViewChunk / kVPT > 0 ? kViewChunk / kVPT : 1;
    for (int32_t v0 = 0; v0 < n; v0 += kC) {
        int32_t pix[kVPT][kC];
        float pzh[kVPT][kC], pzl[kVPT][kC], D[kVPT][kC], raw[kVPT][kC];
#pragma unroll
        for (int j = 0; j < kVPT; ++j)
#pragma unroll
            for (int q = 0; q < kC; ++q) {
                pix[j][q] = -1;
                pzh[j][q] = pzl[j][q] = 0.f;
                if (v0 + q < n && live[j] && vg[j].ok)
                    pix[j][q] = project<kContracted>(sv[v0 + q], vg[j], F.z_near, pzh[j][q], pzl[j][q]);
            }
#pragma unroll
        for (int j = 0; j < kVPT; ++j)
#pragma unroll
            for (int q = 0; q < kC; ++q)
                if (v0 + q < n) load_raster(sv[v0 + q], pix[j][q], D[j][q], raw[j][q]);
#pragma unroll
        for (int j = 0; j < kVPT; ++j)
#pragma unroll
            for (int q = 0; q < kC; ++q) {
                if (v0 + q >= n) break;
                const ViewC& V = sv[v0 + q];
                float e;
                if (gates<kContracted>(V, vg[j], F, pix[j][q], pzh[j][q], pzl[j][q], D[j][q],
                                       raw[j][q], e)) {
                    float m, w;
                    weight(V, vg[j], F, raw[j][q], e, m, w);
                    W[j] = __fmaf_rn(m, w, W[j]);
                    Z[j] = __fadd_rn(Z[j], w);
                    bits[j] |= V.bit;
                }
            }
    }
}

}  // namespace divas
