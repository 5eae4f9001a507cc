// fuse_math.cuh -- per-voxel, per-view arithmetic of the thick-path fusion.
//
// One __device__ function (`vote`) evaluates one (voxel, view) pair exactly
// as Algorithms A.2 / B.5 state the thick path (Sec. 3.5): project the voxel
// centre, read depth and mask at the pixel, gate on the mask (m >= tau) and
// on depth consistency (|p_z - D| <= gamma h_v), and add the Gaussian depth
// weight w = exp(-alpha1 (e / Delta)^2) (Eq. gs-depthweight with the depth
// band [D - Delta, D + Delta]) to W and Z (Eq. vmask).  Every kernel that
// folds views in (single view, many views, batched sessions, the adjoint)
// calls these functions, and the library is compiled with -fmad=false, so
// all of them produce bitwise identical results.
//
// Precision.  The decisions (pixel index, gates) and the weights must agree
// with a double-precision evaluation.  Plain FP32 would not do: p_z ~ 2.5 is
// rounded to ~2.4e-7 while the depth residual e = p_z - D is compared with
// Delta ~ 8e-3, so e / Delta would carry ~4e-5 relative error.  The camera
// coordinates are therefore evaluated as unevaluated sums hi + lo of two
// floats (error-free products via FMA and error-free sums, i.e. the
// compensated dot product of Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005), and e is formed as (p_z,hi - D) +
// p_z,lo, where p_z,hi - D is exact by Sterbenz's lemma whenever the gate can
// pass.  Voxel centres are likewise kept as hi + lo pairs, including the
// inverse scene contraction of contracted grids.
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda_fp16.h>

namespace divas {

constexpr int kMaxViews = 32;

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
struct ViewC {  // one view, passed by value inside kernel parameters
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float Wf, Hf;    // raster size as floats (frame test)
    int32_t W;       // row pitch in elements
    int32_t mask_type;
    uint32_t bit;    // 1 << view index, 0 from view 32 on
    int32_t pad;
    const float* depth;
    const void* mask;
};

struct ViewBatch {
    int32_t n;
    int32_t pad;
    ViewC v[kMaxViews];
};

struct GridC {
    float origin[3];
    float h;
    int32_t g;
    int32_t contracted;
};

struct FuseC {
    float gamma, alpha1, tau_m, logit_tau, z_near, eps, tau_cons;
    int32_t pad;
};

enum : int32_t { kMaskF32 = 0, kMaskF16 = 1, kMaskLogit = 2 };

// ---------------------------------------------------------------------------
// voxel centre (hi + lo per axis) and its depth tolerance Delta = gamma h_v
// ---------------------------------------------------------------------------
struct VoxelGeom {
    float xh[3], xl[3];
    float Delta, invDelta;
    bool ok;  // false: contracted centre with |c| >= 2 (no world position)
};

__device__ __forceinline__ VoxelGeom voxel_geom(int32_t lin, const GridC& G, float gamma) {
    VoxelGeom vg;
    const int32_t g = G.g;
    const int32_t i = lin % g;
    const int32_t r = lin / g;
    const int32_t j = r % g;
    const int32_t k = r / g;
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
    vg.ok = true;
    if (!G.contracted) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { vg.xh[a] = ch[a]; vg.xl[a] = cl[a]; }
    } else {
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
        if (outside) {
            vg.ok = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) { vg.xh[a] = ch[a]; vg.xl[a] = cl[a]; }
        } else if (inner) {
#pragma unroll
            for (int a = 0; a < 3; ++a) { vg.xh[a] = ch[a]; vg.xl[a] = cl[a]; }
        } else {
            // rho = sqrt(n2) as hi + lo
            const float rh = __fsqrt_rn(n2h);
            const float rl = __fdiv_rn(__fadd_rn(__fmaf_rn(-rh, rh, n2h), n2l), __fmul_rn(2.f, rh));
            // d = 2 - rho (2 - rh is exact for rh in [1, 2])
            float dh, dl;
            two_sum(__fsub_rn(2.f, rh), -rl, dh, dl);
            // den = rho d
            float qh, ql;
            two_prod(rh, dh, qh, ql);
            ql = __fadd_rn(ql, __fadd_rn(__fmul_rn(rh, dl), __fmul_rn(rl, dh)));
            two_sum(qh, ql, qh, ql);
            // sc = 1 / den
            const float sh = __frcp_rn(qh);
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
            hv = __fdiv_rn(G.h, __fmul_rn(d, d));  // largest stretch of the inverse contraction
        }
    }
    vg.Delta = __fmul_rn(gamma, hv);
    vg.invDelta = __frcp_rn(vg.Delta);
    return vg;
}

// ---------------------------------------------------------------------------
// projection: pixel index, and camera depth p_z as hi + lo
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool project_voxel(const ViewC& V, const VoxelGeom& vg, float z_near,
                                              int32_t& pix, float& pzh, float& pzl) {
    dot3c(V.R[6], V.R[7], V.R[8], vg.xh, vg.xl, V.t[2], pzh, pzl);
    if (!(pzh > z_near)) return false;
    float pxh, pxl, pyh, pyl;
    dot3c(V.R[0], V.R[1], V.R[2], vg.xh, vg.xl, V.t[0], pxh, pxl);
    dot3c(V.R[3], V.R[4], V.R[5], vg.xh, vg.xl, V.t[1], pyh, pyl);
    const float inv = __frcp_rn(pzh);
    const float u = __fmaf_rn(V.fx, __fmul_rn(pxh, inv), V.cx);
    const float v = __fmaf_rn(V.fy, __fmul_rn(pyh, inv), V.cy);
    if (!(u >= 0.f && u < V.Wf && v >= 0.f && v < V.Hf)) return false;
    pix = (int32_t)v * V.W + (int32_t)u;  // u, v >= 0: truncation is floor
    return true;
}

// mask probability m at pix and whether it passes the thick-path gate
__device__ __forceinline__ bool read_mask(const ViewC& V, int32_t pix, const FuseC& F, float& m) {
    if (V.mask_type == kMaskF16) {
        const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(V.mask) + pix);
        m = __half2float(__ushort_as_half(b));
        return m >= F.tau_m;
    }
    const float raw = __ldg(reinterpret_cast<const float*>(V.mask) + pix);
    if (V.mask_type == kMaskLogit) {
        m = __frcp_rn(__fadd_rn(1.f, expf(-raw)));
        return raw >= F.logit_tau;
    }
    m = raw;
    return m >= F.tau_m;
}

// One accepted thick-path vote: everything the adjoint needs.
struct Vote {
    int32_t pix;
    float m, w, e;
};

__device__ __forceinline__ bool eval_vote(const ViewC& V, const VoxelGeom& vg, const FuseC& F,
                                          Vote& out) {
    int32_t pix;
    float pzh, pzl;
    if (!project_voxel(V, vg, F.z_near, pix, pzh, pzl)) return false;
    const float D = __ldg(V.depth + pix);
    if (!(D > 0.f && D <= FLT_MAX)) return false;  // +inf, NaN, <= 0: no surface
    float m;
    if (!read_mask(V, pix, F, m)) return false;
    const float e = __fadd_rn(__fsub_rn(pzh, D), pzl);
    if (!(fabsf(e) <= vg.Delta)) return false;
    const float r = __fmul_rn(e, vg.invDelta);
    out.pix = pix;
    out.m = m;
    out.e = e;
    out.w = expf(-__fmul_rn(F.alpha1, __fmul_rn(r, r)));
    return true;
}

__device__ __forceinline__ void vote(const ViewC& V, const VoxelGeom& vg, const FuseC& F,
                                     float& W, float& Z, uint32_t& bits) {
    Vote vt;
    if (!eval_vote(V, vg, F, vt)) return;
    W = __fmaf_rn(vt.m, vt.w, W);
    Z = __fadd_rn(Z, vt.w);
    bits |= V.bit;
}

}  // namespace divas
