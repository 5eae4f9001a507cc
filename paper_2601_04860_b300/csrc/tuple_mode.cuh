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
    const uint32_t* sat1;            // (H + 1) x (W + 1) integral image of n_samp (mod 2^32)
    const unsigned long long* sat2;  // same of n_samp^2 (mod 2^64)
    float R[9], t[3];                // world -> camera (unprojection)
    float st_thr;                    // gamma_st * d_cam (see-through threshold on d_med)
    float pad;
};

struct TViewBatch {
    int32_t n;
    int32_t pad;
    TViewC v[kMaxTupleViews];
};
static_assert(sizeof(TViewBatch) <= 3800, "a tuple view batch and the other arguments fit 4 KB");

struct TupleC {
    float beta, tau_thin, rho_cover, rho_occ, n_abs, dist_gate, behind_margin, k_dg;
    int32_t thin_on;
    int32_t pad;
};

// camera depth (hi + lo) and pixel coordinates of a lattice point (plain
// grids: n = 2 idx + 1 + corner offset) or a world point (contracted grids:
// hi + lo); false when it is not in front of the camera
template <bool kContracted>
__device__ __forceinline__ bool project_uv(const ViewC& V, const float* nh, const float* nl,
                                           float z_near, float& pzh, float& pzl, float& u,
                                           float& v) {
    float pz;
    if (!kContracted) {
        lattice_row(V.A + 6, V.B, V.C[2], V.E, nh, pzh, pzl);
        pz = __fadd_rn(pzh, pzl);
        const bool front = pz > z_near && pz <= FLT_MAX;
        const float inv = rcp_nr(front ? pz : 1.f);
        const float pu = __fmaf_rn(V.A[0], nh[0], __fmaf_rn(V.A[1], nh[1], __fmaf_rn(V.A[2], nh[2], V.C[0])));
        const float pv = __fmaf_rn(V.A[3], nh[0], __fmaf_rn(V.A[4], nh[1], __fmaf_rn(V.A[5], nh[2], V.C[1])));
        u = __fmul_rn(pu, inv);
        v = __fmul_rn(pv, inv);
        return front;
    }
    dot3c(V.A[6], V.A[7], V.A[8], nh, nl, V.C[2], pzh, pzl);
    pz = pzh;
    const float px = __fmaf_rn(V.A[0], nh[0], __fmaf_rn(V.A[1], nh[1], __fmaf_rn(
        V.A[2], nh[2], __fmaf_rn(V.A[0], nl[0], __fmaf_rn(V.A[1], nl[1], __fmaf_rn(
        V.A[2], nl[2], V.C[0]))))));
    const float py = __fmaf_rn(V.A[3], nh[0], __fmaf_rn(V.A[4], nh[1], __fmaf_rn(
        V.A[5], nh[2], __fmaf_rn(V.A[3], nl[0], __fmaf_rn(V.A[4], nl[1], __fmaf_rn(
        V.A[5], nl[2], V.C[1]))))));
    const bool front = pz > z_near && pz <= FLT_MAX;
    const float inv = rcp_nr(front ? pz : 1.f);
    u = __fmaf_rn(V.K[0], __fmul_rn(px, inv), V.K[2]);
    v = __fmaf_rn(V.K[1], __fmul_rn(py, inv), V.K[3]);
    return front;
}

// n > mean + sigma over a footprint of A pixels with sums S1 = sum n, S2 =
// sum n^2: n A - S1 > 0 and (n A - S1)^2 > A S2 - S1^2, in exact integers
__device__ __forceinline__ bool layered_exact(uint32_t n, int64_t A, uint32_t S1,
                                              unsigned long long S2) {
    const long long d = (long long)n * A - (long long)S1;
    if (d <= 0) return false;
    const __int128 lhs = (__int128)d * d;
    const __int128 rhs = (__int128)A * (__int128)S2 - (__int128)S1 * (__int128)S1;
    return lhs > rhs;
}

__device__ __forceinline__ float tmask_prob(const ViewC& V, int32_t q, bool& half) {
    if (V.mask_type == kMaskF16) {
        const float m = __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(V.mask) + q)));
        half = m > 0.5f;
        return m;
    }
    const float raw = __ldg(reinterpret_cast<const float*>(V.mask) + q);
    if (V.mask_type == kMaskLogit) {
        half = raw > 0.f;
        return __frcp_rn(__fadd_rn(1.f, expf(-raw)));
    }
    half = raw > 0.5f;
    return raw;
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

template <bool kContracted>
__global__ void __launch_bounds__(kThreads) k_fuse_tuple(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, GridC G, FuseC F,
    const __grid_constant__ TViewBatch TB, TupleC TP, int32_t accumulate, float* __restrict__ W,
    float* __restrict__ Z, uint32_t* __restrict__ bits) {
    const int32_t n = *d_n;
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const uint32_t pk = __ldg(active + a);
        const VoxelGeom vg = voxel_geom<kContracted>(pk, G, F.gamma);
        float Ws = 0.f, Zs = 0.f;
        uint32_t b = 0;
        if (accumulate) {
            Ws = W[a];
            Zs = Z[a];
            b = bits[a];
        }
        if (vg.ok) {
            const float hv = vg.hv;  // world edge h_v
            // the voxel centre in world coordinates (unprojection distances)
            float xw[3];
#pragma unroll
            for (int q = 0; q < 3; ++q)
                xw[q] = kContracted ? __fadd_rn(vg.xh[q], vg.xl[q])
                                    : __fmaf_rn(__fmul_rn(0.5f, G.h), vg.xh[q], G.origin[q]);
            for (int32_t i = 0; i < TB.n; ++i) {
                const TViewC& T = TB.v[i];
                const ViewC& V = T.base;
                float pzh, pzl, u, v;
                if (!project_uv<kContracted>(V, vg.xh, vg.xl, F.z_near, pzh, pzl, u, v)) continue;
                const int32_t pix = pixel_index(V, true, u, v);
                if (pix < 0) continue;
                // footprint: the corners' pixel box
                float umin = FLT_MAX, umax = -FLT_MAX, vmin = FLT_MAX, vmax = -FLT_MAX;
                bool corners = true;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float ch[3], cl[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float s = ((c >> q) & 1) ? 1.f : -1.f;
                        if (kContracted) {
                            ch[q] = __fmaf_rn(s * 0.5f, hv, vg.xh[q]);
                            cl[q] = vg.xl[q];
                        } else {
                            ch[q] = __fadd_rn(vg.xh[q], s);  // lattice n +- 1: exact
                            cl[q] = 0.f;
                        }
                    }
                    float zh, zl, cu, cv;
                    corners = corners && project_uv<kContracted>(V, ch, cl, F.z_near, zh, zl, cu, cv);
                    umin = fminf(umin, cu); umax = fmaxf(umax, cu);
                    vmin = fminf(vmin, cv); vmax = fmaxf(vmax, cv);
                }
                if (!corners) continue;
                const float Wf = (float)V.W, Hf = (float)V.H;
                // pixel box, clamped to the image before the integer conversions
                const int i0 = (int)fminf(fmaxf(floorf(umin), 0.f), Wf);
                const int i1 = (int)fmaxf(fminf(floorf(umax), Wf - 1.f), -1.f);
                const int j0 = (int)fminf(fmaxf(floorf(vmin), 0.f), Hf);
                const int j1 = (int)fmaxf(fminf(floorf(vmax), Hf - 1.f), -1.f);
                if (!(i0 <= i1 && j0 <= j1)) continue;  // (cannot happen: the centre is in frame)
                const int64_t A = (int64_t)(i1 - i0 + 1) * (j1 - j0 + 1);
                const int32_t sw = V.W + 1;
                const uint32_t S1 = __ldg(T.sat1 + (j1 + 1) * sw + i1 + 1) - __ldg(T.sat1 + j0 * sw + i1 + 1) -
                                    __ldg(T.sat1 + (j1 + 1) * sw + i0) + __ldg(T.sat1 + j0 * sw + i0);
                const unsigned long long S2 =
                    __ldg(T.sat2 + (j1 + 1) * sw + i1 + 1) - __ldg(T.sat2 + j0 * sw + i1 + 1) -
                    __ldg(T.sat2 + (j1 + 1) * sw + i0) + __ldg(T.sat2 + j0 * sw + i0);
                const float mean = __fdiv_rn((float)S1, (float)A);
                // centre pixel
                const float dmin = __ldg(V.depth + pix), dmed = __ldg(T.d_med + pix),
                            dmax = __ldg(T.d_max + pix);
                const uint32_t nc = __ldg(T.n_samp + pix);
                bool half;
                const float m = tmask_prob(V, pix, half);
                const float raw_gate = V.mask_type == kMaskLogit
                                           ? __ldg(reinterpret_cast<const float*>(V.mask) + pix)
                                           : m;
                const bool pass = raw_gate >= (V.mask_type == kMaskLogit ? F.logit_tau : F.tau_m);
                const float xd = __fadd_rn(pzh, pzl);
                const float du = __fdiv_rn(__fsub_rn(u, V.K[2]), V.K[0]);
                const float dv = __fdiv_rn(__fsub_rn(v, V.K[3]), V.K[1]);
                const float ray = __fsqrt_rn(__fadd_rn(1.f, __fmaf_rn(du, du, __fmul_rn(dv, dv))));
                const bool trusted = dmin <= dmed;
                const bool seethru = dmed > T.st_thr;
                const bool front = (layered_exact(nc, A, S1, S2) || seethru) && trusted;
                bool check_thin = true;
                if (pass && trusted && dmin > 0.f && dmin <= FLT_MAX && dmed > 0.f &&
                    dmed <= FLT_MAX && dmax > 0.f && dmax <= FLT_MAX) {
                    const float dref = front ? dmin : dmed;
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
                    const float tdep = __fdiv_rn(__fmul_rn(F.gamma, hv), __fmaf_rn(TP.beta, E, 1.f));
                    const float e_med = __fadd_rn(__fsub_rn(pzh, dmed), pzl);
                    const bool vd = front ? (e_min <= tdep) : (fabsf(e_med) <= tdep);
                    if (__fmul_rn(ray, dist) <= tau_sp && vd) {
                        const float hw_p = __fmul_rn(0.5f, __fsub_rn(dmax, dmin));
                        const float hw_r = fmaxf(__fmul_rn(hw_p, ray), F.eps);
                        const float r = __fdiv_rn(__fmul_rn(ray, __fsub_rn(s_off, hw_p)), hw_r);
                        const float w = expf(-__fmul_rn(F.alpha1, __fmul_rn(r, r)));
                        Ws = __fmaf_rn(m, w, Ws);
                        Zs = __fadd_rn(Zs, w);
                        b |= V.bit;
                        check_thin = false;
                    }
                }
                const float dsurf = (trusted && seethru) ? dmin : dmed;
                const float e_surf = __fadd_rn(__fsub_rn(pzh, dsurf), pzl);
                const bool behind = e_surf > __fmul_rn(TP.behind_margin, hv);
                if (!check_thin || behind || !TP.thin_on) continue;
                // thin path: the footprint's pixels
                int n_depth = 0, n_md = 0;
                float m_max = 0.f, d2 = FLT_MAX;
                bool any_d2 = false;
                for (int yy = j0; yy <= j1; ++yy) {
                    for (int xx = i0; xx <= i1; ++xx) {
                        const int32_t q = yy * V.W + xx;
                        const float qmed = __ldg(T.d_med + q);
                        if (qmed < F.eps) continue;
                        const float qmin = __ldg(V.depth + q);
                        const uint32_t nq = __ldg(T.n_samp + q);
                        const float Eq = fmaxf(__fsub_rn((float)nq, mean), 0.f);
                        const float tq = __fdiv_rn(__fmul_rn(F.gamma, hv), __fmaf_rn(TP.beta, Eq, 1.f));
                        const bool fq = (layered_exact(nq, A, S1, S2) || qmed > T.st_thr) && qmin <= qmed;
                        const float lhs = fq ? __fadd_rn(__fsub_rn(pzh, qmin), pzl)
                                             : fabsf(__fadd_rn(__fsub_rn(pzh, qmed), pzl));
                        if (!(lhs <= tq)) continue;
                        ++n_depth;
                        bool hq;
                        const float mq = tmask_prob(V, q, hq);
                        if (!hq) continue;
                        ++n_md;
                        m_max = fmaxf(m_max, mq);
                        const float dq = fq ? qmin : qmed;
                        const float cx = __fmul_rn(__fdiv_rn(__fsub_rn((float)xx + 0.5f, V.K[2]), V.K[0]), dq);
                        const float cy = __fmul_rn(__fdiv_rn(__fsub_rn((float)yy + 0.5f, V.K[3]), V.K[1]), dq);
                        const float pc[3] = {__fsub_rn(cx, T.t[0]), __fsub_rn(cy, T.t[1]), __fsub_rn(dq, T.t[2])};
                        float dd = 0.f;
#pragma unroll
                        for (int r = 0; r < 3; ++r) {  // world = R^T (p_c - t)
                            const float pw = __fmaf_rn(T.R[r], pc[0], __fmaf_rn(T.R[3 + r], pc[1], __fmul_rn(T.R[6 + r], pc[2])));
                            const float df = __fsub_rn(pw, xw[r]);
                            dd = __fmaf_rn(df, df, dd);
                        }
                        d2 = fminf(d2, dd);
                        any_d2 = true;
                    }
                }
                const float cu0 = fmaxf(umin, 0.f), cu1 = fminf(umax, Wf);
                const float cv0 = fmaxf(vmin, 0.f), cv1 = fminf(vmax, Hf);
                const float AB = __fmul_rn(__fsub_rn(cu1, cu0), __fsub_rn(cv1, cv0));
                const float n_min = fmaxf(TP.n_abs, ceilf(__fmul_rn(TP.rho_occ, AB)));
                const float gate = __fmul_rn(TP.dist_gate, hv);
                const float tt = ((float)n_depth >= n_min &&
                                  (float)n_md >= __fmul_rn(TP.rho_cover, (float)n_depth) && any_d2 &&
                                  d2 <= __fmul_rn(gate, gate))
                                     ? m_max
                                     : 0.f;
                if (tt >= TP.tau_thin) {
                    Ws = __fadd_rn(Ws, tt);
                    Zs = __fadd_rn(Zs, 1.f);
                    b |= V.bit;
                }
            }
        }
        W[a] = Ws;
        Z[a] = Zs;
        bits[a] = b;
    }
}

// integral images of one view's n_samp: rows first (one warp per row), then
// columns (one thread per column); out (H + 1) x (W + 1) with a zero first
// row and column, uint32 sums of n and uint64 sums of n^2 (both modular)
__global__ void __launch_bounds__(kThreads) k_sat_rows(const uint16_t* __restrict__ n, int32_t W,
                                                       int32_t H, uint32_t* __restrict__ s1,
                                                       unsigned long long* __restrict__ s2) {
    const int lane = threadIdx.x & 31;
    const int32_t sw = W + 1;
    for (int32_t y = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; y <= H;
         y += (gridDim.x * blockDim.x) >> 5) {
        if (y == 0) {
            for (int32_t x = lane; x < sw; x += 32) {
                s1[x] = 0u;
                s2[x] = 0ull;
            }
            continue;
        }
        uint32_t c1 = 0u;
        unsigned long long c2 = 0ull;
        if (lane == 0) {
            s1[(int64_t)y * sw] = 0u;
            s2[(int64_t)y * sw] = 0ull;
        }
        for (int32_t x0 = 0; x0 < W; x0 += 32) {
            const int32_t x = x0 + lane;
            uint32_t v1 = x < W ? (uint32_t)__ldg(n + (int64_t)(y - 1) * W + x) : 0u;
            unsigned long long v2 = (unsigned long long)v1 * v1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t a1 = __shfl_up_sync(0xffffffffu, v1, o);
                const unsigned long long a2 = __shfl_up_sync(0xffffffffu, v2, o);
                if (lane >= o) {
                    v1 += a1;
                    v2 += a2;
                }
            }
            if (x < W) {
                s1[(int64_t)y * sw + x + 1] = c1 + v1;
                s2[(int64_t)y * sw + x + 1] = c2 + v2;
            }
            c1 += __shfl_sync(0xffffffffu, v1, 31);
            c2 += __shfl_sync(0xffffffffu, v2, 31);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_sat_cols(int32_t W, int32_t H,
                                                       uint32_t* __restrict__ s1,
                                                       unsigned long long* __restrict__ s2) {
    const int32_t sw = W + 1;
    for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < sw; x += gridDim.x * blockDim.x) {
        uint32_t c1 = 0u;
        unsigned long long c2 = 0ull;
        for (int32_t y = 1; y <= H; ++y) {
            c1 += s1[(int64_t)y * sw + x];
            c2 += s2[(int64_t)y * sw + x];
            s1[(int64_t)y * sw + x] = c1;
            s2[(int64_t)y * sw + x] = c2;
        }
    }
}

}  // namespace

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
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (!views || !tp || n_views < 1 || n_views > kMaxViews)
        return fail(c, DIVAS_E_INVALID, "n_views must be in 1..32, views and tp non-NULL");
    if (!(tp->beta >= 0.f) || !(tp->rho_cover >= 0.f) || !(tp->rho_occ >= 0.f) ||
        !(tp->n_abs >= 0.f) || !(tp->dist_gate >= 0.f) || !(tp->behind_margin >= 0.f) ||
        !(tp->k_dg >= 0.f) || !(tp->tau_thin == tp->tau_thin) || !(tp->gamma_st == tp->gamma_st) ||
        !(tp->rho_thin == tp->rho_thin))
        return fail(c, DIVAS_E_INVALID, "tuple params out of range");
    size_t need = 0;
    for (int32_t k = 0; k < n_views; ++k) {
        divas_status st = check_camera(c, &views[k].cam);
        if (st != DIVAS_OK) return st;
        const divas_tuple_view& v = views[k];
        if (!v.d_min || !v.d_med || !v.d_max || !v.n_samp || !v.mask)
            return fail(c, DIVAS_E_INVALID, "a tuple raster is NULL");
        if (v.mask_type < 0 || v.mask_type > 2) return fail(c, DIVAS_E_INVALID, "bad mask_type");
        if (!(v.d_cam == v.d_cam)) return fail(c, DIVAS_E_INVALID, "d_cam is NaN");
        need += (size_t)(v.cam.W + 1) * (v.cam.H + 1) * 12 + 256;
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
    unsigned char* cur = static_cast<unsigned char*>(c->sat);
    for (int32_t k0 = 0; k0 < n_views; k0 += kMaxTupleViews) {
        TViewBatch tb;
        memset(&tb, 0, sizeof(tb));
        tb.n = std::min<int32_t>(kMaxTupleViews, n_views - k0);
        for (int32_t j = 0; j < tb.n; ++j) {
            const divas_tuple_view& v = views[k0 + j];
            TViewC& t = tb.v[j];
            t.base = make_view(v.cam, c->G, v.d_min, v.mask, v.mask_type, c->n_views + k0 + j);
            t.d_med = v.d_med;
            t.d_max = v.d_max;
            t.n_samp = v.n_samp;
            const size_t cells = (size_t)(v.cam.W + 1) * (v.cam.H + 1);
            t.sat2 = reinterpret_cast<const unsigned long long*>(cur);
            t.sat1 = reinterpret_cast<const uint32_t*>(cur + cells * 8);
            cur += cells * 12 + 256 - (cells * 12) % 256;
            memcpy(t.R, v.cam.R, sizeof(t.R));
            memcpy(t.t, v.cam.t, sizeof(t.t));
            t.st_thr = (float)((double)tp->gamma_st * (double)v.d_cam);
            const int rows_blocks = (int)std::min<int64_t>((v.cam.H + 1 + 7) / 8, c->sm_count * 8);
            k_sat_rows<<<rows_blocks, kThreads, 0, s>>>(
                v.n_samp, v.cam.W, v.cam.H, const_cast<uint32_t*>(t.sat1),
                const_cast<unsigned long long*>(t.sat2));
            DIVAS_LAUNCHED(c, "k_sat_rows");
            k_sat_cols<<<(v.cam.W + 1 + kThreads - 1) / kThreads, kThreads, 0, s>>>(
                v.cam.W, v.cam.H, const_cast<uint32_t*>(t.sat1),
                const_cast<unsigned long long*>(t.sat2));
            DIVAS_LAUNCHED(c, "k_sat_cols");
        }
        const int blocks = grid_for(c->cap, c->sm_count);
        const int32_t acc = c->n_views + k0 > 0 ? 1 : 0;
        if (c->G.contracted)
            k_fuse_tuple<true><<<blocks, kThreads, 0, s>>>(c->active, c->d_n, c->G, c->F, tb, T, acc,
                                                           c->W, c->Z, c->bits);
        else
            k_fuse_tuple<false><<<blocks, kThreads, 0, s>>>(c->active, c->d_n, c->G, c->F, tb, T, acc,
                                                            c->W, c->Z, c->bits);
        DIVAS_LAUNCHED(c, "k_fuse_tuple");
    }
    c->n_views += n_views;
    return DIVAS_OK;
}

}  // extern "C"
