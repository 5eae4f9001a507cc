// nerf_mode.cuh -- the NeRF variant of the depth-tuple fusion (appendix
// "NeRF-Backbone 3D Fusion Details": Eqs. distance_cond, dist_tol,
// depth_tol, nerf-accept, nerf-vote, nerf-thindepth .. nerf-thin; Algorithms
// "Thick-Structure Segmentation via Depth-Weighted Voxel Aggregation" and
// "Thin-Structure Segmentation via Footprint-Based Coverage Analysis"),
// included by divas_fuse.cu after tuple_mode.cuh (it reuses its view
// constants, projections, corner boxes and mask-tile maps).
//
// Per view the caller hands over the NeRF depth tuple (d_min, d_exp, d_max
// planar FP32, the ray-sample count n_samp as uint16) with the mask, and
// optionally the dense FP32 density grid.  Per voxel and view, in order:
//
//   - thick path at the centre pixel (mask m >= tau_m, finite positive
//     depths): the voxel against the pixel-centre ray k = ((x + 1/2 - cx) /
//     fx, (y + 1/2 - cy) / fy, 1): z_c = clip(<p, k> / |k|^2, d_min, d_max),
//     delta = |p - k z_c| <= Delta pi_dg + lambda_range |k| (d_max - d_min)
//     and |p_z - d_exp| <= (gamma + min(beta n, b_max)) Delta; the vote m w,
//     w = exp(-alpha1 r^2), r = |z_c - (d_min + d_max)/2| / max((d_max -
//     d_min)/2, eps).  Everything is taken as an offset from p_z: with the
//     projection's sub-pixel offsets e = ((u - x - 1/2) / fx, (v - y - 1/2)
//     / fy), p = p_z (k + e) exactly, so z_proj - p_z = p_z <k, e> / |k|^2
//     and p - k z_c = (p_z e_x - k_x s, p_z e_y - k_y s, -s) with s = z_c -
//     p_z: small quantities formed from exact differences.  On contracted
//     grids (camera depths up to hundreds of voxel edges) e comes from the
//     hi + lo camera coordinates instead of the rounded u, v.
//   - thin path where the thick path did not vote, m > m_thin and density
//     >= rho_thin: the box of the 8 projected corners (N pixels, clipped),
//     the supportive pixels (m > 1/2 and |p_z - d_exp(q)| <= (2 gamma +
//     min(beta n(q), b_max)) Delta) and the peak mask over the box; t =
//     m_max when n_valid >= rho_cover N; t >= tau_thin votes (W += t, Z += 1).
//
// Two launches per batch of up to 16 views, as in the 2DGS variant: a scan
// (one thread per active voxel) computes the thick votes and finds the thin
// candidates; voxels without one are finished there, the others go to a
// heavy list whose pass recomputes their views (a half-warp per voxel, a
// lane per view) with the footprint loops, and adds the votes in view order.
#pragma once

namespace {

struct NerfC {
    float gamma, beta, b_max, lambda_range, rho_cover, tau_thin, rho_thin, k_dg;
    float m_thin;   // thin eligibility on probability masks: m > m_thin
    float l_thin;   // the same on logits: l > l_thin (FP32 logit of m_thin)
    int32_t thin_on;
    int32_t pad;
};

// the centre evaluation's projection, reused by the thin path
struct NerfCentre {
    float pzh, pzl, r0, r1, u, v;
    int32_t pix;
};

// (f p - d z) / (f z) for p, z given as hi + lo: the angle between the ray
// through (p, z) and the pixel ray at offset d from the principal point (d
// exact), the numerator from exact products (f p and d z nearly cancel).
__device__ __forceinline__ float sub_pixel_offset(float f, float ph, float pl, float d, float zh,
                                                  float zl) {
    float a, ae, b, be;
    two_prod(f, ph, a, ae);
    two_prod(d, zh, b, be);
    const float tail = __fadd_rn(__fsub_rn(ae, be), __fsub_rn(__fmul_rn(f, pl), __fmul_rn(d, zl)));
    return __fdiv_rn(__fadd_rn(__fsub_rn(a, b), tail), __fmul_rn(f, __fadd_rn(zh, zl)));
}

// The thick path's spatial gate in FP64, with the operations of the FP64
// definition: p = R x + t, k = the centre pixel's ray, z_c = clip(<p, k> /
// |k|^2, d_min, d_max), delta = |p - k z_c| against h_v pi + lambda_range
// |k| (d_max - d_min) (the re-evaluation of a decision near the gate).
__device__ __noinline__ bool nerf_spatial_exact(const TViewC& T, const double* x, int ix, int iy,
                                                float dmin, float dmax, float hv, float pi,
                                                float lambda) {
    const ViewC& V = T.base;
    double p[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        p[r] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)T.R[3 * r], x[0]),
                                             __dmul_rn((double)T.R[3 * r + 1], x[1])),
                                   __dmul_rn((double)T.R[3 * r + 2], x[2])),
                         (double)T.t[r]);
    const double k0 = __ddiv_rn(__dsub_rn(__dadd_rn((double)ix, 0.5), (double)V.K[2]), (double)V.K[0]);
    const double k1 = __ddiv_rn(__dsub_rn(__dadd_rn((double)iy, 0.5), (double)V.K[3]), (double)V.K[1]);
    const double k2 = __dadd_rn(__dadd_rn(__dmul_rn(k0, k0), __dmul_rn(k1, k1)), 1.0);
    const double zp = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(p[0], k0), __dmul_rn(p[1], k1)), p[2]), k2);
    const double lo = (double)dmin, hi = (double)dmax;
    const double zc = zp < lo ? lo : (zp > hi ? hi : zp);
    const double e0 = __dsub_rn(p[0], __dmul_rn(k0, zc)), e1 = __dsub_rn(p[1], __dmul_rn(k1, zc));
    const double e2 = __dsub_rn(p[2], zc);
    const double delta =
        __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2)));
    const double tau = __dadd_rn(__dmul_rn((double)hv, (double)pi),
                                 __dmul_rn(__dmul_rn((double)lambda, __dsqrt_rn(k2)), __dsub_rn(hi, lo)));
    return delta <= tau;
}

// View T at the voxel's centre pixel: 0 = neither path can vote, 1 = thick
// vote (x = m, y = w), 2 = thin candidate (rho_v is the voxel's density; a
// candidate also needs a mask key >= key_thr in the dilated tile map around
// the centre when the view has one).  A spatial distance within the FP32
// rounding bound of its gate is decided again in FP64 when kExact; otherwise
// it counts as no thick vote and sets undecided (the caller hands the voxel
// to the pass that decides it exactly).
template <bool kC, int kMT = -1, bool kExact = true>
__device__ __forceinline__ int nerf_centre(const TViewC& T, const VoxelGeom& vg, const GridC& G,
                                           const FuseC& F, const NerfC& N, float rho_v, float& x,
                                           float& y, NerfCentre& c, bool& undecided) {
    undecided = false;
    const ViewC& V = T.base;
    if (!project_uv<kC>(V, vg.xh, vg.xl, F.z_near, c.pzh, c.pzl, c.r0, c.r1, c.u, c.v)) return 0;
    const int32_t pix = pixel_index(V, true, c.u, c.v);
    if (pix < 0) return 0;
    c.pix = pix;
    const uint32_t mraw = mask_bits<kMT>(V, pix);
    bool half;
    const float m = mask_from_bits<kMT>(V, mraw, half);
    const bool logit = mask_type_of<kMT>(V) == kMaskLogit;
    const float raw = logit ? __uint_as_float(mraw) : m;
    if (raw >= (logit ? F.logit_tau : F.tau_m)) {
        const float dmin = __ldg(V.depth + pix), dexp = __ldg(T.d_med + pix);
        const float dmax = __ldg(T.d_max + pix);
        if (dmin > 0.f && dmin <= FLT_MAX && dexp > 0.f && dexp <= FLT_MAX && dmax > 0.f &&
            dmax <= FLT_MAX) {
            const float hv = vg.hv;
            const float b = fminf(__fmul_rn(N.beta, (float)__ldg(T.n_samp + pix)), N.b_max);
            const float tdep = __fmul_rn(__fadd_rn(N.gamma, b), hv);
            const float e_exp = __fadd_rn(__fsub_rn(c.pzh, dexp), c.pzl);  // x_d - d_exp
            if (fabsf(e_exp) <= tdep) {
                const int32_t ix = pix % V.W, iy = pix / V.W;
                const float cxp = __fadd_rn((float)ix, 0.5f), cyp = __fadd_rn((float)iy, 0.5f);
                const float kx = __fmul_rn(__fsub_rn(cxp, V.K[2]), T.inv_fx);
                const float ky = __fmul_rn(__fsub_rn(cyp, V.K[3]), T.inv_fy);
                float ex, ey;
                if (kC) {
                    // far voxels: e from hi + lo camera coordinates (a rounded
                    // u would cost e its relative precision at large depths)
                    float qh, ql;
                    dot3c(V.A[0], V.A[1], V.A[2], vg.xh, vg.xl, V.C[0], qh, ql);
                    ex = sub_pixel_offset(V.K[0], qh, ql, __fsub_rn(cxp, V.K[2]), c.pzh, c.pzl);
                    dot3c(V.A[3], V.A[4], V.A[5], vg.xh, vg.xl, V.C[1], qh, ql);
                    ey = sub_pixel_offset(V.K[1], qh, ql, __fsub_rn(cyp, V.K[3]), c.pzh, c.pzl);
                } else {
                    ex = __fmul_rn(__fsub_rn(c.u, cxp), T.inv_fx);
                    ey = __fmul_rn(__fsub_rn(c.v, cyp), T.inv_fy);
                }
                const float pz = __fadd_rn(c.pzh, c.pzl);
                const float k2 = __fadd_rn(1.f, __fmaf_rn(kx, kx, __fmul_rn(ky, ky)));
                const float s0 = __fdiv_rn(__fmul_rn(pz, __fmaf_rn(kx, ex, __fmul_rn(ky, ey))), k2);
                const float lo = -__fadd_rn(__fsub_rn(c.pzh, dmin), c.pzl);  // d_min - p_z
                const float hi = -__fadd_rn(__fsub_rn(c.pzh, dmax), c.pzl);  // d_max - p_z
                // z_c - p_z = clip(s0, lo, hi): lo below lo, else hi above hi
                // (also when d_max < d_min)
                const float s = s0 < lo ? lo : (s0 > hi ? hi : s0);
                const float dx = __fmaf_rn(-kx, s, __fmul_rn(pz, ex));
                const float dy = __fmaf_rn(-ky, s, __fmul_rn(pz, ey));
                const float delta = __fsqrt_rn(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(s, s))));
                const float band = __fsub_rn(dmax, dmin);
                const float pi = pi_dg(T, ix, iy, N.k_dg);
                const float tau_sp = __fmaf_rn(__fmul_rn(N.lambda_range, __fsqrt_rn(k2)), band,
                                               __fmul_rn(hv, pi));
                bool accept = delta <= tau_sp;
                if (fabsf(__fsub_rn(delta, tau_sp)) <= recheck_band(T, vg, G, pz)) {
                    if (kExact) {
                        double xw[3];
                        centre64(vg, G, xw);
                        accept = nerf_spatial_exact(T, xw, ix, iy, dmin, dmax, hv, pi,
                                                    N.lambda_range);
                    } else {
                        accept = false;
                        undecided = true;
                    }
                }
                if (accept) {
                    // z_c - mid: +-(d_max - d_min)/2 at a clamped end (from the
                    // depths themselves: lo and hi are rounded offsets when the
                    // band lies far from p_z), s - (lo + hi)/2 inside the band
                    const float half_band = __fmul_rn(0.5f, band);
                    const float off = (s0 < lo || s0 > hi)
                                          ? half_band
                                          : __fsub_rn(s, __fmul_rn(0.5f, __fadd_rn(lo, hi)));
                    const float hd = fmaxf(half_band, F.eps);
                    const float r = __fdiv_rn(fabsf(off), hd);
                    x = m;
                    y = expf(-__fmul_rn(F.alpha1, __fmul_rn(r, r)));
                    return 1;
                }
            }
        }
    }
    if (!N.thin_on || !(rho_v >= N.rho_thin)) return 0;
    if (!(logit ? raw > N.l_thin : m > N.m_thin)) return 0;
    if (T.tile_dil)
        return __ldg(T.tile_dil + (pix / V.W / kMaskTile) * T.tiles_w + (pix % V.W) / kMaskTile) >=
                       T.key_thr
                   ? 2
                   : 0;
    return 2;
}

// The thin path of a candidate view: the corner box, the support count and
// the peak mask key over it (kThinGroup pixels at a time, loads issued
// together), stopping once n_valid can no longer reach rho_cover N.  Returns
// t >= tau_thin (the vote t in x), else false.
template <bool kC, int kMT = -1>
__device__ __forceinline__ bool nerf_thin(const TViewC& T, const VoxelGeom& vg, const FuseC& F,
                                          const NerfC& N, const NerfCentre& c, float& x) {
    const ViewC& V = T.base;
    const float hv = vg.hv;
    float umin, umax, vmin, vmax;
    if (!corner_box<kC>(T, hv, F.z_near, c.pzh, c.pzl, c.r0, c.r1, umin, umax, vmin, vmax))
        return false;
    const float Wf = (float)V.W, Hf = (float)V.H;
    const int i0 = (int)fminf(fmaxf(floorf(umin), 0.f), Wf);
    const int i1 = (int)fmaxf(fminf(floorf(umax), Wf - 1.f), -1.f);
    const int j0 = (int)fminf(fmaxf(floorf(vmin), 0.f), Hf);
    const int j1 = (int)fmaxf(fminf(floorf(vmax), Hf - 1.f), -1.f);
    if (!(i0 <= i1 && j0 <= j1)) return false;  // (cannot happen: the centre is in frame)
    const uint32_t A = (uint32_t)(i1 - i0 + 1) * (uint32_t)(j1 - j0 + 1);
    if (!box_may_vote(T, i0, i1, j0, j1)) return false;  // m_max < tau_thin
    const float Af = (float)A;
    const float t2 = __fmul_rn(2.f, N.gamma);
    const bool logit = mask_type_of<kMT>(V) == kMaskLogit;
    uint32_t n_valid = 0u;
    float mkey = -FLT_MAX;
    int xx = i0, yy = j0;
    for (uint32_t p0 = 0; p0 < A; p0 += kThinGroup) {
        // n_valid + (pixels left) < rho_cover N: no vote (exact: both < 2^24)
        if (__fmaf_rn(-N.rho_cover, Af, (float)(n_valid + (A - p0))) < 0.f) return false;
        float gexp[kThinGroup];
        uint32_t gn[kThinGroup], gm[kThinGroup];
        bool live[kThinGroup];
#pragma unroll
        for (int k = 0; k < kThinGroup; ++k) {
            live[k] = p0 + k < A;
            gexp[k] = FLT_MAX;
            gn[k] = 0u;
            gm[k] = 0u;
            if (live[k]) {
                const int32_t q = yy * V.W + xx;
                gexp[k] = __ldg(T.d_med + q);
                gn[k] = __ldg(T.n_samp + q);
                gm[k] = mask_bits<kMT>(V, q);
            }
            if (++xx > i1) {
                xx = i0;
                ++yy;
            }
        }
#pragma unroll
        for (int k = 0; k < kThinGroup; ++k) {
            float key;
            bool hq;
            if (mask_type_of<kMT>(V) == kMaskF16) {
                key = __half2float(__ushort_as_half((unsigned short)gm[k]));
                hq = key > 0.5f;
            } else {
                key = __uint_as_float(gm[k]);
                hq = logit ? key > 0.f : key > 0.5f;
            }
            const float bq = fminf(__fmul_rn(N.beta, (float)gn[k]), N.b_max);
            const float tq = __fmul_rn(__fadd_rn(t2, bq), hv);
            const float e = __fadd_rn(__fsub_rn(c.pzh, gexp[k]), c.pzl);
            n_valid += (live[k] && hq && fabsf(e) <= tq) ? 1u : 0u;
            mkey = live[k] ? fmaxf(mkey, key) : mkey;
        }
    }
    if (__fmaf_rn(-N.rho_cover, Af, (float)n_valid) < 0.f) return false;
    const float m_max = logit ? __frcp_rn(__fadd_rn(1.f, expf(-mkey))) : mkey;
    if (!(m_max >= N.tau_thin)) return false;
    x = m_max;
    return true;
}

__device__ __forceinline__ float voxel_density(const float* __restrict__ rho, uint32_t pk, int32_t g) {
    return rho ? __ldg(rho + packed_lin(pk, g)) : 1.f;
}

// Pass 1, one thread per active voxel: every view's thick vote and thin
// candidacy from the centre pixels.  Voxels without a thin candidate add
// their thick votes in view order here; the others go to the heavy list
// (entry: voxel, views with a thick vote | thin candidates << 16).
template <bool kC, int kN, int kMT = -1>
__global__ void __launch_bounds__(kThreads, kC ? 4 : 6) k_nerf_scan(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, GridC G, FuseC F,
    const __grid_constant__ TViewBatch TB, NerfC N, const float* __restrict__ density,
    int32_t accumulate, float* __restrict__ W, float* __restrict__ Z, uint32_t* __restrict__ bits,
    uint2* __restrict__ heavy, int32_t* __restrict__ n_heavy) {
    static_assert(kMaxTupleViews <= 16, "an entry holds 16 thick and 16 thin bits");
    const int32_t n = *d_n;
    const int lane = threadIdx.x & 31;
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < n; base += stride) {
        const int32_t a = base + lane;
        uint32_t thick = 0u, thin = 0u;
        bool heavy_only = false;
        if (a < n) {
            const uint32_t pk = __ldg(active + a);
            const VoxelGeom vg = voxel_geom<kC>(pk, G, F.gamma);
            float Ws = 0.f, Zs = 0.f;
            uint32_t b = 0u;
            if (accumulate) {
                Ws = W[a];
                Zs = Z[a];
                b = bits[a];
            }
            if (vg.ok) {
                const float rho_v = N.thin_on ? voxel_density(density, pk, G.g) : 0.f;
#pragma unroll
                for (int i = 0; i < kN; ++i) {
                    if (i >= TB.n) break;
                    float x = 0.f, y = 0.f;
                    NerfCentre c;
                    bool undecided;
                    const int kind = nerf_centre<kC, kMT, false>(TB.v[i], vg, G, F, N, rho_v, x,
                                                                 y, c, undecided);
                    if (kind == 1) {
                        thick |= 1u << i;
                        Ws = __fmaf_rn(x, y, Ws);
                        Zs = __fadd_rn(Zs, y);
                        b |= TB.v[i].base.bit;
                    } else if (kind == 2) {
                        thin |= 1u << i;
                    }
                    // a spatial decision near its gate: the heavy pass takes the view
                    // again (thick bit) and decides it exactly
                    if (undecided) {
                        thick |= 1u << i;
                        heavy_only = true;
                    }
                }
            }
            if (!thin && !heavy_only) {
                W[a] = Ws;
                Z[a] = Zs;
                bits[a] = b;
            } else if (!accumulate) {
                W[a] = 0.f;
                Z[a] = 0.f;
                bits[a] = 0u;
            }
        }
        const bool to_heavy = thin != 0u || heavy_only;
        const unsigned hb = __ballot_sync(0xffffffffu, to_heavy);
        if (hb) {
            const int lead = __ffs(hb) - 1;
            int32_t slot = 0;
            if (lane == lead) slot = atomicAdd(n_heavy, __popc(hb));
            slot = __shfl_sync(0xffffffffu, slot, lead);
            if (to_heavy)
                heavy[slot + __popc(hb & ((1u << lane) - 1u))] = make_uint2((uint32_t)a, thick | (thin << 16));
        }
    }
}

// Pass 2: a half-warp per listed voxel, lane i = view i: thick views
// recomputed, thin candidates through the footprint loop; the half's first
// lane adds the votes in view order (the scan's FMA and additions).
template <bool kC, int kMT = -1>
__global__ void __launch_bounds__(kThreads) k_nerf_heavy(
    const uint32_t* __restrict__ active, const uint2* __restrict__ heavy,
    const int32_t* __restrict__ n_heavy, GridC G, FuseC F, const __grid_constant__ TViewBatch TB,
    NerfC N, float* __restrict__ W, float* __restrict__ Z, uint32_t* __restrict__ bits) {
    static_assert(sizeof(TViewC) % 8 == 0 && alignof(TViewC) == 8, "view constants copy as 8-byte words");
    constexpr int kIn = (int)(sizeof(TViewC) / 8);
    constexpr int kWords = kIn | 1;  // odd stride: the 16 lanes read 16 banks
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
    for (int32_t s0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 4; s0 - ((threadIdx.x >> 4) & 1) < n;
         s0 += halves) {
        const bool live = s0 < n;
        uint2 h = make_uint2(0u, 0u);
        if (live) h = heavy[s0];
        int kind = 0;
        float x = 0.f, y = 0.f;
        const bool is_thick = (h.y >> l) & 1u, is_thin = (h.y >> (16 + l)) & 1u;
        if (live && (is_thick || is_thin)) {
            const VoxelGeom vg = voxel_geom<kC>(__ldg(active + h.x), G, F.gamma);
            const TViewC& T = *reinterpret_cast<const TViewC*>(sv + l * kWords);
            NerfCentre c;
            // the scan's outcome for this view, recomputed (a thin candidate
            // passed the density test there)
            bool undecided;
            kind = nerf_centre<kC, kMT>(T, vg, G, F, N, is_thin ? FLT_MAX : 0.f, x, y, c, undecided);
            if (kind == 2) kind = nerf_thin<kC, kMT>(T, vg, F, N, c, x) ? 2 : 0;
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

}  // namespace

template <bool kC, int kMT>
static divas_status launch_nerf_scan(int nv, int blocks, cudaStream_t s, divas_ctx* c,
                                     const TViewBatch& tb, const NerfC& N, const float* density,
                                     int32_t acc, uint2* heavy, int32_t* n_heavy) {
#define DIVAS_NERF_SCAN(K)                                                                         \
    k_nerf_scan<kC, K, kMT><<<blocks, kThreads, 0, s>>>(c->active, c->d_n, c->G, c->F, tb, N,      \
                                                       density, acc, c->W, c->Z, c->bits, heavy,  \
                                                       n_heavy)
    if (nv <= 4) DIVAS_NERF_SCAN(4);
    else if (nv <= 8) DIVAS_NERF_SCAN(8);
    else DIVAS_NERF_SCAN(16);
#undef DIVAS_NERF_SCAN
    DIVAS_LAUNCHED(c, "k_nerf_scan");
    return DIVAS_OK;
}

extern "C" {

divas_nerf_params divas_default_nerf_params(int32_t preset) {
    divas_nerf_params p;
    const bool mip = preset == DIVAS_NERF_MIP360;
    p.gamma = mip ? 0.5f : 4.f;
    p.beta = 0.2f;
    p.b_max = mip ? 1.f : 10.f;
    p.lambda_range = mip ? 5.f : 0.05f;
    p.rho_thin = mip ? 30.f : 50.f;
    p.rho_cover = mip ? 0.3f : 0.2f;
    p.tau_thin = 0.6f;
    p.m_thin = 0.1f;
    p.k_dg = 0.f;
    p.reserved = 0;
    return p;
}

divas_status divas_fuse_add_views_nerf(divas_ctx* c, const divas_tuple_view* views, int32_t n_views,
                                       const divas_nerf_params* np, const float* density,
                                       void* stream) {
    return divas_fuse_add_views_nerf_profiled(c, views, n_views, np, density, nullptr, stream);
}

divas_status divas_fuse_add_views_nerf_profiled(divas_ctx* c, const divas_tuple_view* views,
                                                int32_t n_views, const divas_nerf_params* np,
                                                const float* density, void* const* stage_events,
                                                void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (!views || !np || n_views < 1 || n_views > kMaxViews)
        return fail(c, DIVAS_E_INVALID, "n_views must be in 1..32, views and params non-NULL");
    if (!(np->gamma >= 0.f) || !(np->beta >= 0.f) || !(np->b_max >= 0.f) ||
        !(np->lambda_range >= 0.f) || !(np->rho_cover >= 0.f) || !(np->tau_thin > 0.f) ||
        !(np->m_thin >= 0.f && np->m_thin < 1.f) || !(np->k_dg >= 0.f) ||
        !(np->rho_thin == np->rho_thin))
        return fail(c, DIVAS_E_INVALID, "NeRF params out of range");
    if (density && reinterpret_cast<uintptr_t>(density) % 4 != 0)
        return fail(c, DIVAS_E_INVALID, "density must be 4-byte aligned");
    const size_t heavy_bytes = ((size_t)c->cap * 8 + 256 + 255) / 256 * 256;
    size_t need = heavy_bytes;
    float half_u[kMaxViews], half_v[kMaxViews];
    for (int32_t k = 0; k < n_views; ++k) {
        divas_status st = check_camera(c, &views[k].cam);
        if (st != DIVAS_OK) return st;
        const divas_tuple_view& v = views[k];
        if (!v.d_min || !v.d_med || !v.d_max || !v.n_samp || !v.mask)
            return fail(c, DIVAS_E_INVALID, "a tuple raster is NULL");
        if (v.mask_type < 0 || v.mask_type > 2) return fail(c, DIVAS_E_INVALID, "bad mask_type");
        int64_t pixels = 0;
        footprint_bound(v.cam, c->G, c->F.z_near, half_u[k], half_v[k], pixels);
        need += tile_bytes_of(v.cam.W, v.cam.H);
    }
    cudaStream_t s = S(stream);
    if (need > c->sat_bytes) {  // scratch shared with the 2DGS variant, grown on demand
        if (capturing(s))
            return fail(c, DIVAS_E_STATE, "tuple scratch must grow outside a stream capture");
        DIVAS_CUDA(c, cudaStreamSynchronize(s));
        if (c->sat) cudaFree(c->sat);
        c->sat = nullptr;
        c->sat_bytes = 0;
        DIVAS_CUDA(c, cudaMalloc(&c->sat, need));
        c->sat_bytes = need;
    }
    NerfC N;
    N.gamma = np->gamma;
    N.beta = np->beta;
    N.b_max = np->b_max;
    N.lambda_range = np->lambda_range;
    N.rho_cover = np->rho_cover;
    N.tau_thin = np->tau_thin;
    N.rho_thin = np->rho_thin;
    N.k_dg = np->k_dg;
    N.m_thin = np->m_thin;
    N.l_thin = np->m_thin > 0.f ? (float)std::log((double)np->m_thin / (1.0 - (double)np->m_thin))
                                : -std::numeric_limits<float>::infinity();
    // without a density grid every voxel has density 1
    N.thin_on = density || np->rho_thin <= 1.f ? 1 : 0;
    N.pad = 0;
    divas_status st = record_stage(c, stage_events, 0, s);
    if (st != DIVAS_OK) return st;
    unsigned char* cur = static_cast<unsigned char*>(c->sat);
    int32_t* n_heavy = reinterpret_cast<int32_t*>(cur);
    uint2* heavy = reinterpret_cast<uint2*>(cur + 256);
    cur += heavy_bytes;
    TileJobs tj;
    st = launch_tile_maps(c, views, n_views, cur, tj, s);
    if (st != DIVAS_OK) return st;
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
            memcpy(t.R, v.cam.R, sizeof(t.R));
            memcpy(t.t, v.cam.t, sizeof(t.t));
            t.d_med = v.d_med;  // d_exp
            t.d_max = v.d_max;
            t.n_samp = v.n_samp;
            t.sat1 = nullptr;
            t.sat2 = nullptr;
            for (int q = 0; q < 3; ++q) {
                if (c->G.contracted) {
                    for (int r = 0; r < 3; ++r) t.cd[3 * r + q] = v.cam.R[3 * r + q];
                } else {
                    t.cd[q] = t.base.A[q];
                    t.cd[3 + q] = t.base.A[3 + q];
                    t.cd[6 + q] = (float)((double)t.base.A[6 + q] + (double)t.base.B[q]);
                }
            }
            t.st_thr = 0.f;
            t.inv_fx = (float)(1.0 / (double)v.cam.fx);
            t.inv_fy = (float)(1.0 / (double)v.cam.fy);
            t.tile_max = tj.j[k0 + j].out;
            const bool near = half_u[k0 + j] > 0.f && half_u[k0 + j] <= (float)kMaskTile &&
                              half_v[k0 + j] <= (float)kMaskTile;
            t.tile_dil = near ? tj.j[k0 + j].dil : nullptr;
            t.tiles_w = tj.j[k0 + j].tiles_w;
            t.key_thr = thin_key_threshold(v.mask_type, np->tau_thin);
        }
        const int blocks = grid_for(c->cap, c->sm_count);
        const int32_t acc = c->n_views + k0 > 0 ? 1 : 0;
        DIVAS_CUDA(c, cudaMemsetAsync(n_heavy, 0, sizeof(int32_t), s));
        const bool f16 = batch_all_f16(tb);
        if (c->G.contracted)
            st = f16 ? launch_nerf_scan<true, kMaskF16>(tb.n, blocks, s, c, tb, N, density, acc, heavy,
                                                        n_heavy)
                     : launch_nerf_scan<true, -1>(tb.n, blocks, s, c, tb, N, density, acc, heavy,
                                                  n_heavy);
        else
            st = f16 ? launch_nerf_scan<false, kMaskF16>(tb.n, blocks, s, c, tb, N, density, acc, heavy,
                                                         n_heavy)
                     : launch_nerf_scan<false, -1>(tb.n, blocks, s, c, tb, N, density, acc, heavy,
                                                   n_heavy);
        if (st != DIVAS_OK) return st;
        if (last) {
            st = record_stage(c, stage_events, 2, s);
            if (st != DIVAS_OK) return st;
        }
#define DIVAS_NERF_HEAVY(KC, MT)                                                                   \
    k_nerf_heavy<KC, MT><<<blocks, kThreads, 0, s>>>(c->active, heavy, n_heavy, c->G, c->F, tb, N,   \
                                                     c->W, c->Z, c->bits)
        if (c->G.contracted) {
            if (f16) DIVAS_NERF_HEAVY(true, kMaskF16);
            else DIVAS_NERF_HEAVY(true, -1);
        } else {
            if (f16) DIVAS_NERF_HEAVY(false, kMaskF16);
            else DIVAS_NERF_HEAVY(false, -1);
        }
#undef DIVAS_NERF_HEAVY
        DIVAS_LAUNCHED(c, "k_nerf_heavy");
    }
    c->n_views += n_views;
    return record_stage(c, stage_events, 3, s);
}

divas_status divas_density_floor(const float* density, int64_t n, float rho_thresh, uint8_t* occ,
                                 void* stream) {
    if (n == 0) return DIVAS_OK;
    if (!density || !occ || n < 0 || !(rho_thresh == rho_thresh)) return DIVAS_E_INVALID;
    if (reinterpret_cast<uintptr_t>(density) % 16 != 0 || reinterpret_cast<uintptr_t>(occ) % 4 != 0)
        return DIVAS_E_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return DIVAS_E_CUDA;
    }
    const cudaStream_t s = S(stream);
    k_density_floor<<<(int)std::min<int64_t>((n / 4 + kOccThreads - 1) / kOccThreads + 1, 16 * (int64_t)sms),
                      kOccThreads, 0, s>>>(density, n, rho_thresh, occ);
    return cudaGetLastError() == cudaSuccess ? DIVAS_OK : DIVAS_E_CUDA;
}

}  // extern "C"
