// surfels.cuh -- the voxel-to-surfel mapping for 2DGS, Passes 1-3 (Sec. 3.6
// "Voxel-to-Surfel Mapping and Aggregation"; Algorithm "Voxel-to-Surfel
// Mapping for 2DGS"; Eqs. pass1, aspect, needle, pass-needle, cov-atomics,
// kappa, final-F), included by divas_fuse.cu after the label kernels.
//
// Pass 1 is the label lookup of the context's seg bitfield (the cell of the
// surfel's centre); Pass 2 culls aspects above their exact 99th percentile
// (select.cuh); Pass 3 gives each surviving surfel, in every view whose bit is
// set in its voxel's view mask (the context's vote bits, found by a binary
// search of the ascending active list), the count of pixels of its 1-sigma
// box that pass the 3-sigma Cramer test in tangent coordinates and of those
// whose mask reaches tau_M, and keeps it when some view's foreground fraction
// reaches tau_kappa.  One thread owns a surfel's counters and walks its box
// in every view, so no atomics and no tile sort are needed (the paper's tile
// sort is rasterizer scaffolding for ordered blending; coverage counting has
// no order).
#pragma once

#include "select.cuh"

namespace {

constexpr int kSurfThreads = 256;

struct SView {
    float R[9], t[3];
    float fx, fy, cx, cy;
    int32_t W, H;
    const void* mask;
};

struct SViews {
    int32_t n, mask_type;
    float tau_m, logit_m;  // mask gate: probability >= tau_m, or logit >= logit_m
    SView v[kMaxViews];
};
static_assert(sizeof(SViews) <= 3400, "the surfel views fit the kernel parameter space");

// Eq. aspect in FP64 (eps = 1e-8), stored as FP32; NaN scales give NaN
__global__ void __launch_bounds__(kSurfThreads) k_surfel_aspect(const float* __restrict__ s,
                                                                int32_t m, float eps,
                                                                float* __restrict__ a) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double s0 = (double)__ldg(s + 2 * (int64_t)i), s1 = (double)__ldg(s + 2 * (int64_t)i + 1);
        const bool nan = s0 != s0 || s1 != s1;
        const double hi = fmax(s0, s1), lo = fmin(s0, s1);
        a[i] = nan ? __int_as_float(0x7fc00000) : (float)__ddiv_rn(hi, __dadd_rn(lo, (double)eps));
    }
}

__device__ __forceinline__ bool surf_front(const SView& V, const float (&X)[3], float z_near,
                                           float& u, float& v) {
    const float px = __fmaf_rn(V.R[0], X[0], __fmaf_rn(V.R[1], X[1], __fmaf_rn(V.R[2], X[2], V.t[0])));
    const float py = __fmaf_rn(V.R[3], X[0], __fmaf_rn(V.R[4], X[1], __fmaf_rn(V.R[5], X[2], V.t[1])));
    const float pz = __fmaf_rn(V.R[6], X[0], __fmaf_rn(V.R[7], X[1], __fmaf_rn(V.R[8], X[2], V.t[2])));
    if (!(pz > z_near)) return false;
    u = __fmaf_rn(V.fx, __fdiv_rn(px, pz), V.cx);
    v = __fmaf_rn(V.fy, __fdiv_rn(py, pz), V.cy);
    return true;
}

// (total, mask) of a surfel in one view; false when a point is behind
__device__ bool surfel_view(const SView& V, const float (&m)[3], const float (&t0)[3],
                            const float (&t1)[3], int32_t mask_type, float gate, float z_near,
                            uint32_t& total, uint32_t& msk) {
    total = msk = 0u;
    float X[3], cu, cv, u0p, v0p, u0m, v0m, u1p, v1p, u1m, v1m;
    bool ok = surf_front(V, m, z_near, cu, cv);
#pragma unroll
    for (int q = 0; q < 3; ++q) X[q] = __fadd_rn(m[q], t0[q]);
    ok = ok && surf_front(V, X, z_near, u0p, v0p);
#pragma unroll
    for (int q = 0; q < 3; ++q) X[q] = __fsub_rn(m[q], t0[q]);
    ok = ok && surf_front(V, X, z_near, u0m, v0m);
#pragma unroll
    for (int q = 0; q < 3; ++q) X[q] = __fadd_rn(m[q], t1[q]);
    ok = ok && surf_front(V, X, z_near, u1p, v1p);
#pragma unroll
    for (int q = 0; q < 3; ++q) X[q] = __fsub_rn(m[q], t1[q]);
    ok = ok && surf_front(V, X, z_near, u1m, v1m);
    if (!ok) return false;
    const float a0x = __fmul_rn(0.5f, __fsub_rn(u0p, u0m)), a0y = __fmul_rn(0.5f, __fsub_rn(v0p, v0m));
    const float a1x = __fmul_rn(0.5f, __fsub_rn(u1p, u1m)), a1y = __fmul_rn(0.5f, __fsub_rn(v1p, v1m));
    const float det = __fsub_rn(__fmul_rn(a0x, a1y), __fmul_rn(a0y, a1x));
    if (det == 0.f) return true;  // edge-on: no pixel
    const float inv = __frcp_rn(det);
    const float ex = fmaxf(fabsf(a0x), fabsf(a1x)), ey = fmaxf(fabsf(a0y), fabsf(a1y));
    // pixel centres x + 1/2 inside [cu - ex, cu + ex], clipped to the frame
    const int x0 = (int)fmaxf(ceilf(__fsub_rn(__fsub_rn(cu, ex), 0.5f)), 0.f);
    const int x1 = (int)fminf(floorf(__fsub_rn(__fadd_rn(cu, ex), 0.5f)), (float)(V.W - 1));
    const int y0 = (int)fmaxf(ceilf(__fsub_rn(__fsub_rn(cv, ey), 0.5f)), 0.f);
    const int y1 = (int)fminf(floorf(__fsub_rn(__fadd_rn(cv, ey), 0.5f)), (float)(V.H - 1));
    for (int y = y0; y <= y1; ++y) {
        const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), cv);
        for (int x = x0; x <= x1; ++x) {
            const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), cu);
            const float uu = __fmul_rn(__fsub_rn(__fmul_rn(dx, a1y), __fmul_rn(dy, a1x)), inv);
            const float vv = __fmul_rn(__fsub_rn(__fmul_rn(a0x, dy), __fmul_rn(a0y, dx)), inv);
            if (__fadd_rn(__fmul_rn(uu, uu), __fmul_rn(vv, vv)) <= 9.f) {
                ++total;
                const int32_t q = y * V.W + x;
                const float mv = mask_type == kMaskF16
                    ? __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(V.mask) + q)))
                    : __ldg(reinterpret_cast<const float*>(V.mask) + q);
                msk += mv >= gate ? 1u : 0u;
            }
        }
    }
    return true;
}

// the active-list index of packed cell pk (ascending list), or -1
__device__ __forceinline__ int32_t active_find(const uint32_t* __restrict__ active, int32_t n,
                                               uint32_t pk) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(active + mid) < pk) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && __ldg(active + lo) == pk ? lo : -1;
}

// Passes 1-3 per surfel: f (final), f2 (after the needle cull), kappa
__global__ void __launch_bounds__(kSurfThreads) k_surfel_pass(
    const float* __restrict__ mu, const float* __restrict__ scales, const float* __restrict__ quats,
    const float* __restrict__ aspect, int32_t m, GridC G, const uint32_t* __restrict__ seg_bits,
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n,
    const uint32_t* __restrict__ vbits, const SelState* __restrict__ st,
    const __grid_constant__ SViews SV, float tau_kappa, float z_near, uint8_t* __restrict__ f_out,
    uint8_t* __restrict__ f2_out, float* __restrict__ kappa_out) {
    const float tau_a = (float)sel_value(st[0], 0.99);
    const int32_t n_act = *d_n;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int32_t idx[3];
        bool f2 = false, f = false;
        float kappa = 0.f;
        if (point_cell(mu, i, G, idx)) {
            const int64_t lin = ((int64_t)idx[2] * G.g + idx[1]) * G.g + idx[0];
            const bool f1 = (__ldg(seg_bits + (lin >> 5)) >> (lin & 31)) & 1u;
            f2 = f1 && __ldg(aspect + i) <= tau_a;
            const uint32_t pk = (uint32_t)idx[0] | ((uint32_t)idx[1] << 10) | ((uint32_t)idx[2] << 20);
            const int32_t ai = f2 ? active_find(active, n_act, pk) : -1;
            const uint32_t vb = ai >= 0 ? __ldg(vbits + ai) : 0u;
            if (vb) {
                // tangent semi-axes: the scales on the rotation's first two columns
                const float qw = __ldg(quats + 4 * (int64_t)i), qx = __ldg(quats + 4 * (int64_t)i + 1);
                const float qy = __ldg(quats + 4 * (int64_t)i + 2), qz = __ldg(quats + 4 * (int64_t)i + 3);
                const float rn = __frsqrt_rn(__fmaf_rn(qw, qw, __fmaf_rn(qx, qx, __fmaf_rn(qy, qy, __fmul_rn(qz, qz)))));
                const float w = __fmul_rn(qw, rn), x = __fmul_rn(qx, rn), y = __fmul_rn(qy, rn),
                            z = __fmul_rn(qz, rn);
                const float s0 = __ldg(scales + 2 * (int64_t)i), s1 = __ldg(scales + 2 * (int64_t)i + 1);
                const float c0[3] = {__fsub_rn(1.f, __fmul_rn(2.f, __fmaf_rn(y, y, __fmul_rn(z, z)))),
                                     __fmul_rn(2.f, __fmaf_rn(x, y, __fmul_rn(w, z))),
                                     __fmul_rn(2.f, __fsub_rn(__fmul_rn(x, z), __fmul_rn(w, y)))};
                const float c1[3] = {__fmul_rn(2.f, __fsub_rn(__fmul_rn(x, y), __fmul_rn(w, z))),
                                     __fsub_rn(1.f, __fmul_rn(2.f, __fmaf_rn(x, x, __fmul_rn(z, z)))),
                                     __fmul_rn(2.f, __fmaf_rn(y, z, __fmul_rn(w, x)))};
                float t0[3], t1[3];
                const float mm[3] = {__ldg(mu + 3 * (int64_t)i), __ldg(mu + 3 * (int64_t)i + 1),
                                     __ldg(mu + 3 * (int64_t)i + 2)};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    t0[q] = __fmul_rn(s0, c0[q]);
                    t1[q] = __fmul_rn(s1, c1[q]);
                }
                const float gate = SV.mask_type == kMaskLogit ? SV.logit_m : SV.tau_m;
                for (int32_t s = 0; s < SV.n; ++s) {
                    if (!((vb >> s) & 1u)) continue;
                    uint32_t tot, msk;
                    if (!surfel_view(SV.v[s], mm, t0, t1, SV.mask_type, gate, z_near, tot, msk)) continue;
                    const uint32_t den = max(tot, 1u);
                    kappa = fmaxf(kappa, __fdiv_rn((float)msk, (float)den));
                    f = f || (double)msk >= (double)tau_kappa * (double)den;
                }
            }
        }
        f_out[i] = (uint8_t)(f2 && f);
        if (f2_out) f2_out[i] = (uint8_t)f2;
        if (kappa_out) kappa_out[i] = kappa;
    }
}

}  // namespace

extern "C" {

divas_surfel_params divas_default_surfel_params(void) {
    divas_surfel_params p;
    p.tau_m = 0.5f;
    p.tau_kappa = 0.5f;
    p.eps_aspect = 1e-8f;
    p.reserved = 0;
    return p;
}

divas_status divas_surfel_labels(divas_ctx* c, const float* mu, const float* scales,
                                 const float* quats, int64_t m, const divas_camera* cams,
                                 const void* const* masks, int32_t mask_type, int32_t n_views,
                                 const divas_surfel_params* p, uint8_t* f_out, uint8_t* f2_out,
                                 float* kappa_out, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (!mu || !scales || !quats || !f_out || !p || m < 1 || m > INT32_MAX / 4)
        return fail(c, DIVAS_E_INVALID, "surfel arrays NULL or m out of range");
    if (n_views < 0 || n_views > kMaxViews || (n_views > 0 && (!cams || !masks)))
        return fail(c, DIVAS_E_INVALID, "n_views must be in 0..32 with cameras and masks");
    if (mask_type < 0 || mask_type > 2) return fail(c, DIVAS_E_INVALID, "bad mask_type");
    if (!(p->tau_m > 0.f && p->tau_m < 1.f) || !(p->tau_kappa >= 0.f) || !(p->eps_aspect > 0.f))
        return fail(c, DIVAS_E_INVALID, "surfel params out of range");
    SViews SV;
    memset(&SV, 0, sizeof(SV));
    SV.n = n_views;
    SV.mask_type = mask_type;
    SV.tau_m = p->tau_m;
    SV.logit_m = logit_threshold(p->tau_m);
    for (int32_t k = 0; k < n_views; ++k) {
        divas_status st = check_camera(c, &cams[k]);
        if (st != DIVAS_OK) return st;
        if (!masks[k]) return fail(c, DIVAS_E_INVALID, "a mask is NULL");
        SView& v = SV.v[k];
        memcpy(v.R, cams[k].R, sizeof(v.R));
        memcpy(v.t, cams[k].t, sizeof(v.t));
        v.fx = cams[k].fx;
        v.fy = cams[k].fy;
        v.cx = cams[k].cx;
        v.cy = cams[k].cy;
        v.W = cams[k].W;
        v.H = cams[k].H;
        v.mask = masks[k];
    }
    // scratch (the weighting's): aspects, then one selection job
    const int32_t n = (int32_t)m;
    const size_t arr = ((size_t)n * 4 + 255) / 256 * 256;
    const size_t need = arr + sel_scratch_bytes(1);
    cudaStream_t s = S(stream);
    if (need > c->wt_bytes) {
        if (capturing(s))
            return fail(c, DIVAS_E_STATE, "surfel scratch must grow outside a stream capture");
        DIVAS_CUDA(c, cudaStreamSynchronize(s));
        if (c->wt) cudaFree(c->wt);
        c->wt = nullptr;
        c->wt_bytes = 0;
        DIVAS_CUDA(c, cudaMalloc(&c->wt, need));
        c->wt_bytes = need;
    }
    float* aspect = static_cast<float*>(c->wt);
    void* sel = static_cast<unsigned char*>(c->wt) + arr;
    const int blocks = (int)std::min<int64_t>((n + kSurfThreads - 1) / kSurfThreads, 16 * (int64_t)c->sm_count);
    k_surfel_aspect<<<blocks, kSurfThreads, 0, s>>>(scales, n, p->eps_aspect, aspect);
    DIVAS_LAUNCHED(c, "k_surfel_aspect");
    SelJobs J;
    memset(&J, 0, sizeof(J));
    J.n = 1;
    J.j[0] = {aspect, n, 1, 0.99};
    DIVAS_CUDA(c, sel_launch(J, sel, sel_blocks(n, 1, c->sm_count), s));
    k_surfel_pass<<<blocks, kSurfThreads, 0, s>>>(mu, scales, quats, aspect, n, c->G, c->seg_bits,
                                                  c->active, c->d_n, c->bits,
                                                  static_cast<const SelState*>(sel), SV, p->tau_kappa,
                                                  c->F.z_near, f_out, f2_out, kappa_out);
    DIVAS_LAUNCHED(c, "k_surfel_pass");
    return DIVAS_OK;
}

}  // extern "C"
