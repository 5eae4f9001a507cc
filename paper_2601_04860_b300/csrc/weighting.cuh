// weighting.cuh -- depth-weighted mask refinement (Sec. 3.4 "Depth-weighting:
// bounded normalization (NeRF) vs. band-pass (2DGS)"; Eq. nerf-depthweight,
// Eqs. depthband and gs-bandpass), included by divas_fuse.cu.
//
// Per view the weighted mask M~ = M w(D) is written as FP32 probabilities, to
// be folded like any FP32 mask (thick or tuple mode):
//   NeRF min-max:  w = 1 - (D - min D) / (max D - min D)
//   2DGS band:     w = 1 - clip((max(d_min - D, 0) + max(D - d_max, 0)) /
//                               max(d_far - d_max, 1e-6), 0, 1),
//                  [d_min, d_max] = the range of D at the prompts and the
//                  view centre, d_far = P98(D).
// Non-finite depth is no surface: w = 0 there, and it takes no part in min,
// max or the percentile.  P98 is the linear-interpolation percentile between
// the order statistics of ranks k = floor(0.98 (n - 1)) and k + 1 of the n
// finite values, found exactly by the radix select of select.cuh.  All views
// of a call run in one launch per pass (blockIdx.y = view).
#pragma once

#include "select.cuh"

namespace {

constexpr int kWeightPrompts = DIVAS_MAX_PROMPTS + 1;  // + the view centre
constexpr int kWeightThreads = 256;
constexpr int kUnroll = 4;                             // pixels per thread with loads in flight

struct WJob {
    const float* depth;
    const void* mask;
    float* out;
    int32_t mask_type, W, H, n_samples;   // samples: the prompts and the centre
    int32_t sample_pix[kWeightPrompts];   // pixel indices y W + x
};

struct WJobs {
    int32_t n, mode;
    WJob j[kMaxViews];
};
static_assert(sizeof(WJobs) <= 3800, "the weighting jobs fit the kernel parameter space");

// mask probability at pixel i
__device__ __forceinline__ float weight_mask(const WJob& jb, int32_t i) {
    if (jb.mask_type == kMaskF16)
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(jb.mask) + i)));
    const float x = __ldg(reinterpret_cast<const float*>(jb.mask) + i);
    return jb.mask_type == kMaskLogit ? __frcp_rn(__fadd_rn(1.f, expf(-x))) : x;
}

// The view's weighting constants, then M~ per pixel.  stats (nullable):
// views x 4 floats, (min, max, n, 0) or (d_min, d_max, d_far, n).
__global__ void __launch_bounds__(kWeightThreads) k_weight_apply(const __grid_constant__ WJobs J,
                                                                 const SelState* __restrict__ st,
                                                                 float* __restrict__ stats) {
    const WJob& jb = J.j[blockIdx.y];
    const SelState& S = st[blockIdx.y];
    __shared__ float s_a, s_b, s_den;
    __shared__ int s_kind;  // 0: weight 1 on finite pixels, 1: min-max, 2: band
    if (threadIdx.x == 0) {
        const uint32_t n = __ldcg(&S.n_fin);
        float a = 0.f, b = 0.f, den = 1.f, far = __int_as_float(0x7fc00000);
        int kind = 0;
        if (J.mode == DIVAS_WEIGHT_NERF_MINMAX) {
            if (n) {
                a = key_float(__ldcg(&S.lo_key));
                b = key_float(__ldcg(&S.hi_key));
            }
            if (b > a) {
                kind = 1;
                den = __fsub_rn(b, a);
            }
            if (!n) a = b = __int_as_float(0x7fc00000);
        } else {
            float mn = FLT_MAX, mx = -FLT_MAX;
            bool any = false;
            for (int q = 0; q < jb.n_samples; ++q) {
                const float d = __ldg(jb.depth + jb.sample_pix[q]);
                if (!finite_f(d)) continue;
                mn = fminf(mn, d);
                mx = fmaxf(mx, d);
                any = true;
            }
            if (any) {
                kind = 2;
                a = mn;
                b = mx;
                const double dfar = n ? sel_value(S, 0.98) : (double)mx;
                far = (float)dfar;
                den = fmaxf(__fsub_rn(far, mx), 1e-6f);
            } else {
                a = b = __int_as_float(0x7fc00000);
            }
        }
        s_a = a;
        s_b = b;
        s_den = den;
        s_kind = kind;
        if (stats && blockIdx.x == 0) {
            float* o = stats + 4 * blockIdx.y;
            const bool minmax = J.mode == DIVAS_WEIGHT_NERF_MINMAX;
            o[0] = a;
            o[1] = b;
            o[2] = minmax ? (float)n : far;
            o[3] = minmax ? 0.f : (float)n;
        }
    }
    __syncthreads();
    const float a = s_a, b = s_b, den = s_den;
    const int kind = s_kind;
    const int32_t npix = jb.W * jb.H;
    const int32_t stride = gridDim.x * kWeightThreads;
    for (int32_t b0 = blockIdx.x * kWeightThreads + threadIdx.x; b0 < npix; b0 += kUnroll * stride) {
        float d[kUnroll], m[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t i = b0 + u * stride;
            d[u] = i < npix ? __ldg(jb.depth + i) : 0.f;
            m[u] = i < npix ? weight_mask(jb, i) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t i = b0 + u * stride;
            float w = 0.f;
            if (finite_f(d[u])) {
                if (kind == 1) {
                    w = __fsub_rn(1.f, __fdiv_rn(__fsub_rn(d[u], a), den));
                } else if (kind == 2) {
                    const float dm = fmaxf(__fsub_rn(a, d[u]), 0.f), dp = fmaxf(__fsub_rn(d[u], b), 0.f);
                    const float band = fminf(fmaxf(__fdiv_rn(__fadd_rn(dm, dp), den), 0.f), 1.f);
                    w = __fsub_rn(1.f, band);
                } else {
                    w = 1.f;
                }
            }
            if (i < npix) jb.out[i] = __fmul_rn(m[u], w);
        }
    }
}

}  // namespace

extern "C" {

divas_status divas_depth_weight(divas_ctx* c, const divas_weight_view* views, int32_t n_views,
                                int32_t mode, float* stats_out, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (!views || n_views < 1 || n_views > kMaxViews)
        return fail(c, DIVAS_E_INVALID, "n_views must be in 1..32 and views non-NULL");
    if (mode != DIVAS_WEIGHT_NERF_MINMAX && mode != DIVAS_WEIGHT_GS_BAND)
        return fail(c, DIVAS_E_INVALID, "unknown weighting mode");
    WJobs J;
    memset(&J, 0, sizeof(J));
    J.n = n_views;
    J.mode = mode;
    int64_t max_pix = 0;
    for (int32_t k = 0; k < n_views; ++k) {
        const divas_weight_view& v = views[k];
        if (!v.depth || !v.mask || !v.out) return fail(c, DIVAS_E_INVALID, "a raster is NULL");
        if (v.mask_type < 0 || v.mask_type > 2) return fail(c, DIVAS_E_INVALID, "bad mask_type");
        if (v.W < 1 || v.H < 1 || (int64_t)v.W * v.H > INT32_MAX)
            return fail(c, DIVAS_E_INVALID, "bad raster size");
        if (v.n_prompts < 0 || v.n_prompts > DIVAS_MAX_PROMPTS)
            return fail(c, DIVAS_E_INVALID, "n_prompts out of range");
        WJob& jb = J.j[k];
        jb.depth = v.depth;
        jb.mask = v.mask;
        jb.out = v.out;
        jb.mask_type = v.mask_type;
        jb.W = v.W;
        jb.H = v.H;
        for (int32_t q = 0; q < v.n_prompts; ++q) {
            const int32_t x = v.prompt_xy[2 * q], y = v.prompt_xy[2 * q + 1];
            if (x < 0 || x >= v.W || y < 0 || y >= v.H)
                return fail(c, DIVAS_E_INVALID, "a prompt is outside its view");
            jb.sample_pix[q] = y * v.W + x;
        }
        jb.sample_pix[v.n_prompts] = (v.H / 2) * v.W + v.W / 2;  // the view centre
        jb.n_samples = v.n_prompts + 1;
        max_pix = std::max<int64_t>(max_pix, (int64_t)v.W * v.H);
    }
    // the selection jobs: each view's depth raster (count and min / max for
    // min-max, the 98th percentile for the band)
    SelJobs SJ;
    memset(&SJ, 0, sizeof(SJ));
    SJ.n = n_views;
    SJ.minmax = mode == DIVAS_WEIGHT_NERF_MINMAX ? 1 : 0;
    for (int32_t k = 0; k < n_views; ++k) {
        SJ.j[k].x = views[k].depth;
        SJ.j[k].n = views[k].W * views[k].H;
        SJ.j[k].stride = 1;
        SJ.j[k].q = mode == DIVAS_WEIGHT_GS_BAND ? 0.98 : -1.0;
    }
    const size_t need = sel_scratch_bytes(n_views);
    cudaStream_t s = S(stream);
    if (need > c->wt_bytes) {
        if (capturing(s))
            return fail(c, DIVAS_E_STATE, "weighting scratch must grow outside a stream capture");
        DIVAS_CUDA(c, cudaStreamSynchronize(s));
        if (c->wt) cudaFree(c->wt);
        c->wt = nullptr;
        c->wt_bytes = 0;
        DIVAS_CUDA(c, cudaMalloc(&c->wt, need));
        c->wt_bytes = need;
    }
    const int per_view = sel_blocks(max_pix, n_views, c->sm_count);
    DIVAS_CUDA(c, sel_launch(SJ, c->wt, per_view, s));
    const SelState* st = static_cast<const SelState*>(c->wt);
    const dim3 grid(per_view, n_views);
    k_weight_apply<<<grid, kWeightThreads, 0, s>>>(J, st, stats_out);
    DIVAS_LAUNCHED(c, "k_weight_apply");
    return DIVAS_OK;
}

}  // extern "C"
