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

// The view's weighting constants: kind 0 (weight 1 on finite pixels), 1
// (min-max: a = min D, den = max D - min D) or 2 (band [a, b], den = max(d_far
// - b, 1e-6)); the stats row (min, max, n, 0) or (d_min, d_max, d_far, n).
struct WConsts {
    float a, b, den;
    int32_t kind;
};

__device__ __forceinline__ WConsts weight_consts(const WJob& jb, const SelState& S, int32_t mode,
                                                 float* stats_row) {
    const uint32_t n = __ldcg(&S.n_fin);
    float a = 0.f, b = 0.f, den = 1.f, far = __int_as_float(0x7fc00000);
    int kind = 0;
    if (mode == DIVAS_WEIGHT_NERF_MINMAX) {
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
    if (stats_row) {
        const bool minmax = mode == DIVAS_WEIGHT_NERF_MINMAX;
        stats_row[0] = a;
        stats_row[1] = b;
        stats_row[2] = minmax ? (float)n : far;
        stats_row[3] = minmax ? 0.f : (float)n;
    }
    WConsts c;
    c.a = a;
    c.b = b;
    c.den = den;
    c.kind = kind;
    return c;
}

// the weight w(D) of one pixel's depth (0 where D is not finite)
__device__ __forceinline__ float weight_of(const WConsts& c, float d) {
    if (!finite_f(d)) return 0.f;
    if (c.kind == 1) return __fsub_rn(1.f, __fdiv_rn(__fsub_rn(d, c.a), c.den));
    if (c.kind == 2) {
        const float dm = fmaxf(__fsub_rn(c.a, d), 0.f), dp = fmaxf(__fsub_rn(d, c.b), 0.f);
        const float band = fminf(fmaxf(__fdiv_rn(__fadd_rn(dm, dp), c.den), 0.f), 1.f);
        return __fsub_rn(1.f, band);
    }
    return 1.f;
}

// The view's weighting constants, then M~ per pixel.  stats (nullable):
// views x 4 floats, (min, max, n, 0) or (d_min, d_max, d_far, n).
__global__ void __launch_bounds__(kWeightThreads) k_weight_apply(const __grid_constant__ WJobs J,
                                                                 const SelState* __restrict__ st,
                                                                 float* __restrict__ stats) {
    const WJob& jb = J.j[blockIdx.y];
    const SelState& S = st[blockIdx.y];
    __shared__ WConsts s_c;
    if (threadIdx.x == 0)
        s_c = weight_consts(jb, S, J.mode,
                            stats && blockIdx.x == 0 ? stats + 4 * blockIdx.y : nullptr);
    __syncthreads();
    const WConsts wc = s_c;
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
            if (i < npix) jb.out[i] = __fmul_rn(m[u], weight_of(wc, d[u]));
        }
    }
}

// per view of a call, its weighting constants (one thread per view)
__global__ void k_weight_consts(const __grid_constant__ WJobs J, const SelState* __restrict__ st,
                                WConsts* __restrict__ out, float* __restrict__ stats) {
    const int v = threadIdx.x;
    if (v < J.n) out[v] = weight_consts(J.j[v], st[v], J.mode, stats ? stats + 4 * v : nullptr);
}

// The thick-path fold with the depth weight applied to the mask value each
// vote reads: m~ = m w(D) (m the mask probability, w the view's weight of the
// depth at the pixel), gated m~ >= tau_m and voted with m~.  Per vote this is
// the arithmetic of folding divas_depth_weight's weighted raster as an FP32
// mask, so the two give the same accumulators bit for bit; no weighted raster
// is written.  (0 <= m < tau_m cannot pass: w lies in [0, 1], so the weight
// is only computed for the other votes.)
template <bool kContracted, int kChunks>
__global__ void __launch_bounds__(kThreads) k_fuse_weighted(
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n, GridC G, FuseC F,
    const __grid_constant__ ViewBatch VB, const WConsts* __restrict__ consts, int32_t accumulate,
    float* __restrict__ W, float* __restrict__ Z, uint32_t* __restrict__ bits) {
    __shared__ WConsts sc[kMaxViews];
    if (threadIdx.x < VB.n) sc[threadIdx.x] = consts[threadIdx.x];
    __syncthreads();
    const int32_t n = *d_n;
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const VoxelGeom vg = voxel_geom<kContracted>(__ldg(active + a), G, F.gamma);
        float w = 0.f, z = 0.f;
        uint32_t b = 0;
        if (accumulate) {
            w = W[a];
            z = Z[a];
            b = bits[a];
        }
        if (vg.ok) {
#pragma unroll
            for (int c = 0; c < kChunks; ++c) {
                int32_t pix[kViewChunk];
                float pzh[kViewChunk], pzl[kViewChunk], D[kViewChunk], raw[kViewChunk];
#pragma unroll
                for (int q = 0; q < kViewChunk; ++q) {
                    pix[q] = -1;
                    if (c * kViewChunk + q < VB.n)
                        pix[q] = project<kContracted>(VB.v[c * kViewChunk + q], vg, F.z_near,
                                                      pzh[q], pzl[q]);
                }
#pragma unroll
                for (int q = 0; q < kViewChunk; ++q)
                    if (c * kViewChunk + q < VB.n)
                        load_raster(VB.v[c * kViewChunk + q], pix[q], D[q], raw[q]);
#pragma unroll
                for (int q = 0; q < kViewChunk; ++q) {
                    const int v = c * kViewChunk + q;
                    if (v >= VB.n) break;
                    const ViewC& V = VB.v[v];
                    if (!(pix[q] >= 0 && D[q] > 0.f && D[q] <= FLT_MAX &&
                          depth_screen<kContracted>(V, vg, pzh[q], D[q])))
                        continue;
                    const float e = depth_error<kContracted>(V, vg, pzh[q], pzl[q], D[q]);
                    const float m = V.mask_type == kMaskLogit
                                        ? __frcp_rn(__fadd_rn(1.f, expf(-raw[q])))
                                        : raw[q];
                    if (fabsf(e) <= vg.Delta && !(m >= 0.f && m < F.tau_m)) {
                        const float mt = __fmul_rn(m, weight_of(sc[v], D[q]));
                        if (mt >= F.tau_m) {
                            const float r = __fmul_rn(e, vg.invDelta);
                            const float ww = expf(-__fmul_rn(F.alpha1, __fmul_rn(r, r)));
                            w = __fmaf_rn(mt, ww, w);
                            z = __fadd_rn(z, ww);
                            b |= V.bit;
                        }
                    }
                }
            }
        }
        W[a] = w;
        Z[a] = z;
        bits[a] = b;
    }
}

template <bool kContracted, int kChunks = 1>
cudaError_t launch_fuse_weighted(int chunks, int blocks, cudaStream_t s, const divas_ctx* c,
                                 const ViewBatch& vb, const WConsts* consts, int32_t acc) {
    if constexpr (kChunks < kMaxViews / kViewChunk) {
        if (chunks > kChunks)
            return launch_fuse_weighted<kContracted, kChunks + 1>(chunks, blocks, s, c, vb, consts,
                                                                  acc);
    }
    k_fuse_weighted<kContracted, kChunks><<<blocks, kThreads, 0, s>>>(
        c->active, c->d_n, c->G, c->F, vb, consts, acc, c->W, c->Z, c->bits);
    return cudaGetLastError();
}

// weighting jobs of n views (depth, mask, prompts and the view centre); false
// with the reason for an invalid prompt
bool weight_jobs(const divas_weight_view* views, int32_t n_views, int32_t mode, WJobs& J,
                 const char** why) {
    memset(&J, 0, sizeof(J));
    J.n = n_views;
    J.mode = mode;
    for (int32_t k = 0; k < n_views; ++k) {
        const divas_weight_view& v = views[k];
        if (v.n_prompts < 0 || v.n_prompts > DIVAS_MAX_PROMPTS) {
            *why = "n_prompts out of range";
            return false;
        }
        WJob& jb = J.j[k];
        jb.depth = v.depth;
        jb.mask = v.mask;
        jb.out = v.out;
        jb.mask_type = v.mask_type;
        jb.W = v.W;
        jb.H = v.H;
        for (int32_t q = 0; q < v.n_prompts; ++q) {
            const int32_t x = v.prompt_xy[2 * q], y = v.prompt_xy[2 * q + 1];
            if (x < 0 || x >= v.W || y < 0 || y >= v.H) {
                *why = "a prompt is outside its view";
                return false;
            }
            jb.sample_pix[q] = y * v.W + x;
        }
        jb.sample_pix[v.n_prompts] = (v.H / 2) * v.W + v.W / 2;  // the view centre
        jb.n_samples = v.n_prompts + 1;
    }
    return true;
}

// the selection scratch (and room for the per-view constants after it)
divas_status weight_scratch(divas_ctx* c, int32_t n_views, cudaStream_t s, size_t extra) {
    const size_t need = sel_scratch_bytes(n_views) + extra;
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
    return DIVAS_OK;
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
    int64_t max_pix = 0;
    for (int32_t k = 0; k < n_views; ++k) {
        const divas_weight_view& v = views[k];
        if (!v.depth || !v.mask || !v.out) return fail(c, DIVAS_E_INVALID, "a raster is NULL");
        if (v.mask_type < 0 || v.mask_type > 2) return fail(c, DIVAS_E_INVALID, "bad mask_type");
        if (v.W < 1 || v.H < 1 || (int64_t)v.W * v.H > INT32_MAX)
            return fail(c, DIVAS_E_INVALID, "bad raster size");
        max_pix = std::max<int64_t>(max_pix, (int64_t)v.W * v.H);
    }
    WJobs J;
    const char* why = nullptr;
    if (!weight_jobs(views, n_views, mode, J, &why)) return fail(c, DIVAS_E_INVALID, why);
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
    cudaStream_t s = S(stream);
    divas_status st0 = weight_scratch(c, n_views, s, 0);
    if (st0 != DIVAS_OK) return st0;
    const int per_view = sel_blocks(max_pix, n_views, c->sm_count);
    DIVAS_CUDA(c, sel_launch(SJ, c->wt, per_view, s));
    const SelState* st = static_cast<const SelState*>(c->wt);
    const dim3 grid(per_view, n_views);
    k_weight_apply<<<grid, kWeightThreads, 0, s>>>(J, st, stats_out);
    DIVAS_LAUNCHED(c, "k_weight_apply");
    return DIVAS_OK;
}

divas_status divas_fuse_add_views_weighted(divas_ctx* c, const divas_view* views,
                                           const divas_weight_view* prompts, int32_t n_views,
                                           int32_t mode, float* stats_out, void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (mode != DIVAS_WEIGHT_NERF_MINMAX && mode != DIVAS_WEIGHT_GS_BAND)
        return fail(c, DIVAS_E_INVALID, "unknown weighting mode");
    if (mode == DIVAS_WEIGHT_GS_BAND && !prompts)
        return fail(c, DIVAS_E_INVALID, "the band-pass weight needs the prompts");
    ViewBatch vb;
    divas_status st = make_batch(c, views, n_views, c->n_views, vb);
    if (st != DIVAS_OK) return st;
    // the weighting jobs read the views' own depth and mask
    divas_weight_view wv[kMaxViews];
    int64_t max_pix = 0;
    for (int32_t k = 0; k < n_views; ++k) {
        memset(&wv[k], 0, sizeof(wv[k]));
        if (prompts) wv[k] = prompts[k];
        wv[k].depth = views[k].depth;
        wv[k].mask = views[k].mask;
        wv[k].out = nullptr;
        wv[k].mask_type = views[k].mask_type;
        wv[k].W = views[k].cam.W;
        wv[k].H = views[k].cam.H;
        if (mode == DIVAS_WEIGHT_NERF_MINMAX) wv[k].n_prompts = 0;
        max_pix = std::max<int64_t>(max_pix, (int64_t)wv[k].W * wv[k].H);
    }
    WJobs J;
    const char* why = nullptr;
    if (!weight_jobs(wv, n_views, mode, J, &why)) return fail(c, DIVAS_E_INVALID, why);
    SelJobs SJ;
    memset(&SJ, 0, sizeof(SJ));
    SJ.n = n_views;
    SJ.minmax = mode == DIVAS_WEIGHT_NERF_MINMAX ? 1 : 0;
    for (int32_t k = 0; k < n_views; ++k) {
        SJ.j[k].x = views[k].depth;
        SJ.j[k].n = wv[k].W * wv[k].H;
        SJ.j[k].stride = 1;
        SJ.j[k].q = mode == DIVAS_WEIGHT_GS_BAND ? 0.98 : -1.0;
    }
    cudaStream_t s = S(stream);
    const size_t sel_bytes = (sel_scratch_bytes(n_views) + 255) / 256 * 256;
    st = weight_scratch(c, n_views, s, sel_bytes - sel_scratch_bytes(n_views) +
                                           kMaxViews * sizeof(WConsts));
    if (st != DIVAS_OK) return st;
    DIVAS_CUDA(c, sel_launch(SJ, c->wt, sel_blocks(max_pix, n_views, c->sm_count), s));
    const SelState* sst = static_cast<const SelState*>(c->wt);
    WConsts* wc = reinterpret_cast<WConsts*>(static_cast<char*>(c->wt) + sel_bytes);
    k_weight_consts<<<1, 32, 0, s>>>(J, sst, wc, stats_out);
    DIVAS_LAUNCHED(c, "k_weight_consts");
    const int chunks = (vb.n + kViewChunk - 1) / kViewChunk;
    const int blocks = grid_for(c->cap, c->sm_count);
    const int32_t acc = c->n_views > 0 ? 1 : 0;
    cudaError_t e = c->G.contracted
                        ? launch_fuse_weighted<true>(chunks, blocks, s, c, vb, wc, acc)
                        : launch_fuse_weighted<false>(chunks, blocks, s, c, vb, wc, acc);
    if (e != cudaSuccess) return cuda_fail(c, e, "k_fuse_weighted");
    c->n_views += vb.n;
    return DIVAS_OK;
}

}  // extern "C"
