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
// finite values, found exactly by a radix select on order-preserving 32-bit
// keys: digits of 11, 11 and 10 bits (one counting pass each), then a pass
// for the count of keys <= x_k and the smallest key above it.  All views of a
// call run in one launch per pass (blockIdx.y = view).
#pragma once

namespace {

constexpr int kWeightPrompts = DIVAS_MAX_PROMPTS + 1;  // + the view centre
constexpr int kRadixBins = 2048;                       // 11-bit digits
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

// per-view selection state (device scratch, set by k_weight_init per call);
// each pass writes its own fields, read only by later launches
struct WState {
    uint32_t n_fin;              // finite pixels
    uint32_t lo_key, hi_key;     // min / max keys (NeRF)
    uint32_t prefix1, rank1;     // after the first digit: key bits fixed, rank left within them
    uint32_t prefix2, rank2;     // after the second digit
    uint32_t c_le, m_gt;         // keys <= x_k, smallest key > x_k
    uint32_t key_k;              // x_k's key
};

// the states' identities and zeroed histograms
__global__ void __launch_bounds__(kWeightThreads) k_weight_init(WState* __restrict__ st, int32_t n,
                                                                uint32_t* __restrict__ hist,
                                                                int64_t hist_words) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        WState z;
        memset(&z, 0, sizeof(z));
        z.lo_key = 0xffffffffu;
        z.m_gt = 0xffffffffu;
        st[t] = z;
    }
    for (int64_t w = t; w < hist_words; w += (int64_t)gridDim.x * blockDim.x) hist[w] = 0u;
}

// finite float -> key whose unsigned order is the float order
__device__ __forceinline__ uint32_t float_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ bool finite_f(float f) { return fabsf(f) <= FLT_MAX; }

// digit pass p (0, 1, 2): bits [shift, shift + width) of the key
__device__ __forceinline__ int digit_shift(int p) { return p == 0 ? 21 : p == 1 ? 10 : 0; }
__device__ __forceinline__ int digit_width(int p) { return p == 2 ? 10 : 11; }

// the rank k = floor(0.98 (n - 1)) and r - k of a view's n finite values
__device__ __forceinline__ uint32_t p98_rank(uint32_t n, double& frac) {
    const double r = 0.98 * (double)(n - 1u);
    const double k = floor(r);
    frac = r - k;
    return (uint32_t)k;
}

// block-wide: the bin of rank `rank` in hist (kRadixBins counts) and the rank
// left within that bin; every thread gets them
__device__ void hist_find(const uint32_t* __restrict__ hist, uint32_t rank, uint32_t& bin,
                          uint32_t& rank_in) {
    __shared__ uint32_t s_bin, s_rank;
    if (threadIdx.x == 0) {
        s_bin = 0u;
        s_rank = 0u;
    }
    __syncthreads();
    constexpr int kPer = kRadixBins / kWeightThreads;
    uint32_t v[kPer], sum = 0u;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        v[q] = __ldcg(hist + threadIdx.x * kPer + q);
        sum += v[q];
    }
    uint32_t total;
    uint32_t before = block_exclusive_scan(sum, &total);
    if (rank >= before && rank < before + sum) {
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            if (rank < before + v[q]) {
                s_bin = threadIdx.x * kPer + q;
                s_rank = rank - before;
                break;
            }
            before += v[q];
        }
    }
    __syncthreads();
    bin = s_bin;
    rank_in = s_rank;
    __syncthreads();
}

// merge a block's shared histogram into the global one (nonzero bins only)
__device__ __forceinline__ void hist_merge(const uint32_t* sh, uint32_t* __restrict__ g) {
    for (int b = threadIdx.x; b < kRadixBins; b += kWeightThreads)
        if (sh[b]) atomicAdd(g + b, sh[b]);
}

// warp-aggregated shared-memory histogram increment
__device__ __forceinline__ void hist_add(uint32_t* sh, bool on, uint32_t bin) {
    const unsigned act = __ballot_sync(0xffffffffu, on);
    if (!on) return;
    const unsigned peers = __match_any_sync(act, bin);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(sh + bin, __popc(peers));
}

// Pass 1: finite count, min / max keys (NeRF) or the first digit's histogram
// (band).  hist: views x 3 x kRadixBins.
__global__ void __launch_bounds__(kWeightThreads) k_weight_pass1(const __grid_constant__ WJobs J,
                                                                 WState* __restrict__ st,
                                                                 uint32_t* __restrict__ hist) {
    const WJob& jb = J.j[blockIdx.y];
    __shared__ uint32_t sh[kRadixBins];
    __shared__ uint32_t s_n, s_lo, s_hi;
    const bool band = J.mode == DIVAS_WEIGHT_GS_BAND;
    for (int b = threadIdx.x; b < kRadixBins; b += kWeightThreads) sh[b] = 0u;
    if (threadIdx.x == 0) {
        s_n = 0u;
        s_lo = 0xffffffffu;
        s_hi = 0u;
    }
    __syncthreads();
    const int32_t npix = jb.W * jb.H;
    uint32_t cnt = 0u, lo = 0xffffffffu, hi = 0u;
    const int32_t stride = gridDim.x * kWeightThreads;
    // warp-uniform loop (the histogram step shuffles), kUnroll loads in flight
    for (int32_t b0 = (blockIdx.x * kWeightThreads + threadIdx.x) & ~31; b0 < npix; b0 += kUnroll * stride) {
        float d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t i = b0 + (threadIdx.x & 31) + u * stride;
            d[u] = i < npix ? __ldg(jb.depth + i) : __int_as_float(0x7fc00000);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const bool fin = finite_f(d[u]);
            const uint32_t key = fin ? float_key(d[u]) : 0u;
            cnt += fin ? 1u : 0u;
            if (fin) {
                lo = min(lo, key);
                hi = max(hi, key);
            }
            if (band) hist_add(sh, fin, key >> 21);
        }
    }
    // block reductions
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_n, cnt);
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
    }
    __syncthreads();
    WState& S = st[blockIdx.y];
    if (threadIdx.x == 0) {
        if (s_n) {
            atomicAdd(&S.n_fin, s_n);
            atomicMin(&S.lo_key, s_lo);
            atomicMax(&S.hi_key, s_hi);
        }
    }
    if (band) hist_merge(sh, hist + (size_t)blockIdx.y * 3 * kRadixBins);
}

// Pass 2 / 3 (P = 1, 2): fix digit P - 1 from its histogram (block 0 keeps
// the prefix for the next pass), then count digit P of the keys that match.
template <int P>
__global__ void __launch_bounds__(kWeightThreads) k_weight_digit(const __grid_constant__ WJobs J,
                                                                 WState* __restrict__ st,
                                                                 uint32_t* __restrict__ hist) {
    const WJob& jb = J.j[blockIdx.y];
    WState& S = st[blockIdx.y];
    const uint32_t n = __ldcg(&S.n_fin);
    if (n == 0u) return;  // whole block: nothing to select
    uint32_t* H = hist + (size_t)blockIdx.y * 3 * kRadixBins;
    uint32_t rank, prefix;
    if (P == 1) {
        double frac;
        rank = p98_rank(n, frac);
        prefix = 0u;
    } else {
        rank = __ldcg(&S.rank1);
        prefix = __ldcg(&S.prefix1);
    }
    uint32_t bin, rin;
    hist_find(H + (P - 1) * kRadixBins, rank, bin, rin);
    prefix |= bin << digit_shift(P - 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (P == 1) {
            S.prefix1 = prefix;
            S.rank1 = rin;
        } else {
            S.prefix2 = prefix;
            S.rank2 = rin;
        }
    }
    __shared__ uint32_t sh[kRadixBins];
    for (int b = threadIdx.x; b < kRadixBins; b += kWeightThreads) sh[b] = 0u;
    __syncthreads();
    const int hi_shift = digit_shift(P - 1);
    const int sh_p = digit_shift(P);
    const uint32_t dmask = (1u << digit_width(P)) - 1u;
    const int32_t npix = jb.W * jb.H;
    const int32_t stride = gridDim.x * kWeightThreads;
    for (int32_t b0 = (blockIdx.x * kWeightThreads + threadIdx.x) & ~31; b0 < npix; b0 += kUnroll * stride) {
        float d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t i = b0 + (threadIdx.x & 31) + u * stride;
            d[u] = i < npix ? __ldg(jb.depth + i) : __int_as_float(0x7fc00000);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const bool fin = finite_f(d[u]);
            const uint32_t key = fin ? float_key(d[u]) : 0u;
            const bool match = fin && (key >> hi_shift) == (prefix >> hi_shift);
            hist_add(sh, match, (key >> sh_p) & dmask);
        }
    }
    __syncthreads();
    hist_merge(sh, H + P * kRadixBins);
}

// Pass 4: fix the last digit (x_k's key), then count the keys <= x_k and
// take the smallest key > x_k.
__global__ void __launch_bounds__(kWeightThreads) k_weight_final(const __grid_constant__ WJobs J,
                                                                 WState* __restrict__ st,
                                                                 const uint32_t* __restrict__ hist) {
    const WJob& jb = J.j[blockIdx.y];
    WState& S = st[blockIdx.y];
    if (__ldcg(&S.n_fin) == 0u) return;
    uint32_t bin, rin;
    hist_find(hist + (size_t)blockIdx.y * 3 * kRadixBins + 2 * kRadixBins, __ldcg(&S.rank2), bin,
              rin);
    const uint32_t key_k = __ldcg(&S.prefix2) | bin;
    if (blockIdx.x == 0 && threadIdx.x == 0) S.key_k = key_k;
    __shared__ uint32_t s_le, s_gt;
    if (threadIdx.x == 0) {
        s_le = 0u;
        s_gt = 0xffffffffu;
    }
    __syncthreads();
    uint32_t le = 0u, gt = 0xffffffffu;
    const int32_t npix = jb.W * jb.H;
    const int32_t stride = gridDim.x * kWeightThreads;
    for (int32_t b0 = blockIdx.x * kWeightThreads + threadIdx.x; b0 < npix; b0 += kUnroll * stride) {
        float d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t i = b0 + u * stride;
            d[u] = i < npix ? __ldg(jb.depth + i) : __int_as_float(0x7fc00000);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (!finite_f(d[u])) continue;
            const uint32_t key = float_key(d[u]);
            if (key <= key_k) ++le;
            else gt = min(gt, key);
        }
    }
    le = __reduce_add_sync(0xffffffffu, le);
    gt = __reduce_min_sync(0xffffffffu, gt);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_le, le);
        atomicMin(&s_gt, gt);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&S.c_le, s_le);
        atomicMin(&S.m_gt, s_gt);
    }
}

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
                                                                 const WState* __restrict__ st,
                                                                 float* __restrict__ stats) {
    const WJob& jb = J.j[blockIdx.y];
    const WState& S = st[blockIdx.y];
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
                double dfar = (double)mx;
                if (n) {
                    double frac;
                    const uint32_t k = p98_rank(n, frac);
                    const uint32_t key_k = __ldcg(&S.key_k);
                    const double xk = (double)key_float(key_k);
                    double xk1 = xk;
                    if (k + 1u < n && __ldcg(&S.c_le) < k + 2u) xk1 = (double)key_float(__ldcg(&S.m_gt));
                    dfar = xk + frac * (xk1 - xk);
                }
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
    // scratch: states, then the three histograms of each view
    const size_t st_bytes = ((size_t)n_views * sizeof(WState) + 255) / 256 * 256;
    const size_t need = st_bytes + (size_t)n_views * 3 * kRadixBins * 4;
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
    WState* st = static_cast<WState*>(c->wt);
    uint32_t* hist = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(c->wt) + st_bytes);
    const int64_t hist_words = (int64_t)n_views * 3 * kRadixBins;
    k_weight_init<<<(unsigned)((hist_words + kWeightThreads - 1) / kWeightThreads), kWeightThreads, 0, s>>>(
        st, n_views, hist, hist_words);
    DIVAS_LAUNCHED(c, "k_weight_init");
    // about 8 blocks per SM over all views, at least kUnroll pixels per thread
    const int per_view = (int)std::max<int64_t>(1, std::min<int64_t>(
        (max_pix + kWeightThreads * kUnroll - 1) / (kWeightThreads * kUnroll),
        (8 * c->sm_count + n_views - 1) / n_views));
    const dim3 grid(per_view, n_views);
    k_weight_pass1<<<grid, kWeightThreads, 0, s>>>(J, st, hist);
    DIVAS_LAUNCHED(c, "k_weight_pass1");
    if (mode == DIVAS_WEIGHT_GS_BAND) {
        k_weight_digit<1><<<grid, kWeightThreads, 0, s>>>(J, st, hist);
        DIVAS_LAUNCHED(c, "k_weight_digit");
        k_weight_digit<2><<<grid, kWeightThreads, 0, s>>>(J, st, hist);
        DIVAS_LAUNCHED(c, "k_weight_digit");
        k_weight_final<<<grid, kWeightThreads, 0, s>>>(J, st, hist);
        DIVAS_LAUNCHED(c, "k_weight_final");
    }
    k_weight_apply<<<grid, kWeightThreads, 0, s>>>(J, st, stats_out);
    DIVAS_LAUNCHED(c, "k_weight_apply");
    return DIVAS_OK;
}

}  // extern "C"
