// select.cuh -- exact order statistics of FP32 arrays, many arrays per launch,
// included by divas_fuse.cu.  For each job (an array x[i * stride], i < n)
// the pass over its finite values gives their count and, on request, their
// minimum and maximum; the linear-interpolation quantile q (Hyndman and Fan
// type 7: r = q (n - 1), k = floor(r), s[k] + (r - k) (s[k + 1] - s[k]) over
// the ascending finite values s) is found exactly by a radix select on
// order-preserving 32-bit keys: digits of 11, 11 and 10 bits (one counting
// pass each, shared-memory histograms merged per block), then a pass for the
// count of keys <= s[k] and the smallest key above it (s[k + 1]).  The value
// itself is formed in FP64 by sel_value.  blockIdx.y = job; 256 threads, four
// elements per thread with their loads in flight.
#pragma once

namespace {

constexpr int kSelThreads = 256;
constexpr int kSelUnroll = 4;
constexpr int kRadixBins = 2048;  // 11-bit digits
constexpr int kMaxSelJobs = 32;

struct SelJob {
    const float* x;
    int32_t n, stride;
    double q;  // the quantile in [0, 1]; < 0: no selection (count, min / max only)
};

struct SelJobs {
    int32_t n;
    int32_t minmax;  // also the min / max keys
    SelJob j[kMaxSelJobs];
};

// per-job state (device scratch, set by k_sel_init); each pass writes its own
// fields, read only by later launches
struct SelState {
    uint32_t n_fin;           // finite values
    uint32_t lo_key, hi_key;  // min / max keys
    uint32_t prefix1, rank1;  // after the first digit: key bits fixed, rank left within them
    uint32_t prefix2, rank2;  // after the second digit
    uint32_t c_le, m_gt;      // keys <= s[k], smallest key > s[k]
    uint32_t key_k;           // s[k]'s key
};

__global__ void __launch_bounds__(kSelThreads) k_sel_init(SelState* __restrict__ st, int32_t n,
                                                          uint32_t* __restrict__ hist,
                                                          int64_t hist_words) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        SelState z;
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

// digit p (0, 1, 2): bits [shift, shift + width) of the key
__device__ __forceinline__ int digit_shift(int p) { return p == 0 ? 21 : p == 1 ? 10 : 0; }
__device__ __forceinline__ int digit_width(int p) { return p == 2 ? 10 : 11; }

// the rank k = floor(q (n - 1)) and r - k of n finite values (FP64)
__device__ __forceinline__ uint32_t sel_rank(uint32_t n, double q, double& frac) {
    const double r = q * (double)(n - 1u);
    const double k = floor(r);
    frac = r - k;
    return (uint32_t)k;
}

// the quantile's value in FP64 from a finished state (NaN without finite values)
__device__ __forceinline__ double sel_value(const SelState& S, double q) {
    const uint32_t n = __ldcg(&S.n_fin);
    if (n == 0u) return __longlong_as_double(0x7ff8000000000000ll);
    double frac;
    const uint32_t k = sel_rank(n, q, frac);
    const double xk = (double)key_float(__ldcg(&S.key_k));
    double xk1 = xk;
    if (k + 1u < n && __ldcg(&S.c_le) < k + 2u) xk1 = (double)key_float(__ldcg(&S.m_gt));
    return xk + frac * (xk1 - xk);
}

// block-wide: the bin of rank `rank` in hist (kRadixBins counts) and the rank
// left within it; every thread gets them
__device__ void hist_find(const uint32_t* __restrict__ hist, uint32_t rank, uint32_t& bin,
                          uint32_t& rank_in) {
    __shared__ uint32_t s_bin, s_rank;
    if (threadIdx.x == 0) {
        s_bin = 0u;
        s_rank = 0u;
    }
    __syncthreads();
    constexpr int kPer = kRadixBins / kSelThreads;
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
    for (int b = threadIdx.x; b < kRadixBins; b += kSelThreads)
        if (sh[b]) atomicAdd(g + b, sh[b]);
}

// warp-aggregated shared-memory histogram increment
__device__ __forceinline__ void hist_add(uint32_t* sh, bool on, uint32_t bin) {
    const unsigned act = __ballot_sync(0xffffffffu, on);
    if (!on) return;
    const unsigned peers = __match_any_sync(act, bin);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(sh + bin, __popc(peers));
}

// the kSelUnroll elements of a warp-uniform step starting at b0 (NaN past n)
__device__ __forceinline__ void sel_load(const SelJob& jb, int32_t b0, int32_t stride_all,
                                         int lane, float (&d)[kSelUnroll]) {
#pragma unroll
    for (int u = 0; u < kSelUnroll; ++u) {
        const int32_t i = b0 + lane + u * stride_all;
        d[u] = i < jb.n ? __ldg(jb.x + (int64_t)i * jb.stride) : __int_as_float(0x7fc00000);
    }
}

// Pass 1: finite count, min / max keys, the first digit's histogram.
// hist: jobs x 3 x kRadixBins.
__global__ void __launch_bounds__(kSelThreads) k_sel_pass1(const __grid_constant__ SelJobs J,
                                                           SelState* __restrict__ st,
                                                           uint32_t* __restrict__ hist) {
    const SelJob& jb = J.j[blockIdx.y];
    __shared__ uint32_t sh[kRadixBins];
    __shared__ uint32_t s_n, s_lo, s_hi;
    const bool sel = jb.q >= 0.0;
    for (int b = threadIdx.x; b < kRadixBins; b += kSelThreads) sh[b] = 0u;
    if (threadIdx.x == 0) {
        s_n = 0u;
        s_lo = 0xffffffffu;
        s_hi = 0u;
    }
    __syncthreads();
    uint32_t cnt = 0u, lo = 0xffffffffu, hi = 0u;
    const int32_t all = gridDim.x * kSelThreads;
    // warp-uniform loop (the histogram step votes across the warp)
    for (int32_t b0 = (blockIdx.x * kSelThreads + threadIdx.x) & ~31; b0 < jb.n; b0 += kSelUnroll * all) {
        float d[kSelUnroll];
        sel_load(jb, b0, all, threadIdx.x & 31, d);
#pragma unroll
        for (int u = 0; u < kSelUnroll; ++u) {
            const bool fin = finite_f(d[u]);
            const uint32_t key = fin ? float_key(d[u]) : 0u;
            cnt += fin ? 1u : 0u;
            if (fin) {
                lo = min(lo, key);
                hi = max(hi, key);
            }
            if (sel) hist_add(sh, fin, key >> 21);
        }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_n, cnt);
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
    }
    __syncthreads();
    SelState& S = st[blockIdx.y];
    if (threadIdx.x == 0 && s_n) {
        atomicAdd(&S.n_fin, s_n);
        if (J.minmax) {
            atomicMin(&S.lo_key, s_lo);
            atomicMax(&S.hi_key, s_hi);
        }
    }
    if (sel) hist_merge(sh, hist + (size_t)blockIdx.y * 3 * kRadixBins);
}

// Pass 2 / 3 (P = 1, 2): fix digit P - 1 from its histogram (block 0 keeps
// the prefix for the next pass), then count digit P of the keys that match.
template <int P>
__global__ void __launch_bounds__(kSelThreads) k_sel_digit(const __grid_constant__ SelJobs J,
                                                           SelState* __restrict__ st,
                                                           uint32_t* __restrict__ hist) {
    const SelJob& jb = J.j[blockIdx.y];
    SelState& S = st[blockIdx.y];
    const uint32_t n = __ldcg(&S.n_fin);
    if (n == 0u || jb.q < 0.0) return;  // whole block: nothing to select
    uint32_t* H = hist + (size_t)blockIdx.y * 3 * kRadixBins;
    uint32_t rank, prefix;
    if (P == 1) {
        double frac;
        rank = sel_rank(n, jb.q, frac);
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
    for (int b = threadIdx.x; b < kRadixBins; b += kSelThreads) sh[b] = 0u;
    __syncthreads();
    const int hi_shift = digit_shift(P - 1);
    const int sh_p = digit_shift(P);
    const uint32_t dmask = (1u << digit_width(P)) - 1u;
    const int32_t all = gridDim.x * kSelThreads;
    for (int32_t b0 = (blockIdx.x * kSelThreads + threadIdx.x) & ~31; b0 < jb.n; b0 += kSelUnroll * all) {
        float d[kSelUnroll];
        sel_load(jb, b0, all, threadIdx.x & 31, d);
#pragma unroll
        for (int u = 0; u < kSelUnroll; ++u) {
            const bool fin = finite_f(d[u]);
            const uint32_t key = fin ? float_key(d[u]) : 0u;
            const bool match = fin && (key >> hi_shift) == (prefix >> hi_shift);
            hist_add(sh, match, (key >> sh_p) & dmask);
        }
    }
    __syncthreads();
    hist_merge(sh, H + P * kRadixBins);
}

// Pass 4: fix the last digit (s[k]'s key), then count the keys <= s[k] and
// take the smallest key > s[k].
__global__ void __launch_bounds__(kSelThreads) k_sel_final(const __grid_constant__ SelJobs J,
                                                           SelState* __restrict__ st,
                                                           const uint32_t* __restrict__ hist) {
    const SelJob& jb = J.j[blockIdx.y];
    SelState& S = st[blockIdx.y];
    if (__ldcg(&S.n_fin) == 0u || jb.q < 0.0) return;
    uint32_t bin, rin;
    hist_find(hist + (size_t)blockIdx.y * 3 * kRadixBins + 2 * kRadixBins, __ldcg(&S.rank2), bin, rin);
    const uint32_t key_k = __ldcg(&S.prefix2) | bin;
    if (blockIdx.x == 0 && threadIdx.x == 0) S.key_k = key_k;
    __shared__ uint32_t s_le, s_gt;
    if (threadIdx.x == 0) {
        s_le = 0u;
        s_gt = 0xffffffffu;
    }
    __syncthreads();
    uint32_t le = 0u, gt = 0xffffffffu;
    const int32_t all = gridDim.x * kSelThreads;
    for (int32_t b0 = (blockIdx.x * kSelThreads + threadIdx.x) & ~31; b0 < jb.n; b0 += kSelUnroll * all) {
        float d[kSelUnroll];
        sel_load(jb, b0, all, threadIdx.x & 31, d);
#pragma unroll
        for (int u = 0; u < kSelUnroll; ++u) {
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

// scratch of n_jobs states and histograms
inline size_t sel_state_bytes(int32_t n_jobs) {
    return ((size_t)n_jobs * sizeof(SelState) + 255) / 256 * 256;
}
inline size_t sel_scratch_bytes(int32_t n_jobs) {
    return sel_state_bytes(n_jobs) + (size_t)n_jobs * 3 * kRadixBins * 4;
}

// blocks per job: about 8 per SM over all jobs, at least kSelUnroll elements per thread
inline int sel_blocks(int64_t max_n, int32_t n_jobs, int32_t sm_count) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(
        (max_n + kSelThreads * kSelUnroll - 1) / (kSelThreads * kSelUnroll),
        (8 * (int64_t)sm_count + n_jobs - 1) / n_jobs));
}

// the passes of one selection round (scratch: sel_scratch_bytes(J.n) bytes);
// returns the first launch error
inline cudaError_t sel_launch(const SelJobs& J, void* scratch, int blocks, cudaStream_t s) {
    SelState* st = static_cast<SelState*>(scratch);
    uint32_t* hist = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(scratch) + sel_state_bytes(J.n));
    const int64_t hist_words = (int64_t)J.n * 3 * kRadixBins;
    bool any = false;
    for (int32_t k = 0; k < J.n; ++k) any = any || J.j[k].q >= 0.0;
    k_sel_init<<<(unsigned)((hist_words + kSelThreads - 1) / kSelThreads), kSelThreads, 0, s>>>(
        st, J.n, hist, hist_words);
    const dim3 grid(blocks, J.n);
    k_sel_pass1<<<grid, kSelThreads, 0, s>>>(J, st, hist);
    if (any) {
        k_sel_digit<1><<<grid, kSelThreads, 0, s>>>(J, st, hist);
        k_sel_digit<2><<<grid, kSelThreads, 0, s>>>(J, st, hist);
        k_sel_final<<<grid, kSelThreads, 0, s>>>(J, st, hist);
    }
    return cudaGetLastError();
}

}  // namespace
