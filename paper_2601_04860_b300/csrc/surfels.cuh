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
// no order); a surfel whose box in some view holds more than kSurfelSmallBox
// pixels (a large or elongated disc) is listed and counted by a whole block,
// its box's pixels spread over the threads.
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

// a surfel's footprint in one view: the centre, the projected tangent
// vectors, 1 / det, the 1-sigma pixel box (clipped to the frame)
struct SFoot {
    float cu, cv, a0x, a0y, a1x, a1y, inv;
    int x0, x1, y0, y1;
    bool any;  // a pixel can be accepted (in front, not edge-on, box non-empty)
};

// false when the centre or a tip is behind the camera (the view is skipped)
__device__ bool surfel_foot(const SView& V, const float (&m)[3], const float (&t0)[3],
                            const float (&t1)[3], float z_near, SFoot& F) {
    float X[3], u0p, v0p, u0m, v0m, u1p, v1p, u1m, v1m;
    F.any = false;
    bool ok = surf_front(V, m, z_near, F.cu, F.cv);
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
    F.a0x = __fmul_rn(0.5f, __fsub_rn(u0p, u0m));
    F.a0y = __fmul_rn(0.5f, __fsub_rn(v0p, v0m));
    F.a1x = __fmul_rn(0.5f, __fsub_rn(u1p, u1m));
    F.a1y = __fmul_rn(0.5f, __fsub_rn(v1p, v1m));
    const float det = __fsub_rn(__fmul_rn(F.a0x, F.a1y), __fmul_rn(F.a0y, F.a1x));
    if (det == 0.f) return true;  // edge-on: no pixel
    F.inv = __frcp_rn(det);
    const float ex = fmaxf(fabsf(F.a0x), fabsf(F.a1x)), ey = fmaxf(fabsf(F.a0y), fabsf(F.a1y));
    // pixel centres x + 1/2 inside [cu - ex, cu + ex], clipped to the frame
    F.x0 = (int)fmaxf(ceilf(__fsub_rn(__fsub_rn(F.cu, ex), 0.5f)), 0.f);
    F.x1 = (int)fminf(floorf(__fsub_rn(__fadd_rn(F.cu, ex), 0.5f)), (float)(V.W - 1));
    F.y0 = (int)fmaxf(ceilf(__fsub_rn(__fsub_rn(F.cv, ey), 0.5f)), 0.f);
    F.y1 = (int)fminf(floorf(__fsub_rn(__fadd_rn(F.cv, ey), 0.5f)), (float)(V.H - 1));
    F.any = F.x0 <= F.x1 && F.y0 <= F.y1;
    return true;
}

// the 3-sigma Cramer test and the mask at pixel (x, y): adds to (total, mask)
__device__ __forceinline__ void surfel_pixel(const SView& V, const SFoot& F, int x, int y,
                                             int32_t mask_type, float gate, uint32_t& total,
                                             uint32_t& msk) {
    const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), F.cu);
    const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), F.cv);
    const float uu = __fmul_rn(__fsub_rn(__fmul_rn(dx, F.a1y), __fmul_rn(dy, F.a1x)), F.inv);
    const float vv = __fmul_rn(__fsub_rn(__fmul_rn(F.a0x, dy), __fmul_rn(F.a0y, dx)), F.inv);
    if (__fadd_rn(__fmul_rn(uu, uu), __fmul_rn(vv, vv)) <= 9.f) {
        ++total;
        const int32_t q = y * V.W + x;
        const float mv = mask_type == kMaskF16
            ? __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(V.mask) + q)))
            : __ldg(reinterpret_cast<const float*>(V.mask) + q);
        msk += mv >= gate ? 1u : 0u;
    }
}

// the box's pixel count (64-bit)
__device__ __forceinline__ int64_t foot_area(const SFoot& F) {
    return F.any ? (int64_t)(F.x1 - F.x0 + 1) * (F.y1 - F.y0 + 1) : 0;
}

constexpr int64_t kSurfelSmallBox = 256;  // larger boxes go to the block-per-surfel pass
constexpr int kSurfBigThreads = 512;       // threads of a block of that pass

// a surfel's tangent semi-axes and centre
__device__ __forceinline__ void surfel_axes(const float* __restrict__ mu,
                                            const float* __restrict__ scales,
                                            const float* __restrict__ quats, int32_t i,
                                            float (&mm)[3], float (&t0)[3], float (&t1)[3]) {
    const float qw = __ldg(quats + 4 * (int64_t)i), qx = __ldg(quats + 4 * (int64_t)i + 1);
    const float qy = __ldg(quats + 4 * (int64_t)i + 2), qz = __ldg(quats + 4 * (int64_t)i + 3);
    const float rn = __frsqrt_rn(__fmaf_rn(qw, qw, __fmaf_rn(qx, qx, __fmaf_rn(qy, qy, __fmul_rn(qz, qz)))));
    const float w = __fmul_rn(qw, rn), x = __fmul_rn(qx, rn), y = __fmul_rn(qy, rn), z = __fmul_rn(qz, rn);
    const float s0 = __ldg(scales + 2 * (int64_t)i), s1 = __ldg(scales + 2 * (int64_t)i + 1);
    const float c0[3] = {__fsub_rn(1.f, __fmul_rn(2.f, __fmaf_rn(y, y, __fmul_rn(z, z)))),
                         __fmul_rn(2.f, __fmaf_rn(x, y, __fmul_rn(w, z))),
                         __fmul_rn(2.f, __fsub_rn(__fmul_rn(x, z), __fmul_rn(w, y)))};
    const float c1[3] = {__fmul_rn(2.f, __fsub_rn(__fmul_rn(x, y), __fmul_rn(w, z))),
                         __fsub_rn(1.f, __fmul_rn(2.f, __fmaf_rn(x, x, __fmul_rn(z, z)))),
                         __fmul_rn(2.f, __fmaf_rn(y, z, __fmul_rn(w, x)))};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        mm[q] = __ldg(mu + 3 * (int64_t)i + q);
        t0[q] = __fmul_rn(s0, c0[q]);
        t1[q] = __fmul_rn(s1, c1[q]);
    }
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

// Passes 1-3 per surfel: f (final), f2 (after the needle cull), kappa.  A
// surfel whose 1-sigma box in some scored view holds more than
// kSurfelSmallBox pixels is appended to `big` (with its view bits) and left
// to k_surfel_big.
__global__ void __launch_bounds__(kSurfThreads, 6) k_surfel_pass(
    const float* __restrict__ mu, const float* __restrict__ scales, const float* __restrict__ quats,
    const float* __restrict__ aspect, int32_t m, GridC G, const uint32_t* __restrict__ seg_bits,
    const uint32_t* __restrict__ active, const int32_t* __restrict__ d_n,
    const uint32_t* __restrict__ vbits, const SelState* __restrict__ st,
    const __grid_constant__ SViews SV, float tau_kappa, float z_near, uint8_t* __restrict__ f_out,
    uint8_t* __restrict__ f2_out, float* __restrict__ kappa_out, uint2* __restrict__ big,
    int32_t* __restrict__ n_big) {
    const float tau_a = (float)sel_value(st[0], 0.99);
    const int32_t n_act = *d_n;
    const float gate = SV.mask_type == kMaskLogit ? SV.logit_m : SV.tau_m;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int32_t idx[3];
        bool f2 = false, f = false, large = false;
        float kappa = 0.f;
        uint32_t vb = 0u;
        if (point_cell(mu, i, G, idx)) {
            const int64_t lin = ((int64_t)idx[2] * G.g + idx[1]) * G.g + idx[0];
            const bool f1 = (__ldg(seg_bits + (lin >> 5)) >> (lin & 31)) & 1u;
            f2 = f1 && __ldg(aspect + i) <= tau_a;
            const uint32_t pk = (uint32_t)idx[0] | ((uint32_t)idx[1] << 10) | ((uint32_t)idx[2] << 20);
            const int32_t ai = f2 ? active_find(active, n_act, pk) : -1;
            vb = ai >= 0 ? __ldg(vbits + ai) : 0u;
            if (vb) {
                float mm[3], t0[3], t1[3];
                surfel_axes(mu, scales, quats, i, mm, t0, t1);
                for (int32_t s = 0; s < SV.n && !large; ++s) {
                    if (!((vb >> s) & 1u)) continue;
                    SFoot F;
                    if (!surfel_foot(SV.v[s], mm, t0, t1, z_near, F)) continue;
                    if (foot_area(F) > kSurfelSmallBox) {
                        large = true;
                        break;
                    }
                    uint32_t tot = 0u, msk = 0u;
                    if (F.any)
                        for (int y = F.y0; y <= F.y1; ++y)
                            for (int x = F.x0; x <= F.x1; ++x)
                                surfel_pixel(SV.v[s], F, x, y, SV.mask_type, gate, tot, msk);
                    const uint32_t den = max(tot, 1u);
                    kappa = fmaxf(kappa, __fdiv_rn((float)msk, (float)den));
                    f = f || (double)msk >= (double)tau_kappa * (double)den;
                }
            }
        }
        if (f2_out) f2_out[i] = (uint8_t)f2;
        if (large) {
            big[atomicAdd(n_big, 1)] = make_uint2((uint32_t)i, vb);  // at most m entries
            continue;
        }
        f_out[i] = (uint8_t)(f2 && f);
        if (kappa_out) kappa_out[i] = kappa;
    }
}

// A box larger than kSliceArea pixels is cut into slices of whole rows (about
// kSliceArea pixels each): the block that meets it takes the first slice and
// queues the others for k_surfel_slices, their counts meeting in a split slot
// whose last slice (remaining -> 0) decides the view.  When the queue or the
// slots are full, the block takes the whole box itself.
constexpr int64_t kSliceArea = 16384;
constexpr int32_t kSplitCap = 1 << 16;  // split slots per call
constexpr int32_t kSliceCap = 1 << 20;  // queued slices per call

struct SplitSlot {
    int32_t e, s;        // listed surfel, view
    uint32_t tot, msk;   // counts of the slices done
    int32_t remaining;   // slices not yet counted
    int32_t pad;
};

struct SliceQueue {
    SplitSlot* slots;
    int32_t* n_slots;
    uint2* slices;       // (slot, slice index)
    int32_t* n_slices;
};

// rows per slice of a box of the given width
__device__ __forceinline__ int32_t slice_rows(const SFoot& F) {
    const int64_t w = (int64_t)(F.x1 - F.x0 + 1);
    const int64_t r = kSliceArea / w;
    return (int32_t)(r < 1 ? 1 : r);
}

// the view's fraction for listed surfel e into its accumulator (kappa: the
// largest fraction, as non-negative float bits; y: some view reached tau_kappa)
__device__ __forceinline__ void surfel_view_done(uint2* __restrict__ acc, int32_t e, uint32_t tot,
                                                 uint32_t msk, float tau_kappa) {
    const uint32_t den = max(tot, 1u);
    atomicMax(&acc[e].x, __float_as_uint(__fdiv_rn((float)msk, (float)den)));
    if ((double)msk >= (double)tau_kappa * (double)den) atomicOr(&acc[e].y, 1u);
}

// the box rows [ya, yb] of footprint F over the block (warps take rows, lanes
// columns: consecutive mask words); the block's counts in (s_tot, s_msk)
__device__ __forceinline__ void surfel_rows(const SView& V, const SFoot& F, int ya, int yb,
                                            int32_t mask_type, float gate, uint32_t* s_tot,
                                            uint32_t* s_msk) {
    uint32_t tot = 0u, msk = 0u;
    const int nwarps = (int)(blockDim.x >> 5), lane = (int)(threadIdx.x & 31);
    for (int y = ya + (int)(threadIdx.x >> 5); y <= yb; y += nwarps)
        for (int x = F.x0 + lane; x <= F.x1; x += 32)
            surfel_pixel(V, F, x, y, mask_type, gate, tot, msk);
    tot = __reduce_add_sync(0xffffffffu, tot);
    msk = __reduce_add_sync(0xffffffffu, msk);
    if (lane == 0) {
        atomicAdd(s_tot, tot);
        atomicAdd(s_msk, msk);
    }
}

// a split slot's counts after one slice: the slice that finishes the box
// decides the view
__device__ __forceinline__ void slice_done(SplitSlot* slot, uint32_t tot, uint32_t msk,
                                           uint2* __restrict__ acc, float tau_kappa) {
    atomicAdd(&slot->tot, tot);
    atomicAdd(&slot->msk, msk);
    __threadfence();
    if (atomicSub(&slot->remaining, 1) == 1) {
        __threadfence();
        const uint32_t t = atomicAdd(&slot->tot, 0u), m = atomicAdd(&slot->msk, 0u);
        surfel_view_done(acc, slot->e, t, m, tau_kappa);
    }
}

// The listed surfels: one block per (listed surfel, view) (blockIdx.y =
// view); the footprint (one thread), then the box's pixels spread over the
// block and the counts reduced (a box above kSliceArea pixels: its first
// slice, the others queued); per surfel, the largest fraction (atomicMax on
// its non-negative bits) and whether some view reached tau_kappa (atomicOr)
// go to acc (zeroed).
__global__ void __launch_bounds__(kSurfBigThreads) k_surfel_big(
    const float* __restrict__ mu, const float* __restrict__ scales, const float* __restrict__ quats,
    const uint2* __restrict__ big, const int32_t* __restrict__ n_big,
    const __grid_constant__ SViews SV, float tau_kappa, float z_near, uint2* __restrict__ acc,
    SliceQueue Q) {
    __shared__ SFoot sF;
    __shared__ bool s_ok;
    __shared__ int32_t s_slot, s_rows;
    __shared__ uint32_t s_tot, s_msk;
    const float gate = SV.mask_type == kMaskLogit ? SV.logit_m : SV.tau_m;
    const int32_t nb = *n_big;
    const int32_t s = blockIdx.y;
    for (int32_t e = blockIdx.x; e < nb; e += gridDim.x) {
        const uint2 it = big[e];
        if (!((it.y >> s) & 1u)) continue;  // block-uniform
        const int32_t i = (int32_t)it.x;
        if (threadIdx.x == 0) {
            float mm[3], t0[3], t1[3];
            surfel_axes(mu, scales, quats, i, mm, t0, t1);
            s_ok = surfel_foot(SV.v[s], mm, t0, t1, z_near, sF);
            s_tot = 0u;
            s_msk = 0u;
            s_slot = -1;
            s_rows = sF.y1 - sF.y0 + 1;
            if (s_ok && sF.any && foot_area(sF) > kSliceArea) {
                // queue slices 1 .. S - 1; slice 0 is this block's
                const int32_t R = slice_rows(sF);
                const int32_t S = (sF.y1 - sF.y0 + R) / R;
                const int32_t slot = atomicAdd(Q.n_slots, 1);
                const int32_t first = slot < kSplitCap ? atomicAdd(Q.n_slices, S - 1) : kSliceCap;
                if (slot < kSplitCap && first + (S - 1) <= kSliceCap) {
                    Q.slots[slot] = SplitSlot{e, s, 0u, 0u, S, 0};
                    for (int32_t k = 1; k < S; ++k) Q.slices[first + k - 1] = make_uint2((uint32_t)slot, (uint32_t)k);
                    s_slot = slot;
                    s_rows = R;
                } else {
                    // no room: the whole box here; the part of the reservation
                    // inside the queue is marked empty
                    for (int32_t k = first; k < kSliceCap && k < first + (S - 1); ++k)
                        Q.slices[k] = make_uint2(0xffffffffu, 0u);
                }
            }
        }
        __syncthreads();
        if (s_ok && sF.any)
            surfel_rows(SV.v[s], sF, sF.y0, min(sF.y1, sF.y0 + s_rows - 1), SV.mask_type, gate,
                        &s_tot, &s_msk);
        __syncthreads();
        if (threadIdx.x == 0 && s_ok) {
            if (s_slot >= 0) {
                __threadfence();  // the slot's fields before the slices' counts
                slice_done(Q.slots + s_slot, s_tot, s_msk, acc, tau_kappa);
            } else {
                surfel_view_done(acc, e, s_tot, s_msk, tau_kappa);
            }
        }
        __syncthreads();
    }
}

// the queued slices of the split boxes, one at a time per block
__global__ void __launch_bounds__(kSurfBigThreads) k_surfel_slices(
    const float* __restrict__ mu, const float* __restrict__ scales, const float* __restrict__ quats,
    const uint2* __restrict__ big, const __grid_constant__ SViews SV, float tau_kappa,
    float z_near, uint2* __restrict__ acc, SliceQueue Q) {
    __shared__ SFoot sF;
    __shared__ uint32_t s_tot, s_msk;
    const float gate = SV.mask_type == kMaskLogit ? SV.logit_m : SV.tau_m;
    const int32_t n = min(*Q.n_slices, kSliceCap);
    for (int32_t q = blockIdx.x; q < n; q += gridDim.x) {
        const uint2 sl = Q.slices[q];
        if (sl.x >= (uint32_t)kSplitCap) continue;  // an empty entry (block-uniform)
        SplitSlot* slot = Q.slots + sl.x;
        const int32_t e = slot->e, s = slot->s;
        if (threadIdx.x == 0) {
            float mm[3], t0[3], t1[3];
            surfel_axes(mu, scales, quats, (int32_t)big[e].x, mm, t0, t1);
            surfel_foot(SV.v[s], mm, t0, t1, z_near, sF);  // as when the box was split
            s_tot = 0u;
            s_msk = 0u;
        }
        __syncthreads();
        const int32_t R = slice_rows(sF);
        const int ya = sF.y0 + (int)sl.y * R;
        surfel_rows(SV.v[s], sF, ya, min(sF.y1, ya + R - 1), SV.mask_type, gate, &s_tot, &s_msk);
        __syncthreads();
        if (threadIdx.x == 0) slice_done(slot, s_tot, s_msk, acc, tau_kappa);
        __syncthreads();
    }
}

// the listed surfels' outputs from their accumulators
__global__ void __launch_bounds__(kSurfThreads) k_surfel_big_out(
    const uint2* __restrict__ big, const int32_t* __restrict__ n_big, const uint2* __restrict__ acc,
    uint8_t* __restrict__ f_out, float* __restrict__ kappa_out) {
    const int32_t nb = *n_big;
    for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)big[e].x;
        f_out[i] = (uint8_t)(acc[e].y != 0u);  // listed surfels passed Pass 2
        if (kappa_out) kappa_out[i] = __uint_as_float(acc[e].x);
    }
}

// The back-projected overlay of a view (Sec. 3.7 "Iterative Mask
// Propagation"): each pixel centre unprojected at its planar depth,
// x = R^T (((u + 1/2 - cx) / fx) d, ((v + 1/2 - cy) / fy) d, d) - R^T t, and
// the seg bit of the cell holding x (0 for no surface or outside the grid).
// The point is formed in FP32; where its cell coordinate (q - origin) / h (q
// = x, or contract(x)) lies within the FP32 rounding bound of an integer, the
// pixel is evaluated again in FP64 with the operations of the FP64
// definition, so that the cell agrees with it away from 1e-6 (relative) of a
// boundary.
struct OverlayView {
    float R[9], t[3];
    float fx, fy, cx, cy;
    int32_t W, H;
};

// the cell of pixel (x, y) at depth d in FP64; false outside the grid
__device__ __noinline__ bool overlay_cell64(const OverlayView& V, const GridC& G, int x, int y,
                                            float d, int32_t (&idx)[3]) {
    const double dd = (double)d;
    const double pc[3] = {
        __dmul_rn(__ddiv_rn(__dsub_rn(__dadd_rn((double)x, 0.5), (double)V.cx), (double)V.fx), dd),
        __dmul_rn(__ddiv_rn(__dsub_rn(__dadd_rn((double)y, 0.5), (double)V.cy), (double)V.fy), dd),
        dd};
    double X[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        X[r] = __dadd_rn(__dadd_rn(__dmul_rn(__dsub_rn(pc[0], (double)V.t[0]), (double)V.R[r]),
                                   __dmul_rn(__dsub_rn(pc[1], (double)V.t[1]), (double)V.R[3 + r])),
                         __dmul_rn(__dsub_rn(pc[2], (double)V.t[2]), (double)V.R[6 + r]));
    if (G.contracted) {  // contract(x) = (2 - 1/|x|) x / |x| beyond the unit ball
        const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(X[0], X[0]), __dmul_rn(X[1], X[1])),
                                              __dmul_rn(X[2], X[2])));
        if (r > 1.0) {
            const double sc = __ddiv_rn(__dsub_rn(2.0, __ddiv_rn(1.0, r)), r);
#pragma unroll
            for (int q = 0; q < 3; ++q) X[q] = __dmul_rn(X[q], sc);
        }
    }
    bool inside = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double s = __ddiv_rn(__dsub_rn(X[q], (double)G.origin[q]), (double)G.h);
        inside = inside && s >= 0.0 && s < (double)G.g;
        idx[q] = inside ? (int32_t)floor(s) : 0;
    }
    return inside;
}

__global__ void __launch_bounds__(kSurfThreads) k_overlay(OverlayView V, const float* __restrict__ depth,
                                                          GridC G, const uint32_t* __restrict__ seg_bits,
                                                          uint8_t* __restrict__ out) {
    const int32_t npix = V.W * V.H;
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < npix; q += gridDim.x * blockDim.x) {
        const float d = __ldg(depth + q);
        uint8_t lab = 0;
        if (d > 0.f && d <= FLT_MAX) {
            const int x = q % V.W, y = q / V.W;
            const float pc[3] = {
                __fsub_rn(__fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn((float)x, 0.5f), V.cx), V.fx), d), V.t[0]),
                __fsub_rn(__fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn((float)y, 0.5f), V.cy), V.fy), d), V.t[1]),
                __fsub_rn(d, V.t[2])};
            float X[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)  // world = R^T (p_c - t)
                X[r] = __fmaf_rn(V.R[r], pc[0], __fmaf_rn(V.R[3 + r], pc[1], __fmul_rn(V.R[6 + r], pc[2])));
            // the cell coordinate in FP32 and its distance to the nearest integer
            float Q[3] = {X[0], X[1], X[2]};
            float mag = fabsf(pc[0]) + fabsf(pc[1]) + fabsf(pc[2]) + fabsf(V.t[0]) +
                        fabsf(V.t[1]) + fabsf(V.t[2]);
            if (G.contracted) {
                const float r = __fsqrt_rn(__fmaf_rn(X[0], X[0], __fmaf_rn(X[1], X[1], __fmul_rn(X[2], X[2]))));
                if (r > 1.f) {
                    const float sc = __fdiv_rn(__fsub_rn(2.f, __frcp_rn(r)), r);
#pragma unroll
                    for (int k = 0; k < 3; ++k) Q[k] = __fmul_rn(X[k], sc);
                }
            }
            bool near = false;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float sk = __fdiv_rn(__fsub_rn(Q[k], G.origin[k]), G.h);
                const float band = __fmul_rn(0x1p-15f, __fadd_rn(__fdiv_rn(mag, G.h), fabsf(sk)));
                near = near || fabsf(__fsub_rn(sk, rintf(sk))) <= band;
            }
            int32_t idx[3];
            const bool in = near ? overlay_cell64(V, G, x, y, d, idx) : point_cell(X, 0, G, idx);
            if (in) {
                const int64_t lin = ((int64_t)idx[2] * G.g + idx[1]) * G.g + idx[0];
                lab = (uint8_t)((__ldg(seg_bits + (lin >> 5)) >> (lin & 31)) & 1u);
            }
        }
        out[q] = lab;
    }
}

}  // namespace

extern "C" {

divas_status divas_overlay(divas_ctx* c, const divas_camera* cam, const float* depth, uint8_t* out,
                           void* stream) {
    if (!c) return fail(nullptr, DIVAS_E_INVALID, "ctx is NULL");
    if (!cam || !depth || !out) return fail(c, DIVAS_E_INVALID, "camera, depth and out are required");
    divas_status st = check_camera(c, cam);
    if (st != DIVAS_OK) return st;
    OverlayView V;
    memcpy(V.R, cam->R, sizeof(V.R));
    memcpy(V.t, cam->t, sizeof(V.t));
    V.fx = cam->fx;
    V.fy = cam->fy;
    V.cx = cam->cx;
    V.cy = cam->cy;
    V.W = cam->W;
    V.H = cam->H;
    const int64_t npix = (int64_t)cam->W * cam->H;
    k_overlay<<<(int)std::min<int64_t>((npix + kSurfThreads - 1) / kSurfThreads, 16 * (int64_t)c->sm_count),
                kSurfThreads, 0, S(stream)>>>(V, depth, c->G, c->seg_bits, out);
    DIVAS_LAUNCHED(c, "k_overlay");
    return DIVAS_OK;
}

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
    // scratch (the weighting's): aspects, the large-footprint list and its
    // count, then one selection job
    const int32_t n = (int32_t)m;
    const size_t arr = ((size_t)n * 4 + 255) / 256 * 256;
    const size_t lst = ((size_t)n * 16 + 256 + 255) / 256 * 256;  // list + accumulators
    const size_t spl = (size_t)kSplitCap * sizeof(SplitSlot) + (size_t)kSliceCap * sizeof(uint2) + 256;
    const size_t need = arr + lst + spl + sel_scratch_bytes(1);
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
    int32_t* n_big = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(c->wt) + arr);
    uint2* big = reinterpret_cast<uint2*>(static_cast<unsigned char*>(c->wt) + arr + 256);
    uint2* acc = big + n;
    unsigned char* sp = static_cast<unsigned char*>(c->wt) + arr + lst;
    SliceQueue Q;
    Q.n_slots = reinterpret_cast<int32_t*>(sp);
    Q.n_slices = reinterpret_cast<int32_t*>(sp) + 1;
    Q.slots = reinterpret_cast<SplitSlot*>(sp + 256);
    Q.slices = reinterpret_cast<uint2*>(sp + 256 + (size_t)kSplitCap * sizeof(SplitSlot));
    void* sel = static_cast<unsigned char*>(c->wt) + arr + lst + spl;
    DIVAS_CUDA(c, cudaMemsetAsync(n_big, 0, sizeof(int32_t), s));
    DIVAS_CUDA(c, cudaMemsetAsync(sp, 0, 2 * sizeof(int32_t), s));
    DIVAS_CUDA(c, cudaMemsetAsync(acc, 0, (size_t)n * sizeof(uint2), s));
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
                                                  c->F.z_near, f_out, f2_out, kappa_out, big,
                                                  n_big);
    DIVAS_LAUNCHED(c, "k_surfel_pass");
    if (n_views > 0) {
        k_surfel_big<<<dim3(std::max(1, 4 * c->sm_count / n_views), n_views), kSurfBigThreads, 0, s>>>(
            mu, scales, quats, big, n_big, SV, p->tau_kappa, c->F.z_near, acc, Q);
        DIVAS_LAUNCHED(c, "k_surfel_big");
        k_surfel_slices<<<4 * c->sm_count, kSurfBigThreads, 0, s>>>(mu, scales, quats, big, SV,
                                                                   p->tau_kappa, c->F.z_near,
                                                                   acc, Q);
        DIVAS_LAUNCHED(c, "k_surfel_slices");
        k_surfel_big_out<<<c->sm_count, kSurfThreads, 0, s>>>(big, n_big, acc, f_out, kappa_out);
        DIVAS_LAUNCHED(c, "k_surfel_big_out");
    }
    return DIVAS_OK;
}

}  // extern "C"
