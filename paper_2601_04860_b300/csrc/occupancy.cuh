// occupancy.cuh -- the 2DGS occupancy construction (Sec. 3.5 "Occupancy by
// Morton-scattered opacity"; Appendix "Occupancy grid construction"; Eqs.
// scene-norm and voxel-size), included by divas_fuse.cu.
//
// divas_scene_frame_from_gaussians: each surfel's larger scale, then one
// selection launch set (select.cuh) for the three coordinate medians of the
// centres and the median larger scale, the radial distances |mu - c| (FP64,
// stored as FP32) and a second selection for their 99th percentile; the host
// then applies the frame rules in FP64: b = max(ceil(1.05 r_fg), 1),
// h = max(alpha_v s_bar, beta_v r_fg / g0), g = the smallest power of two
// >= 2 b / h capped at g_max (h raised to 2 b / g_max when the cap binds).
// divas_occupancy_from_gaussians: the opacity scatter-add into a dense FP32
// density grid (cube test and voxel index in FP64, FP32 atomics; the
// paper's Morton layout is a memory order of the same set, the grid here is
// linear, x fastest), then the tau_TF floor into the fusion's uint8 prior.
#pragma once

#include "select.cuh"

namespace {

constexpr int kOccThreads = 256;

// the larger of each surfel's two scales (NaN if either is NaN)
__global__ void __launch_bounds__(kOccThreads) k_gauss_smax(const float* __restrict__ s, int32_t m,
                                                            float* __restrict__ smax) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const float a = __ldg(s + 2 * (int64_t)i), b = __ldg(s + 2 * (int64_t)i + 1);
        smax[i] = (a != a || b != b) ? __int_as_float(0x7fc00000) : fmaxf(a, b);
    }
}

// |mu_i - c| in FP64 ((dx dx + dy dy) + dz dz), stored as FP32; c = the
// coordinate medians of the first selection round (states 0..2)
__global__ void __launch_bounds__(kOccThreads) k_gauss_dist(const float* __restrict__ mu, int32_t m,
                                                            const SelState* __restrict__ st,
                                                            float* __restrict__ dist) {
    __shared__ double c[3];
    if (threadIdx.x < 3) c[threadIdx.x] = sel_value(st[threadIdx.x], 0.5);
    __syncthreads();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double dx = __dsub_rn((double)__ldg(mu + 3 * (int64_t)i), c[0]);
        const double dy = __dsub_rn((double)__ldg(mu + 3 * (int64_t)i + 1), c[1]);
        const double dz = __dsub_rn((double)__ldg(mu + 3 * (int64_t)i + 2), c[2]);
        dist[i] = (float)__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                              __dmul_rn(dz, dz)));
    }
}

// the frame's selected values: c[0..2] and s_bar (first selection), r_fg (second)
__global__ void k_gauss_frame(const SelState* __restrict__ st1, const SelState* __restrict__ st2,
                              double* __restrict__ out) {
    const int t = threadIdx.x;
    if (t < 4) out[t] = sel_value(st1[t], 0.5);
    if (t == 4) out[4] = sel_value(st2[0], 0.99);
}

struct OccFrame {
    double c[3];
    double b, h;
    int32_t g;
    int32_t pad;
};

// opacity scatter-add of the surfels inside the half-open cube c +- b
__global__ void __launch_bounds__(kOccThreads) k_gauss_scatter(const float* __restrict__ mu,
                                                               const float* __restrict__ alpha,
                                                               int32_t m, OccFrame f,
                                                               float* __restrict__ rho) {
    const double two_b = __dmul_rn(2.0, f.b);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int32_t idx[3];
        bool in = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = __dadd_rn(__dsub_rn((double)__ldg(mu + 3 * (int64_t)i + a), f.c[a]), f.b);
            in = in && x >= 0.0 && x < two_b;
            idx[a] = in ? min((int32_t)floor(__ddiv_rn(x, f.h)), f.g - 1) : 0;
        }
        if (!in) continue;
        const int64_t lin = ((int64_t)idx[2] * f.g + idx[1]) * f.g + idx[0];
        atomicAdd(rho + lin, __ldg(alpha + i));
    }
}

// occ = rho >= tau (1 / 0)
__global__ void __launch_bounds__(kOccThreads) k_density_floor(const float* __restrict__ rho, int64_t n,
                                                               float tau, uint8_t* __restrict__ occ) {
    const int64_t n4 = n / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(rho) + q);
        const uint32_t w = (v.x >= tau ? 1u : 0u) | (v.y >= tau ? 1u << 8 : 0u) |
                           (v.z >= tau ? 1u << 16 : 0u) | (v.w >= tau ? 1u << 24 : 0u);
        reinterpret_cast<uint32_t*>(occ)[q] = w;
    }
    for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        occ[i] = rho[i] >= tau ? 1 : 0;
}

}  // namespace

extern "C" {

divas_occupancy_params divas_default_occupancy_params(void) {
    divas_occupancy_params p;
    p.alpha_v = 3.0;
    p.beta_v = 1.0;
    p.pad = 1.05;
    p.g0 = 256;
    p.g_max = 512;
    p.tau_tf = 0.5f;
    p.reserved = 0;
    return p;
}

divas_status divas_scene_frame_from_gaussians(const float* mu, const float* scales, int64_t m,
                                              const divas_occupancy_params* p,
                                              divas_scene_frame* out, void* stream) {
    if (!mu || !scales || !p || !out || m < 1 || m > INT32_MAX / 3) return DIVAS_E_INVALID;
    if (!(p->alpha_v >= 0.0) || !(p->beta_v >= 0.0) || p->g0 < 1 || p->g_max < 1 ||
        p->g_max > 2048 || (p->g_max & (p->g_max - 1)) != 0 || !(p->pad > 0.0))
        return DIVAS_E_INVALID;
    const cudaStream_t s = S(stream);
    const int32_t n = (int32_t)m;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // scratch: smax, dist (n floats each), two selection rounds, 5 doubles
    const size_t arr = ((size_t)n * 4 + 255) / 256 * 256;
    const size_t sel1 = sel_scratch_bytes(4), sel2 = sel_scratch_bytes(1);
    unsigned char* scr = nullptr;
    if (cudaMalloc(&scr, 2 * arr + sel1 + sel2 + 256) != cudaSuccess) {
        (void)cudaGetLastError();
        return DIVAS_E_CUDA;
    }
    float* smax = reinterpret_cast<float*>(scr);
    float* dist = reinterpret_cast<float*>(scr + arr);
    void* s1 = scr + 2 * arr;
    void* s2 = scr + 2 * arr + sel1;
    double* vals = reinterpret_cast<double*>(scr + 2 * arr + sel1 + sel2);
    const int blocks = (int)std::min<int64_t>((n + kOccThreads - 1) / kOccThreads, 8 * (int64_t)sms);
    k_gauss_smax<<<blocks, kOccThreads, 0, s>>>(scales, n, smax);
    SelJobs J1;
    memset(&J1, 0, sizeof(J1));
    J1.n = 4;
    for (int a = 0; a < 3; ++a) J1.j[a] = {mu + a, n, 3, 0.5};
    J1.j[3] = {smax, n, 1, 0.5};
    cudaError_t e = sel_launch(J1, s1, sel_blocks(n, 4, sms), s);
    if (e == cudaSuccess) {
        k_gauss_dist<<<blocks, kOccThreads, 0, s>>>(mu, n, static_cast<const SelState*>(s1), dist);
        SelJobs J2;
        memset(&J2, 0, sizeof(J2));
        J2.n = 1;
        J2.j[0] = {dist, n, 1, 0.99};
        e = sel_launch(J2, s2, sel_blocks(n, 1, sms), s);
    }
    double v[5] = {0, 0, 0, 0, 0};
    if (e == cudaSuccess) {
        k_gauss_frame<<<1, 32, 0, s>>>(static_cast<const SelState*>(s1), static_cast<const SelState*>(s2),
                                       vals);
        e = cudaMemcpyAsync(v, vals, sizeof(v), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scr);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return DIVAS_E_CUDA;
    }
    // the frame rules (FP64, as written in Eqs. scene-norm and voxel-size)
    memset(out, 0, sizeof(*out));
    for (int a = 0; a < 3; ++a) out->c[a] = v[a];
    out->s_bar = v[3];
    out->r_fg = v[4];
    if (!(std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]) && std::isfinite(v[3]) &&
          std::isfinite(v[4])))
        return DIVAS_E_INVALID;  // no finite centres or scales
    out->b = std::max(std::ceil(p->pad * v[4]), 1.0);
    double h = std::max(p->alpha_v * v[3], p->beta_v * v[4] / (double)p->g0);
    if (!(h > 0.0)) return DIVAS_E_INVALID;  // zero scales and radius: no voxel edge
    const double need = 2.0 * out->b / h;
    int32_t g = 1;
    while (g < need && g < p->g_max) g *= 2;
    if (need > p->g_max) {
        g = p->g_max;
        h = 2.0 * out->b / p->g_max;
    }
    out->h = h;
    out->g = g;
    for (int a = 0; a < 3; ++a) out->origin[a] = out->c[a] - out->b;
    return DIVAS_OK;
}

divas_status divas_occupancy_from_gaussians(const float* mu, const float* alpha, int64_t m,
                                            const divas_scene_frame* f, float tau_tf,
                                            float* density, uint8_t* occ_out, void* stream) {
    if (!mu || !alpha || !f || !density || !occ_out || m < 0 || m > INT32_MAX / 3)
        return DIVAS_E_INVALID;
    if (f->g < 1 || f->g > 2048 || !(f->h > 0.0) || !(f->b > 0.0) || tau_tf != tau_tf)
        return DIVAS_E_INVALID;
    if (reinterpret_cast<uintptr_t>(density) % 16 != 0 || reinterpret_cast<uintptr_t>(occ_out) % 4 != 0)
        return DIVAS_E_INVALID;  // the floor pass reads 16-byte words and writes 4-byte words
    const cudaStream_t s = S(stream);
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cells = (int64_t)f->g * f->g * f->g;
    if (cudaMemsetAsync(density, 0, (size_t)cells * 4, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return DIVAS_E_CUDA;
    }
    OccFrame F;
    memset(&F, 0, sizeof(F));
    for (int a = 0; a < 3; ++a) F.c[a] = f->c[a];
    F.b = f->b;
    F.h = f->h;
    F.g = f->g;
    if (m > 0)
        k_gauss_scatter<<<(int)std::min<int64_t>((m + kOccThreads - 1) / kOccThreads, 16 * (int64_t)sms),
                          kOccThreads, 0, s>>>(mu, alpha, (int32_t)m, F, density);
    k_density_floor<<<(int)std::min<int64_t>((cells / 4 + kOccThreads - 1) / kOccThreads + 1, 16 * (int64_t)sms),
                      kOccThreads, 0, s>>>(density, cells, tau_tf, occ_out);
    return cudaGetLastError() == cudaSuccess ? DIVAS_OK : DIVAS_E_CUDA;
}

}  // extern "C"
