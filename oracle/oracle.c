/*
 * oracle.c -- plain, slow, double-precision CPU reference of depth-weighted
 * multi-view voxel fusion (DivAS, arXiv 2601.04860).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, loads or calls
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * What it computes, per voxel v of the occupied set (Sec. 3.5 "Shared
 * voxel-voting concept"; Algorithm "Thick-Structure Segmentation for 2DGS"
 * in Appendix B.5; Algorithm "Thick-Structure Segmentation via
 * Depth-Weighted Voxel Aggregation" in Appendix A.2):
 *
 *   W = Z = 0, bits = 0
 *   for each view i in index order:
 *     p = R_i x_v + t_i                       (world -> camera)
 *     skip unless p_z > z_near
 *     u = fx p_x / p_z + cx,  v = fy p_y / p_z + cy          (pi_i, Sec. A.2)
 *     skip unless 0 <= u < W and 0 <= v < H  ("out-of-frame voxels skip view i")
 *     D = depth_i[floor v][floor u],  m = mask_i[floor v][floor u]
 *     skip unless D finite and D > 0          (no rendered surface)
 *     skip unless m >= tau_m                  (thick-path entry, m >= 0.5)
 *     Delta = gamma h_v,  e = p_z - D         (depth tolerance t_depth, Eq. tightening
 *                                             with eta = 1; planar/ray factors cancel)
 *     skip unless |e| <= Delta                (symmetric branch of Eq. asym-gate)
 *     w = exp(-alpha1 (e / Delta)^2)          (Eq. gs-depthweight with the band
 *                                             [D - Delta, D + Delta])
 *     W += m w,  Z += w,  bits |= 1 << i      (Eq. vmask)
 *   P = W / Z if Z > eps else 0               (Eq. compact-fusion, thick terms)
 *   seg = P >= tau_cons;  vmask = seg ? bits : 0
 *
 * and labels a point x by the segmentation bit of the voxel that contains
 * it (Eq. pass1), 0 outside the grid, for NaN, or for an unoccupied voxel.
 * For a contracted grid (unbounded scenes, Sec. A.2 "mapped through scene
 * contraction") voxel centres are uncontracted before projection and points
 * are contracted before lookup.
 *
 * Next to every decision it records how close the decision was to flipping
 * (relative margin below ORACLE_MARGIN sets a per-voxel / per-point flag):
 * such items are excluded from exact comparisons against FP32 code.
 *
 * parity: pinned by the closed-form, invariant and brute-force tests of the
 * test suite (single view, alpha1 = 0 mean, view-order invariance, analytic
 * scenes, independent NumPy re-implementation with analytic depth, central
 * finite differences for the adjoint).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MARGIN 1e-6

enum {
    FLAG_PIX = 1,      /* pixel index / in-frame decision near an integer */
    FLAG_DEPTH = 2,    /* |e| near Delta */
    FLAG_ZNEAR = 4,    /* p_z near z_near */
    FLAG_CONS = 8,     /* P near tau_cons */
    FLAG_CONTRACT = 16 /* |c| near the contraction's branch radius 1 */
};

enum { MASK_F32 = 0, MASK_F16 = 1, MASK_LOGIT_F32 = 2 };

typedef struct {
    double tau_m, gamma, alpha1, tau_cons, eps, z_near;
    double logit_tau; /* gate threshold for logit masks, lhs >= logit_tau */
} oracle_params;

/* One view: camera as float32 values (widened exactly), rasters as given. */
typedef struct {
    float R[9], t[3], fx, fy, cx, cy;
    int32_t W, H;
    const float* depth;
    const void* mask;
} oracle_view;

/* Exact value of an IEEE binary16 bit pattern. */
static double half_to_double(uint16_t b) {
    int sign = (b >> 15) & 1;
    int e = (b >> 10) & 0x1f;
    int m = b & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);
    else if (e == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp((double)(m | 0x400), e - 25);
    return sign ? -v : v;
}

/* Mask value at pixel p: probability m, and the quantity the gate compares. */
static void mask_at(const oracle_view* vw, int mask_type, int64_t p, const oracle_params* pr,
                    double* m, int* pass) {
    if (mask_type == MASK_F16) {
        *m = half_to_double(((const uint16_t*)vw->mask)[p]);
        *pass = *m >= pr->tau_m;
    } else if (mask_type == MASK_LOGIT_F32) {
        double l = ((const float*)vw->mask)[p];
        *m = 1.0 / (1.0 + exp(-l));
        *pass = l >= pr->logit_tau;
    } else {
        *m = ((const float*)vw->mask)[p];
        *pass = *m >= pr->tau_m;
    }
}

static double dist_to_int(double a) {
    double f = a - floor(a);
    return f < 1.0 - f ? f : 1.0 - f;
}

/*
 * Voxel centre in world space and its world edge h_v.
 * Plain grid: x = origin + (idx + 1/2) h.  Contracted grid: c = that point in
 * contracted space; x = c for |c| <= 1, c / (|c| (2 - |c|)) for 1 < |c| < 2
 * (inverse of contract(x) = (2 - 1/|x|) x/|x|); h_v = h / (2 - |c|)^2 there,
 * the largest stretch of the inverse contraction.  Returns 0 for |c| >= 2.
 */
static int voxel_centre(int64_t lin, int g, const double* origin, double h, int contracted,
                        double* x, double* hv, uint32_t* flags) {
    int64_t i = lin % g, j = (lin / g) % g, k = lin / ((int64_t)g * g);
    double c[3] = {origin[0] + (i + 0.5) * h, origin[1] + (j + 0.5) * h,
                   origin[2] + (k + 0.5) * h};
    if (!contracted) {
        x[0] = c[0]; x[1] = c[1]; x[2] = c[2];
        *hv = h;
        return 1;
    }
    double rho = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (fabs(rho - 1.0) < ORACLE_MARGIN) *flags |= FLAG_CONTRACT;
    if (rho >= 2.0) return 0;
    if (rho <= 1.0) {
        x[0] = c[0]; x[1] = c[1]; x[2] = c[2];
        *hv = h;
        return 1;
    }
    double s = 1.0 / (rho * (2.0 - rho));
    x[0] = c[0] * s; x[1] = c[1] * s; x[2] = c[2] * s;
    *hv = h / ((2.0 - rho) * (2.0 - rho));
    return 1;
}

/*
 * Projection of world point x into view vw.  Returns 1 and the pixel
 * (ix, iy) when the point is in front of the camera and in frame; also
 * returns p (camera coordinates) and raises flags for near decisions.
 */
static int project(const oracle_view* vw, const double* x, double z_near, double* p, int* ix,
                   int* iy, uint32_t* flags) {
    const float* R = vw->R;
    for (int r = 0; r < 3; ++r)
        p[r] = (double)R[3 * r] * x[0] + (double)R[3 * r + 1] * x[1] +
               (double)R[3 * r + 2] * x[2] + (double)vw->t[r];
    double zscale = fabs((double)R[6] * x[0]) + fabs((double)R[7] * x[1]) +
                    fabs((double)R[8] * x[2]) + fabs((double)vw->t[2]);
    if (fabs(p[2] - z_near) < ORACLE_MARGIN * (zscale + 1e-30)) *flags |= FLAG_ZNEAR;
    if (!(p[2] > z_near)) return 0;
    double qx = p[0] / p[2], qy = p[1] / p[2];
    double u = (double)vw->fx * qx + (double)vw->cx;
    double v = (double)vw->fy * qy + (double)vw->cy;
    double su = 1.0 + fabs((double)vw->cx) + fabs((double)vw->fx * qx);
    double sv = 1.0 + fabs((double)vw->cy) + fabs((double)vw->fy * qy);
    if (dist_to_int(u) < ORACLE_MARGIN * su || dist_to_int(v) < ORACLE_MARGIN * sv)
        *flags |= FLAG_PIX;
    if (!(u >= 0.0 && u < (double)vw->W && v >= 0.0 && v < (double)vw->H)) return 0;
    *ix = (int)floor(u);
    *iy = (int)floor(v);
    return 1;
}

/*
 * Fusion of n_views views into the voxels lin[0..n_vox).
 * Outputs (each may be NULL): W, Z, P (double); seg (uint8); bits (raw view
 * bits of accepted votes); vmask (bits if seg else 0); flags; pix
 * (n_vox x n_views, pixel index iy*W + ix or -1 when the view was skipped
 * before the raster read).
 */
void oracle_fuse(int g, const double* origin, double h, int contracted, int64_t n_vox,
                 const int64_t* lin, int n_views, const oracle_view* views, int mask_type,
                 const oracle_params* pr, double* W_out, double* Z_out, double* P_out,
                 uint8_t* seg_out, uint32_t* bits_out, uint32_t* vmask_out, uint32_t* flags_out,
                 int32_t* pix_out) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t a = 0; a < n_vox; ++a) {
        uint32_t flags = 0, bits = 0;
        double Wsum = 0.0, Zsum = 0.0;
        double x[3], hv;
        int ok = voxel_centre(lin[a], g, origin, h, contracted, x, &hv, &flags);
        for (int i = 0; i < n_views; ++i) {
            if (pix_out) pix_out[a * n_views + i] = -1;
            if (!ok) continue;
            const oracle_view* vw = &views[i];
            double p[3];
            int ix, iy;
            if (!project(vw, x, pr->z_near, p, &ix, &iy, &flags)) continue;
            int64_t pix = (int64_t)iy * vw->W + ix;
            if (pix_out) pix_out[a * n_views + i] = (int32_t)pix;
            double D = vw->depth[pix];
            if (!(isfinite(D) && D > 0.0)) continue;
            double m;
            int pass;
            mask_at(vw, mask_type, pix, pr, &m, &pass);
            if (!pass) continue;
            double Delta = pr->gamma * hv;
            double e = p[2] - D;
            double sc = fabs(p[2]) > fabs(D) ? fabs(p[2]) : fabs(D);
            if (fabs(fabs(e) - Delta) < ORACLE_MARGIN * sc) flags |= FLAG_DEPTH;
            if (!(fabs(e) <= Delta)) continue;
            double r = e / Delta;
            double w = exp(-pr->alpha1 * r * r);
            Wsum += m * w;
            Zsum += w;
            if (i < 32) bits |= 1u << i;
        }
        double P = Zsum > pr->eps ? Wsum / Zsum : 0.0;
        if (Zsum > pr->eps && fabs(P - pr->tau_cons) < ORACLE_MARGIN) flags |= FLAG_CONS;
        int seg = P >= pr->tau_cons;
        if (W_out) W_out[a] = Wsum;
        if (Z_out) Z_out[a] = Zsum;
        if (P_out) P_out[a] = P;
        if (seg_out) seg_out[a] = (uint8_t)seg;
        if (bits_out) bits_out[a] = bits;
        if (vmask_out) vmask_out[a] = seg ? bits : 0u;
        if (flags_out) flags_out[a] = flags;
    }
}

/*
 * Adjoint of the fusion for a voxel-space cotangent gP = dL/dP.
 * With the gates held fixed (they are piecewise constant), per accepted vote
 *   dP/dm = w / Z,        dP/dw = (m - P) / Z,
 *   dw/dD = w * 2 alpha1 e / Delta^2      (e = p_z - D),
 *   dm/dl = m (1 - m)                     (logit masks; 1 for probability masks)
 * and the pixel (iy, ix) that supplied m and D receives
 *   gM[pix] += gP * (w / Z) * dm/dl,   gD[pix] += gP * ((m - P) / Z) * dw/dD.
 * gM and gD are per-view double rasters (H x W), accumulated into.
 */
void oracle_fuse_grad(int g, const double* origin, double h, int contracted, int64_t n_vox,
                      const int64_t* lin, int n_views, const oracle_view* views, int mask_type,
                      const oracle_params* pr, const double* gP, double* const* gM,
                      double* const* gD) {
    for (int64_t a = 0; a < n_vox; ++a) {
        if (gP[a] == 0.0) continue;
        uint32_t flags = 0;
        double x[3], hv;
        if (!voxel_centre(lin[a], g, origin, h, contracted, x, &hv, &flags)) continue;
        /* forward pass of this voxel, keeping the accepted votes */
        double wv[64], mv[64], ev[64];
        int64_t pv[64];
        int iv[64];
        int nv = 0;
        double Wsum = 0.0, Zsum = 0.0;
        double Delta = pr->gamma * hv;
        for (int i = 0; i < n_views && nv < 64; ++i) {
            const oracle_view* vw = &views[i];
            double p[3];
            int ix, iy;
            if (!project(vw, x, pr->z_near, p, &ix, &iy, &flags)) continue;
            int64_t pix = (int64_t)iy * vw->W + ix;
            double D = vw->depth[pix];
            if (!(isfinite(D) && D > 0.0)) continue;
            double m;
            int pass;
            mask_at(vw, mask_type, pix, pr, &m, &pass);
            if (!pass) continue;
            double e = p[2] - D;
            if (!(fabs(e) <= Delta)) continue;
            double r = e / Delta;
            double w = exp(-pr->alpha1 * r * r);
            Wsum += m * w;
            Zsum += w;
            wv[nv] = w; mv[nv] = m; ev[nv] = e; pv[nv] = pix; iv[nv] = i;
            ++nv;
        }
        if (!(Zsum > pr->eps)) continue;
        double P = Wsum / Zsum;
        for (int k = 0; k < nv; ++k) {
            double dmdl = mask_type == MASK_LOGIT_F32 ? mv[k] * (1.0 - mv[k]) : 1.0;
            double dwdD = wv[k] * 2.0 * pr->alpha1 * ev[k] / (Delta * Delta);
            gM[iv[k]][pv[k]] += gP[a] * (wv[k] / Zsum) * dmdl;
            gD[iv[k]][pv[k]] += gP[a] * ((mv[k] - P) / Zsum) * dwdD;
        }
    }
}

/*
 * Pass 1 label lookup (Eq. pass1): index = floor((q - origin) / h) per axis,
 * q = x (plain grid) or contract(x) (contracted grid); label = seg of that
 * voxel if 0 <= index < g on every axis, else 0; NaN coordinates give 0.
 * seg_dense: g^3 uint8 (x fastest), 1 = segmented.  flags: 1 when some
 * (q - origin)/h lies within ORACLE_MARGIN (relative) of an integer.
 */
void oracle_label(int g, const double* origin, double h, int contracted,
                  const uint8_t* seg_dense, int64_t n, const float* xyz, uint8_t* labels,
                  uint32_t* flags) {
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        double x[3] = {xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
        uint32_t f = 0;
        labels[a] = 0;
        if (isnan(x[0]) || isnan(x[1]) || isnan(x[2])) {
            if (flags) flags[a] = 0;
            continue;
        }
        double q[3] = {x[0], x[1], x[2]};
        if (contracted) {
            double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            if (r > 1.0) {
                double s = (2.0 - 1.0 / r) / r;
                q[0] = x[0] * s; q[1] = x[1] * s; q[2] = x[2] * s;
            }
        }
        int64_t idx[3];
        int inside = 1;
        for (int ax = 0; ax < 3; ++ax) {
            double s = (q[ax] - origin[ax]) / h;
            double sc = fabs(s) > 1.0 ? fabs(s) : 1.0;
            if (dist_to_int(s) < ORACLE_MARGIN * sc) f |= 1u;
            if (!(s >= 0.0 && s < (double)g)) {
                inside = 0;
                continue;
            }
            idx[ax] = (int64_t)floor(s);
        }
        if (flags) flags[a] = f;
        if (!inside) continue;
        labels[a] = seg_dense[(idx[2] * g + idx[1]) * g + idx[0]];
    }
}

/* Pixel projection of every voxel in one view (-1 = skipped); same rule as above. */
void oracle_project(int g, const double* origin, double h, int contracted, int64_t n_vox,
                    const int64_t* lin, const oracle_view* view, double z_near, int32_t* pix_out,
                    uint32_t* flags_out) {
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n_vox; ++a) {
        uint32_t flags = 0;
        double x[3], hv, p[3];
        int ix, iy;
        pix_out[a] = -1;
        if (voxel_centre(lin[a], g, origin, h, contracted, x, &hv, &flags) &&
            project(view, x, z_near, p, &ix, &iy, &flags))
            pix_out[a] = (int32_t)((int64_t)iy * view->W + ix);
        if (flags_out) flags_out[a] = flags;
    }
}

/* Thread count for the OpenMP loops above (the CPU baseline states it). */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
