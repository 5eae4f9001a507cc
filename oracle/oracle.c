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

/* ==========================================================================
 * Depth-tuple mode (Sec. 3.5 "Footprint statistics" .. "Thin-structure
 * path"; Algorithm "Thick-Structure Segmentation for 2DGS" and Algorithm
 * "Thin-Structure Segmentation for 2DGS" in Appendix B.5).
 *
 * Per voxel v (centre x, edge h_v, density rho_v) and view i in index order,
 * with o_i the camera centre, x_d = p_z the voxel's planar depth, t* = |x - o_i|
 * its distance along the ray through its own projection (the ray direction
 * d_hat runs through the projected point, so x lies on it and the planar-to-ray
 * factor is 1 / cos(theta) = t* / x_d):
 *
 *   skip unless the centre and all 8 corners x +- h_v/2 are in front
 *   (p_z > z_near) and the centre projects in frame;
 *   footprint B = pixels floor(u_min)..floor(u_max) x floor(v_min)..floor(v_max)
 *     of the corners' projections, clipped to the image; A = |B|,
 *     S1 = sum n_samp, S2 = sum n_samp^2 over B (the four-corner integral-image
 *     query); A_B = (u_max - u_min)(v_max - v_min) of the box clipped to
 *     [0, W] x [0, H];
 *   layered(n) = n > mean + sigma (mean = S1/A, sigma^2 = S2/A - mean^2), decided
 *     exactly on integers: n A - S1 > 0 and (n A - S1)^2 > A S2 - S1^2;
 *   E(n) = max(n - mean, 0);  t_depth(n) = gamma h_v / (1 + beta E(n))  (Eq. tightening)
 *   at the centre pixel: trusted = d_min <= d_med, seethru = d_med > gamma_st d_cam,
 *     front = (layered(n) or seethru) and trusted              (Eq. seethrough)
 *   thick path (m >= tau_m, trusted, all three depths finite and > 0):
 *     d_ref = front ? d_min : d_med;  t_hat = clip(t*, d_min^ray, d_ref^ray);
 *     spatial: |t* - t_hat| <= h_v pi_dg   (Eq. gs-spatial; |x - (o + t_hat d_hat)|)
 *     depth:   front ? x_d - d_min <= t_depth : |x_d - d_med| <= t_depth  (Eq. asym-gate)
 *     vote:    w = exp(-alpha1 ((t_hat - d_ctr) / d_hw)^2), d_ctr = (d_min^ray + d_max^ray)/2,
 *              d_hw = max((d_max^ray - d_min^ray)/2, eps)         (Eq. gs-depthweight)
 *              W += m w, Z += w, bits |= 1 << i                   (Eq. vmask)
 *   behind: d_surf = (trusted and seethru) ? d_min : d_med;
 *           behind_fail = x_d > d_surf + behind_margin h_v        (Eq. behind-gate)
 *   thin path (no thick vote, not behind_fail, rho_v >= rho_thin):
 *     per pixel q of B with not (d_med(q) < eps): front(q) as above with q's own
 *     values; valid = front(q) ? x_d - d_min(q) <= t_depth(n(q)) : |x_d - d_med(q)|
 *     <= t_depth(n(q)); valid -> n_depth += 1; valid and m(q) > 1/2 -> n_md += 1,
 *     m_max = max(m_max, m(q)), d2 = min(d2, |unproject(q, front(q) ? d_min(q) :
 *     d_med(q)) - x|^2) (pixel centre, planar depth)         (Eq. thin-d2min)
 *     t = m_max if n_depth >= max(n_abs, ceil(rho_occ A_B)), n_md >= rho_cover n_depth
 *         and d2 <= (dist_gate h_v)^2, else 0        (Eqs. thin-nmin, gs-coverage, thin-tthin-gs)
 *     t >= tau_thin -> W += t, Z += 1, bits |= 1 << i         (Eq. compact-fusion)
 *   pi_dg at pixel (x, y) = exp(-k G), G = g_x^2 + g_y^2 of c = (d_min + d_max)/2 by
 *   central differences, clamped at the border; G = inf (pi = 0) when a used c is
 *   not finite; pi = 1 when k = 0 (App. D).
 *
 * parity: pinned by the tuple-mode tests (closed-form single-voxel cases of
 * every gate, exact integer footprint statistics, an independent NumPy
 * statement on small scenes).
 * ========================================================================== */

enum { FLAG_TUPLE = 32 }; /* a tuple-mode gate (spatial, depth, behind, thin, footprint) near flipping */

typedef struct {
    float R[9], t[3], fx, fy, cx, cy;
    int32_t W, H;
    const float* d_min;
    const float* d_med;
    const float* d_max;
    const uint16_t* n_samp;
    const void* mask;
    double d_cam;
} oracle_tview;

typedef struct {
    double beta, gamma_st, tau_thin, rho_cover, rho_occ, n_abs, dist_gate, behind_margin, k_dg,
        rho_thin;
} oracle_tparams;

/* mask probability at p (and the thick-entry gate m >= tau_m) */
static void tmask_at(const oracle_tview* vw, int mask_type, int64_t p, const oracle_params* pr,
                     double* m, int* pass, int* half) {
    if (mask_type == MASK_F16) {
        *m = half_to_double(((const uint16_t*)vw->mask)[p]);
        *pass = *m >= pr->tau_m;
        *half = *m > 0.5;
    } else if (mask_type == MASK_LOGIT_F32) {
        double l = ((const float*)vw->mask)[p];
        *m = 1.0 / (1.0 + exp(-l));
        *pass = l >= pr->logit_tau;
        *half = l > 0.0; /* sigmoid(l) > 1/2 exactly when l > 0 */
    } else {
        *m = ((const float*)vw->mask)[p];
        *pass = *m >= pr->tau_m;
        *half = *m > 0.5;
    }
}

static double centre_depth(const oracle_tview* vw, int x, int y) {
    if (x < 0) x = 0;
    if (x > vw->W - 1) x = vw->W - 1;
    if (y < 0) y = 0;
    if (y > vw->H - 1) y = vw->H - 1;
    int64_t q = (int64_t)y * vw->W + x;
    return 0.5 * ((double)vw->d_min[q] + (double)vw->d_max[q]);
}

static double pi_dg(const oracle_tview* vw, int x, int y, double k) {
    if (k == 0.0) return 1.0;
    double a = centre_depth(vw, x + 1, y), b = centre_depth(vw, x - 1, y);
    double c = centre_depth(vw, x, y + 1), d = centre_depth(vw, x, y - 1);
    if (!(isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d))) return 0.0;
    double gx = a - b, gy = c - d;
    return exp(-k * (gx * gx + gy * gy));
}

/* n > mean + sigma over a footprint of A pixels with sums S1, S2, exactly */
static int layered_exact(int64_t n, int64_t A, int64_t S1, int64_t S2) {
    int64_t d = n * A - S1;
    if (d <= 0) return 0;
    return (__int128)d * d > (__int128)A * S2 - (__int128)S1 * S1;
}

static void near_flag(double lhs, double rhs, double scale, uint32_t* flags) {
    if (fabs(lhs - rhs) < ORACLE_MARGIN * (scale + 1e-30)) *flags |= FLAG_TUPLE;
}

void oracle_fuse_tuple(int g, const double* origin, double h, int contracted, int64_t n_vox,
                       const int64_t* lin, const double* rho, int n_views,
                       const oracle_tview* views, int mask_type, const oracle_params* pr,
                       const oracle_tparams* tp, double* W_out, double* Z_out, double* P_out,
                       uint8_t* seg_out, uint32_t* bits_out, uint32_t* flags_out,
                       uint8_t* kind_out, double* thin_out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < n_vox; ++a) {
        uint32_t flags = 0, bits = 0;
        double Wsum = 0.0, Zsum = 0.0;
        double x[3], hv;
        int ok = voxel_centre(lin[a], g, origin, h, contracted, x, &hv, &flags);
        double rho_v = rho ? rho[a] : 1.0;
        for (int i = 0; i < n_views; ++i) {
            if (kind_out) kind_out[a * n_views + i] = 0;
            if (thin_out) thin_out[a * n_views + i] = 0.0;
            if (!ok) continue;
            const oracle_tview* vw = &views[i];
            const float* R = vw->R;
            /* centre: camera coordinates and pixel */
            double p[3];
            int ix, iy;
            oracle_view pv = {{0}, {0}, vw->fx, vw->fy, vw->cx, vw->cy, vw->W, vw->H, NULL, NULL};
            memcpy(pv.R, vw->R, sizeof(pv.R));
            memcpy(pv.t, vw->t, sizeof(pv.t));
            int in = project(&pv, x, pr->z_near, p, &ix, &iy, &flags);
            /* corners: all in front, the footprint box of their projections */
            double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
            int corners_ok = 1;
            for (int c = 0; c < 8; ++c) {
                double xc[3] = {x[0] + ((c & 1) ? 0.5 : -0.5) * hv,
                                x[1] + ((c & 2) ? 0.5 : -0.5) * hv,
                                x[2] + ((c & 4) ? 0.5 : -0.5) * hv};
                double q[3];
                for (int r = 0; r < 3; ++r)
                    q[r] = (double)R[3 * r] * xc[0] + (double)R[3 * r + 1] * xc[1] +
                           (double)R[3 * r + 2] * xc[2] + vw->t[r];
                near_flag(q[2], pr->z_near, fabs(q[2]) + 1.0, &flags);
                if (!(q[2] > pr->z_near)) { corners_ok = 0; break; }
                double u = (double)vw->fx * q[0] / q[2] + (double)vw->cx;
                double v = (double)vw->fy * q[1] / q[2] + (double)vw->cy;
                umin = fmin(umin, u); umax = fmax(umax, u);
                vmin = fmin(vmin, v); vmax = fmax(vmax, v);
            }
            if (!in || !corners_ok) continue;
            /* the box edges decide which pixel rows and columns it covers: only
               an edge near an integer inside the frame (the floor is clamped to
               the frame outside it) can flip that */
            {
                const double ext[4] = {umin, umax, vmin, vmax};
                for (int e = 0; e < 4; ++e) {
                    double lim = e < 2 ? (double)vw->W : (double)vw->H;
                    double c = e < 2 ? (double)vw->cx : (double)vw->cy;
                    double s = 1.0 + fabs(c) + fabs(ext[e] - c);
                    if (ext[e] > -0.5 && ext[e] < lim + 0.5 && dist_to_int(ext[e]) < ORACLE_MARGIN * s)
                        flags |= FLAG_TUPLE;
                }
            }
            double cu0 = fmax(umin, 0.0), cu1 = fmin(umax, (double)vw->W);
            double cv0 = fmax(vmin, 0.0), cv1 = fmin(vmax, (double)vw->H);
            int i0 = (int)fmax(floor(umin), 0.0), i1 = (int)fmin(floor(umax), vw->W - 1.0);
            int j0 = (int)fmax(floor(vmin), 0.0), j1 = (int)fmin(floor(vmax), vw->H - 1.0);
            int64_t A = (int64_t)(i1 - i0 + 1) * (j1 - j0 + 1), S1 = 0, S2 = 0;
            for (int yy = j0; yy <= j1; ++yy)
                for (int xx = i0; xx <= i1; ++xx) {
                    int64_t nn = vw->n_samp[(int64_t)yy * vw->W + xx];
                    S1 += nn;
                    S2 += nn * nn;
                }
            double mean = (double)S1 / (double)A;
            double A_B = (cu1 - cu0) * (cv1 - cv0);
            /* centre pixel */
            int64_t pix = (int64_t)iy * vw->W + ix;
            double dmin = vw->d_min[pix], dmed = vw->d_med[pix], dmax = vw->d_max[pix];
            int64_t n = vw->n_samp[pix];
            double m;
            int pass, half;
            tmask_at(vw, mask_type, pix, pr, &m, &pass, &half);
            double xd = p[2];
            double oc[3];
            for (int r = 0; r < 3; ++r)  /* o = -R^T t */
                oc[r] = -((double)R[r] * vw->t[0] + (double)R[3 + r] * vw->t[1] +
                          (double)R[6 + r] * vw->t[2]);
            double tstar = sqrt((x[0] - oc[0]) * (x[0] - oc[0]) + (x[1] - oc[1]) * (x[1] - oc[1]) +
                                (x[2] - oc[2]) * (x[2] - oc[2]));
            double ray = tstar / xd; /* 1 / cos(theta) */
            int trusted = dmin <= dmed;
            int seethru = dmed > tp->gamma_st * vw->d_cam;
            near_flag(dmed, tp->gamma_st * vw->d_cam, fabs(dmed), &flags);
            int layered = layered_exact(n, A, S1, S2);
            int front = (layered || seethru) && trusted;
            int check_thin = 1;
            if (pass && trusted && isfinite(dmin) && isfinite(dmed) && isfinite(dmax) &&
                dmin > 0.0 && dmed > 0.0 && dmax > 0.0) {
                double dref = front ? dmin : dmed;
                double lo = dmin * ray, hi = dref * ray;
                double that = tstar < lo ? lo : (tstar > hi ? hi : tstar);
                double delta = fabs(tstar - that);
                double tau_sp = hv * pi_dg(vw, ix, iy, tp->k_dg);
                double E = fmax((double)n - mean, 0.0);
                double tdep = pr->gamma * hv / (1.0 + tp->beta * E);
                double lhs = front ? xd - dmin : fabs(xd - dmed);
                near_flag(delta, tau_sp, tstar, &flags);
                near_flag(lhs, tdep, fabs(xd), &flags);
                if (delta <= tau_sp && lhs <= tdep) {
                    double dctr = 0.5 * (dmin + dmax) * ray;
                    double dhw = fmax(0.5 * (dmax - dmin) * ray, pr->eps);
                    double r = (that - dctr) / dhw;
                    double w = exp(-pr->alpha1 * r * r);
                    Wsum += m * w;
                    Zsum += w;
                    bits |= i < 32 ? 1u << i : 0u;
                    check_thin = 0;
                    if (kind_out) kind_out[a * n_views + i] = 1;
                }
            }
            double dsurf = (trusted && seethru) ? dmin : dmed;
            near_flag(xd, dsurf + tp->behind_margin * hv, fabs(xd), &flags);
            int behind_fail = xd > dsurf + tp->behind_margin * hv;
            if (!check_thin || behind_fail || !(rho_v >= tp->rho_thin)) continue;
            /* thin path over the footprint */
            int64_t n_depth = 0, n_md = 0;
            double m_max = 0.0, d2 = INFINITY;
            for (int yy = j0; yy <= j1; ++yy)
                for (int xx = i0; xx <= i1; ++xx) {
                    int64_t q = (int64_t)yy * vw->W + xx;
                    double qmin = vw->d_min[q], qmed = vw->d_med[q];
                    if (qmed < pr->eps) continue;
                    int64_t nq = vw->n_samp[q];
                    double Eq = fmax((double)nq - mean, 0.0);
                    double tq = pr->gamma * hv / (1.0 + tp->beta * Eq);
                    int tr_q = qmin <= qmed;
                    int st_q = qmed > tp->gamma_st * vw->d_cam;
                    int fr_q = (layered_exact(nq, A, S1, S2) || st_q) && tr_q;
                    double lhs = fr_q ? xd - qmin : fabs(xd - qmed);
                    near_flag(lhs, tq, fabs(xd), &flags);
                    near_flag(qmed, tp->gamma_st * vw->d_cam, fabs(qmed), &flags);
                    if (!(lhs <= tq)) continue;
                    ++n_depth;
                    double mq;
                    int pq, hq;
                    tmask_at(vw, mask_type, q, pr, &mq, &pq, &hq);
                    if (!hq) continue;
                    ++n_md;
                    if (mq > m_max) m_max = mq;
                    double dq = fr_q ? qmin : qmed;
                    double pc[3] = {((double)xx + 0.5 - (double)vw->cx) / (double)vw->fx * dq,
                                    ((double)yy + 0.5 - (double)vw->cy) / (double)vw->fy * dq, dq};
                    double pw[3];
                    for (int r = 0; r < 3; ++r)  /* world = R^T (pc - t) */
                        pw[r] = (double)R[r] * (pc[0] - vw->t[0]) +
                                (double)R[3 + r] * (pc[1] - vw->t[1]) +
                                (double)R[6 + r] * (pc[2] - vw->t[2]);
                    double dd = (pw[0] - x[0]) * (pw[0] - x[0]) + (pw[1] - x[1]) * (pw[1] - x[1]) +
                                (pw[2] - x[2]) * (pw[2] - x[2]);
                    if (dd < d2) d2 = dd;
                }
            double n_min = fmax(tp->n_abs, ceil(tp->rho_occ * A_B));
            double gate = tp->dist_gate * hv;
            /* the distance gate: near it within 1e-6 of the gate itself */
            near_flag(sqrt(d2), gate, gate, &flags);
            {   /* ceil near an integer step: flag when the two candidate counts
                   would decide this voxel differently */
                double k = round(tp->rho_occ * A_B);
                if (fabs(tp->rho_occ * A_B - k) < ORACLE_MARGIN * (A_B + 1.0) &&
                    ((double)n_depth >= fmax(tp->n_abs, k)) != ((double)n_depth >= fmax(tp->n_abs, k + 1.0)))
                    flags |= FLAG_TUPLE;
            }
            double t = ((double)n_depth >= n_min && (double)n_md >= tp->rho_cover * (double)n_depth &&
                        d2 <= gate * gate)
                           ? m_max
                           : 0.0;
            if (thin_out) thin_out[a * n_views + i] = t;
            near_flag(t, tp->tau_thin, 1.0, &flags);
            if (t >= tp->tau_thin) {
                Wsum += t;
                Zsum += 1.0;
                bits |= i < 32 ? 1u << i : 0u;
                if (kind_out) kind_out[a * n_views + i] = 2;
            }
        }
        double P = (Zsum > pr->eps) ? Wsum / Zsum : 0.0;
        if (Zsum > pr->eps && fabs(P - pr->tau_cons) < ORACLE_MARGIN) flags |= FLAG_CONS;
        int seg = (P >= pr->tau_cons);
        if (W_out) W_out[a] = Wsum;
        if (Z_out) Z_out[a] = Zsum;
        if (P_out) P_out[a] = P;
        if (seg_out) seg_out[a] = (uint8_t)seg;
        if (bits_out) bits_out[a] = bits;
        if (flags_out) flags_out[a] = flags;
    }
}

/* ==========================================================================
 * NeRF variant of the depth-tuple fusion (Appendix "NeRF-Backbone 3D Fusion
 * Details": Eqs. distance_cond, dist_tol, depth_tol, nerf-accept, nerf-vote,
 * nerf-thindepth, nerf-support, nerf-counters, nerf-coverage, nerf-thin;
 * Algorithms "Thick-Structure Segmentation via Depth-Weighted Voxel
 * Aggregation" and "Thin-Structure Segmentation via Footprint-Based Coverage
 * Analysis"), per voxel x (centre x_c, edge Delta = h_v) and view i in order:
 *
 *   centre pixel (x_p, y_p) of the projection (in frame, in front of z_near);
 *   m = mask probability there; check_thin = 1;
 *   thick entry m >= tau_m (logits l >= logit(tau_m)) with d_min, d_exp,
 *   d_max finite and positive (planar depths of the tuple at the centre
 *   pixel), n = n_samp there:
 *     the pixel's ray through its centre, camera-space direction
 *     k = ((x_p + 1/2 - cx)/fx, (y_p + 1/2 - cy)/fy, 1), |k| = 1/cos theta;
 *     a planar depth d on it is the point k d (ray distance |k| d);
 *     closest point of the band: z_proj = <p, k> / |k|^2 (p = camera-space
 *     x_c), z_c = clip(z_proj, d_min, d_max), delta = |p - k z_c|;
 *     tau_spatial = Delta pi_dg + lambda_range |k| (d_max - d_min);
 *     b = min(beta n, b_max), tau_depth = (gamma + b) Delta;
 *     x_d = p_z; accept when delta <= tau_spatial and |x_d - d_exp| <=
 *     tau_depth: mu = (d_min + d_max)/2, h_d = max((d_max - d_min)/2, eps),
 *     r = |z_c - mu| / h_d (the ray-space ratio: |k| cancels),
 *     w = exp(-alpha1 r^2), W += m w, Z += w, check_thin = 0;
 *   thin fallback when check_thin, m > m_thin (logits l > logit(m_thin) in
 *   FP32) and rho_x >= rho_thin: the 8 corners x_c +- Delta/2 (all in front
 *   of z_near), the pixel box of their projections clipped to the frame (N
 *   pixels); per box pixel q: b_q = min(beta n(q), b_max), support = m(q) >
 *   1/2 and |x_d - d_exp(q)| <= (2 gamma + b_q) Delta; n_valid = the
 *   supports, m_max = max of m(q) over the whole box; t = m_max when n_valid
 *   >= rho_cover N, else 0; t >= tau_thin -> W += t, Z += 1.
 *   P = W / Z if Z > eps else 0; seg = P >= tau_cons.
 *
 * Near-boundary flags as in the 2DGS variant: the spatial gate within 1e-6
 * of tau_spatial itself, the depth gates against 1e-6 |x_d|, box edges near
 * an integer, tau_thin, z_near.
 *
 * parity: pinned by the NeRF-variant tests (single-voxel closed forms of
 * every gate and of the weight, an independent NumPy statement in ray space).
 * ========================================================================== */

typedef struct {
    double gamma, beta, b_max, lambda_range, rho_thin, rho_cover, tau_thin, m_thin, k_dg;
} oracle_nparams;

void oracle_fuse_nerf(int g, const double* origin, double h, int contracted, int64_t n_vox,
                      const int64_t* lin, const double* rho, int n_views,
                      const oracle_tview* views, int mask_type, const oracle_params* pr,
                      const oracle_nparams* np, double* W_out, double* Z_out, double* P_out,
                      uint8_t* seg_out, uint32_t* bits_out, uint32_t* flags_out,
                      uint8_t* kind_out, double* thin_out) {
    /* the thin eligibility m > m_thin on logits: l > logit(m_thin), as FP32 */
    double l_thin = (np->m_thin <= 0.0) ? -INFINITY
                  : (np->m_thin >= 1.0) ? INFINITY
                  : (double)(float)log(np->m_thin / (1.0 - np->m_thin));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < n_vox; ++a) {
        uint32_t flags = 0, bits = 0;
        double Wsum = 0.0, Zsum = 0.0;
        double x[3], hv;
        int ok = voxel_centre(lin[a], g, origin, h, contracted, x, &hv, &flags);
        double rho_v = rho ? rho[a] : 1.0;
        for (int i = 0; i < n_views; ++i) {
            if (kind_out) kind_out[a * n_views + i] = 0;
            if (thin_out) thin_out[a * n_views + i] = 0.0;
            if (!ok) continue;
            const oracle_tview* vw = &views[i];
            const float* R = vw->R;
            double p[3];
            int ix, iy;
            oracle_view pv = {{0}, {0}, vw->fx, vw->fy, vw->cx, vw->cy, vw->W, vw->H, NULL, NULL};
            memcpy(pv.R, vw->R, sizeof(pv.R));
            memcpy(pv.t, vw->t, sizeof(pv.t));
            if (!project(&pv, x, pr->z_near, p, &ix, &iy, &flags)) continue;
            int64_t pix = (int64_t)iy * vw->W + ix;
            double m;
            int pass, half;
            tmask_at(vw, mask_type, pix, pr, &m, &pass, &half);
            double xd = p[2];
            int check_thin = 1;
            /* thick path (Eqs. distance_cond .. nerf-vote) */
            double dmin = vw->d_min[pix], dexp = vw->d_med[pix], dmax = vw->d_max[pix];
            int64_t n = vw->n_samp[pix];
            if (pass && isfinite(dmin) && isfinite(dexp) && isfinite(dmax) && dmin > 0.0 &&
                dexp > 0.0 && dmax > 0.0) {
                double k[3] = {((double)ix + 0.5 - (double)vw->cx) / (double)vw->fx,
                               ((double)iy + 0.5 - (double)vw->cy) / (double)vw->fy, 1.0};
                double k2 = k[0] * k[0] + k[1] * k[1] + 1.0;
                double zproj = (p[0] * k[0] + p[1] * k[1] + p[2]) / k2;
                double zc = zproj < dmin ? dmin : (zproj > dmax ? dmax : zproj);
                double e0 = p[0] - k[0] * zc, e1 = p[1] - k[1] * zc, e2 = p[2] - zc;
                double delta = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
                double tau_sp = hv * pi_dg(vw, ix, iy, np->k_dg) +
                                np->lambda_range * sqrt(k2) * (dmax - dmin);
                double b = fmin(np->beta * (double)n, np->b_max);
                double tau_d = (np->gamma + b) * hv;
                near_flag(delta, tau_sp, tau_sp, &flags);
                near_flag(fabs(xd - dexp), tau_d, fabs(xd), &flags);
                if (delta <= tau_sp && fabs(xd - dexp) <= tau_d) {
                    double mu = 0.5 * (dmin + dmax);
                    double hd = fmax(0.5 * (dmax - dmin), pr->eps);
                    double r = fabs(zc - mu) / hd;
                    double w = exp(-pr->alpha1 * r * r);
                    Wsum += m * w;
                    Zsum += w;
                    bits |= i < 32 ? 1u << i : 0u;
                    check_thin = 0;
                    if (kind_out) kind_out[a * n_views + i] = 1;
                }
            }
            /* thin fallback (Eqs. nerf-thindepth .. nerf-thin) */
            int eligible;
            if (mask_type == MASK_LOGIT_F32)
                eligible = (double)((const float*)vw->mask)[pix] > l_thin;
            else
                eligible = m > np->m_thin;
            if (!check_thin || !eligible || !(rho_v >= np->rho_thin)) continue;
            double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
            int corners_ok = 1;
            for (int c = 0; c < 8; ++c) {
                double xc[3] = {x[0] + ((c & 1) ? 0.5 : -0.5) * hv,
                                x[1] + ((c & 2) ? 0.5 : -0.5) * hv,
                                x[2] + ((c & 4) ? 0.5 : -0.5) * hv};
                double q[3];
                for (int r = 0; r < 3; ++r)
                    q[r] = (double)R[3 * r] * xc[0] + (double)R[3 * r + 1] * xc[1] +
                           (double)R[3 * r + 2] * xc[2] + vw->t[r];
                near_flag(q[2], pr->z_near, fabs(q[2]) + 1.0, &flags);
                if (!(q[2] > pr->z_near)) { corners_ok = 0; break; }
                double u = (double)vw->fx * q[0] / q[2] + (double)vw->cx;
                double v = (double)vw->fy * q[1] / q[2] + (double)vw->cy;
                umin = fmin(umin, u); umax = fmax(umax, u);
                vmin = fmin(vmin, v); vmax = fmax(vmax, v);
            }
            if (!corners_ok) continue;
            {
                const double ext[4] = {umin, umax, vmin, vmax};
                for (int e = 0; e < 4; ++e) {
                    double lim = e < 2 ? (double)vw->W : (double)vw->H;
                    double c = e < 2 ? (double)vw->cx : (double)vw->cy;
                    double s = 1.0 + fabs(c) + fabs(ext[e] - c);
                    if (ext[e] > -0.5 && ext[e] < lim + 0.5 && dist_to_int(ext[e]) < ORACLE_MARGIN * s)
                        flags |= FLAG_TUPLE;
                }
            }
            int i0 = (int)fmax(floor(umin), 0.0), i1 = (int)fmin(floor(umax), vw->W - 1.0);
            int j0 = (int)fmax(floor(vmin), 0.0), j1 = (int)fmin(floor(vmax), vw->H - 1.0);
            int64_t N = (int64_t)(i1 - i0 + 1) * (j1 - j0 + 1), n_valid = 0;
            double m_max = 0.0;
            for (int yy = j0; yy <= j1; ++yy)
                for (int xx = i0; xx <= i1; ++xx) {
                    int64_t q = (int64_t)yy * vw->W + xx;
                    double mq;
                    int pq, hq;
                    tmask_at(vw, mask_type, q, pr, &mq, &pq, &hq);
                    if (mq > m_max) m_max = mq;
                    double bq = fmin(np->beta * (double)vw->n_samp[q], np->b_max);
                    double tq = (2.0 * np->gamma + bq) * hv;
                    double e = fabs(xd - (double)vw->d_med[q]);
                    near_flag(e, tq, fabs(xd), &flags);
                    if (hq && e <= tq) ++n_valid;
                }
            double t = ((double)n_valid >= np->rho_cover * (double)N) ? m_max : 0.0;
            if (thin_out) thin_out[a * n_views + i] = t;
            near_flag(t, np->tau_thin, 1.0, &flags);
            if (t >= np->tau_thin) {
                Wsum += t;
                Zsum += 1.0;
                bits |= i < 32 ? 1u << i : 0u;
                if (kind_out) kind_out[a * n_views + i] = 2;
            }
        }
        double P = (Zsum > pr->eps) ? Wsum / Zsum : 0.0;
        if (Zsum > pr->eps && fabs(P - pr->tau_cons) < ORACLE_MARGIN) flags |= FLAG_CONS;
        int seg = (P >= pr->tau_cons);
        if (W_out) W_out[a] = Wsum;
        if (Z_out) Z_out[a] = Zsum;
        if (P_out) P_out[a] = P;
        if (seg_out) seg_out[a] = (uint8_t)seg;
        if (bits_out) bits_out[a] = bits;
        if (flags_out) flags_out[a] = flags;
    }
}
