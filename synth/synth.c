/*
 * Seeded synthetic scenes for the depth-weighted voxel fusion workloads.
 *
 * This file holds none of the fusion method's arithmetic. It renders the
 * inputs the method consumes, the way a trained NeRF / 2DGS backbone would
 * hand them to the fusion stage (Sec. 3.1 "Preliminaries": a per-pixel
 * rendered depth, Sec. 3.4: a per-view mask), from analytic primitives:
 *
 *   - planar camera-Z depth of the nearest hit along the ray through each
 *     pixel centre (+inf on a miss), and the id of the primitive hit;
 *   - occupancy priors (Sec. 3.5 "Occupancy", Appendix B.1): voxels near a
 *     surface, by several recipes;
 *   - soft masks: indicator -> separable Gaussian blur -> + noise -> clamp ->
 *     IEEE binary16 (round to nearest even).
 *
 * Random numbers are drawn by the Python side (numpy PCG64) and passed in;
 * nothing here draws any.  All arithmetic is double precision.
 *
 * Conventions: cameras are OpenCV world->camera (x right, y down, z forward),
 * R row-major, camera centre C = -R^T t; pixel (i, j) has its centre at
 * (i + 1/2, j + 1/2).  An ellipsoid is {x : |M (x - c)| = 1} with
 * M = A^-1 R_e^T (A the semi-axes, R_e the axes as columns).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static inline void matvec3(const double* M, const double* v, double* out) {
    out[0] = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
    out[1] = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
    out[2] = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
}

/* Nearest positive ray parameter of |M(o + t d - c)| = 1, or +inf. */
static inline double hit_ellipsoid(const double* c, const double* M,
                                   const double* o, const double* d) {
    double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
    double op[3], dp[3];
    matvec3(M, oc, op);
    matvec3(M, d, dp);
    double a = dot3(dp, dp);
    double b = 2.0 * dot3(op, dp);
    double q = dot3(op, op) - 1.0;
    if (q <= 0.0) return INFINITY; /* origin inside: not used by the scenes */
    if (b >= 0.0) return INFINITY; /* both roots behind the origin */
    double disc = b * b - 4.0 * a * q;
    if (disc < 0.0) return INFINITY;
    /* stable near root: 2q / (-b + sqrt(disc)) */
    double t = 2.0 * q / (-b + sqrt(disc));
    return t > 0.0 ? t : INFINITY;
}

/* Both positive ray parameters of |M(o + t d - c)| = 1 (entry t0, exit t1);
 * returns 0 when the ray misses or the object lies behind the origin. */
static inline int hit_ellipsoid2(const double* c, const double* M, const double* o,
                                 const double* d, double* t0, double* t1) {
    double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
    double op[3], dp[3];
    matvec3(M, oc, op);
    matvec3(M, d, dp);
    double a = dot3(dp, dp);
    double b = 2.0 * dot3(op, dp);
    double q = dot3(op, op) - 1.0;
    if (q <= 0.0 || b >= 0.0) return 0;
    double disc = b * b - 4.0 * a * q;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double qq = -0.5 * (b - sq); /* b < 0: no cancellation */
    double r0 = q / qq, r1 = qq / a;
    *t0 = fmin(r0, r1);
    *t1 = fmax(r0, r1);
    return *t0 > 0.0;
}

/* Conservative pixel bounding box of a sphere (camera-space centre cc, radius r). */
static void sphere_bbox(const double* cc, double r, double fx, double fy, double cx,
                        double cy, int W, int H, int* box) {
    if (cc[2] - r <= 1e-6) { /* touches or crosses the camera plane */
        box[0] = 0; box[1] = W - 1; box[2] = 0; box[3] = H - 1;
        return;
    }
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int sx = -1; sx <= 1; sx += 2)
        for (int sz = -1; sz <= 1; sz += 2) {
            double q = (cc[0] + sx * r) / (cc[2] + sz * r);
            umin = fmin(umin, q); umax = fmax(umax, q);
        }
    for (int sy = -1; sy <= 1; sy += 2)
        for (int sz = -1; sz <= 1; sz += 2) {
            double q = (cc[1] + sy * r) / (cc[2] + sz * r);
            vmin = fmin(vmin, q); vmax = fmax(vmax, q);
        }
    umin = fx * umin + cx; umax = fx * umax + cx;
    vmin = fy * vmin + cy; vmax = fy * vmax + cy;
    /* pixel centres in [umin, umax], one pixel of slack either side */
    double i0 = ceil(umin - 0.5) - 1.0, i1 = floor(umax - 0.5) + 1.0;
    double j0 = ceil(vmin - 0.5) - 1.0, j1 = floor(vmax - 0.5) + 1.0;
    box[0] = (int)fmax(i0, 0.0);
    box[1] = (int)fmin(i1, (double)(W - 1));
    box[2] = (int)fmax(j0, 0.0);
    box[3] = (int)fmin(j1, (double)(H - 1));
}

/*
 * Planar depth and hit id for one view.
 * ell_*: n_ell ellipsoids (centre 3, M 9, bounding radius 1, id 1)
 * pl_*:  n_pl planes n.x = d (normal 3, offset 1, id 1); disc radius
 *        pl_rad (<= 0: unbounded) about the origin's projection.
 * depth: H*W float32, +inf on a miss;  hit: H*W int32, -1 on a miss.
 */
void synth_render(int n_ell, const double* ell_c, const double* ell_M,
                  const double* ell_brad, const int32_t* ell_id, int n_pl,
                  const double* pl_n, const double* pl_d, const double* pl_rad,
                  const int32_t* pl_id, const double* R, const double* t, double fx,
                  double fy, double cx, double cy, int W, int H, float* depth,
                  int32_t* hit) {
    double C[3] = {-(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]),
                   -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]),
                   -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2])};
    int* box = (int*)malloc(sizeof(int) * 4 * (size_t)(n_ell > 0 ? n_ell : 1));
    for (int e = 0; e < n_ell; ++e) {
        double cc[3];
        matvec3(R, ell_c + 3 * e, cc);
        cc[0] += t[0]; cc[1] += t[1]; cc[2] += t[2];
        sphere_bbox(cc, ell_brad[e], fx, fy, cx, cy, W, H, box + 4 * e);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            depth[(size_t)j * W + i] = INFINITY;
            hit[(size_t)j * W + i] = -1;
        }
        double* best = (double*)malloc(sizeof(double) * W);
        for (int i = 0; i < W; ++i) best[i] = INFINITY;
        int32_t* bid = hit + (size_t)j * W;
        double yc = ((double)j + 0.5 - cy) / fy;
        for (int e = 0; e < n_ell; ++e) {
            const int* b = box + 4 * e;
            if (j < b[2] || j > b[3] || b[0] > b[1]) continue;
            for (int i = b[0]; i <= b[1]; ++i) {
                double dc[3] = {((double)i + 0.5 - cx) / fx, yc, 1.0};
                double d[3] = {R[0] * dc[0] + R[3] * dc[1] + R[6] * dc[2],
                               R[1] * dc[0] + R[4] * dc[1] + R[7] * dc[2],
                               R[2] * dc[0] + R[5] * dc[1] + R[8] * dc[2]};
                double th = hit_ellipsoid(ell_c + 3 * e, ell_M + 9 * e, C, d);
                if (th < best[i]) { best[i] = th; bid[i] = ell_id[e]; }
            }
        }
        for (int p = 0; p < n_pl; ++p) {
            const double* n = pl_n + 3 * p;
            for (int i = 0; i < W; ++i) {
                double dc[3] = {((double)i + 0.5 - cx) / fx, yc, 1.0};
                double d[3] = {R[0] * dc[0] + R[3] * dc[1] + R[6] * dc[2],
                               R[1] * dc[0] + R[4] * dc[1] + R[7] * dc[2],
                               R[2] * dc[0] + R[5] * dc[1] + R[8] * dc[2]};
                double nd = dot3(n, d);
                if (nd == 0.0) continue;
                double th = (pl_d[p] - dot3(n, C)) / nd;
                if (!(th > 0.0) || !(th < best[i])) continue;
                if (pl_rad[p] > 0.0) {
                    double x[3] = {C[0] + th * d[0], C[1] + th * d[1], C[2] + th * d[2]};
                    double off = dot3(n, x);
                    double r2 = dot3(x, x) - off * off;
                    if (r2 > pl_rad[p] * pl_rad[p]) continue;
                }
                best[i] = th;
                bid[i] = pl_id[p];
            }
        }
        for (int i = 0; i < W; ++i) depth[(size_t)j * W + i] = (float)best[i];
        free(best);
    }
    free(box);
}

/*
 * Sphere-shell occupancy: voxel occupied iff min_k | |x - c_k| - r_k | <= band,
 * x the voxel centre origin + (idx + 1/2) h.  occ: g^3 uint8, x fastest.
 */
void synth_occ_sphere_band(int n_sph, const double* c, const double* r, double band,
                           int g, const double* origin, double h, uint8_t* occ) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g; ++k)
        for (int j = 0; j < g; ++j)
            for (int i = 0; i < g; ++i) {
                double x[3] = {origin[0] + (i + 0.5) * h, origin[1] + (j + 0.5) * h,
                               origin[2] + (k + 0.5) * h};
                double best = INFINITY;
                for (int s = 0; s < n_sph; ++s) {
                    double dx = x[0] - c[3 * s], dy = x[1] - c[3 * s + 1],
                           dz = x[2] - c[3 * s + 2];
                    double dist = fabs(sqrt(dx * dx + dy * dy + dz * dz) - r[s]);
                    if (dist < best) best = dist;
                }
                occ[((size_t)k * g + j) * g + i] = best <= band ? 1 : 0;
            }
}

/*
 * Surface-straddle occupancy: voxel occupied iff the implicit function of some
 * ellipsoid (|M(x-c)|^2 - 1) or plane (n.x - d) changes sign over its 8
 * corners.  Corners are origin + (idx + {0,1}) h.
 */
void synth_occ_corner_sign(int n_ell, const double* ell_c, const double* ell_M,
                           const double* ell_brad, int n_pl, const double* pl_n,
                           const double* pl_d, int g, const double* origin, double h,
                           uint8_t* occ) {
    memset(occ, 0, (size_t)g * g * g);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < g; ++k) {
        double z0 = origin[2] + k * h, z1 = z0 + h;
        for (int e = 0; e < n_ell; ++e) {
            const double* c = ell_c + 3 * e;
            const double* M = ell_M + 9 * e;
            double br = ell_brad[e];
            if (z1 < c[2] - br || z0 > c[2] + br) continue;
            int i0 = (int)floor((c[0] - br - origin[0]) / h) - 1;
            int i1 = (int)floor((c[0] + br - origin[0]) / h) + 1;
            int j0 = (int)floor((c[1] - br - origin[1]) / h) - 1;
            int j1 = (int)floor((c[1] + br - origin[1]) / h) + 1;
            if (i0 < 0) i0 = 0;
            if (j0 < 0) j0 = 0;
            if (i1 > g - 1) i1 = g - 1;
            if (j1 > g - 1) j1 = g - 1;
            for (int j = j0; j <= j1; ++j)
                for (int i = i0; i <= i1; ++i) {
                    int npos = 0;
                    for (int q = 0; q < 8; ++q) {
                        double x[3] = {origin[0] + (i + (q & 1)) * h - c[0],
                                       origin[1] + (j + ((q >> 1) & 1)) * h - c[1],
                                       origin[2] + (k + ((q >> 2) & 1)) * h - c[2]};
                        double y[3];
                        matvec3(M, x, y);
                        npos += dot3(y, y) - 1.0 > 0.0;
                    }
                    if (npos != 0 && npos != 8) occ[((size_t)k * g + j) * g + i] = 1;
                }
        }
        for (int p = 0; p < n_pl; ++p) {
            const double* n = pl_n + 3 * p;
            for (int j = 0; j < g; ++j)
                for (int i = 0; i < g; ++i) {
                    int npos = 0;
                    for (int q = 0; q < 8; ++q) {
                        double x[3] = {origin[0] + (i + (q & 1)) * h,
                                       origin[1] + (j + ((q >> 1) & 1)) * h,
                                       origin[2] + (k + ((q >> 2) & 1)) * h};
                        npos += dot3(n, x) - pl_d[p] > 0.0;
                    }
                    if (npos != 0 && npos != 8) occ[((size_t)k * g + j) * g + i] = 1;
                }
        }
    }
}

/* IEEE binary16 bits of a float, round to nearest even (finite, |x| small). */
static uint16_t half_bits_rne(float f) {
    union { float f; uint32_t u; } v = {f};
    uint32_t sign = (v.u >> 16) & 0x8000u;
    uint32_t a = v.u & 0x7fffffffu;
    if (a >= 0x7f800000u) return (uint16_t)(sign | 0x7c00u | (a > 0x7f800000u ? 0x200u : 0));
    if (a >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u); /* overflow -> inf */
    if (a < 0x38800000u) {                                    /* subnormal half */
        /* value = a_float; half subnormal unit = 2^-24 */
        double x = (double)v.f;
        if (x < 0) x = -x;
        double q = x * 16777216.0; /* in units of 2^-24 */
        double fl = floor(q);
        double rem = q - fl;
        uint32_t m = (uint32_t)fl;
        if (rem > 0.5 || (rem == 0.5 && (m & 1u))) m += 1;
        return (uint16_t)(sign | m);
    }
    uint32_t exp = ((a >> 23) - 127 + 15);
    uint32_t mant = a & 0x7fffffu;
    uint32_t hm = mant >> 13;
    uint32_t rest = mant & 0x1fffu;
    uint32_t out = (exp << 10) | hm;
    if (rest > 0x1000u || (rest == 0x1000u && (hm & 1u))) out += 1;
    return (uint16_t)(sign | out);
}

/*
 * Soft mask: separable normalised Gaussian blur (sigma, radius, clamp-to-edge)
 * of a 0/1 indicator, + noise (one float per pixel), clamp to [0,1], stored
 * as binary16 bits (round to nearest even).
 */
void synth_soft_mask(const uint8_t* ind, int W, int H, double sigma, int radius,
                     const float* noise, uint16_t* out) {
    int K = 2 * radius + 1;
    double* w = (double*)malloc(sizeof(double) * K);
    double s = 0.0;
    for (int k = -radius; k <= radius; ++k) {
        w[k + radius] = exp(-0.5 * (double)k * k / (sigma * sigma));
        s += w[k + radius];
    }
    for (int k = 0; k < K; ++k) w[k] /= s;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)W * H);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            double acc = 0.0;
            for (int k = -radius; k <= radius; ++k) {
                int ii = i + k;
                ii = ii < 0 ? 0 : (ii >= W ? W - 1 : ii);
                acc += w[k + radius] * ind[(size_t)j * W + ii];
            }
            tmp[(size_t)j * W + i] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            double acc = 0.0;
            for (int k = -radius; k <= radius; ++k) {
                int jj = j + k;
                jj = jj < 0 ? 0 : (jj >= H ? H - 1 : jj);
                acc += w[k + radius] * tmp[(size_t)jj * W + i];
            }
            double m = acc + (double)noise[(size_t)j * W + i];
            m = m < 0.0 ? 0.0 : (m > 1.0 ? 1.0 : m);
            out[(size_t)j * W + i] = half_bits_rne((float)m);
        }
    free(tmp);
    free(w);
}

/*
 * Contracted-grid surface distance for the unbounded scene.
 * The grid covers contracted space [-2,2]^3 with g voxels per side
 * (h_c = 4/g).  For each voxel centre q (|q| < 2) this returns the distance,
 * in units of h_c, from q to the nearest contracted surface: the ground
 * plane (q_z = 0 inside the disc |q_xy| <= plane_rc) and the contracted
 * ellipsoids, the latter to first order, |G| / |grad_q G| with
 * G(q) = |M(u(q) - c)| - 1 and u the inverse contraction.  Voxels whose
 * distance exceeds s_max (or with |q| >= 2) get +inf.
 *
 * Inverse contraction: u(q) = q for |q| <= 1, q / (|q| (2 - |q|)) otherwise.
 * Each ellipsoid only visits the contracted cube of half-width
 * L*brad + (s_max + 2) h_c about contract(c); L bounds the stretch of the
 * contraction on the world ball about c (1-Lipschitz inside, 2/r outside).
 */
static void contract3(const double* x, double* q) {
    double r = sqrt(dot3(x, x));
    if (r <= 1.0) { q[0] = x[0]; q[1] = x[1]; q[2] = x[2]; return; }
    double s = (2.0 - 1.0 / r) / r;
    q[0] = x[0] * s; q[1] = x[1] * s; q[2] = x[2] * s;
}

void synth_contracted_distance(int n_ell, const double* ell_c, const double* ell_M,
                               const double* ell_brad, double plane_rc, int g,
                               double s_max, float* nd) {
    const double hc = 4.0 / g;
    const size_t n = (size_t)g * g * g;
#pragma omp parallel for schedule(static)
    for (size_t v = 0; v < n; ++v) nd[v] = INFINITY;
    /* ground plane q_z = 0: only the two layers next to it can be within s_max */
    int kz0 = (int)floor(g / 2 - s_max - 1), kz1 = (int)ceil(g / 2 + s_max + 1);
    if (kz0 < 0) kz0 = 0;
    if (kz1 > g - 1) kz1 = g - 1;
#pragma omp parallel for schedule(static)
    for (int k = kz0; k <= kz1; ++k)
        for (int j = 0; j < g; ++j)
            for (int i = 0; i < g; ++i) {
                double q[3] = {-2.0 + (i + 0.5) * hc, -2.0 + (j + 0.5) * hc,
                               -2.0 + (k + 0.5) * hc};
                if (dot3(q, q) >= 4.0) continue;
                if (q[0] * q[0] + q[1] * q[1] > plane_rc * plane_rc) continue;
                double d = fabs(q[2]) / hc;
                if (d <= s_max) nd[((size_t)k * g + j) * g + i] = (float)d;
            }
    /* ellipsoids: serial over ellipsoids, parallel over the z-slices of each box */
    for (int e = 0; e < n_ell; ++e) {
        const double* c = ell_c + 3 * e;
        const double* M = ell_M + 9 * e;
        double rc = sqrt(dot3(c, c));
        double rmin = rc - ell_brad[e];
        double L = 1.0;
        if (rmin > 1.0) L = fmax(1.0 / (rmin * rmin), (2.0 - 1.0 / rmin) / rmin);
        double qc[3];
        contract3(c, qc);
        double half = L * ell_brad[e] + (s_max + 2.0) * hc;
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)floor((qc[a] - half + 2.0) / hc);
            hi[a] = (int)floor((qc[a] + half + 2.0) / hc);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > g - 1) hi[a] = g - 1;
        }
        /* M^T M for the world gradient */
        double MtM[9];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s)
                MtM[3 * r + s] = M[r] * M[s] + M[3 + r] * M[3 + s] + M[6 + r] * M[6 + s];
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    double q[3] = {-2.0 + (i + 0.5) * hc, -2.0 + (j + 0.5) * hc,
                                   -2.0 + (k + 0.5) * hc};
                    double rho2 = dot3(q, q);
                    if (rho2 >= 4.0) continue;
                    double rho = sqrt(rho2);
                    double x[3], a = 1.0, beta = 0.0;
                    if (rho <= 1.0) {
                        x[0] = q[0]; x[1] = q[1]; x[2] = q[2];
                    } else {
                        a = 1.0 / (rho * (2.0 - rho));
                        /* d a / d q = -(2 - 2 rho) / (rho (2-rho))^2 * q / rho */
                        beta = -(2.0 - 2.0 * rho) / (rho * rho * (2.0 - rho) * (2.0 - rho) * rho);
                        x[0] = a * q[0]; x[1] = a * q[1]; x[2] = a * q[2];
                    }
                    double dx[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
                    double y[3];
                    matvec3(M, dx, y);
                    double ny = sqrt(dot3(y, y));
                    if (ny == 0.0) continue;
                    double G = ny - 1.0;
                    double gw[3];
                    matvec3(MtM, dx, gw); /* world gradient times |y| */
                    gw[0] /= ny; gw[1] /= ny; gw[2] /= ny;
                    /* J_u^T gw, J_u = a I + beta q q^T (symmetric) */
                    double qg = dot3(q, gw);
                    double gq[3] = {a * gw[0] + beta * q[0] * qg, a * gw[1] + beta * q[1] * qg,
                                    a * gw[2] + beta * q[2] * qg};
                    double ng = sqrt(dot3(gq, gq));
                    if (ng == 0.0) continue;
                    double d = fabs(G) / ng / hc;
                    size_t v = ((size_t)k * g + j) * g + i;
                    if (d <= s_max && d < nd[v]) nd[v] = (float)d;
                }
    }
}

/*
 * Depth tuple of one view (the per-pixel outputs a 2DGS / NeRF renderer hands
 * to the fusion stage in depth-tuple mode, Sec. 3.5): planar depth of the
 * nearest hit (front), planar depth where the ray leaves that primitive
 * (back; = front for planes), number of primitive surfaces the ray crosses
 * over its whole length (2 per ellipsoid it passes through, 1 per plane it
 * hits), and the id of the nearest primitive.  Same scene arguments as
 * synth_render; front/back: H*W float32 (+inf on a miss), cross: H*W int32.
 */
void synth_render_tuple(int n_ell, const double* ell_c, const double* ell_M,
                        const double* ell_brad, const int32_t* ell_id, int n_pl,
                        const double* pl_n, const double* pl_d, const double* pl_rad,
                        const int32_t* pl_id, const double* R, const double* t, double fx,
                        double fy, double cx, double cy, int W, int H, float* front,
                        float* back, int32_t* cross, int32_t* hit) {
    double C[3] = {-(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]),
                   -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]),
                   -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2])};
    int* box = (int*)malloc(sizeof(int) * 4 * (size_t)(n_ell > 0 ? n_ell : 1));
    for (int e = 0; e < n_ell; ++e) {
        double cc[3];
        matvec3(R, ell_c + 3 * e, cc);
        cc[0] += t[0]; cc[1] += t[1]; cc[2] += t[2];
        sphere_bbox(cc, ell_brad[e], fx, fy, cx, cy, W, H, box + 4 * e);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < H; ++j) {
        double* best = (double*)malloc(sizeof(double) * W);
        double* bexit = (double*)malloc(sizeof(double) * W);
        int32_t* nc = cross + (size_t)j * W;
        int32_t* bid = hit + (size_t)j * W;
        for (int i = 0; i < W; ++i) {
            best[i] = INFINITY;
            bexit[i] = INFINITY;
            nc[i] = 0;
            bid[i] = -1;
        }
        double yc = ((double)j + 0.5 - cy) / fy;
        for (int e = 0; e < n_ell; ++e) {
            const int* b = box + 4 * e;
            if (j < b[2] || j > b[3] || b[0] > b[1]) continue;
            for (int i = b[0]; i <= b[1]; ++i) {
                double dc[3] = {((double)i + 0.5 - cx) / fx, yc, 1.0};
                double d[3] = {R[0] * dc[0] + R[3] * dc[1] + R[6] * dc[2],
                               R[1] * dc[0] + R[4] * dc[1] + R[7] * dc[2],
                               R[2] * dc[0] + R[5] * dc[1] + R[8] * dc[2]};
                double t0, t1;
                if (!hit_ellipsoid2(ell_c + 3 * e, ell_M + 9 * e, C, d, &t0, &t1)) continue;
                nc[i] += 2;
                if (t0 < best[i]) { best[i] = t0; bexit[i] = t1; bid[i] = ell_id[e]; }
            }
        }
        for (int p = 0; p < n_pl; ++p) {
            const double* n = pl_n + 3 * p;
            for (int i = 0; i < W; ++i) {
                double dc[3] = {((double)i + 0.5 - cx) / fx, yc, 1.0};
                double d[3] = {R[0] * dc[0] + R[3] * dc[1] + R[6] * dc[2],
                               R[1] * dc[0] + R[4] * dc[1] + R[7] * dc[2],
                               R[2] * dc[0] + R[5] * dc[1] + R[8] * dc[2]};
                double nd = dot3(n, d);
                if (nd == 0.0) continue;
                double th = (pl_d[p] - dot3(n, C)) / nd;
                if (!(th > 0.0)) continue;
                if (pl_rad[p] > 0.0) {
                    double x[3] = {C[0] + th * d[0], C[1] + th * d[1], C[2] + th * d[2]};
                    double off = dot3(n, x);
                    double r2 = dot3(x, x) - off * off;
                    if (r2 > pl_rad[p] * pl_rad[p]) continue;
                }
                nc[i] += 1;
                if (th < best[i]) { best[i] = th; bexit[i] = th; bid[i] = pl_id[p]; }
            }
        }
        for (int i = 0; i < W; ++i) {
            front[(size_t)j * W + i] = (float)best[i];
            back[(size_t)j * W + i] = (float)bexit[i];
        }
        free(best);
        free(bexit);
    }
    free(box);
}
