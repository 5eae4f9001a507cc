"""Independent NumPy brute force of the thick-path fusion (test infrastructure).

TEST INFRASTRUCTURE ONLY.  A second, separately written FP64 statement of
the same rule as ``oracle.c`` (Sec. 3.5, Eq. compact-fusion, Eq.
gs-depthweight, Eq. vmask), used to pin the C oracle.  It differs from the
oracle in where the depth comes from: instead of reading the stored FP32
depth raster it re-casts the ray through the centre of the pixel the voxel
projects to and intersects it analytically with the scene's spheres,
ellipsoids and planes (planar depth: the ray direction has camera-z 1).

It also flags voxels whose pixel ray grazes a surface (near-zero
discriminant) or nearly ties between two surfaces, where the stored raster
and the analytic cast can disagree on which surface was hit.
"""
from __future__ import annotations

import numpy as np


def voxel_centres(grid, lin):
    """World centres (N, 3) and world edges (N,) of voxels with linear indices lin.

    Returns also a boolean array, False where a contracted centre has
    |c| >= 2 (no world position)."""
    g = int(grid.g)
    lin = np.asarray(lin, np.int64)
    idx = np.stack([lin % g, (lin // g) % g, lin // (g * g)], axis=1).astype(np.float64)
    o = np.asarray(grid.origin, np.float32).astype(np.float64)
    h = float(np.float32(grid.h))
    c = o + (idx + 0.5) * h
    ok = np.ones(len(lin), bool)
    hv = np.full(len(lin), h)
    if not grid.contracted:
        return c, hv, ok
    rho = np.linalg.norm(c, axis=1)
    ok = rho < 2.0
    outer = (rho > 1.0) & ok
    x = c.copy()
    s = np.ones_like(rho)
    s[outer] = 1.0 / (rho[outer] * (2.0 - rho[outer]))
    x = c * s[:, None]
    hv[outer] = h / (2.0 - rho[outer]) ** 2
    return x, hv, ok


def cast(scene, C, d):
    """Nearest positive hit parameter t (inf on a miss), hit id (-1), and a
    boolean 'ambiguous' (grazing or near tie) for rays C + t d (d: (N, 3))."""
    n = len(d)
    best = np.full(n, np.inf)
    second = np.full(n, np.inf)
    bid = np.full(n, -1, np.int64)
    graze = np.zeros(n, bool)
    for e in range(len(scene.ell_c)):
        A_inv = np.diag(1.0 / scene.ell_axes[e])
        M = A_inv @ scene.ell_rot[e].T
        op = M @ (C - scene.ell_c[e])
        dp = d @ M.T
        a = np.einsum("ij,ij->i", dp, dp)
        b = 2.0 * dp @ op
        q = op @ op - 1.0
        disc = b * b - 4.0 * a * q
        hit = (disc >= 0.0) & (b < 0.0) & (q > 0.0)
        with np.errstate(invalid="ignore", divide="ignore"):
            t = np.where(hit, 2.0 * q / (-b + np.sqrt(np.maximum(disc, 0.0))), np.inf)
        graze |= np.abs(disc) < 1e-9 * (b * b + 1e-300)
        closer = t < best
        second = np.where(closer, best, np.minimum(second, t))
        bid = np.where(closer, scene.ell_id[e], bid)
        best = np.where(closer, t, best)
    for p in range(len(scene.pl_d)):
        nrm = scene.pl_n[p]
        nd = d @ nrm
        with np.errstate(invalid="ignore", divide="ignore"):
            t = (scene.pl_d[p] - nrm @ C) / nd
        t = np.where((nd != 0.0) & (t > 0.0), t, np.inf)
        if scene.pl_rad[p] > 0:
            x = C + np.where(np.isfinite(t), t, 0.0)[:, None] * d
            off = x @ nrm
            r2 = np.einsum("ij,ij->i", x, x) - off * off
            t = np.where(np.isfinite(t) & (r2 <= scene.pl_rad[p] ** 2), t, np.inf)
        closer = t < best
        second = np.where(closer, best, np.minimum(second, t))
        bid = np.where(closer, scene.pl_id[p], bid)
        best = np.where(closer, t, best)
    with np.errstate(invalid="ignore"):
        tie = np.isfinite(second) & (np.abs(second - best) < 1e-7 * np.maximum(best, 1.0))
    return best, bid, graze | tie


def fuse(grid, lin, cams, masks, scene, tau_m=0.5, gamma=1.0, alpha1=0.5, tau_cons=0.5,
         eps=1e-12, z_near=1e-6, mask_kind="f32"):
    """Brute-force fusion with analytic depth.  ``masks`` are the stored mask
    rasters (float32 probabilities, or binary16 bits with mask_kind='f16').

    Returns dict(W, Z, P, seg, bits, ambiguous, pix) with float64 scores."""
    x, hv, ok = voxel_centres(grid, lin)
    n = len(x)
    W = np.zeros(n)
    Z = np.zeros(n)
    bits = np.zeros(n, np.uint64)
    amb = np.zeros(n, bool)
    pix_all = np.full((n, len(cams)), -1, np.int64)
    for i, cam in enumerate(cams):
        R = np.asarray(cam.R, np.float32).astype(np.float64)
        t = np.asarray(cam.t, np.float32).astype(np.float64)
        p = x @ R.T + t
        front = ok & (p[:, 2] > z_near)
        with np.errstate(invalid="ignore", divide="ignore"):
            u = cam.fx * (p[:, 0] / p[:, 2]) + cam.cx
            v = cam.fy * (p[:, 1] / p[:, 2]) + cam.cy
        inside = front & (u >= 0) & (u < cam.W) & (v >= 0) & (v < cam.H)
        sel = np.flatnonzero(inside)
        ix = np.floor(u[sel]).astype(np.int64)
        iy = np.floor(v[sel]).astype(np.int64)
        pix_all[sel, i] = iy * cam.W + ix
        # ray through the pixel centre, planar parameterisation (camera-z = 1)
        dc = np.stack([(ix + 0.5 - cam.cx) / cam.fx, (iy + 0.5 - cam.cy) / cam.fy,
                       np.ones(len(sel))], axis=1)
        dw = dc @ R
        C = -R.T @ t
        D, _, ambig = cast(scene, C, dw)
        amb[sel] |= ambig
        mk = np.asarray(masks[i])
        if mask_kind == "f16":
            m = mk.view(np.float16).astype(np.float64)[iy, ix]
        else:
            m = mk.astype(np.float64)[iy, ix]
        valid = np.isfinite(D) & (D > 0) & (m >= tau_m)
        Delta = gamma * hv[sel]
        e = p[sel, 2] - D
        acc = valid & (np.abs(e) <= Delta)
        r = np.where(acc, e / Delta, 0.0)
        w = np.exp(-alpha1 * r * r)
        s2 = sel[acc]
        W[s2] += m[acc] * w[acc]
        Z[s2] += w[acc]
        if i < 32:
            bits[s2] |= np.uint64(1 << i)
    P = np.where(Z > eps, W / np.where(Z > eps, Z, 1.0), 0.0)
    seg = (P >= tau_cons).astype(np.uint8)
    return dict(W=W, Z=Z, P=P, seg=seg, bits=bits.astype(np.uint32), ambiguous=amb,
                pix=pix_all)


def label(grid, seg_dense, xyz):
    """Per-point Pass 1 lookup, one point at a time (brute force)."""
    g = int(grid.g)
    o = np.asarray(grid.origin, np.float32).astype(np.float64)
    h = float(np.float32(grid.h))
    out = np.zeros(len(xyz), np.uint8)
    for a, pt in enumerate(np.asarray(xyz, np.float32).astype(np.float64)):
        if np.isnan(pt).any():
            continue
        q = pt
        if grid.contracted:
            r = float(np.sqrt(pt @ pt))
            if r > 1.0:
                q = (2.0 - 1.0 / r) * pt / r
        s = (q - o) / h
        if np.any(s < 0) or np.any(s >= g):
            continue
        i, j, k = (int(np.floor(c)) for c in s)
        out[a] = seg_dense[(k * g + j) * g + i]
    return out
