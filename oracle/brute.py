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


def _mask_prob(mask, mask_type):
    """Per-pixel probability and the strict half test, as float64 arrays."""
    if mask_type == 1:    # binary16 bits
        m = mask.view(np.float16).astype(np.float64) if mask.dtype != np.float16 \
            else mask.astype(np.float64)
        return m, m > 0.5
    if mask_type == 2:    # logits
        lg = mask.astype(np.float64)
        return 1.0 / (1.0 + np.exp(-lg)), lg > 0.0
    m = mask.astype(np.float64)
    return m, m > 0.5


def fuse_tuple(grid, lin, cams, tup, masks, mask_type, tau_m=0.5, gamma=1.0, alpha1=0.5,
               tau_cons=0.5, eps=1e-12, z_near=1e-6, beta=0.05, gamma_st=1.5, tau_thin=0.6,
               rho_cover=0.5, rho_occ=0.1, n_abs=25.0, dist_gate=1.5, behind_margin=2.0,
               k_dg=0.0, rho_thin=1.0, rho=None):
    """Depth-tuple-mode fusion written out per voxel and view with NumPy
    slices (Sec. 3.5, Algorithms "Thick-Structure Segmentation for 2DGS" and
    "Thin-Structure Segmentation for 2DGS", App. B.5): footprint statistics
    by summing the footprint slice (no integral image), the layered test as
    n > mean + std in float64, the ray geometry through explicit vectors
    (camera centre, unit ray direction, closest clamped point), unprojection
    through the inverse intrinsics.  Small inputs only (a Python loop).

    Returns W, Z, P, seg, bits, kind (n x views: 0 / 1 thick / 2 thin)."""
    x, hvs, ok = voxel_centres(grid, lin)
    n_v = len(cams)
    N = len(lin)
    W = np.zeros(N)
    Z = np.zeros(N)
    bits = np.zeros(N, np.uint32)
    kind = np.zeros((N, n_v), np.uint8)
    logit_tau = -np.inf if tau_m <= 0 else (np.inf if tau_m >= 1 else
                                            float(np.float32(np.log(tau_m / (1 - tau_m)))))
    per_view = []
    for i, cam in enumerate(cams):
        R = np.asarray(cam.R, np.float32).astype(np.float64).reshape(3, 3)
        t = np.asarray(cam.t, np.float32).astype(np.float64)
        o = -R.T @ t
        mprob, mhalf = _mask_prob(np.asarray(masks[i]), mask_type)
        raw = np.asarray(masks[i])
        if mask_type == 1:
            gate = mprob >= tau_m
        elif mask_type == 2:
            gate = raw.astype(np.float64) >= logit_tau
        else:
            gate = mprob >= tau_m
        dmin = tup["d_min"][i].astype(np.float64)
        dmax = tup["d_max"][i].astype(np.float64)
        cen = 0.5 * (dmin + dmax)
        cp = np.pad(cen, 1, mode="edge")
        gx = cp[1:-1, 2:] - cp[1:-1, :-2]
        gy = cp[2:, 1:-1] - cp[:-2, 1:-1]
        fin = np.isfinite(cp[1:-1, 2:]) & np.isfinite(cp[1:-1, :-2]) & \
            np.isfinite(cp[2:, 1:-1]) & np.isfinite(cp[:-2, 1:-1])
        with np.errstate(invalid="ignore", over="ignore"):
            pig = np.where(fin, np.exp(-k_dg * (gx * gx + gy * gy)), 0.0) if k_dg else \
                np.ones_like(cen)
        per_view.append((R, t, o, mprob, mhalf, gate, dmin, tup["d_med"][i].astype(np.float64),
                         dmax, tup["n_samp"][i].astype(np.int64), pig,
                         float(np.float32(tup["d_cam"][i]))))
    signs = np.array([[sx, sy, sz] for sz in (-0.5, 0.5) for sy in (-0.5, 0.5)
                      for sx in (-0.5, 0.5)])
    for a in range(N):
        if not ok[a]:
            continue
        hv = hvs[a]
        xc = x[a]
        rv = 1.0 if rho is None else float(rho[a])
        for i, cam in enumerate(cams):
            R, t, o, mprob, mhalf, gate, dmin, dmed, dmax, ns, pig, dcam = per_view[i]
            fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
            pc = R @ xc + t
            corners = R @ (xc[None, :] + signs * hv).T + t[:, None]
            if pc[2] <= z_near or np.any(corners[2] <= z_near):
                continue
            u = fx * pc[0] / pc[2] + cx
            v = fy * pc[1] / pc[2] + cy
            if not (0 <= u < cam.W and 0 <= v < cam.H):
                continue
            cu = fx * corners[0] / corners[2] + cx
            cv = fy * corners[1] / corners[2] + cy
            i0, i1 = max(int(np.floor(cu.min())), 0), min(int(np.floor(cu.max())), cam.W - 1)
            j0, j1 = max(int(np.floor(cv.min())), 0), min(int(np.floor(cv.max())), cam.H - 1)
            area = (min(cu.max(), cam.W) - max(cu.min(), 0.0)) * \
                (min(cv.max(), cam.H) - max(cv.min(), 0.0))
            fp = ns[j0:j1 + 1, i0:i1 + 1].astype(np.float64)
            mean = fp.mean()
            std = np.sqrt(max((fp * fp).mean() - mean * mean, 0.0))
            ix, iy = int(np.floor(u)), int(np.floor(v))
            d_lo, d_me, d_hi, n_c = dmin[iy, ix], dmed[iy, ix], dmax[iy, ix], ns[iy, ix]
            trusted = d_lo <= d_me
            seethru = d_me > gamma_st * dcam
            front = (n_c > mean + std or seethru) and trusted
            xd = pc[2]
            dist = np.linalg.norm(xc - o)
            dhat = (xc - o) / dist
            cos = float(R[2] @ dhat)
            voted = False
            if gate[iy, ix] and trusted and all(np.isfinite([d_lo, d_me, d_hi])) and \
                    min(d_lo, d_me, d_hi) > 0:
                ref = d_lo if front else d_me
                th = min(max(dist, d_lo / cos), ref / cos)
                closest = o + th * dhat
                tdep = gamma * hv / (1.0 + beta * max(n_c - mean, 0.0))
                ok_d = (xd - d_lo <= tdep) if front else (abs(xd - d_me) <= tdep)
                if np.linalg.norm(xc - closest) <= hv * pig[iy, ix] and ok_d:
                    ctr = 0.5 * (d_lo + d_hi) / cos
                    hw = max(0.5 * (d_hi - d_lo) / cos, eps)
                    w = np.exp(-alpha1 * ((th - ctr) / hw) ** 2)
                    W[a] += mprob[iy, ix] * w
                    Z[a] += w
                    bits[a] |= np.uint32(1 << i) if i < 32 else np.uint32(0)
                    kind[a, i] = 1
                    voted = True
            surf = d_lo if (trusted and seethru) else d_me
            if voted or xd > surf + behind_margin * hv or not (rv >= rho_thin):
                continue
            n_depth = n_md = 0
            m_max = 0.0
            d2 = np.inf
            Kinv = np.array([[1 / fx, 0, -cx / fx], [0, 1 / fy, -cy / fy], [0, 0, 1]])
            for yy in range(j0, j1 + 1):
                for xx in range(i0, i1 + 1):
                    q_lo, q_me, nq = dmin[yy, xx], dmed[yy, xx], ns[yy, xx]
                    if q_me < eps:
                        continue
                    tq = gamma * hv / (1.0 + beta * max(nq - mean, 0.0))
                    fq = (nq > mean + std or q_me > gamma_st * dcam) and q_lo <= q_me
                    ok_q = (xd - q_lo <= tq) if fq else (abs(xd - q_me) <= tq)
                    if not ok_q:
                        continue
                    n_depth += 1
                    if not mhalf[yy, xx]:
                        continue
                    n_md += 1
                    m_max = max(m_max, mprob[yy, xx])
                    dq = q_lo if fq else q_me
                    pcam = Kinv @ np.array([xx + 0.5, yy + 0.5, 1.0]) * dq
                    pw = R.T @ (pcam - t)
                    d2 = min(d2, float(np.sum((pw - xc) ** 2)))
            tt = m_max if (n_depth >= max(n_abs, np.ceil(rho_occ * area)) and
                           n_md >= rho_cover * n_depth and d2 <= (dist_gate * hv) ** 2) else 0.0
            if tt >= tau_thin:
                W[a] += tt
                Z[a] += 1.0
                bits[a] |= np.uint32(1 << i) if i < 32 else np.uint32(0)
                kind[a, i] = 2
    P = np.where(Z > eps, W / np.where(Z > eps, Z, 1.0), 0.0)
    return dict(W=W, Z=Z, P=P, seg=(P >= tau_cons).astype(np.uint8), bits=bits, kind=kind)


def fuse_nerf(grid, lin, cams, tup, masks, mask_type, rho=None, tau_m=0.5, alpha1=0.5,
              tau_cons=0.5, eps=1e-12, z_near=1e-6, gamma=4.0, beta=0.2, b_max=10.0,
              lambda_range=0.05, rho_thin=50.0, rho_cover=0.2, tau_thin=0.6, m_thin=0.1,
              k_dg=0.0):
    """NeRF-variant fusion written out per voxel and view in ray space
    (appendix "NeRF-Backbone 3D Fusion Details", Algorithms "Thick-Structure
    Segmentation via Depth-Weighted Voxel Aggregation" and "Thin-Structure
    Segmentation via Footprint-Based Coverage Analysis"): the centre pixel's
    ray as the camera centre o and a unit world direction d through the pixel
    centre, the planar band [d_min, d_max] turned into the ray segment
    [d_min, d_max] / cos theta, the projection t_proj = <x_c - o, d> clamped
    to it, the closest point o + t_c d and its distance; the weight from the
    ray-space mid-point and half-width; the thin path's footprint as a NumPy
    slice of the box of the eight projected corners.  Small inputs only.

    Returns W, Z, P, seg, bits, kind (n x views: 0 / 1 thick / 2 thin)."""
    x, hvs, ok = voxel_centres(grid, lin)
    n_v = len(cams)
    N = len(lin)
    W = np.zeros(N)
    Z = np.zeros(N)
    bits = np.zeros(N, np.uint32)
    kind = np.zeros((N, n_v), np.uint8)

    def logit32(p):
        return -np.inf if p <= 0 else (np.inf if p >= 1 else
                                       float(np.float32(np.log(p / (1 - p)))))
    per_view = []
    for i, cam in enumerate(cams):
        R = np.asarray(cam.R, np.float32).astype(np.float64).reshape(3, 3)
        t = np.asarray(cam.t, np.float32).astype(np.float64)
        mprob, mhalf = _mask_prob(np.asarray(masks[i]), mask_type)
        raw = np.asarray(masks[i]).astype(np.float64)
        if mask_type == 2:
            gate, elig = raw >= logit32(tau_m), raw > logit32(m_thin)
        else:
            gate, elig = mprob >= tau_m, mprob > m_thin
        dmin = tup["d_min"][i].astype(np.float64)
        dmax = tup["d_max"][i].astype(np.float64)
        cen = 0.5 * (dmin + dmax)
        cp = np.pad(cen, 1, mode="edge")
        gx = cp[1:-1, 2:] - cp[1:-1, :-2]
        gy = cp[2:, 1:-1] - cp[:-2, 1:-1]
        fin = np.isfinite(cp[1:-1, 2:]) & np.isfinite(cp[1:-1, :-2]) & \
            np.isfinite(cp[2:, 1:-1]) & np.isfinite(cp[:-2, 1:-1])
        with np.errstate(invalid="ignore", over="ignore"):
            pig = np.where(fin, np.exp(-k_dg * (gx * gx + gy * gy)), 0.0) if k_dg else \
                np.ones_like(cen)
        per_view.append((R, t, -R.T @ t, mprob, mhalf, gate, elig, dmin,
                         tup["d_exp"][i].astype(np.float64), dmax,
                         tup["n_samp"][i].astype(np.int64), pig))
    signs = np.array([[sx, sy, sz] for sz in (-0.5, 0.5) for sy in (-0.5, 0.5)
                      for sx in (-0.5, 0.5)])
    for a in range(N):
        if not ok[a]:
            continue
        hv = hvs[a]
        xc = x[a]
        rv = 1.0 if rho is None else float(rho[a])
        for i, cam in enumerate(cams):
            R, t, o, mprob, mhalf, gate, elig, dmin, dexp, dmax, ns, pig = per_view[i]
            fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
            pc = R @ xc + t
            if pc[2] <= z_near:
                continue
            u = fx * pc[0] / pc[2] + cx
            v = fy * pc[1] / pc[2] + cy
            if not (0 <= u < cam.W and 0 <= v < cam.H):
                continue
            ix, iy = int(np.floor(u)), int(np.floor(v))
            xd = pc[2]
            voted = False
            lo, ex, hi, nc = dmin[iy, ix], dexp[iy, ix], dmax[iy, ix], ns[iy, ix]
            if gate[iy, ix] and np.all(np.isfinite([lo, ex, hi])) and min(lo, ex, hi) > 0:
                kcam = np.array([(ix + 0.5 - cx) / fx, (iy + 0.5 - cy) / fy, 1.0])
                sec = np.linalg.norm(kcam)           # 1 / cos(theta)
                d = R.T @ (kcam / sec)               # unit world direction
                t_proj = float(np.dot(xc - o, d))
                t_c = min(max(t_proj, lo * sec), hi * sec)
                delta = np.linalg.norm(xc - (o + t_c * d))
                tau_sp = hv * pig[iy, ix] + lambda_range * (hi - lo) * sec
                b = min(beta * nc, b_max)
                if delta <= tau_sp and abs(xd - ex) <= (gamma + b) * hv:
                    mu = 0.5 * (lo + hi) * sec
                    hd = max(0.5 * (hi - lo) * sec, eps * sec)
                    w = np.exp(-alpha1 * ((t_c - mu) / hd) ** 2)
                    W[a] += mprob[iy, ix] * w
                    Z[a] += w
                    bits[a] |= np.uint32(1 << i) if i < 32 else np.uint32(0)
                    kind[a, i] = 1
                    voted = True
            if voted or not elig[iy, ix] or not (rv >= rho_thin):
                continue
            corners = R @ (xc[None, :] + signs * hv).T + t[:, None]
            if np.any(corners[2] <= z_near):
                continue
            cu = fx * corners[0] / corners[2] + cx
            cv = fy * corners[1] / corners[2] + cy
            i0, i1 = max(int(np.floor(cu.min())), 0), min(int(np.floor(cu.max())), cam.W - 1)
            j0, j1 = max(int(np.floor(cv.min())), 0), min(int(np.floor(cv.max())), cam.H - 1)
            box = (slice(j0, j1 + 1), slice(i0, i1 + 1))
            tol = (2.0 * gamma + np.minimum(beta * ns[box], b_max)) * hv
            with np.errstate(invalid="ignore"):
                support = mhalf[box] & (np.abs(xd - dexp[box]) <= tol)
            m_max = float(mprob[box].max())
            tt = m_max if support.sum() >= rho_cover * support.size else 0.0
            if tt >= tau_thin:
                W[a] += tt
                Z[a] += 1.0
                bits[a] |= np.uint32(1 << i) if i < 32 else np.uint32(0)
                kind[a, i] = 2
    P = np.where(Z > eps, W / np.where(Z > eps, Z, 1.0), 0.0)
    return dict(W=W, Z=Z, P=P, seg=(P >= tau_cons).astype(np.uint8), bits=bits, kind=kind)
