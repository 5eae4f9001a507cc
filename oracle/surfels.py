"""FP64 statement of the voxel-to-surfel mapping, Passes 2 and 3 (test
infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests/ and the CPU legs of bench.py, never
by the library.  Plain NumPy and Python loops, one function per step
(Sec. 3.6 "Voxel-to-Surfel Mapping and Aggregation"; Algorithm "Voxel-to-
Surfel Mapping for 2DGS"; Appendix "Voxel-to-Surfel Mapping: Implementation
Details"):

  Pass 1 (Eq. pass1): F1 = the seg bit of the surfel's voxel (the label
    lookup of the thick path, oracle.label).
  Pass 2 (Eqs. aspect, needle, pass-needle): a = max(s1, s2) / (min(s1, s2)
    + eps), tau_a = P99(a), F2 = F1 and a <= tau_a.
  Pass 3 (Eqs. cov-atomics, kappa, final-F), per view s in which the bit s
    of the surfel voxel's view mask is set: the tangent semi-axes
    t0 = s1 R[:, 0], t1 = s2 R[:, 1] (R from the unit quaternion), the centre
    c = pi(mu) and the projected tangent vectors alpha_k = (pi(mu + t_k) -
    pi(mu - t_k)) / 2; the 1-sigma box c +- e, e = max(|alpha_0|, |alpha_1|)
    per image axis; for every pixel centre (x + 1/2, y + 1/2) in the box
    (and in frame) the 3-sigma Cramer test: d = pixel - c, u = det(d,
    alpha_1) / det(alpha_0, alpha_1), v = det(alpha_0, d) / det(alpha_0,
    alpha_1), accepted when u^2 + v^2 <= 9; total += 1, mask += 1 where
    M >= tau_M; kappa_s = mask / max(total, 1), kappa = max_s kappa_s;
    F = F2 and kappa >= tau_kappa.

Readings (where the paper is silent):
  - eps = 1e-8; the aspects are formed in FP64 and stored as FP32 (the
    array the selection reads); tau_a is their linear-interpolation P99;
  - quaternions are (w, x, y, z), normalised; the surfel's tangent plane is
    spanned by the rotation's first two columns;
  - alpha_k is the half difference of the two tips' projections (symmetric);
    a view counts only when the centre and the four tips are in front of
    z_near; det(alpha_0, alpha_1) = 0 (edge-on) accepts no pixel;
  - pixel (x, y) covers [x, x + 1) x [y, y + 1) and is visited when its
    centre lies in the closed box; M >= tau_M on the mask probability
    (logits: l >= logit(tau_M));
  - kappa_s >= tau_kappa is decided as mask >= tau_kappa max(total, 1).

Near-boundary flags (the GPU projects in FP32): a visited or bordering
pixel whose u^2 + v^2 lies within 0.02 of 9, a pixel centre within 1e-3
pixel of a box edge, or a tip or centre near z_near may go either way;
such surfels are flagged (the counts are integers, so kappa_s >= tau_kappa
is exact once they agree).

The back-projected overlay (Sec. 3.7 "Iterative Mask Propagation": the
fused 3D mask shown on the next view): each pixel centre unprojected at its
planar depth, x = R^T (((u + 1/2 - cx) / fx) d, ((v + 1/2 - cy) / fy) d, d)
- R^T t in FP64, and the seg bit of its cell floor((q - origin) / h) (q = x,
or contract(x) on a contracted grid; the Pass 1 lookup rule, taken on the
FP64 point); 0 where the depth is not finite and positive or the point is
outside the grid.  Pixels whose (q - origin) / h lies within 1e-6
(relative, as for point labels) of an integer are flagged.

parity: pinned by tests/test_oracle_surfels.py (closed forms for a
fronto-parallel disc, gating, the aspect threshold, a per-pixel brute force
over the whole image, a constructed overlay, planted mistakes).
"""
from __future__ import annotations

import math

import numpy as np

from .weighting import mask_probability, percentile_linear

EPS_ASPECT = 1e-8


def quat_to_rot(q) -> np.ndarray:
    """Rotation matrix of the quaternion (w, x, y, z) (normalised first)."""
    w, x, y, z = (float(v) for v in q)
    n = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / n, x / n, y / n, z / n
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def aspects(scales: np.ndarray) -> np.ndarray:
    """Eq. aspect in FP64, stored as FP32."""
    s = np.asarray(scales, np.float32).astype(np.float64)
    return (np.maximum(s[:, 0], s[:, 1]) / (np.minimum(s[:, 0], s[:, 1]) + EPS_ASPECT)).astype(np.float32)


def _project(cam, X):
    p = np.asarray(cam.R, np.float64) @ X + np.asarray(cam.t, np.float64)
    return p, np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


def surfel_view_counts(mu, s, q, cam, mask_p, tau_m=0.5, z_near=1e-6):
    """(total, mask, flagged) of one surfel in one view (Pass 3 (ii)-(iv))."""
    R = quat_to_rot(q)
    m = np.asarray(mu, np.float32).astype(np.float64)
    t0 = float(np.float32(s[0])) * R[:, 0]
    t1 = float(np.float32(s[1])) * R[:, 1]
    pts = [m, m + t0, m - t0, m + t1, m - t1]
    proj = [_project(cam, X) for X in pts]
    flag = False
    for p, _ in proj:
        if abs(p[2] - z_near) < 1e-6 * (abs(p[2]) + 1.0):
            flag = True
        if not p[2] > z_near:
            return 0, 0, flag
    c = proj[0][1]
    a0 = 0.5 * (proj[1][1] - proj[2][1])
    a1 = 0.5 * (proj[3][1] - proj[4][1])
    det = a0[0] * a1[1] - a0[1] * a1[0]
    if det == 0.0:
        return 0, 0, True
    ex = max(abs(a0[0]), abs(a1[0]))
    ey = max(abs(a0[1]), abs(a1[1]))
    x0, x1 = math.ceil(c[0] - ex - 0.5), math.floor(c[0] + ex - 0.5)
    y0, y1 = math.ceil(c[1] - ey - 0.5), math.floor(c[1] + ey - 0.5)
    for e in (c[0] - ex - 0.5, c[0] + ex - 0.5, c[1] - ey - 0.5, c[1] + ey - 0.5):
        if abs(e - round(e)) < 1e-3:
            flag = True
    total = msk = 0
    H, W = mask_p.shape
    for y in range(max(y0, 0), min(y1, H - 1) + 1):
        for x in range(max(x0, 0), min(x1, W - 1) + 1):
            dx, dy = x + 0.5 - c[0], y + 0.5 - c[1]
            u = (dx * a1[1] - dy * a1[0]) / det
            v = (a0[0] * dy - a0[1] * dx) / det
            r2 = u * u + v * v
            if abs(r2 - 9.0) < 0.02:
                flag = True
            if r2 <= 9.0:
                total += 1
                if mask_p[y, x] >= tau_m:
                    msk += 1
    return total, msk, flag


def surfel_labels(mu, scales, quats, F1, voxel_bits, cams, masks, mask_type, tau_m=0.5,
                  tau_kappa=0.5, z_near=1e-6):
    """Passes 2 and 3 given Pass 1 (F1) and each surfel's voxel view mask
    (voxel_bits, 0 where the voxel is not active): F2, F, kappa, tau_a and
    the per-surfel flags."""
    a = aspects(scales)
    tau_a = percentile_linear(a, 0.99)
    F2 = np.asarray(F1, bool) & (a <= np.float32(tau_a))
    probs = []
    for mk in masks:
        p = mask_probability(mk, mask_type)
        if mask_type == 2:  # logits gate as l >= logit(tau_M), exactly
            lt = np.float32(math.log(tau_m / (1.0 - tau_m)))
            p = np.where(np.asarray(mk, np.float32) >= lt, 1.0, 0.0)
        probs.append(p)
    thr = 1.0 if mask_type == 2 else tau_m
    kappa = np.zeros(len(a))
    keep = np.zeros(len(a), bool)
    flags = np.zeros(len(a), bool)
    for i in np.nonzero(F2)[0]:
        for sidx, cam in enumerate(cams):
            if not (int(voxel_bits[i]) >> sidx) & 1 or sidx >= 32:
                continue
            tot, msk, fl = surfel_view_counts(mu[i], scales[i], quats[i], cam, probs[sidx],
                                              thr, z_near)
            flags[i] |= fl
            kappa[i] = max(kappa[i], msk / max(tot, 1))
            if msk >= tau_kappa * max(tot, 1):
                keep[i] = True
    return {"F2": F2, "F": F2 & keep, "kappa": kappa, "tau_a": tau_a, "flags": flags}


def overlay(grid, seg_dense, cam, depth):
    """The overlay of one view: (uint8 H x W, the near-boundary flags per pixel)."""
    D = np.asarray(depth, np.float32).astype(np.float64)
    H, W = D.shape
    ys, xs = np.mgrid[0:H, 0:W]
    ok = np.isfinite(D) & (D > 0)
    Dz = np.where(ok, D, 1.0)
    pc = np.stack([((xs + 0.5 - float(cam.cx)) / float(cam.fx)) * Dz,
                   ((ys + 0.5 - float(cam.cy)) / float(cam.fy)) * Dz, Dz], axis=-1).reshape(-1, 3)
    R = np.asarray(cam.R, np.float32).astype(np.float64).reshape(3, 3)
    t = np.asarray(cam.t, np.float32).astype(np.float64)
    X = (pc - t) @ R                              # R^T (p_c - t), row vectors
    if getattr(grid, "contracted", False):        # contract(x) = (2 - 1/|x|) x / |x|
        r = np.sqrt((X * X).sum(axis=1))
        sc = np.where(r > 1.0, (2.0 - 1.0 / np.where(r > 1.0, r, 1.0)) / np.where(r > 1.0, r, 1.0),
                      1.0)
        X = X * sc[:, None]
    g = int(grid.g)
    h = float(np.float32(grid.h))
    org = np.asarray(grid.origin, np.float32).astype(np.float64)
    s = (X - org) / h
    f = s - np.floor(s)
    near = np.any(np.minimum(f, 1.0 - f) < 1e-6 * np.maximum(1.0, np.abs(s)), axis=1)
    inside = np.all((s >= 0.0) & (s < g), axis=1) & ok.ravel()
    idx = np.where(inside[:, None], np.floor(s), 0).astype(np.int64)
    seg = np.asarray(seg_dense, np.uint8).ravel()
    lab = np.where(inside, seg[(idx[:, 2] * g + idx[:, 1]) * g + idx[:, 0]], 0).astype(np.uint8)
    fl = np.where(ok.ravel(), near, False).astype(np.uint32)
    return lab.reshape(H, W), fl.reshape(H, W)
