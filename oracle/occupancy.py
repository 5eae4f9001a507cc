"""FP64 statement of the 2DGS occupancy construction (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests/ and the CPU legs of bench.py, never
by the library.  Plain NumPy, one function per step (Sec. 3.5 "Occupancy by
Morton-scattered opacity"; Appendix "Occupancy grid construction"):

  Eq. scene-norm:  c = median_i(mu_i) (coordinate-wise),
                   r_fg = P99(|mu_i - c|),  b = ceil(1.05 r_fg)
  Eq. voxel-size:  h_v = max(alpha_v s_bar, beta_v r_scene / g0),
                   (alpha_v, beta_v, g0) = (3, 1, 256); g = the smallest power
                   of two with g >= 2 b / h_v, capped at g_max
  AABB filter to the cube c +- b; voxel index floor((mu - c + b) / h_v);
  rho[voxel] += alpha_i (opacity scatter-add); active = {rho >= tau_TF},
  tau_TF = 0.5.

Readings (where the paper is silent):
  - medians and P99 are the linear-interpolation quantile of
    oracle.weighting.percentile_linear (the median of an even count is the
    mean of the two middle values);
  - the radial distances are formed in FP64 from the FP32 centres and the
    FP64 centre c, (dx dx + dy dy) + dz dz, square-rooted, then stored as
    FP32 (the array a device selection reads); r_fg is their P99;
  - s_bar is the median over surfels of their larger scale max(s_u, s_v)
    (the "median Gaussian footprint" of the hyper-parameter table);
  - r_scene = r_fg (the robust scene radius);
  - b = max(ceil(1.05 r_fg), 1) (an integer number of world units, at least
    one);
  - when the cap binds (2 b / h_v > g_max), h_v = 2 b / g_max so that the
    grid still covers the cube;
  - the cube is half-open, c - b <= mu < c + b per axis; the index is
    clamped to g - 1 (only rounding can reach g);
  - the voxel order of the result is the linear one (x fastest); the paper's
    Morton order is a memory layout of the same set;
  - rho >= tau_TF is inclusive.

Near-boundary flags: a voxel whose FP64 opacity sum lies within
2^-22 n sum|alpha| of tau_TF (n surfels; an FP32 sum of n terms in any order
is that close) may go either way on the GPU.

parity: pinned by tests/test_oracle_occupancy.py (closed forms of the frame
rules on constructed clouds, a brute-force per-voxel sum, translation
invariance, planted mistakes).
"""
from __future__ import annotations

import math

import numpy as np

from .weighting import percentile_linear

DEFAULTS = {"alpha_v": 3.0, "beta_v": 1.0, "g0": 256, "g_max": 512, "pad": 1.05, "tau_tf": 0.5}


def radial_distances(mu: np.ndarray, c) -> np.ndarray:
    """|mu_i - c| in FP64, stored as FP32."""
    m = np.asarray(mu, np.float32).astype(np.float64)
    dx, dy, dz = m[:, 0] - c[0], m[:, 1] - c[1], m[:, 2] - c[2]
    return np.sqrt((dx * dx + dy * dy) + dz * dz).astype(np.float32)


def scene_frame(mu: np.ndarray, scales: np.ndarray, alpha_v=3.0, beta_v=1.0, g0=256, g_max=512,
                pad=1.05) -> dict:
    """Eqs. scene-norm and voxel-size: the grid's frame from the surfel cloud."""
    mu = np.asarray(mu, np.float32)
    c = [percentile_linear(mu[:, a], 0.5) for a in range(3)]
    r_fg = percentile_linear(radial_distances(mu, c), 0.99)
    b = max(math.ceil(pad * r_fg), 1)
    smax = np.maximum(np.asarray(scales, np.float32)[:, 0], np.asarray(scales, np.float32)[:, 1])
    s_bar = percentile_linear(smax, 0.5)
    h = max(alpha_v * s_bar, beta_v * r_fg / g0)
    need = 2.0 * b / h
    g = 1
    while g < need and g < g_max:
        g *= 2
    if need > g_max:
        g = g_max
        h = 2.0 * b / g_max
    return {"c": c, "r_fg": r_fg, "b": float(b), "s_bar": s_bar, "h": h, "g": g,
            "origin": [c[a] - b for a in range(3)]}


def occupancy(mu: np.ndarray, alpha: np.ndarray, frame: dict, tau_tf: float = 0.5) -> dict:
    """AABB filter, voxel index, opacity scatter-add, tau_TF floor: the dense
    active mask (g^3, x fastest), the FP64 density, per-voxel counts and the
    near-threshold flags."""
    m = np.asarray(mu, np.float32).astype(np.float64)
    a = np.asarray(alpha, np.float32).astype(np.float64)
    c, b, h, g = frame["c"], frame["b"], frame["h"], frame["g"]
    x = np.stack([m[:, k] - c[k] + b for k in range(3)], axis=1)
    keep = np.all((x >= 0.0) & (x < 2.0 * b), axis=1)
    idx = np.minimum(np.floor(x[keep] / h).astype(np.int64), g - 1)
    lin = (idx[:, 2] * g + idx[:, 1]) * g + idx[:, 0]
    rho = np.bincount(lin, weights=a[keep], minlength=g ** 3)
    cnt = np.bincount(lin, minlength=g ** 3)
    mag = np.bincount(lin, weights=np.abs(a[keep]), minlength=g ** 3)
    active = rho >= tau_tf
    near = (cnt > 0) & (np.abs(rho - tau_tf) <= 2.0 ** -22 * cnt * mag + 1e-30)
    return {"active": active, "rho": rho, "count": cnt, "near": near, "n_kept": int(keep.sum())}
