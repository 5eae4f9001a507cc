"""FP64 statement of the depth-weighted mask refinement (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU legs of
bench.py, never by the library.  Plain NumPy, no blocking or reordering, one
function per equation:

  Eq. nerf-depthweight (Sec. 3.4, "Depth-weighting: bounded normalization
  (NeRF) vs. band-pass (2DGS)"):
      M~ = M (1 - Z^),  Z^ = (D_exp - min D_exp) / (max D_exp - min D_exp)

  Eq. depthband and Eq. gs-bandpass (same paragraph):
      D_s = {D_med at every positive prompt} U {D_med at the view centre},
      d_min = min D_s, d_max = max D_s, d_far = P98(D_med),
      Delta- = max(d_min - D_med, 0), Delta+ = max(D_med - d_max, 0),
      D_band = clip((Delta- + Delta+) / max(d_far - d_max, 1e-6), 0, 1),
      M~ = M (1 - D_band)

Readings (where the paper is silent):
  - M is the mask probability: binary16 and FP32 masks as given, logits
    through the sigmoid; M~ is an FP32-representable probability.
  - Non-finite depth means no surface: M~ = 0 there, and such pixels take
    no part in min / max / the percentile.  NaN and +-inf alike.
  - min / max / P98 run over the finite pixels of the raster; with no finite
    pixel, or max == min, Z^ = 0 on the finite pixels.
  - P98 is the linear-interpolation percentile (Hyndman and Fan type 7):
    s the ascending finite values, r = 0.98 (n - 1), k = floor(r),
    P98 = s[k] + (r - k) (s[k + 1] - s[k]) (s[k] when k + 1 = n).
  - The view centre is pixel (floor(W / 2), floor(H / 2)); a prompt is a
    pixel (x, y); samples with non-finite depth are dropped; with no finite
    sample there is no band and the weight is 1 on finite pixels.
  - With no finite pixel at all, d_far = d_max (the floored denominator).

parity: pinned by tests/test_oracle_weighting.py (closed forms at the band
edges, at d_far and at the raster's min / max; the percentile of
permutations and of repeated values against its order-statistic definition
and the mean of the two middle values).
"""
from __future__ import annotations

import math

import numpy as np

MASK_F16, MASK_F32, MASK_LOGIT_F32 = 1, 0, 2  # the library's mask_type codes


def mask_probability(mask: np.ndarray, mask_type: int) -> np.ndarray:
    """The mask as FP64 probabilities (binary16 bits, FP32 values or FP32 logits)."""
    if mask_type == MASK_F16:
        return np.asarray(mask).view(np.float16).astype(np.float64)
    m = np.asarray(mask, np.float32).astype(np.float64)
    if mask_type == MASK_LOGIT_F32:
        return 1.0 / (1.0 + np.exp(-m))
    return m


def percentile_linear(values: np.ndarray, q: float) -> float:
    """The linear-interpolation percentile of the finite values (q in [0, 1])."""
    s = np.sort(np.asarray(values, np.float64)[np.isfinite(values)])
    n = len(s)
    if n == 0:
        return math.nan
    r = q * (n - 1)
    k = int(math.floor(r))
    if k + 1 >= n:
        return float(s[k])
    return float(s[k] + (r - k) * (s[k + 1] - s[k]))


def nerf_minmax(depth: np.ndarray, mask: np.ndarray, mask_type: int):
    """Eq. nerf-depthweight: (M~, (min, max, n_finite))."""
    D = np.asarray(depth, np.float32).astype(np.float64)
    fin = np.isfinite(D)
    n = int(fin.sum())
    lo = float(D[fin].min()) if n else 0.0
    hi = float(D[fin].max()) if n else 0.0
    zhat = np.zeros_like(D)
    if hi > lo:
        zhat[fin] = (D[fin] - lo) / (hi - lo)
    w = np.where(fin, 1.0 - zhat, 0.0)
    return mask_probability(mask, mask_type) * w, (lo, hi, n)


def band_samples(d_med: np.ndarray, prompts) -> list:
    """Eq. depthband: D_med at the prompts (x, y) and at the view centre."""
    D = np.asarray(d_med, np.float32)
    H, W = D.shape
    pts = [(int(x), int(y)) for x, y in prompts] + [(W // 2, H // 2)]
    return [float(D[y, x]) for x, y in pts if math.isfinite(float(D[y, x]))]


def gs_band(d_med: np.ndarray, mask: np.ndarray, mask_type: int, prompts):
    """Eqs. depthband and gs-bandpass: (M~, (d_min, d_max, d_far, n_finite))."""
    D = np.asarray(d_med, np.float32).astype(np.float64)
    fin = np.isfinite(D)
    n = int(fin.sum())
    s = band_samples(d_med, prompts)
    m = mask_probability(mask, mask_type)
    if not s:
        return np.where(fin, m, 0.0), (math.nan, math.nan, math.nan, n)
    d_min, d_max = min(s), max(s)
    d_far = percentile_linear(D, 0.98) if n else d_max
    den = max(d_far - d_max, 1e-6)
    with np.errstate(invalid="ignore"):
        dm = np.maximum(d_min - D, 0.0)
        dp = np.maximum(D - d_max, 0.0)
        band = np.clip((dm + dp) / den, 0.0, 1.0)
    w = np.where(fin, 1.0 - band, 0.0)
    return m * w, (d_min, d_max, d_far, n)
