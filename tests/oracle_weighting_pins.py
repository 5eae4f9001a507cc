"""Pins of the depth-weighting oracle (oracle/weighting.py) to closed forms
and definitions, each a function of the module so that planted mistakes can
be checked against them (Eqs. nerf-depthweight, depthband, gs-bandpass)."""
import math

import numpy as np

F32 = 0


def pin_percentile_of_permutations(W):
    """s[k] = k for a permutation of 0..n-1, so P_q = q (n - 1) exactly."""
    rng = np.random.Generator(np.random.PCG64(5))
    for n in (1, 2, 3, 7, 51, 100, 1001):
        v = rng.permutation(n).astype(np.float64)
        for q in (0.0, 0.5, 0.98, 1.0):
            got = W.percentile_linear(v, q)
            assert math.isclose(got, q * (n - 1), rel_tol=0, abs_tol=1e-9), (n, q, got)


def pin_percentile_median_and_ties(W):
    """q = 1/2 is the median (middle value, or the mean of the two middle
    values); repeated values give that value; non-finite values are ignored."""
    rng = np.random.Generator(np.random.PCG64(6))
    for n in (5, 6, 101, 100):
        v = rng.normal(size=n)
        s = sorted(v)
        med = s[n // 2] if n % 2 else 0.5 * (s[n // 2 - 1] + s[n // 2])
        assert math.isclose(W.percentile_linear(v, 0.5), med, rel_tol=1e-12, abs_tol=1e-12)
    assert W.percentile_linear(np.full(37, 2.5), 0.98) == 2.5
    v = np.array([1.0, np.nan, 2.0, np.inf, 3.0, -np.inf, 4.0, 5.0])
    assert math.isclose(W.percentile_linear(v, 0.98), 4.0 + 0.92 * 1.0, rel_tol=1e-12)
    assert math.isnan(W.percentile_linear(np.array([np.nan, np.inf]), 0.98))


def pin_percentile_against_library(W):
    """numpy's linear percentile on random data (a second statement)."""
    rng = np.random.Generator(np.random.PCG64(7))
    for n in (2, 10, 999, 4096):
        v = rng.lognormal(size=n)
        assert math.isclose(W.percentile_linear(v, 0.98), float(np.percentile(v, 98.0)),
                            rel_tol=1e-12)


def pin_nerf_closed_form(W):
    """Z^ = 0 at the nearest finite pixel (weight 1), 1 at the farthest
    (weight 0), 1/2 halfway; non-finite depth weighs 0; a constant raster
    weighs 1; logits go through the sigmoid."""
    D = np.array([[2.0, 4.0, 3.0], [np.inf, np.nan, 2.5]], np.float32)
    M = np.array([[0.8, 0.6, 1.0], [1.0, 1.0, 0.4]], np.float32)
    out, (lo, hi, n) = W.nerf_minmax(D, M, F32)
    assert (lo, hi, n) == (2.0, 4.0, 4)
    m = M.astype(np.float64)
    want = [[m[0, 0], 0.0, 0.5], [0.0, 0.0, m[1, 2] * 0.75]]
    assert np.allclose(out, want, rtol=0, atol=1e-15)
    out, _ = W.nerf_minmax(np.full((2, 2), 3.0, np.float32), M[:, :2], F32)
    assert np.allclose(out, M[:, :2].astype(np.float64), rtol=0, atol=0)
    L = np.array([[0.0, 2.0]], np.float32)
    out, _ = W.nerf_minmax(np.array([[1.0, 1.0]], np.float32), L, 2)
    assert np.allclose(out, [[0.5, 1.0 / (1.0 + math.exp(-2.0))]], rtol=1e-15)


def _band_case():
    """A 9 x 9 raster: centre (4, 4) at depth 2, prompts at depths 1.5 and
    2.5 (so the band is [1.5, 2.5]); three pixels at 10 and one at 100 put
    P98 of the 80 finite values at 10 (ranks 77 and 78 are both 10)."""
    D = np.full((9, 9), 2.0, np.float32)
    D[1, 1] = 1.5                 # prompt (x = 1, y = 1)
    D[7, 2] = 2.5                 # prompt (x = 2, y = 7)
    D[0, 0:3] = [3.0, 4.0, 0.5]   # outside the band: above and below
    D[8, 0:3] = 10.0              # the far tail
    D[8, 8] = 100.0
    D[8, 7] = np.inf              # no surface
    return D, [(1, 1), (2, 7)]


def pin_band_closed_form(W):
    """Inside [d_min, d_max] the weight is 1; outside it falls linearly with
    slope 1 / (d_far - d_max) on both sides; at or past d_far it is 0;
    non-finite depth weighs 0."""
    D, prompts = _band_case()
    M = np.ones_like(D)
    out, (dmn, dmx, dfar, n) = W.gs_band(D, M, F32, prompts)
    assert (dmn, dmx, n) == (1.5, 2.5, 80)
    assert dfar == 10.0
    den = 7.5
    assert out[4, 4] == 1.0 and out[1, 1] == 1.0 and out[7, 2] == 1.0
    assert math.isclose(out[0, 0], 1.0 - 0.5 / den, rel_tol=1e-15)    # 3.0 = d_max + 0.5
    assert math.isclose(out[0, 1], 1.0 - 1.5 / den, rel_tol=1e-15)    # 4.0 = d_max + 1.5
    assert math.isclose(out[0, 2], 1.0 - 1.0 / den, rel_tol=1e-15)    # 0.5 = d_min - 1
    assert out[8, 0] == 0.0 and out[8, 8] == 0.0 and out[8, 7] == 0.0


def pin_band_samples_and_degenerate(W):
    """The band comes from the prompts and the centre pixel (floor(W/2),
    floor(H/2)); non-finite samples are dropped; no finite sample: weight 1
    on finite pixels; d_far <= d_max: the floored denominator makes the
    weight an inside / outside indicator."""
    D = np.array([[5.0, 5.0, 5.0, 5.0], [5.0, 5.0, 1.0, 5.0], [5.0, 5.0, 5.0, 5.0]], np.float32)
    M = np.full(D.shape, 0.5, np.float32)
    out, (dmn, dmx, _, _) = W.gs_band(D, M, F32, [])
    assert (dmn, dmx) == (1.0, 1.0)   # centre (2, 1) alone
    assert np.all(out[D == 5.0] == 0.0) and out[1, 2] == 0.5   # d_far = 5 = the far values
    out, (dmn, dmx, _, _) = W.gs_band(D, M, F32, [(0, 0)])
    assert (dmn, dmx) == (1.0, 5.0) and np.all(out == 0.5)
    Dn = D.copy()
    Dn[1, 2] = np.nan
    out, (dmn, _, _, _) = W.gs_band(Dn, M, F32, [(3, 2)])
    assert dmn == 5.0 and out[1, 2] == 0.0 and np.all(out[np.isfinite(Dn)] == 0.5)
    out, b = W.gs_band(Dn, M, F32, [])
    assert math.isnan(b[0]) and np.all(out[np.isfinite(Dn)] == 0.5) and out[1, 2] == 0.0


ALL_PINS = [pin_percentile_of_permutations, pin_percentile_median_and_ties,
            pin_percentile_against_library, pin_nerf_closed_form, pin_band_closed_form,
            pin_band_samples_and_degenerate]
