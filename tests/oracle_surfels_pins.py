"""Pins of the voxel-to-surfel oracle (oracle/surfels.py, Passes 2 and 3) to
closed forms, a brute force and the gating rule, each a function of the
module so that planted mistakes can be checked against them (Eqs. aspect,
needle, pass-needle, cov-atomics, kappa, final-F)."""
import math

import numpy as np


class _Cam:
    def __init__(self, f=100.0, W=64, H=48):
        self.R = np.eye(3, dtype=np.float32)
        self.t = np.zeros(3, np.float32)
        self.fx = self.fy = np.float32(f)
        self.cx, self.cy = np.float32(W / 2), np.float32(H / 2)
        self.W, self.H = W, H


def pin_rotation(S):
    """Identity, a quarter turn about z, and scale invariance of q."""
    assert np.allclose(S.quat_to_rot([1, 0, 0, 0]), np.eye(3), atol=0)
    Rz = S.quat_to_rot([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    assert np.allclose(Rz, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)
    assert np.allclose(S.quat_to_rot([2, 0, 0, 2]), Rz, atol=1e-15)


def pin_aspect_threshold(S):
    """a = max / (min + 1e-8); tau_a = P99 of 101 aspects 1..101 = 100; the
    surfel with aspect 101 is the one culled."""
    k = np.arange(1, 102, dtype=np.float64)
    sc = np.stack([np.ones(101), k], axis=1).astype(np.float32)
    a = S.aspects(sc)
    assert np.allclose(a, k / (1 + 1e-8), rtol=1e-7)
    r = S.surfel_labels(np.zeros((101, 3), np.float32), sc, np.tile([1, 0, 0, 0], (101, 1)),
                        np.ones(101, bool), np.zeros(101, np.uint32), [], [], 0)
    assert math.isclose(r["tau_a"], float(a[99]), rel_tol=1e-12)
    assert r["F2"].sum() == 100 and not r["F2"][100]


def _fronto(S, s=0.025, z=1.0, mask_cols=3):
    """A disc parallel to the image plane at depth 1, f = 100, radius s: its
    1-sigma half-extent is f s / z = 2.5 px and its centre a pixel centre, so
    the box holds the 5 x 5 pixel centres at offsets -2..2 (all inside the
    3-sigma circle); the mask covers `mask_cols` of those 5 columns."""
    cam = _Cam()
    mu = np.array([(32.5 - 32) / 100.0, (24.5 - 24) / 100.0, z], np.float32)
    mask = np.zeros((48, 64), np.float32)
    mask[:, 30:30 + mask_cols] = 1.0
    return cam, mu, np.array([s, s], np.float32), np.array([1, 0, 0, 0], np.float32), mask


def pin_fronto_parallel_counts(S):
    cam, mu, s, q, mask = _fronto(S)
    tot, msk, _ = S.surfel_view_counts(mu, s, q, cam, mask)
    assert (tot, msk) == (25, 15)
    cam, mu, s, q, mask = _fronto(S, mask_cols=2)
    r = S.surfel_labels(mu[None], s[None], q[None], [True], np.array([1], np.uint32), [cam],
                        [mask], 0)
    assert math.isclose(r["kappa"][0], 10 / 25) and not r["F"][0]
    cam, mu, s, q, mask = _fronto(S, mask_cols=3)
    r = S.surfel_labels(mu[None], s[None], q[None], [True], np.array([1], np.uint32), [cam],
                        [mask], 0)
    assert math.isclose(r["kappa"][0], 15 / 25) and r["F"][0]


def pin_coverage_at_threshold(S):
    """A disc centred on a pixel corner with a 2-pixel half-extent visits the
    4 x 4 pixel centres at offsets +-0.5, +-1.5; a mask over two of the four
    columns gives kappa = 8 / 16 = tau_kappa exactly, which is kept."""
    cam = _Cam()
    mu = np.array([0.0, 0.0, 1.0], np.float32)
    s = np.array([0.02, 0.02], np.float32)
    q = np.array([1, 0, 0, 0], np.float32)
    mask = np.zeros((48, 64), np.float32)
    mask[:, 30:32] = 1.0
    tot, msk, _ = S.surfel_view_counts(mu, s, q, cam, mask)
    assert (tot, msk) == (16, 8)
    r = S.surfel_labels(mu[None], s[None], q[None], [True], np.array([1], np.uint32), [cam],
                        [mask], 0)
    assert r["kappa"][0] == 0.5 and r["F"][0]


def pin_gating_and_max(S):
    """A view whose bit is not set is not scored; kappa is the maximum over
    the scored views (one clean view suffices)."""
    cam, mu, s, q, mask = _fronto(S, mask_cols=5)
    empty = np.zeros_like(mask)
    r = S.surfel_labels(mu[None], s[None], q[None], [True], np.array([0b10], np.uint32),
                        [cam, cam], [mask, empty], 0)
    assert r["kappa"][0] == 0.0 and not r["F"][0]
    r = S.surfel_labels(mu[None], s[None], q[None], [True], np.array([0b11], np.uint32),
                        [cam, cam], [empty, mask], 0)
    assert r["kappa"][0] == 1.0 and r["F"][0]


def pin_brute_force_whole_image(S):
    """Tilted, elongated surfels against a scan of every pixel of the image
    with the same box and ellipse rule."""
    rng = np.random.Generator(np.random.PCG64(12))
    cam = _Cam(f=120.0, W=80, H=60)
    mask = (rng.uniform(size=(60, 80)) < 0.5).astype(np.float32)
    for _ in range(20):
        mu = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.15, 0.15), rng.uniform(0.8, 1.5)],
                      np.float32)
        s = rng.uniform(0.005, 0.03, size=2).astype(np.float32)
        q = rng.normal(size=4).astype(np.float32)
        tot, msk, _ = S.surfel_view_counts(mu, s, q, cam, mask)
        R = S.quat_to_rot(q)
        m = mu.astype(np.float64)
        P = lambda X: np.array([cam.fx * X[0] / X[2] + cam.cx, cam.fy * X[1] / X[2] + cam.cy])
        c = P(m)
        a0 = 0.5 * (P(m + float(s[0]) * R[:, 0]) - P(m - float(s[0]) * R[:, 0]))
        a1 = 0.5 * (P(m + float(s[1]) * R[:, 1]) - P(m - float(s[1]) * R[:, 1]))
        det = a0[0] * a1[1] - a0[1] * a1[0]
        ex, ey = max(abs(a0[0]), abs(a1[0])), max(abs(a0[1]), abs(a1[1]))
        bt = bm = 0
        for y in range(60):
            for x in range(80):
                px, py = x + 0.5, y + 0.5
                if abs(px - c[0]) > ex or abs(py - c[1]) > ey:
                    continue
                u = ((px - c[0]) * a1[1] - (py - c[1]) * a1[0]) / det
                v = (a0[0] * (py - c[1]) - a0[1] * (px - c[0])) / det
                if u * u + v * v <= 9.0:
                    bt += 1
                    bm += int(mask[y, x] >= 0.5)
        assert (tot, msk) == (bt, bm)


def pin_overlay_constructed(S):
    """A fronto-parallel plane at depth 1 seen by an identity camera (f = 100,
    64 x 48) through a 4^3 grid of edge 0.25 over [-0.5, 0.5]^2 x [0.5, 1.5]
    whose one segmented voxel is (2, 2, 2) (x, y in [0, 0.25), z in
    [1, 1.25)): the overlay is 1 exactly on the pixels whose centres
    unproject into [0, 0.25)^2, i.e. columns 32..56 and rows 24..48 clipped
    to the frame; no-surface pixels are 0."""
    class G:
        g, origin, h, contracted = 4, (-0.5, -0.5, 0.5), 0.25, False
    cam = _Cam()
    seg = np.zeros(64, np.uint8)
    seg[(2 * 4 + 2) * 4 + 2] = 1
    D = np.ones((48, 64), np.float32)
    D[0, :] = np.inf
    out, _ = S.overlay(G, seg, cam, D)
    want = np.zeros((48, 64), np.uint8)
    for y in range(48):
        for x in range(64):
            px, py = (x + 0.5 - 32) / 100.0, (y + 0.5 - 24) / 100.0
            want[y, x] = 1 if (0 <= px < 0.25 and 0 <= py < 0.25 and y > 0) else 0
    assert np.array_equal(out, want) and want.sum() == 25 * 24 - 0


ALL_PINS = [pin_rotation, pin_aspect_threshold, pin_fronto_parallel_counts,
            pin_coverage_at_threshold, pin_gating_and_max, pin_brute_force_whole_image,
            pin_overlay_constructed]
