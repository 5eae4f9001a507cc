"""Pins of the occupancy-construction oracle (oracle/occupancy.py) to closed
forms, a brute-force loop and an invariance, each a function of the module
so that planted mistakes can be checked against them (Eqs. scene-norm,
voxel-size; the opacity scatter-add and the tau_TF floor)."""
import math

import numpy as np


def _line_cloud(c0=(10.0, -4.0, 2.5)):
    """101 centres c0 + (o, 0, 0), o = -50..50: coordinate medians c0, radial
    distances 0, 1, 1, 2, 2, ..., 50, 50 (so P99 = s[99] = 50)."""
    o = np.arange(-50, 51, dtype=np.float64)
    mu = np.zeros((101, 3), np.float32)
    mu[:, 0] = c0[0] + o
    mu[:, 1] = c0[1]
    mu[:, 2] = c0[2]
    return mu


def pin_frame_closed_form(O):
    """c = c0, r_fg = 50, b = ceil(52.5) = 53; larger scales 0.1 k (k = 1..101)
    with median 5.1 (FP32), h = 3 s_bar (the surfel term wins), g = 8 (the
    smallest power of two >= 2 b / h = 6.93)."""
    mu = _line_cloud()
    k = np.arange(1, 102, dtype=np.float32)
    scales = np.stack([np.float32(0.1) * k, np.full(101, 0.05, np.float32)], axis=1).astype(np.float32)
    f = O.scene_frame(mu, scales)
    assert f["c"] == [10.0, -4.0, 2.5] and f["r_fg"] == 50.0 and f["b"] == 53.0
    s_bar = float(np.float32(np.float32(0.1) * np.float32(51)))
    assert f["s_bar"] == s_bar and f["h"] == 3.0 * s_bar
    assert f["g"] == 8 and f["origin"] == [10.0 - 53, -4.0 - 53, 2.5 - 53]


def pin_frame_scene_term_and_cap(O):
    """Tiny surfels: h = r_fg / 256 (the scene term); the grid needs
    2 b / h = 2 * 53 * 256 / 50 = 542.72 -> 1024 cells, capped at g_max = 512
    with h raised to 2 b / 512; with g_max = 1024 no cap."""
    mu = _line_cloud()
    scales = np.full((101, 2), 1e-4, np.float32)
    f = O.scene_frame(mu, scales, g_max=1024)
    assert f["h"] == 50.0 / 256 and f["g"] == 1024
    f = O.scene_frame(mu, scales, g_max=512)
    assert f["g"] == 512 and f["h"] == 2 * 53.0 / 512


def pin_frame_median_even_and_floor_b(O):
    """An even count: the median is the mean of the two middle values; a
    cloud of radius 0 still gets b = 1."""
    mu = np.array([[0, 0, 0], [1, 2, 4], [3, 6, 8], [7, 10, 12]], np.float32)
    f = O.scene_frame(mu, np.ones((4, 2), np.float32))
    assert f["c"] == [2.0, 4.0, 6.0]
    f = O.scene_frame(np.zeros((5, 3), np.float32), np.ones((5, 2), np.float32))
    assert f["r_fg"] == 0.0 and f["b"] == 1.0


def pin_occupancy_constructed(O):
    """Opacity sums 0.3 + 0.3 (active), 0.2 + 0.2 (not), 0.5 alone (active:
    the floor is inclusive); a centre at c + b is outside (half-open cube), one
    at c - b is in voxel 0."""
    fr = {"c": [0.0, 0.0, 0.0], "b": 2.0, "h": 1.0, "g": 4}
    mu = np.array([[-0.5, 0.5, -1.5], [-0.25, 0.75, -1.25],     # voxel (1, 2, 0)
                   [1.5, 1.5, 1.5], [1.75, 1.25, 1.5],          # voxel (3, 3, 3)
                   [-2.0, -2.0, -2.0],                          # voxel (0, 0, 0)
                   [2.0, 0.0, 0.0]], np.float32)                # outside
    alpha = np.array([0.3, 0.3, 0.2, 0.2, 0.5, 1.0], np.float32)
    o = O.occupancy(mu, alpha, fr)
    want = np.zeros(64, bool)
    want[(0 * 4 + 2) * 4 + 1] = True
    want[0] = True
    assert np.array_equal(o["active"], want) and o["n_kept"] == 5
    assert o["count"][(3 * 4 + 3) * 4 + 3] == 2 and not o["active"][(3 * 4 + 3) * 4 + 3]


def pin_occupancy_brute_force(O):
    """A random cloud against a per-surfel Python loop of the same rule."""
    rng = np.random.Generator(np.random.PCG64(9))
    mu = rng.normal(0.0, 1.0, size=(3000, 3)).astype(np.float32)
    scales = rng.uniform(0.01, 0.05, size=(3000, 2)).astype(np.float32)
    alpha = rng.uniform(0.0, 0.4, size=3000).astype(np.float32)
    f = O.scene_frame(mu, scales)
    o = O.occupancy(mu, alpha, f)
    sums = {}
    for p, a in zip(mu.astype(np.float64), alpha.astype(np.float64)):
        ijk = []
        for ax in range(3):
            x = p[ax] - f["c"][ax] + f["b"]
            if not (0.0 <= x < 2.0 * f["b"]):
                break
            ijk.append(min(int(math.floor(x / f["h"])), f["g"] - 1))
        else:
            key = (ijk[2] * f["g"] + ijk[1]) * f["g"] + ijk[0]
            sums[key] = sums.get(key, 0.0) + a
    want = np.zeros(f["g"] ** 3, bool)
    for key, s in sums.items():
        want[key] = s >= 0.5
    assert np.array_equal(o["active"], want) and o["active"].sum() > 10


def pin_translation_invariance(O):
    """Centres on a dyadic lattice shifted by an exactly representable vector:
    the frame moves with them, the active set does not change."""
    rng = np.random.Generator(np.random.PCG64(10))
    mu = (rng.integers(-64, 64, size=(2000, 3)) / 8.0).astype(np.float32)
    scales = np.full((2000, 2), 0.125, np.float32)
    alpha = rng.uniform(0.1, 0.4, size=2000).astype(np.float32)
    t = np.array([64.0, -32.0, 16.0], np.float32)
    f0 = O.scene_frame(mu, scales)
    f1 = O.scene_frame(mu + t, scales)
    assert [f1["c"][a] - f0["c"][a] for a in range(3)] == [64.0, -32.0, 16.0]
    assert (f0["r_fg"], f0["b"], f0["h"], f0["g"]) == (f1["r_fg"], f1["b"], f1["h"], f1["g"])
    assert np.array_equal(O.occupancy(mu, alpha, f0)["active"],
                          O.occupancy(mu + t, alpha, f1)["active"])


ALL_PINS = [pin_frame_closed_form, pin_frame_scene_term_and_cap,
            pin_frame_median_even_and_floor_b, pin_occupancy_constructed,
            pin_occupancy_brute_force, pin_translation_invariance]
