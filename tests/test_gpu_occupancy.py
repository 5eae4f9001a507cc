"""Occupancy construction from 2DGS surfels on the GPU against the FP64
oracle: the scene frame (bitwise), the occupancy and the density (exact for
dyadic opacities; near-floor voxels excluded otherwise), and the occupancy
feeding the fusion (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import oracle.occupancy as O
import synth
from paper_2601_04860_b300 import OccupancyParams, VoxelFusion, occupancy, scene_frame
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _cloud(n_points=100_000, dyadic=True, seed=1300):
    wl = synth.config2(g=64, W=224, H=168, n_ell=50, n_points=n_points)
    return wl, synth.gaussians(wl, seed=seed, dyadic=dyadic)


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _frame_equal(f, ref):
    assert list(f.c) == ref["c"], (f.c, ref["c"])
    assert (f.r_fg, f.b, f.s_bar, f.h, f.g) == (ref["r_fg"], ref["b"], ref["s_bar"], ref["h"], ref["g"])
    assert list(f.origin) == ref["origin"]


def _degenerate(mu, scales, alpha, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    mu, scales = mu.copy(), scales.copy()
    m = len(mu)
    mu[rng.choice(m, 50, replace=False), rng.integers(0, 3, 50)] = np.nan
    mu[rng.choice(m, 50, replace=False), rng.integers(0, 3, 50)] = np.inf
    scales[rng.choice(m, 50, replace=False), rng.integers(0, 2, 50)] = np.nan
    dup = rng.choice(m, 2000, replace=False)
    mu[dup] = mu[dup[0]]                      # many identical centres (ties)
    mu[:, 2] -= np.float32(7.25)              # off-centre, negative coordinates
    return mu, scales, alpha


@pytest.mark.parametrize("case", ["scene", "degenerate", "tiny1", "tiny2", "capped"])
def test_frame_matches_oracle_bitwise(case):
    _, (mu, sc, al) = _cloud(20_000)
    params = {}
    if case == "degenerate":
        mu, sc, al = _degenerate(mu, sc, al)
    elif case == "tiny1":
        mu, sc = mu[:1], sc[:1]
    elif case == "tiny2":
        mu, sc = mu[:2], sc[:2]
    elif case == "capped":
        sc = sc * np.float32(1e-3)
        params = {"g_max": 64}
    dmu, dsc = _dev(mu, sc)
    f = scene_frame(dmu, dsc, OccupancyParams(**params))
    _frame_equal(f, O.scene_frame(mu, sc, **params))


@pytest.mark.parametrize("dyadic", [True, False])
def test_occupancy_matches_oracle(dyadic):
    _, (mu, sc, al) = _cloud(100_000, dyadic=dyadic)
    dmu, dsc, dal = _dev(mu, sc, al)
    f = scene_frame(dmu, dsc)
    ref = O.occupancy(mu, al, O.scene_frame(mu, sc))
    occ, rho = occupancy(dmu, dal, f)
    got = occ.cpu().numpy().astype(bool)
    rho = rho.cpu().numpy().astype(np.float64)
    if dyadic:  # FP32 sums of multiples of 1/64 are exact in any order
        assert np.array_equal(got, ref["active"])
        assert np.array_equal(rho, ref["rho"])
        assert (ref["rho"] == 0.5).sum() > 10, "the inclusive floor is not exercised"
    else:
        ok = ~ref["near"]
        assert np.array_equal(got[ok], ref["active"][ok]) and (~ok).sum() < 50
        assert np.allclose(rho, ref["rho"], rtol=1e-5, atol=1e-6)
    assert ref["active"].sum() > 1000


def test_occupancy_feeds_the_fusion():
    """The GPU's occupancy of a surfel cloud in its own frame, fused with the
    scene's views, against the oracle's occupancy fused by the oracle."""
    wl, (mu, sc, al) = _cloud(100_000)
    dmu, dsc, dal = _dev(mu, sc, al)
    f = scene_frame(dmu, dsc)
    occ, _ = occupancy(dmu, dal, f)
    grid = f.grid()
    ref_frame = O.scene_frame(mu, sc)
    ref_occ = O.occupancy(mu, al, ref_frame)["active"].astype(np.uint8)
    assert np.array_equal(occ.cpu().numpy(), ref_occ)
    wl2 = synth.Workload(**{k: getattr(wl, k) for k in wl.__dataclass_fields__})
    wl2.grid = synth.Grid(g=grid.g, origin=grid.origin, h=grid.h, contracted=False)
    wl2.occ = ref_occ
    wl2.coords = None
    d = H.upload(wl2)
    d["occ"] = occ  # the GPU's own occupancy
    got = H.run_gpu(wl2, oracle.Params(), dev_inputs=d, labels=False)
    s = H.compare(wl2, got, oracle.Params(), check_labels=False, max_flagged=0.03)
    assert s["voted"] > 100  # a coarse grid (h about 0.038): a few hundred voting voxels


def test_occupancy_rejects_bad_arguments():
    from paper_2601_04860_b300 import DivasError
    _, (mu, sc, al) = _cloud(2_000)
    dmu, dsc, dal = _dev(mu, sc, al)
    with pytest.raises(DivasError):
        scene_frame(dmu, dsc, OccupancyParams(g_max=500))       # not a power of two
    with pytest.raises(DivasError):
        scene_frame(dmu, dsc, OccupancyParams(pad=0.0))
    f = scene_frame(dmu, dsc)
    n = f.g ** 3
    buf = torch.empty(n + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(DivasError):                               # density not 16-byte aligned
        occupancy(dmu, dal, f, density=buf[1:n + 1])
    with pytest.raises(ValueError):
        occupancy(dmu, dal[:-1], f)
