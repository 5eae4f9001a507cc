"""CUDA path vs the FP64 oracle, element by element (needs a GPU).

Indices, votes, view masks, consensus and labels must be bit-exact except for
items the oracle flags as within 1e-6 of a rounding or threshold boundary;
W, Z and P must agree to 1e-5 relative.  Every call goes through the C ABI.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

P0 = oracle.Params()


def _report(name, s):
    print(f"[parity] {name}: {s}")


@pytest.mark.parametrize("tau_m", [0.5, 0.0])
def test_config1_full(tau_m):
    wl = synth.config1()
    prm = oracle.Params(tau_m=tau_m)
    gpu = H.run_gpu(wl, prm, want_pix=True)
    s = H.compare(wl, gpu, prm)
    _report(f"config1 tau_m={tau_m}", s)
    assert s["voted"] > 100


def test_config2_reduced():
    wl = synth.config2(g=128, W=504, H=378, n_ell=100, n_points=100_000)
    gpu = H.run_gpu(wl, P0, want_pix=True)
    s = H.compare(wl, gpu, P0, max_flagged=0.0133)  # 1.5 x the measured 0.88%
    _report("config2 g=128", s)
    assert s["voted"] > 500


def test_config2_soft_consensus():
    wl = synth.config2(g=96, W=336, H=252, n_ell=60, n_points=20_000)
    prm = oracle.Params(tau_m=0.0, alpha1=1.5, gamma=2.0)
    gpu = H.run_gpu(wl, prm)
    _report("config2 g=96 tau_m=0", H.compare(wl, gpu, prm))


def test_config3_reduced():
    wl = synth.config3(g=128, n_views=8, W=648, H=420, n_ell=300, n_occ=None,
                       n_points=100_000)
    gpu = H.run_gpu(wl, P0, want_pix=True)
    s = H.compare(wl, gpu, P0, max_flagged=0.0263)  # 1.5 x the measured 1.75%
    _report("config3 g=128", s)
    assert s["voted"] > 500


def test_config4_logits_reduced():
    wl = synth.config4(g=96, W=336, H=252, n_ell=60, n_points=20_000)
    gpu = H.run_gpu(wl, P0, want_pix=True)
    _report("config4 g=96", H.compare(wl, gpu, P0))


@pytest.mark.parametrize("maker", ["dense", "sparse"])
def test_incremental_equals_oneshot(maker):
    if maker == "dense":
        wl = synth.config2(g=96, W=336, H=252, n_ell=60, n_points=1000)
    else:
        wl = synth.config3(g=96, n_views=10, W=324, H=210, n_ell=200, n_occ=None,
                           n_points=1000)
    d = H.upload(wl)
    runs = {m: H.run_gpu(wl, P0, mode=m, dev_inputs=d, labels=False)
            for m in ("oneshot", "incremental", "split")}
    for m in ("incremental", "split"):
        for k in ("W", "Z", "bits", "score", "vmask", "seg_dense"):
            assert np.array_equal(runs[m][k], runs["oneshot"][k]), (m, k)


def test_edge_cases():
    # odd g (ragged occupancy words), random sparse prior, with NaN / <=0 depth pixels
    wl = synth.config1(g=37, n_points=5000)
    rng = np.random.Generator(np.random.PCG64(9))
    for d in wl.depth:
        sel = rng.random(d.shape) < 0.01
        d[sel] = np.nan
        d[rng.random(d.shape) < 0.01] = -1.0
        d[rng.random(d.shape) < 0.01] = 0.0
    wl.points[:10] = np.nan
    wl.points[10:20] = 5.0
    gpu = H.run_gpu(wl, P0, want_pix=True)
    _report("g=37", H.compare(wl, gpu, P0))
    # every voxel occupied
    wl2 = synth.config1(g=16, n_points=500)
    wl2.occ[:] = 1
    gpu = H.run_gpu(wl2, P0, want_pix=True)
    _report("all occupied", H.compare(wl2, gpu, P0))
    # a single occupied voxel, and an empty prior
    wl3 = synth.config1(g=16, n_points=100)
    wl3.occ[:] = 0
    wl3.occ[(8 * 16 + 8) * 16 + 8] = 1
    H.compare(wl3, H.run_gpu(wl3, P0, want_pix=True), P0)
    wl3.occ[:] = 0
    gpu = H.run_gpu(wl3, P0)
    assert gpu["n_active"] == 0 and gpu["n_seg"] == 0
    assert not gpu["score"].any() and not gpu["labels"].any()
    # a camera that sees nothing (everything behind it)
    wl4 = synth.config1(g=24, n_points=100)
    c = wl4.cams[0]
    wl4.cams[0] = synth.Camera(c.R, np.array([0, 0, -10], np.float32), c.fx, c.fy, c.cx, c.cy,
                               c.W, c.H)
    H.compare(wl4, H.run_gpu(wl4, P0, want_pix=True), P0)


def test_sparse_duplicates_and_order():
    wl = synth.config3(g=64, n_views=4, W=162, H=105, n_ell=60, n_occ=None, n_points=2000)
    rng = np.random.Generator(np.random.PCG64(2))
    coords = wl.coords
    shuffled = np.concatenate([coords, coords[: len(coords) // 3]])[
        rng.permutation(len(coords) + len(coords) // 3)]
    ref = H.run_gpu(wl, P0, labels=False)
    wl.coords = np.ascontiguousarray(shuffled)
    got = H.run_gpu(wl, P0, labels=False)
    for k in ("W", "Z", "bits", "score", "seg_dense"):
        assert np.array_equal(ref[k], got[k]), k


def test_set_occupancy_reset_and_checkpoint():
    from paper_2601_04860_b300 import VoxelFusion
    wl = synth.config2(g=64, W=252, H=189, n_ell=40, n_points=1000)
    d = H.upload(wl)
    ref = H.run_gpu(wl, P0, dev_inputs=d, labels=False)
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(P0))
    # a smaller prior, then back to the original one
    half = d["occ"].clone()
    half[: half.numel() // 2] = 0
    fu.set_occupancy(occ=half)
    fu.add_views(wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
    fu.set_occupancy(occ=d["occ"])
    fu.sync()
    assert fu.n_active == ref["n_active"]
    fu.add_views(wl.cams[:3], d["depth"][:3], d["mask"][:3], mask_type=wl.mask_type)
    state = fu.export_state()
    state = {k: (v.clone() if isinstance(v, torch.Tensor) else v) for k, v in state.items()}
    fu.close()
    fu2 = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(P0))
    fu2.import_state(state)
    fu2.add_views(wl.cams[3:], d["depth"][3:], d["mask"][3:], mask_type=wl.mask_type)
    out = fu2.finalize(score=True)
    st = fu2.export_state()
    assert np.array_equal(out["score"].cpu().numpy(), ref["score"])
    assert np.array_equal(st["W"].cpu().numpy(), ref["W"])
    assert np.array_equal(st["bits"].cpu().numpy().view(np.uint32), ref["bits"])
    fu2.reset()
    fu2.add_views(wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
    assert np.array_equal(fu2.finalize(score=True)["score"].cpu().numpy(), ref["score"])
    fu2.close()


def test_invalid_arguments_are_rejected():
    from paper_2601_04860_b300 import DivasError, VoxelFusion
    wl = synth.config1(g=16, n_points=10)
    d = H.upload(wl)
    import ctypes

    from paper_2601_04860_b300 import _lib as L
    lib = L.load()
    occ1 = torch.zeros(1, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    prm = H.to_params(P0).c()
    for g, hh, kind in [(0, 0.125, 0), (2048, 0.125, 0), (16, 0.0, 0), (16, float("nan"), 0),
                        (16, 0.125, 5)]:
        grid = L.DivasGrid(kind, g, (ctypes.c_float * 3)(-1, -1, -1), hh, 0)
        st = lib.divas_fuse_init(ctypes.byref(h), ctypes.byref(grid),
                                 ctypes.c_void_p(occ1.data_ptr()), None, 0, ctypes.byref(prm),
                                 None)
        assert st == 1 and not h.value, (g, hh, kind, st)
        assert lib.divas_last_error(None)
    # dense kind with coords, sparse kind with occ
    grid = L.DivasGrid(0, 16, (ctypes.c_float * 3)(-1, -1, -1), 0.125, 0)
    st = lib.divas_fuse_init(ctypes.byref(h), ctypes.byref(grid), None, None, 0,
                             ctypes.byref(prm), None)
    assert st == 1
    coords = torch.tensor([[0, 0, 0], [16, 0, 0]], dtype=torch.int32, device="cuda")
    with pytest.raises(DivasError) as e:
        VoxelFusion(wl.grid, coords=coords)
    assert e.value.status == 1
    fu = VoxelFusion(wl.grid, occ=d["occ"])
    with pytest.raises(DivasError):
        fu.add_view(wl.cams[0], d["depth"][0], d["mask"][0], mask_type=7)
    c = wl.cams[0]
    badcam = synth.Camera(c.R, c.t, c.fx, c.fy, c.cx, c.cy, 0, c.H)
    with pytest.raises(DivasError):
        fu.add_view(badcam, d["depth"][0], d["mask"][0], mask_type=0)
    assert fu.n_views == 0
    fu.close()


# ---------------------------------------------------------------------------
# full sizes, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------
def test_config2_full_size_sampled():
    MAXF = 0.0285  # 1.5 x the measured 1.9%
    wl = synth.config2()
    gpu = H.run_gpu(wl, P0, want_pix=True)
    rng = np.random.Generator(np.random.PCG64(1))
    sample = np.sort(rng.choice(gpu["n_active"], size=min(150_000, gpu["n_active"]),
                                replace=False))
    s = H.compare(wl, gpu, P0, sample=sample, max_flagged=MAXF)
    _report("config2 full (sampled)", s)
    assert s["voted"] > 300


def test_config3_full_size_sampled():
    MAXF = 0.079  # 1.5 x the measured 5.2% (16 views: twice the pixel decisions)
    wl = synth.config3()
    gpu = H.run_gpu(wl, P0)
    rng = np.random.Generator(np.random.PCG64(1))
    sample = np.sort(rng.choice(gpu["n_active"], size=100_000, replace=False))
    s = H.compare(wl, gpu, P0, sample=sample, max_flagged=MAXF)
    _report("config3 full (sampled)", s)
    assert s["voted"] > 1000

