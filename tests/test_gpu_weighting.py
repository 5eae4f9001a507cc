"""Depth-weighted mask refinement (NeRF min-max, 2DGS band-pass) on the GPU
against the FP64 oracle: the per-view constants (min / max, the band and the
98th-percentile far depth, found by exact selection), the weighted masks,
and the fusion of the weighted masks (GPU)."""
import math

import numpy as np
import pytest
import torch

import oracle
import oracle.weighting as OW
import synth
from paper_2601_04860_b300 import VoxelFusion
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _wl(mask_type=oracle.MASK_F16):
    wl = synth.config2(g=64, W=224, H=168, n_ell=50, n_points=100)
    if mask_type == oracle.MASK_F16:
        return wl
    p = [m.view(np.float16).astype(np.float64) for m in wl.mask]
    if mask_type == oracle.MASK_F32:
        wl.mask = [x.astype(np.float32) for x in p]
    else:
        wl.mask = [np.log(np.clip(x, 1e-4, 1 - 1e-4) / (1 - np.clip(x, 1e-4, 1 - 1e-4)))
                   .astype(np.float32) for x in p]
    wl.mask_type = mask_type
    return wl


def _dev_mask(m, mask_type):
    a = np.ascontiguousarray(m)
    return torch.from_numpy(a.view(np.int16) if mask_type == oracle.MASK_F16 else a).cuda()


def _gpu_weight(depths, masks, mask_type, mode, prompts):
    fu = VoxelFusion(synth.Grid(g=8, origin=(-1.0, -1.0, -1.0), h=0.25, contracted=False),
                     occ=torch.ones(512, dtype=torch.uint8, device="cuda"),
                     params=H.to_params(oracle.Params()))
    d = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in depths]
    m = [_dev_mask(x, mask_type) for x in masks]
    out, st = fu.depth_weight(d, m, mask_type, mode=mode, prompts=prompts, stats=True)
    res = [o.cpu().numpy() for o in out], st.cpu().numpy()
    fu.close()
    return res


def _oracle_weight(depths, masks, mask_type, mode, prompts):
    outs, stats = [], []
    for k, (d, m) in enumerate(zip(depths, masks)):
        if mode == "nerf":
            o, s = OW.nerf_minmax(d, m, mask_type)
        else:
            o, s = OW.gs_band(d, m, mask_type, prompts[k])
        outs.append(o)
        stats.append(s)
    return outs, stats


def _check(depths, masks, mask_type, mode, prompts):
    got, gst = _gpu_weight(depths, masks, mask_type, mode, prompts)
    ref, rst = _oracle_weight(depths, masks, mask_type, mode, prompts)
    for k in range(len(depths)):
        if mode == "nerf":
            lo, hi, n = rst[k]
            if n:
                assert gst[k, 0] == np.float32(lo) and gst[k, 1] == np.float32(hi), k
            assert gst[k, 2] == n
        else:
            dmn, dmx, dfar, n = rst[k]
            assert gst[k, 3] == n
            if math.isnan(dmn):
                assert np.isnan(gst[k, :3]).all()
            else:
                assert gst[k, 0] == np.float32(dmn) and gst[k, 1] == np.float32(dmx), k
                # the order statistics are exact; the interpolation is FP64 on
                # both sides, then rounded to FP32
                assert gst[k, 2] == np.float32(dfar), (k, gst[k, 2], dfar)
        fin = np.isfinite(np.asarray(depths[k], np.float32))
        assert (got[k][~fin] == 0).all(), "no-surface pixels must weigh 0"
        err = np.abs(got[k].astype(np.float64) - ref[k])
        assert err.max() <= 2e-6, (k, err.max())
    return got, ref


@pytest.mark.parametrize("mode", ["nerf", "band"])
@pytest.mark.parametrize("mask_type", [oracle.MASK_F16, oracle.MASK_F32, oracle.MASK_LOGIT_F32])
def test_weights_match_oracle(mode, mask_type):
    wl = _wl(mask_type)
    _check(wl.depth, wl.mask, mask_type, mode, synth.prompts(wl))


@pytest.mark.parametrize("shape", [(1, 1), (5, 7), (40, 2100), (840, 1297), (131, 1297)])
def test_percentile_selection_exact(shape):
    """Rasters with many ties, negative values, signed zeros and no-surface
    pixels: the selected order statistics and d_far equal the oracle's."""
    rng = np.random.Generator(np.random.PCG64(shape[0] * 31 + shape[1]))
    views = []
    for kind in range(4):
        if kind == 0:
            d = rng.choice(np.array([0.5, 1.0, 2.0, 2.0, 3.0, 7.5], np.float32), size=shape)
        elif kind == 1:
            d = rng.normal(0.0, 3.0, size=shape).astype(np.float32)
            d.flat[:: 7] = -0.0
            d.flat[3:: 11] = 0.0
        elif kind == 2:
            d = rng.lognormal(0.5, 1.0, size=shape).astype(np.float32)
            d[rng.uniform(size=shape) < 0.3] = np.inf
            d[rng.uniform(size=shape) < 0.1] = np.nan
            d[rng.uniform(size=shape) < 0.05] = -np.inf
        else:
            d = np.full(shape, 4.25, np.float32)
            d[rng.uniform(size=shape) < 0.02] = 1e30
        views.append(np.ascontiguousarray(d))
    masks = [np.ones(shape, np.float32) for _ in views]
    prompts = [[(0, 0)] for _ in views]
    _check(views, masks, oracle.MASK_F32, "band", prompts)
    _check(views, masks, oracle.MASK_F32, "nerf", prompts)


def test_no_finite_pixels_and_constant_depth():
    shape = (9, 13)
    depths = [np.full(shape, np.inf, np.float32), np.full(shape, 2.0, np.float32),
              np.full(shape, np.nan, np.float32)]
    masks = [np.full(shape, 0.7, np.float32) for _ in depths]
    for mode in ("nerf", "band"):
        got, _ = _check(depths, masks, oracle.MASK_F32, mode, [[], [(3, 4)], []])
        assert (got[0] == 0).all() and (got[2] == 0).all()
        assert np.allclose(got[1], 0.7, rtol=0, atol=0)


@pytest.mark.parametrize("mode", ["nerf", "band"])
def test_weighted_fusion_matches_oracle(mode):
    """Fusion of the weighted masks: GPU weights + GPU fusion against oracle
    weights + oracle fusion; voxels whose sampled weighted mask lies within
    1e-6 of the mask gate (where the two independently rounded weights may
    fall on either side) are excluded and counted."""
    wl = _wl(oracle.MASK_F16)
    prm = oracle.Params()
    pr = synth.prompts(wl)
    d = H.upload(wl)
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(prm))
    wm = fu.depth_weight(d["depth"], d["mask"], wl.mask_type, mode=mode, prompts=pr)
    fu.add_views(wl.cams, d["depth"], wm, mask_type=oracle.MASK_F32)
    st = fu.export_state()
    fin = fu.finalize(score=True)
    got = {k: st[k].cpu().numpy() for k in ("W", "Z")}
    got["bits"] = st["bits"].cpu().numpy().view(np.uint32)
    got["score"] = fin["score"].cpu().numpy()
    fu.close()
    ref_m, _ = _oracle_weight(wl.depth, wl.mask, wl.mask_type, mode, pr)
    ref_m32 = [m.astype(np.float32) for m in ref_m]
    lin = wl.active_linear()
    o = oracle.fuse(wl.grid, lin, wl.cams, wl.depth, ref_m32, oracle.MASK_F32, prm, want_pix=True)
    near = np.zeros(len(lin), bool)
    for k in range(wl.n_views):
        p = o["pix"][:, k]
        v = np.where(p >= 0, ref_m[k].ravel()[np.maximum(p, 0)], 0.0)
        near |= (p >= 0) & (np.abs(v - prm.tau_m) < 1e-6)
    ok = (o["flags"] == 0) & ~near
    assert ok.mean() > 0.95 and (o["Z"][ok] > 0).sum() > 100
    assert (got["bits"][ok] == o["bits"][ok]).all(), "votes differ"
    for key in ("W", "Z"):
        a, b = got[key][ok].astype(np.float64), o[key][ok]
        assert not (np.abs(a - b) > H.RTOL * np.abs(b) + 1e-30).any(), key
    a, b = got["score"][lin][ok].astype(np.float64), o["P"][ok]
    assert not (np.abs(a - b) > H.RTOL * np.abs(b) + 1e-30).any(), "scores differ"


def test_weight_rejects_bad_arguments():
    wl = _wl()
    d = H.upload(wl)
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(oracle.Params()))
    with pytest.raises(Exception):
        fu.depth_weight(d["depth"][:1], d["mask"][:1], wl.mask_type, prompts=[[(224, 0)]])
    with pytest.raises(Exception):
        fu.depth_weight(d["depth"][:1], d["mask"][:1], wl.mask_type, prompts=[[(1, 1)] * 16])
    from paper_2601_04860_b300 import _lib as L
    arr = (L.DivasWeightView * 1)()
    assert L.load().divas_depth_weight(fu.handle, arr, 1, 1, None, None) == 1  # NULL rasters
    assert L.load().divas_depth_weight(fu.handle, arr, 1, 3, None, None) == 1  # bad mode
    fu.close()


@pytest.mark.parametrize("mode", ["nerf", "band"])
@pytest.mark.parametrize("mask_type", [oracle.MASK_F16, oracle.MASK_F32, oracle.MASK_LOGIT_F32])
def test_weighted_fusion_in_one_pass(mode, mask_type):
    """The weight folded into the fusion's mask read: the accumulators equal
    bitwise the two-pass path (weighted FP32 rasters, then add_views), and the
    result equals the oracle's fusion of its own weighted masks outside the
    flagged voxels (near-boundary decisions, or a sampled M~ within 1e-6 of the
    mask gate)."""
    wl = _wl(mask_type)
    prm = oracle.Params()
    pr = synth.prompts(wl)
    d = H.upload(wl)
    dm = [_dev_mask(m, mask_type) for m in wl.mask]
    one = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(prm))
    st1 = one.add_views_weighted(wl.cams, d["depth"], dm, mask_type=mask_type, mode=mode,
                                 prompts=pr, stats=True)
    two = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(prm))
    wm, st2 = two.depth_weight(d["depth"], dm, mask_type, mode=mode, prompts=pr, stats=True)
    two.add_views(wl.cams, d["depth"], wm, mask_type=oracle.MASK_F32)
    a, b = one.export_state(), two.export_state()
    for k in ("W", "Z", "bits"):
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(st1.nan_to_num(-7.0), st2.nan_to_num(-7.0))
    got = {k: a[k].cpu().numpy() for k in ("W", "Z")}
    got["bits"] = a["bits"].cpu().numpy().view(np.uint32)
    one.close()
    two.close()
    ref_m, _ = _oracle_weight(wl.depth, wl.mask, mask_type, mode, pr)
    ref_m32 = [m.astype(np.float32) for m in ref_m]
    lin = wl.active_linear()
    o = oracle.fuse(wl.grid, lin, wl.cams, wl.depth, ref_m32, oracle.MASK_F32, prm, want_pix=True)
    near = np.zeros(len(lin), bool)
    for k in range(wl.n_views):
        p = o["pix"][:, k]
        v = np.where(p >= 0, ref_m[k].ravel()[np.maximum(p, 0)], 0.0)
        near |= (p >= 0) & (np.abs(v - prm.tau_m) < 1e-6)
    ok = (o["flags"] == 0) & ~near
    bad = ok & ((got["bits"] != o["bits"]) |
                (np.abs(got["W"].astype(np.float64) - o["W"]) > H.RTOL * np.abs(o["W"]) + 1e-30) |
                (np.abs(got["Z"].astype(np.float64) - o["Z"]) > H.RTOL * np.abs(o["Z"]) + 1e-30))
    H.record(H.current_test(), len(lin), int((~ok).sum()), int(bad.sum()))
    assert (~ok).mean() <= 0.03 and (o["Z"][ok] > 0).sum() > 100
    assert not bad.any()
