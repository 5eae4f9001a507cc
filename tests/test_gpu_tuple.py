"""Depth-tuple mode (thick gates on the depth tuple + thin footprint path) on
the GPU against the FP64 oracle: W, Z and view bits per active voxel, with
the oracle's near-boundary voxels excluded from exact checks (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import TupleParams, VoxelFusion
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _upload_tuple(tw):
    dev = torch.device("cuda")
    t = tw.tuple
    up = {k: [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in t[k]]
          for k in ("d_min", "d_med", "d_max")}
    up["n_samp"] = [torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).to(dev)
                    for a in t["n_samp"]]
    if tw.mask_type == oracle.MASK_F16:
        up["mask"] = [torch.from_numpy(m.view(np.float16)).to(dev) for m in tw.mask]
    else:
        up["mask"] = [torch.from_numpy(m).to(dev) for m in tw.mask]
    up["occ"] = None if tw.occ is None else torch.from_numpy(tw.occ).to(dev)
    up["coords"] = None if tw.coords is None else torch.from_numpy(tw.coords).to(dev)
    return up


def _gpu(tw, prm, tp, splits=None):
    up = _upload_tuple(tw)
    fu = VoxelFusion(tw.grid, occ=up["occ"], coords=up["coords"], params=H.to_params(prm))
    n = tw.n_views
    cuts = [0] + (splits or []) + [n]
    for a, b in zip(cuts[:-1], cuts[1:]):
        fu.add_views_tuple(tw.cams[a:b], up["d_min"][a:b], up["d_med"][a:b], up["d_max"][a:b],
                           up["n_samp"][a:b], up["mask"][a:b], tw.tuple["d_cam"][a:b],
                           tw.mask_type, tparams=TupleParams(**tp.__dict__))
    st = fu.export_state()
    out = {"W": st["W"].cpu().numpy(), "Z": st["Z"].cpu().numpy(),
           "bits": st["bits"].cpu().numpy().view(np.uint32),
           "active": fu.active_coords().cpu().numpy()}
    fin = fu.finalize(score=True)
    out["score"] = fin["score"].cpu().numpy()
    torch.cuda.synchronize()
    fu.close()
    return out


def _compare(tw, got, prm, tp, max_flagged=0.026):
    """Bits exact, W and Z within RTOL outside the oracle's near-boundary
    voxels; max_flagged: ceiling of their fraction (1.5 x the measured one)."""
    lin = tw.active_linear()
    g = tw.grid.g
    act = got["active"].astype(np.int64)
    assert np.array_equal((act[:, 2] * g + act[:, 1]) * g + act[:, 0], lin)
    ref = oracle.fuse_tuple(tw.grid, lin, tw.cams, tw.tuple, tw.mask, tw.mask_type,
                            params=prm.f32(), tparams=tp.f32())
    ok = ref["flags"] == 0
    bad = ok & ((got["bits"] != ref["bits"]) |
                ~np.isclose(got["W"], ref["W"], rtol=H.RTOL, atol=1e-30) |
                ~np.isclose(got["Z"], ref["Z"], rtol=H.RTOL, atol=1e-30))
    H.record(H.current_test(), len(lin), int((~ok).sum()), int(bad.sum()))
    assert (~ok).mean() <= max_flagged, (~ok).mean()
    assert np.array_equal(got["bits"][ok], ref["bits"][ok]), "view bits differ"
    assert np.allclose(got["W"][ok], ref["W"][ok], rtol=H.RTOL, atol=1e-30), "W differs"
    assert np.allclose(got["Z"][ok], ref["Z"][ok], rtol=H.RTOL, atol=1e-30), "Z differs"
    thick = int((ref["kind"][ok] == 1).sum())
    thin = int((ref["kind"][ok] == 2).sum())
    return thick, thin


def _dense(**kw):
    wl = synth.config2(g=64, W=224, H=168, n_ell=50, n_points=100)
    return synth.with_tuple(wl, **kw)


@pytest.mark.parametrize("case", ["thin_on", "paper_defaults", "soft_consensus", "gradient"])
def test_tuple_dense_matches_oracle(case):
    tw = _dense()
    prm, tp = oracle.Params(), oracle.TupleParams(n_abs=4.0)
    if case == "paper_defaults":
        tp = oracle.TupleParams()
    elif case == "soft_consensus":
        prm, tp = oracle.Params(tau_m=0.3, alpha1=1.0), oracle.TupleParams(n_abs=2.0, tau_thin=0.3)
    elif case == "gradient":
        tp = oracle.TupleParams(n_abs=4.0, k_dg=30.0)
    thick, thin = _compare(tw, _gpu(tw, prm, tp), prm, tp)
    assert thick > 100
    if case != "paper_defaults":
        assert thin > 50


def test_tuple_logit_and_f32_masks():
    tw = _dense()
    logits = []
    for m in tw.mask:
        p = np.clip(m.view(np.float16).astype(np.float64), 1e-4, 1 - 1e-4)
        logits.append(np.log(p / (1 - p)).astype(np.float32))
    probs = [m.view(np.float16).astype(np.float32) for m in tw.mask]
    for masks, mt in ((logits, oracle.MASK_LOGIT_F32), (probs, oracle.MASK_F32)):
        tw.mask, tw.mask_type = masks, mt
        thick, thin = _compare(tw, _gpu(tw, oracle.Params(), oracle.TupleParams(n_abs=4.0)),
                               oracle.Params(), oracle.TupleParams(n_abs=4.0))
        assert thick > 100 and thin > 50


def test_tuple_contracted_and_many_views():
    wl = synth.config3(g=48, n_views=20, W=162, H=105, n_ell=80, n_occ=None, n_points=100)
    tw = synth.with_tuple(wl, target=(0.0, 0.0, 0.5))
    prm, tp = oracle.Params(), oracle.TupleParams(n_abs=2.0)
    one = _gpu(tw, prm, tp)                 # 20 views: two launches of <= 16
    thick, _ = _compare(tw, one, prm, tp, max_flagged=0.058)
    assert thick > 100
    split = _gpu(tw, prm, tp, splits=[7, 13])
    for k in ("W", "Z", "bits", "score"):
        assert np.array_equal(one[k], split[k]), f"{k}: split calls differ from one call"


def test_tuple_rejects_bad_arguments():
    import ctypes
    from paper_2601_04860_b300 import _lib as L
    from paper_2601_04860_b300.fusion import tuple_views_c
    tw = synth.with_tuple(synth.config1(g=16, n_points=10))
    up = _upload_tuple(tw)
    fu = VoxelFusion(tw.grid, occ=up["occ"], params=H.to_params(oracle.Params()))
    arr = tuple_views_c(tw.cams[:1], up["d_min"], up["d_med"], up["d_max"], up["n_samp"],
                        up["mask"], tw.tuple["d_cam"], tw.mask_type)
    lib = L.load()
    tp = TupleParams().c()
    assert lib.divas_fuse_add_views_tuple(fu.handle, arr, 0, ctypes.byref(tp), None) == 1
    for bad in (TupleParams(beta=-1.0).c(), TupleParams(tau_thin=0.0).c()):
        assert lib.divas_fuse_add_views_tuple(fu.handle, arr, 1, ctypes.byref(bad), None) == 1
    arr[0].d_med = None
    assert lib.divas_fuse_add_views_tuple(fu.handle, arr, 1, ctypes.byref(tp), None) == 1
    assert fu.n_views == 0
    fu.close()


@pytest.mark.parametrize("W,H,hi", [(1, 1, 9), (33, 65, 40), (1008, 77, 40), (2100, 40, 65535),
                                    (1297, 131, 65535)])
def test_integral_images_exact(W, H, hi):
    """The per-view integral images of n_samp equal NumPy's exact cumulative
    sums (uint32 and uint64, modular), ragged strips and column segments
    included."""
    from paper_2601_04860_b300 import _lib as L
    rng = np.random.Generator(np.random.PCG64(W * 7919 + H))
    n = rng.integers(0, hi + 1, size=(H, W), dtype=np.uint16)
    dn = torch.from_numpy(n.view(np.int16)).cuda()
    s1 = torch.empty((H + 1, W + 1), dtype=torch.int32, device="cuda")
    s2 = torch.empty((H + 1, W + 1), dtype=torch.int64, device="cuda")
    lib = L.load()
    assert lib.divas_debug_integral_images(dn.data_ptr(), W, H, s1.data_ptr(), s2.data_ptr(),
                                           None) == 0
    n64 = n.astype(np.uint64)
    e2 = np.zeros((H + 1, W + 1), np.uint64)
    e2[1:, 1:] = (n64 * n64).cumsum(0).cumsum(1)        # wraps mod 2^64
    e1 = np.zeros((H + 1, W + 1), np.uint64)
    e1[1:, 1:] = n64.cumsum(0).cumsum(1)
    e1 &= np.uint64(0xFFFFFFFF)
    assert np.array_equal(s1.cpu().numpy().view(np.uint32).astype(np.uint64), e1)
    assert np.array_equal(s2.cpu().numpy().view(np.uint64), e2)


def _perturb(tw, seed, frac_nan=0.04, frac_inf=0.04, frac_neg=0.03, frac_zero=0.02,
             untrusted=0.2, big_n=0.1):
    """Degenerate rasters: NaN / +inf / negative / zero depths, many untrusted
    pixels (d_min > d_med) and n_samp at its maximum 65535."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = tw.tuple
    for k in range(tw.n_views):
        dmin, dmed, dmax = t["d_min"][k].copy(), t["d_med"][k].copy(), t["d_max"][k].copy()
        shp = dmin.shape
        dmed[rng.uniform(size=shp) < frac_nan] = np.nan
        dmin[rng.uniform(size=shp) < frac_inf] = np.inf
        dmax[rng.uniform(size=shp) < frac_neg] = -1.0
        dmed[rng.uniform(size=shp) < frac_zero] = 0.0
        un = rng.uniform(size=shp) < untrusted
        dmed[un] = dmin[un] - np.float32(0.01)
        n = t["n_samp"][k].copy()
        n[rng.uniform(size=shp) < big_n] = 65535
        t["d_min"][k], t["d_med"][k], t["d_max"][k], t["n_samp"][k] = dmin, dmed, dmax, n
    return tw


def test_tuple_degenerate_rasters():
    """NaN / inf / non-positive depths, untrusted pixels and n_samp = 65535
    (integer footprint statistics near their limits) match the oracle."""
    tw = _perturb(_dense(), seed=7)
    prm, tp = oracle.Params(), oracle.TupleParams(n_abs=4.0)
    thick, thin = _compare(tw, _gpu(tw, prm, tp), prm, tp)
    assert thick > 50 and thin > 20


def test_tuple_large_footprints_and_wide_counts():
    """A coarse plain grid seen close up: footprints of hundreds of pixels
    (integral images on a plain grid, no one-tile pre-check) with n_samp
    values up to 65535, so that A S2 - S1^2 reaches the 128-bit layered test."""
    wl = synth.config1(g=16, W=320, H=240, f=300.0, n_points=100, band=0.15)
    tw = synth.with_tuple(wl)
    rng = np.random.Generator(np.random.PCG64(11))
    for k in range(tw.n_views):
        n = tw.tuple["n_samp"][k]
        hi = rng.uniform(size=n.shape) < 0.5
        tw.tuple["n_samp"][k] = np.where(hi, np.uint16(65535), n).astype(np.uint16)
    prm, tp = oracle.Params(), oracle.TupleParams(n_abs=4.0)
    # hundreds of pixels per footprint: more per-pixel gates near a tie
    thick, thin = _compare(tw, _gpu(tw, prm, tp), prm, tp, max_flagged=0.193)
    assert thick > 20 and thin > 20


def test_tuple_32_views_two_launches():
    """32 views (two launches of 16; view bit 31 set) against the oracle."""
    wl = synth.config1(g=32, n_views=32, W=128, H=96, f=110.0, n_points=100)
    tw = synth.with_tuple(wl)
    prm, tp = oracle.Params(), oracle.TupleParams(n_abs=2.0)
    got = _gpu(tw, prm, tp)
    thick, _ = _compare(tw, got, prm, tp, max_flagged=0.056)
    assert thick > 100
    assert (got["bits"] >> 31).any(), "no voxel took a vote from view 31"


def test_tuple_no_positive_mask_and_empty_set():
    """Masks with no positive pixel give no votes; an empty occupied set
    folds and finalizes to nothing."""
    tw = _dense()
    tw.mask = [np.zeros_like(m) for m in tw.mask]
    got = _gpu(tw, oracle.Params(), oracle.TupleParams(n_abs=2.0))
    assert not got["W"].any() and not got["bits"].any()
    up = _upload_tuple(tw)
    empty = torch.zeros_like(up["occ"])
    fu = VoxelFusion(tw.grid, occ=empty, params=H.to_params(oracle.Params()))
    assert fu.n_active == 0
    fu.add_views_tuple(tw.cams, up["d_min"], up["d_med"], up["d_max"], up["n_samp"], up["mask"],
                       tw.tuple["d_cam"], tw.mask_type, tparams=TupleParams(n_abs=2.0))
    fin = fu.finalize(score=True)
    assert not fin["score"].any()
    fu.close()
