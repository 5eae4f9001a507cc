"""NeRF variant of the depth-tuple fusion (thick ray-band alignment with the
bonus depth tolerance and Gaussian band weight; thin footprint coverage with
the peak mask) on the GPU against the FP64 oracle: W, Z and view bits per
active voxel, near-boundary voxels excluded from exact checks; the density
floor that builds the occupancy prior, exactly (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import NerfParams, VoxelFusion, density_floor
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

RHO_THRESH = 10.0  # Table kernel_hyperparams, LLFF density_thresh


def _upload(nw, rho):
    dev = torch.device("cuda")
    t = nw.tuple
    up = {k: [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in t[k]]
          for k in ("d_min", "d_exp", "d_max")}
    up["n_samp"] = [torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).to(dev)
                    for a in t["n_samp"]]
    if nw.mask_type == oracle.MASK_F16:
        up["mask"] = [torch.from_numpy(m.view(np.float16)).to(dev) for m in nw.mask]
    else:
        up["mask"] = [torch.from_numpy(np.ascontiguousarray(m)).to(dev) for m in nw.mask]
    up["rho"] = None if rho is None else torch.from_numpy(rho).to(dev)
    return up


def _gpu(nw, prm, npar, rho, splits=None, with_density=True):
    up = _upload(nw, rho)
    if nw.occ is not None:
        occ = density_floor(up["rho"], RHO_THRESH)
        assert np.array_equal(occ.cpu().numpy(), (rho >= np.float32(RHO_THRESH)).astype(np.uint8))
        fu = VoxelFusion(nw.grid, occ=occ, params=H.to_params(prm))
    else:
        fu = VoxelFusion(nw.grid, coords=torch.from_numpy(nw.coords).cuda(), params=H.to_params(prm))
    n = nw.n_views
    cuts = [0] + (splits or []) + [n]
    for a, b in zip(cuts[:-1], cuts[1:]):
        fu.add_views_nerf(nw.cams[a:b], up["d_min"][a:b], up["d_exp"][a:b], up["d_max"][a:b],
                          up["n_samp"][a:b], up["mask"][a:b], nw.mask_type,
                          nparams=NerfParams(**npar.__dict__),
                          density=up["rho"] if with_density else None)
    st = fu.export_state()
    out = {"W": st["W"].cpu().numpy(), "Z": st["Z"].cpu().numpy(),
           "bits": st["bits"].cpu().numpy().view(np.uint32),
           "active": fu.active_coords().cpu().numpy()}
    fin = fu.finalize(score=True)
    out["score"] = fin["score"].cpu().numpy()
    torch.cuda.synchronize()
    fu.close()
    return out


def _compare(nw, got, prm, npar, rho, max_flagged=0.015, with_density=True):
    """Bits exact, W and Z within RTOL outside the oracle's near-boundary
    voxels; max_flagged: ceiling of their fraction (1.5 x the measured one)."""
    lin = nw.active_linear()
    g = nw.grid.g
    act = got["active"].astype(np.int64)
    assert np.array_equal((act[:, 2] * g + act[:, 1]) * g + act[:, 0], lin)
    ref = oracle.fuse_nerf(nw.grid, lin, nw.cams, nw.tuple, nw.mask, nw.mask_type,
                           params=prm.f32(), nparams=npar.f32(),
                           rho=rho[lin].astype(np.float64) if with_density else None)
    ok = ref["flags"] == 0
    bad = ok & ((got["bits"] != ref["bits"]) |
                ~np.isclose(got["W"], ref["W"], rtol=H.RTOL, atol=1e-30) |
                ~np.isclose(got["Z"], ref["Z"], rtol=H.RTOL, atol=1e-30))
    H.record(H.current_test(), len(lin), int((~ok).sum()), int(bad.sum()))
    assert (~ok).mean() <= max_flagged, (~ok).mean()
    assert np.array_equal(got["bits"][ok], ref["bits"][ok]), "view bits differ"
    assert np.allclose(got["W"][ok], ref["W"][ok], rtol=H.RTOL, atol=1e-30), "W differs"
    assert np.allclose(got["Z"][ok], ref["Z"][ok], rtol=H.RTOL, atol=1e-30), "Z differs"
    return int((ref["kind"][ok] == 1).sum()), int((ref["kind"][ok] == 2).sum())


def _dense():
    wl = synth.config2(g=64, W=224, H=168, n_ell=50, n_points=100)
    return synth.with_nerf_tuple(wl), synth.nerf_density(wl)


@pytest.mark.parametrize("case", ["llff", "mip360", "soft", "no_density"])
def test_nerf_dense_matches_oracle(case):
    nw, rho = _dense()
    prm, npar, wd = oracle.Params(), oracle.NerfParams(), True
    if case == "mip360":
        npar = oracle.NerfParams.mip360()
    elif case == "soft":
        prm = oracle.Params(tau_m=0.3, alpha1=1.0)
        npar = oracle.NerfParams(rho_cover=0.4, tau_thin=0.3, k_dg=30.0)
    elif case == "no_density":  # density 1 everywhere: rho_thin = 1 keeps the thin path on
        npar, wd = oracle.NerfParams(rho_thin=1.0), False
    thick, thin = _compare(nw, _gpu(nw, prm, npar, rho, with_density=wd), prm, npar, rho,
                           with_density=wd)
    assert thick > 100 and thin > 20, (thick, thin)


def test_nerf_logit_and_f32_masks():
    nw, rho = _dense()
    logits = []
    for m in nw.mask:
        p = np.clip(m.view(np.float16).astype(np.float64), 1e-4, 1 - 1e-4)
        logits.append(np.log(p / (1 - p)).astype(np.float32))
    probs = [m.view(np.float16).astype(np.float32) for m in nw.mask]
    prm, npar = oracle.Params(), oracle.NerfParams()
    for masks, mt in ((logits, oracle.MASK_LOGIT_F32), (probs, oracle.MASK_F32)):
        nw.mask, nw.mask_type = masks, mt
        thick, thin = _compare(nw, _gpu(nw, prm, npar, rho), prm, npar, rho)
        assert thick > 100 and thin > 20


def test_nerf_contracted_and_many_views():
    """20 views of a contracted grid (two launches of <= 16 views, no
    one-tile pre-check); split calls equal one call bitwise."""
    wl = synth.config3(g=48, n_views=20, W=162, H=105, n_ell=80, n_occ=None, n_points=100)
    nw, rho = synth.with_nerf_tuple(wl), synth.nerf_density(wl)
    prm, npar = oracle.Params(), oracle.NerfParams.mip360()
    one = _gpu(nw, prm, npar, rho)
    thick, _ = _compare(nw, one, prm, npar, rho, max_flagged=0.031)
    assert thick > 100
    split = _gpu(nw, prm, npar, rho, splits=[7, 13])
    for k in ("W", "Z", "bits", "score"):
        assert np.array_equal(one[k], split[k]), f"{k}: split calls differ from one call"


def test_nerf_degenerate_rasters():
    """NaN / +inf / non-positive depths, d_max below d_min, n_samp at 65535
    and masks with no positive pixel in some views."""
    nw, rho = _dense()
    rng = np.random.Generator(np.random.PCG64(5))
    t = nw.tuple
    for k in range(nw.n_views):
        shp = t["d_min"][k].shape
        for key, val, frac in (("d_exp", np.nan, 0.04), ("d_min", np.inf, 0.04),
                               ("d_max", -1.0, 0.03), ("d_exp", 0.0, 0.02)):
            a = t[key][k].copy()
            a[rng.uniform(size=shp) < frac] = val
            t[key][k] = a
        sw = rng.uniform(size=shp) < 0.05          # d_max < d_min
        lo, hi = t["d_min"][k].copy(), t["d_max"][k].copy()
        lo[sw], hi[sw] = t["d_max"][k][sw], t["d_min"][k][sw]
        t["d_min"][k], t["d_max"][k] = lo, hi
        n = t["n_samp"][k].copy()
        n[rng.uniform(size=shp) < 0.1] = 65535
        t["n_samp"][k] = n
    nw.mask[1] = np.zeros_like(nw.mask[1])
    prm, npar = oracle.Params(), oracle.NerfParams()
    thick, thin = _compare(nw, _gpu(nw, prm, npar, rho), prm, npar, rho)
    assert thick > 50 and thin > 10


def test_nerf_large_footprints():
    """A coarse plain grid seen close up: footprints of hundreds of pixels
    (no one-tile pre-check, long coverage loops with early exits)."""
    wl = synth.config1(g=16, W=320, H=240, f=300.0, n_points=100, band=0.15)
    nw, rho = synth.with_nerf_tuple(wl), synth.nerf_density(wl)
    prm = oracle.Params()
    for npar in (oracle.NerfParams(), oracle.NerfParams(rho_cover=0.05, tau_thin=0.3)):
        _compare(nw, _gpu(nw, prm, npar, rho), prm, npar, rho, max_flagged=0.01)


def test_density_floor_exact_and_ragged():
    for n in (0, 1, 3, 4, 1001, 64 ** 3):
        rho = np.random.Generator(np.random.PCG64(n)).uniform(0, 20, n).astype(np.float32)
        if n > 3:
            rho[:3] = (np.nan, np.float32(10.0), np.nextafter(np.float32(10.0), np.float32(0)))
        d = torch.from_numpy(rho).cuda()
        got = density_floor(d, 10.0).cpu().numpy()
        assert np.array_equal(got, (rho >= np.float32(10.0)).astype(np.uint8))


def test_nerf_rejects_bad_arguments():
    import ctypes
    from paper_2601_04860_b300 import _lib as L
    from paper_2601_04860_b300.fusion import tuple_views_c
    wl = synth.config1(g=16, n_points=10)
    nw, rho = synth.with_nerf_tuple(wl), synth.nerf_density(wl)
    up = _upload(nw, rho)
    fu = VoxelFusion(nw.grid, occ=torch.from_numpy(nw.occ).cuda(), params=H.to_params(oracle.Params()))
    arr = tuple_views_c(nw.cams[:1], up["d_min"], up["d_exp"], up["d_max"], up["n_samp"],
                        up["mask"], [0.0], nw.mask_type)
    lib = L.load()
    npr = NerfParams().c()
    assert lib.divas_fuse_add_views_nerf(fu.handle, arr, 0, ctypes.byref(npr), None, None) == 1
    for bad in (NerfParams(tau_thin=0.0), NerfParams(m_thin=1.0), NerfParams(beta=-1.0),
                NerfParams(gamma=float("nan"))):
        assert lib.divas_fuse_add_views_nerf(fu.handle, arr, 1, ctypes.byref(bad.c()), None,
                                             None) == 1
    odd = up["rho"].view(torch.uint8)[1:5]  # misaligned density pointer
    assert lib.divas_fuse_add_views_nerf(fu.handle, arr, 1, ctypes.byref(npr), odd.data_ptr(),
                                         None) == 1
    with pytest.raises(ValueError):
        fu.add_views_nerf(nw.cams[:1], up["d_min"][:1], up["d_exp"][:1], up["d_max"][:1],
                          up["n_samp"][:1], up["mask"][:1], nw.mask_type, density=up["rho"][:-1])
    assert fu.n_views == 0
    assert lib.divas_density_floor(up["rho"].data_ptr() + 4, 8, 10.0,
                                   torch.empty(16, dtype=torch.uint8, device="cuda").data_ptr(),
                                   None) == 1
    fu.close()
