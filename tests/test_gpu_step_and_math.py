"""The one-call step equals the separate calls, and the projection's
reciprocal stays within one ulp of the correctly rounded one (GPU)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import PreparedViews, VoxelFusion, seg_bits_to_bool
from paper_2601_04860_b300 import _lib as L
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def test_reciprocal_within_one_ulp():
    rng = np.random.Generator(np.random.PCG64(3))
    x = np.exp(rng.uniform(np.log(1e-6), np.log(1e30), 2_000_000)).astype(np.float32)
    x = np.concatenate([x, np.float32([1.0, 2.0, 3.0, 0.5, 1e-6, 7.0, 1e30, 2.5])])
    xt = torch.from_numpy(x).cuda()
    nr = torch.empty_like(xt)
    ie = torch.empty_like(xt)
    st = L.load().divas_debug_rcp(ctypes.c_void_p(xt.data_ptr()), len(x),
                                  ctypes.c_void_p(nr.data_ptr()), ctypes.c_void_p(ie.data_ptr()),
                                  None)
    assert st == 0
    a = nr.cpu().numpy().view(np.int32).astype(np.int64)
    b = ie.cpu().numpy().view(np.int32).astype(np.int64)
    assert np.abs(a - b).max() <= 1
    # and the correctly rounded one is the FP64 reciprocal rounded
    ref = (1.0 / x.astype(np.float64)).astype(np.float32).view(np.int32).astype(np.int64)
    assert np.array_equal(b, ref)


@pytest.mark.parametrize("which", ["dense", "dense4", "dense7", "dense12", "dense_f32", "sparse"])
def test_step_equals_separate_calls(which):
    """Bitwise: the one-call step (its fusion kernel takes the binary16,
    full-chunk instance for 4, 8 and 12 FP16 views, the generic one for 7
    views or FP32 masks) against the separate calls' kernels."""
    if which.startswith("dense"):
        nv = {"dense4": 4, "dense7": 7}.get(which, 8)
        wl = synth.config2(g=96, n_views=nv, W=336, H=252, n_ell=60, n_points=20_000)
        if which == "dense12":  # the eight cameras and four of them again
            wl.cams, wl.depth, wl.mask = (wl.cams + wl.cams[:4], wl.depth + wl.depth[:4],
                                          wl.mask + wl.mask[:4])
        if which == "dense_f32":
            wl.mask = [m.view(np.float16).astype(np.float32) for m in wl.mask]
            wl.mask_type = oracle.MASK_F32
    else:
        wl = synth.config3(g=96, n_views=8, W=324, H=210, n_ell=200, n_occ=None,
                           n_points=20_000)
    d = H.upload(wl)
    P0 = H.to_params(oracle.Params())
    ref = H.run_gpu(wl, oracle.Params(), dev_inputs=d)
    fu = VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=P0)
    n_score = fu.n_cells if fu.dense else fu.n_active
    score = torch.full((n_score,), 7.0, device="cuda")
    seg = torch.full(((fu.n_cells + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    lab = torch.empty(len(wl.points), dtype=torch.uint8, device="cuda")
    pv = PreparedViews(wl.cams, d["depth"], d["mask"], wl.mask_type)
    for _ in range(2):  # twice: the second call must not see leftovers of the first
        fu.step(pv, occ=d["occ"], coords=d["coords"], score=score, seg_bits=seg,
                xyz=d["points"], labels=lab)
        torch.cuda.synchronize()
        assert np.array_equal(score.cpu().numpy(), ref["score"])
        assert np.array_equal(seg_bits_to_bool(seg, fu.n_cells).cpu().numpy(), ref["seg_dense"])
        assert np.array_equal(lab.cpu().numpy(), ref["labels"])
    fu.close()

