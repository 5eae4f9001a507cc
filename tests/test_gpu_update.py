"""The one-launch incremental update (divas_fuse_update) equals add_views +
finalize, its seg bits are set and cleared in place, and set_occupancy leaves
the context's seg bitfield clear (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import Batch, PreparedViews, VoxelFusion, seg_bits_to_bool
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _workloads():
    dense = synth.config2(g=96, W=336, H=252, n_ell=60, n_points=20_000)
    sparse = synth.config3(g=96, n_views=8, W=324, H=210, n_ell=200, n_occ=None, n_points=20_000)
    return [("dense", dense), ("sparse", sparse)]


def _reference(wl, d, params, n_first):
    """add_views of the first n_first views, then each later view with
    add_views + finalize; the outputs after every update."""
    fu = VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=H.to_params(params))
    fu.add_views(wl.cams[:n_first], d["depth"][:n_first], d["mask"][:n_first],
                 mask_type=wl.mask_type)
    outs = []
    for k in range(n_first, wl.n_views):
        fu.add_views(wl.cams[k:k + 1], d["depth"][k:k + 1], d["mask"][k:k + 1],
                     mask_type=wl.mask_type)
        o = fu.finalize(score=True, seg_bits=True)
        outs.append((o["score"].cpu().numpy(),
                     seg_bits_to_bool(o["seg_bits"], fu.n_cells).cpu().numpy(),
                     fu.label_points(d["points"]).cpu().numpy()))
    fu.close()
    return outs


@pytest.mark.parametrize("keep", [False, True])
@pytest.mark.parametrize("which", ["dense", "sparse"])
@pytest.mark.parametrize("tau_m", [0.5, 0.0])
def test_update_equals_add_views_then_finalize(which, keep, tau_m):
    wl = dict(_workloads())[which]
    params = oracle.Params(tau_m=tau_m)  # tau_m = 0: seg bits can flip back to 0
    d = H.upload(wl)
    n_first = 3
    ref = _reference(wl, d, params, n_first)
    fu = VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=H.to_params(params))
    fu.add_views(wl.cams[:n_first], d["depth"][:n_first], d["mask"][:n_first],
                 mask_type=wl.mask_type)
    n_score = fu.n_cells if fu.dense else fu.n_active
    words = (fu.n_cells + 31) // 32
    if keep:  # buffers holding this context's earlier result (zeros before the first)
        score = torch.zeros(n_score, dtype=torch.float32, device="cuda")
        seg = torch.zeros(words, dtype=torch.int32, device="cuda")
    else:     # garbage that the update must overwrite
        score = torch.full((n_score,), 7.0, dtype=torch.float32, device="cuda")
        seg = torch.full((words,), -1, dtype=torch.int32, device="cuda")
    flipped = 0
    prev = None
    for j, k in enumerate(range(n_first, wl.n_views)):
        pv = PreparedViews(wl.cams[k:k + 1], d["depth"][k:k + 1], d["mask"][k:k + 1],
                           wl.mask_type)
        fu.update(pv, score=score, seg_bits=seg, keep_zeros=keep)
        got_seg = seg_bits_to_bool(seg, fu.n_cells).cpu().numpy()
        assert np.array_equal(score.cpu().numpy(), ref[j][0]), f"scores differ after view {k}"
        assert np.array_equal(got_seg, ref[j][1]), f"seg differs after view {k}"
        assert np.array_equal(fu.label_points(d["points"]).cpu().numpy(), ref[j][2])
        if prev is not None:
            flipped += int((prev & ~got_seg).sum())
        prev = got_seg
    if tau_m == 0.0:
        assert flipped > 0, "no seg bit went back to 0: the clearing path was not exercised"
    fu.close()


def test_set_occupancy_clears_the_seg_bitfield():
    wl = synth.config1(n_points=5_000)
    d = H.upload(wl)
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(oracle.Params()))
    fu.add_views(wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
    fu.finalize(score=True)
    assert fu.label_points(d["points"]).cpu().numpy().any()
    fu.set_occupancy(occ=d["occ"])
    assert not fu.label_points(d["points"]).cpu().numpy().any()
    fu.close()


def test_batch_finalize_keep_zeros():
    wls = [synth.config1(seed=1001 + k, n_points=2_000) for k in range(3)]
    ds = [H.upload(w) for w in wls]
    refs = [H.run_gpu(w, oracle.Params(), dev_inputs=d, labels=False) for w, d in zip(wls, ds)]
    fus = [VoxelFusion(w.grid, occ=d["occ"], params=H.to_params(oracle.Params()))
           for w, d in zip(wls, ds)]
    scores = [torch.zeros(f.n_cells, dtype=torch.float32, device="cuda") for f in fus]
    b = Batch(max_sessions=8, max_views=64)
    for f, w, d in zip(fus, wls, ds):
        b.queue(f, w.cams, d["depth"], d["mask"], w.mask_type)
    b.fuse()
    b.finalize(scores=scores, keep_zeros=True)
    torch.cuda.synchronize()
    for s, r in zip(scores, refs):
        assert np.array_equal(s.cpu().numpy(), r["score"])
    b.close()
    for f in fus:
        f.close()


def test_update_rejects_unknown_flags_and_bad_views():
    import ctypes
    from paper_2601_04860_b300 import _lib as L
    from paper_2601_04860_b300.fusion import view_c
    wl = synth.config1(g=32, n_points=100)
    d = H.upload(wl)
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(oracle.Params()))
    v = view_c(wl.cams[0], d["depth"][0], d["mask"][0], wl.mask_type)
    lib = L.load()
    assert lib.divas_fuse_update(fu.handle, ctypes.byref(v), 1, None, None, 2, None) == 1
    assert lib.divas_fuse_update(fu.handle, ctypes.byref(v), 0, None, None, 0, None) == 1
    assert lib.divas_fuse_update(fu.handle, None, 1, None, None, 0, None) == 1
    assert fu.n_views == 0  # nothing was folded
    fu.close()
