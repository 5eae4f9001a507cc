"""The allocation-free one-shot entry point against the context-based path (GPU).

divas_fuse_dense_noalloc serves callers that must not allocate device memory
while they run (for example a per-frame plug-in inside a host application that
owns all GPU memory, where an allocation would synchronise the device).  It
keeps its scratch in one device array of the library, shared by every call, so
this test checks two calls in a row -- with different inputs, so that anything
left over from the first call would show -- against the regular
init / add_views / finalize path.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import _lib as L
from paper_2601_04860_b300.fusion import view_c
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _grid_c(grid):
    g = L.DivasGrid()
    g.kind = 0
    g.g = int(grid.g)
    for k in range(3):
        g.origin[k] = float(grid.origin[k])
    g.h = float(grid.h)
    g.contracted = 0
    return g


def _noalloc(wl, d, params):
    lib = L.load()
    n = int(wl.grid.g) ** 3
    score = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    seg = torch.full(((n + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    views = (L.DivasView * wl.n_views)()
    for k in range(wl.n_views):
        views[k] = view_c(wl.cams[k], d["depth"][k], d["mask"][k], wl.mask_type)
    st = lib.divas_fuse_dense_noalloc(
        ctypes.byref(_grid_c(wl.grid)), ctypes.c_void_p(d["occ"].data_ptr()), views, wl.n_views,
        ctypes.byref(H.to_params(params).c()), ctypes.c_void_p(score.data_ptr()),
        ctypes.c_void_p(seg.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.DIVAS_OK, lib.divas_noalloc_last_error()
    torch.cuda.synchronize()
    return score.cpu().numpy(), seg.cpu().numpy().view(np.uint32)


def _reference(wl, d, params):
    ref = H.run_gpu(wl, params, dev_inputs=d, labels=False)
    words = np.packbits(ref["seg_dense"].astype(np.uint8), bitorder="little").view(np.uint32)
    return ref["score"], words


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    first = synth.config1()                                     # 64^3, 4 views, binary masks
    second = synth.config2(g=48, W=252, H=189, n_ell=40, n_points=10)  # soft FP16 masks
    cases = [(first, oracle.Params()), (second, oracle.Params(tau_m=0.0, alpha1=1.0))]
    for wl, prm in cases:
        d = H.upload(wl)
        got_score, got_seg = _noalloc(wl, d, prm)
        ref_score, ref_seg = _reference(wl, d, prm)
        assert np.allclose(got_score, ref_score, rtol=H.RTOL, atol=0), "scores differ"
        assert np.array_equal(got_seg[: len(ref_seg)], ref_seg), "seg bits differ"
        assert (got_score[ref_score == 0] == 0).all()


def test_noalloc_rejects_grids_beyond_its_limit():
    lib = L.load()
    wl = synth.config1(g=16, n_points=10)
    d = H.upload(wl)
    big = synth.Grid(65, (-1.0, -1.0, -1.0), 2.0 / 65)
    views = (L.DivasView * 1)()
    views[0] = view_c(wl.cams[0], d["depth"][0], d["mask"][0], wl.mask_type)
    st = lib.divas_fuse_dense_noalloc(ctypes.byref(_grid_c(big)),
                                      ctypes.c_void_p(d["occ"].data_ptr()), views, 1,
                                      ctypes.byref(H.to_params(oracle.Params()).c()), None, None,
                                      None)
    assert st == 1
    assert b"64^3" in lib.divas_noalloc_last_error()
