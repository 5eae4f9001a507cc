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
import math

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


def _views(wl, d, n=None):
    n = wl.n_views if n is None else n
    views = (L.DivasView * n)()
    for k in range(n):
        views[k] = view_c(wl.cams[k], d["depth"][k], d["mask"][k], wl.mask_type)
    return views


def _noalloc(wl, d, params, want_score=True):
    lib = L.load()
    n = int(wl.grid.g) ** 3
    score = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    seg = torch.full(((n + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    st = lib.divas_fuse_dense_noalloc(
        ctypes.byref(_grid_c(wl.grid)), ctypes.c_void_p(d["occ"].data_ptr()), _views(wl, d),
        wl.n_views, ctypes.byref(H.to_params(params).c()),
        ctypes.c_void_p(score.data_ptr()) if want_score else None,
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


def test_noalloc_seg_bits_without_a_score_buffer():
    wl = synth.config1(n_points=10)
    d = H.upload(wl)
    _, got_seg = _noalloc(wl, d, oracle.Params(), want_score=False)
    _, ref_seg = _reference(wl, d, oracle.Params())
    assert np.array_equal(got_seg[: len(ref_seg)], ref_seg)


def _bad_cases():
    """(name, mutate(grid, views, params) -> n_views, expected message fragment)."""
    def big(g, v, p):
        g.g = 65
        g.h = 2.0 / 65
        return 1, b"64^3"

    def huge(g, v, p):
        g.g = 1 << 22          # its cube would overflow 64-bit products of int32 sides
        return 1, b"64^3"

    def sparse(g, v, p):
        g.kind = 1
        return 1, b"dense"

    def contracted(g, v, p):
        g.contracted = 1
        return 1, b"dense"

    def nan_origin(g, v, p):
        g.origin[1] = math.nan
        return 1, b"origin"

    def no_views(g, v, p):
        return 0, b"n_views"

    def too_many(g, v, p):
        return 33, b"n_views"

    def nan_fx(g, v, p):
        v[0].cam.fx = math.nan
        return 1, b"intrinsics"

    def inf_t(g, v, p):
        v[0].cam.t[2] = math.inf
        return 1, b"camera t"

    def nan_R(g, v, p):
        v[0].cam.R[4] = math.nan
        return 1, b"camera R"

    def nan_tau_cons(g, v, p):
        p.tau_cons = math.nan
        return 1, b"params"

    def nan_tau_mask(g, v, p):
        p.tau_mask = math.nan
        return 1, b"params"

    def inf_alpha(g, v, p):
        p.alpha1 = math.inf
        return 1, b"params"

    def nan_z_near(g, v, p):
        p.z_near = math.nan
        return 1, b"params"

    def bad_mask_type(g, v, p):
        v[0].mask_type = 3
        return 1, b"bad view"

    def null_depth(g, v, p):
        v[0].depth = None
        return 1, b"bad view"

    return [big, huge, sparse, contracted, nan_origin, no_views, too_many, nan_fx, inf_t, nan_R,
            nan_tau_cons, nan_tau_mask, inf_alpha, nan_z_near, bad_mask_type, null_depth]


@pytest.mark.parametrize("case", _bad_cases(), ids=lambda f: f.__name__)
def test_noalloc_rejects_invalid_arguments(case):
    lib = L.load()
    wl = synth.config1(g=16, n_points=10)
    d = H.upload(wl)
    grid = _grid_c(wl.grid)
    views = (L.DivasView * 33)()
    for k in range(33):
        views[k] = view_c(wl.cams[k % wl.n_views], d["depth"][k % wl.n_views],
                          d["mask"][k % wl.n_views], wl.mask_type)
    params = H.to_params(oracle.Params()).c()
    n_views, fragment = case(grid, views, params)
    st = lib.divas_fuse_dense_noalloc(ctypes.byref(grid), ctypes.c_void_p(d["occ"].data_ptr()),
                                      views, n_views, ctypes.byref(params), None, None, None)
    assert st == 1
    assert fragment in lib.divas_noalloc_last_error()
