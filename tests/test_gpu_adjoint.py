"""Adjoint kernel and autograd Function vs the FP64 oracle's analytic gradient (GPU).

The oracle's adjoint is itself pinned by central finite differences
(tests/oracle_pins.py::pin_gradient_fd).  Here the GPU gradient, an FP32
atomic scatter, must match it within 1e-5 relative to the largest gradient.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import MASK_LOGIT_F32, VoxelFusion, fuse
from tests import gpu_helpers as H
from tests.oracle_pins import target_truth

pytestmark = pytest.mark.gpu

P0 = oracle.Params()


def _workload(g, views, W, H_, n_ell):
    wl = synth.config4(g=g, W=W, H=H_, n_ell=n_ell, n_points=10)
    wl.cams = [wl.cams[i] for i in views]
    wl.depth = [wl.depth[i] for i in views]
    wl.mask = [wl.mask[i] for i in views]
    return wl


def _excluded_pixels(wl, lin, flags):
    """Pixels read by voxels the oracle flags as near a decision boundary."""
    bad = [np.zeros(c.W * c.H, bool) for c in wl.cams]
    sel = lin[flags != 0]
    if len(sel):
        o = oracle.fuse(wl.grid, sel, wl.cams, wl.depth, wl.mask, wl.mask_type, P0, want_pix=True)
        for i in range(wl.n_views):
            p = o["pix"][:, i]
            bad[i][p[p >= 0]] = True
    return bad


@pytest.mark.parametrize("shape", [(32, [0, 3, 7], 252, 189, 30), (96, list(range(8)), 336, 252, 60)])
def test_adjoint_matches_oracle(shape):
    g, views, W, H_, n_ell = shape
    wl = _workload(g, views, W, H_, n_ell)
    lin = wl.active_linear()
    y = target_truth(wl, lin)
    ref = oracle.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, MASK_LOGIT_F32, P0)
    _, gP = oracle.bce_loss_grad(ref["P"], y)
    gM_o, gD_o = oracle.fuse_grad(wl.grid, lin, wl.cams, wl.depth, wl.mask, MASK_LOGIT_F32, gP, P0)
    # the same cotangent, on the dense grid, into the GPU adjoint
    d = H.upload(wl)
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(P0))
    fu.add_views(wl.cams, d["depth"], d["mask"], mask_type=MASK_LOGIT_F32)
    dense_g = np.zeros(g ** 3, np.float32)
    dense_g[lin] = gP
    gM = [torch.zeros_like(m) for m in d["mask"]]
    gD = [torch.zeros_like(x) for x in d["depth"]]
    fu.backward(wl.cams, d["depth"], d["mask"], torch.from_numpy(dense_g).cuda(), gM, gD,
                mask_type=MASK_LOGIT_F32)
    torch.cuda.synchronize()
    bad = _excluded_pixels(wl, lin, ref["flags"])
    gmax = max(max(np.abs(a).max() for a in gM_o), max(np.abs(a).max() for a in gD_o))
    assert gmax > 0
    checked = 0
    for i in range(wl.n_views):
        ok = ~bad[i]
        for name, go, gg in (("mask", gM_o[i], gM[i]), ("depth", gD_o[i], gD[i])):
            a = gg.cpu().numpy().reshape(-1)[ok].astype(np.float64)
            b = go.reshape(-1)[ok]
            err = np.abs(a - b).max()
            assert err <= 1e-5 * gmax, (name, i, err, gmax)
            checked += int((b != 0).sum())
    assert checked > 100
    fu.close()


def test_autograd_function_end_to_end():
    wl = _workload(48, [0, 3, 7], 252, 189, 30)
    lin = wl.active_linear()
    y = target_truth(wl, lin)
    d = H.upload(wl)
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=H.to_params(P0))
    logits = [m.clone().requires_grad_(True) for m in d["mask"]]
    depths = [x.clone().requires_grad_(True) for x in d["depth"]]
    P = fuse(fu, wl.cams, logits, depths)
    lin_t = torch.from_numpy(lin).cuda()
    yt = torch.from_numpy(y).cuda().float()
    Pc = P[lin_t].clamp(1e-6, 1 - 1e-6)
    loss = -(yt * torch.log(Pc) + (1 - yt) * torch.log(1 - Pc)).sum()
    loss.backward()
    # oracle: same loss on the oracle's P, its analytic adjoint
    ref = oracle.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, MASK_LOGIT_F32, P0)
    L_o, gP = oracle.bce_loss_grad(ref["P"], y)
    assert abs(float(loss.detach()) - L_o) <= 1e-4 * abs(L_o)
    gM_o, gD_o = oracle.fuse_grad(wl.grid, lin, wl.cams, wl.depth, wl.mask, MASK_LOGIT_F32, gP, P0)
    bad = _excluded_pixels(wl, lin, ref["flags"])
    gmax = max(max(np.abs(a).max() for a in gM_o), max(np.abs(a).max() for a in gD_o))
    for i in range(wl.n_views):
        ok = ~bad[i]
        a = logits[i].grad.cpu().numpy().reshape(-1)[ok]
        b = gM_o[i].reshape(-1)[ok]
        assert np.abs(a - b).max() <= 1e-4 * gmax
        a = depths[i].grad.cpu().numpy().reshape(-1)[ok]
        b = gD_o[i].reshape(-1)[ok]
        assert np.abs(a - b).max() <= 1e-4 * gmax
    fu.close()
