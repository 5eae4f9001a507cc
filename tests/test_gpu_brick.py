"""Brick-major active order (DIVAS_ORDER_BRICKS): the same per-voxel results as
the linear order, bitwise, and the oracle's (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import VoxelFusion, PreparedViews
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

P0 = oracle.Params()


def brick_key(act: np.ndarray, g: int) -> np.ndarray:
    """Position of each (i, j, k) in brick-major order: 8^3 bricks in linear
    brick order, cells of a brick in linear order (x fastest in both)."""
    a = act.astype(np.int64)
    i, j, k = a[:, 0], a[:, 1], a[:, 2]
    nb = g // 8
    b = ((k // 8) * nb + (j // 8)) * nb + (i // 8)
    return b * 512 + ((k % 8) * 8 + (j % 8)) * 8 + (i % 8)


def to_linear(gpu: dict, g: int) -> dict:
    """A sparse context's state with its active-list arrays permuted into
    ascending linear order (the order compare() expects)."""
    act = gpu["active"].astype(np.int64)
    lin = (act[:, 2] * g + act[:, 1]) * g + act[:, 0]
    o = np.argsort(lin, kind="stable")
    out = dict(gpu)
    for k in ("active", "W", "Z", "bits", "vmask", "score"):
        out[k] = gpu[k][o]
    return out


def _plain_sparse():
    """Config 1 (plain 64^3 grid) with its prior given as coordinates."""
    import copy
    wl = copy.copy(synth.config1())
    lin = np.flatnonzero(wl.occ)
    g = wl.grid.g
    wl.coords = np.column_stack([lin % g, (lin // g) % g, lin // (g * g)]).astype(np.int32)
    wl.occ = None
    wl.name = "config1-sparse"
    return wl


def _small3():
    return synth.config3(g=128, n_views=8, W=648, H=420, n_ell=300, n_occ=None,
                         n_points=50_000)


def _sparse_session():
    mix = synth.session_mix(n_sessions=64, scale=0.25)
    return next(synth.session_workload(r) for r in mix
                if not r["dense"] and int(round(r["g"] * r.get("scale", 1.0))) % 8 == 0)


# (workload builder, ceiling of its near-boundary fraction: 1.5 x the measured)
WORKLOADS = [(_small3, 0.0263), (_plain_sparse, 0.0133), (_sparse_session, 0.06)]


def _step(wl, d, brick: bool):
    prm = H.to_params(P0)
    prm.brick_order = brick
    fu = VoxelFusion(wl.grid, coords=d["coords"], params=prm)
    score = torch.empty(fu.n_active, dtype=torch.float32, device="cuda")
    labels = torch.empty(len(d["points"]), dtype=torch.uint8, device="cuda")
    views = PreparedViews(wl.cams, d["depth"], d["mask"], wl.mask_type)
    fu.step(views, coords=d["coords"], score=score, xyz=d["points"], labels=labels)
    torch.cuda.synchronize()
    return fu, H.state_of(fu, score, labels)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_brick_order_matches_linear_order_and_oracle(which):
    build, max_flagged = WORKLOADS[which]
    wl = build()
    d = H.upload(wl)
    fl, lin_state = _step(wl, d, brick=False)
    fb, brick_state = _step(wl, d, brick=True)
    g = wl.grid.g
    key = brick_key(brick_state["active"], g)
    assert (np.diff(key) > 0).all(), "active list not in brick-major order"
    b = to_linear(brick_state, g)
    for k in ("active", "W", "Z", "bits", "vmask", "score"):
        assert np.array_equal(b[k], lin_state[k]), k
    assert np.array_equal(b["seg_dense"], lin_state["seg_dense"])
    assert np.array_equal(brick_state["labels"], lin_state["labels"])
    s = H.compare(wl, b, P0, sample=H.sample_of(fb.n_active, 20_000),
                  name=f"{H.current_test()} {wl.name} g={g}"
                       f"{' contracted' if wl.grid.contracted else ''}",
                  max_flagged=max_flagged)
    assert s["voted"] > 0
    fl.close()
    fb.close()


def test_brick_order_incremental_views():
    """Views folded one call at a time onto a brick-ordered context give the
    one-call result."""
    wl = _small3()
    d = H.upload(wl)
    fb, ref = _step(wl, d, brick=True)
    prm = H.to_params(P0)
    prm.brick_order = True
    fu = VoxelFusion(wl.grid, coords=d["coords"], params=prm)
    h = wl.n_views // 2
    fu.add_views(wl.cams[:h], d["depth"][:h], d["mask"][:h], mask_type=wl.mask_type)
    fu.add_views(wl.cams[h:], d["depth"][h:], d["mask"][h:], mask_type=wl.mask_type)
    score = torch.empty(fu.n_active, dtype=torch.float32, device="cuda")
    fu.finalize(score=score)
    st = H.state_of(fu, score)
    for k in ("active", "W", "Z", "bits", "score"):
        assert np.array_equal(st[k], ref[k]), k
    fu.close()
    fb.close()


def test_brick_order_rejected_unless_g_multiple_of_8():
    wl = synth.config1(g=60)
    d = H.upload(wl)
    prm = H.to_params(P0)
    prm.brick_order = True
    with pytest.raises(Exception):
        VoxelFusion(wl.grid, occ=d["occ"], params=prm)


def _dense_state(fu, score, labels=None):
    st = H.state_of(fu, score, labels)
    return to_linear(dict(st, score=np.zeros(len(st["W"]), np.float32)), fu.g), st["score"]


@pytest.mark.parametrize("build", [lambda: synth.config1(),
                                   lambda: synth.config2(g=128, W=504, H=378)])
def test_dense_brick_order_matches_linear_order_and_oracle(build):
    """A dense prior in brick order (brick-major words built from the uint8
    grid, the score grid zeroed by the count kernel, warp-level culling): the
    one-call step, views folded one call at a time and an update with its
    zero-fill give the linear-order results bitwise."""
    wl = build()
    d = H.upload(wl)
    out = {}
    for brick in (False, True):
        prm = H.to_params(P0)
        prm.brick_order = brick
        fu = VoxelFusion(wl.grid, occ=d["occ"], params=prm)
        score = torch.full((fu.n_cells,), 7.0, dtype=torch.float32, device="cuda")
        labels = torch.empty(len(d["points"]), dtype=torch.uint8, device="cuda")
        views = PreparedViews(wl.cams, d["depth"], d["mask"], wl.mask_type)
        fu.step(views, occ=d["occ"], score=score, xyz=d["points"], labels=labels)
        torch.cuda.synchronize()
        lin_st, sc = _dense_state(fu, score, labels)
        # the same views again through the incremental update (zero-fill path)
        fu2 = VoxelFusion(wl.grid, occ=d["occ"], params=prm)
        h = max(1, wl.n_views // 2)
        fu2.add_views(wl.cams[:h], d["depth"][:h], d["mask"][:h], mask_type=wl.mask_type)
        score2 = torch.full((fu2.n_cells,), 7.0, dtype=torch.float32, device="cuda")
        fu2.update(PreparedViews(wl.cams[h:], d["depth"][h:], d["mask"][h:], wl.mask_type),
                   score=score2)
        torch.cuda.synchronize()
        upd, sc2 = _dense_state(fu2, score2)
        out[brick] = (lin_st, sc, upd, sc2, fu)
        fu2.close()
    a, b = out[False], out[True]
    for k in ("active", "W", "Z", "bits", "vmask"):
        assert np.array_equal(b[0][k], a[0][k]), k
        assert np.array_equal(b[2][k], a[2][k]), ("update", k)
    assert np.array_equal(b[1], a[1]) and np.array_equal(b[3], a[3]), "dense scores"
    assert np.array_equal(b[0]["seg_dense"], a[0]["seg_dense"])
    assert np.array_equal(b[0]["labels"], a[0]["labels"])
    assert (a[0]["Z"] > 0).any()
    lin_b = dict(b[0], score=b[1])
    H.compare(wl, lin_b, P0, sample=H.sample_of(len(lin_b["W"]), 20_000),
              name=f"{H.current_test()} {wl.name} g={wl.grid.g} dense brick", max_flagged=0.03)
    for v in out.values():
        v[4].close()


@pytest.mark.parametrize("mask_type", [oracle.MASK_F32, oracle.MASK_LOGIT_F32])
def test_culling_with_f32_and_logit_masks(mask_type):
    """The culled fusion on FP32 probability and logit masks (the per-view mask
    type read at run time) gives the unculled linear-order result."""
    import copy
    wl = copy.copy(_small3())
    prob = [m.view(np.float16).astype(np.float32) for m in wl.mask]
    if mask_type == oracle.MASK_F32:
        wl.mask = prob
    else:
        with np.errstate(divide="ignore"):
            wl.mask = [np.log(p / (1.0 - p)).astype(np.float32) for p in prob]
    wl.mask_type = mask_type
    d = H.upload(wl)
    fl, lin_state = _step(wl, d, brick=False)
    fb, brick_state = _step(wl, d, brick=True)
    b = to_linear(brick_state, wl.grid.g)
    for k in ("active", "W", "Z", "bits", "vmask", "score"):
        assert np.array_equal(b[k], lin_state[k]), k
    assert np.array_equal(brick_state["labels"], lin_state["labels"])
    assert (lin_state["Z"] > 0).any()
    fl.close()
    fb.close()


def test_batched_brick_sessions_match_linear_sessions_alone():
    """Brick-ordered sessions in one batched launch (their views culled per
    brick) give each session's linear-order result alone, bitwise."""
    from paper_2601_04860_b300 import Batch, Schedule
    mix = synth.session_mix(n_sessions=64, scale=0.25)
    wls = [synth.session_workload(mix[i]) for i in (1, 3, 9, 21)]
    ups = [H.upload(wl) for wl in wls]
    ref = []
    for wl, d in zip(wls, ups):
        fu = VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=H.to_params(P0))
        fu.add_views(wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
        st = H.state_of(fu, torch.zeros(fu.n_cells if fu.dense else fu.n_active,
                                        device="cuda"))
        ref.append(st)
        fu.close()
    for sched in (Schedule(256, 1, 8, 4096), Schedule(128, 2, 4, 1024)):
        fus = []
        for wl, d in zip(wls, ups):
            prm = H.to_params(P0)
            prm.brick_order = wl.grid.g % 8 == 0
            fus.append(VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=prm))
        b = Batch(max_sessions=8, max_views=256)
        for (wl, d), fu in zip(zip(wls, ups), fus):
            b.queue(fu, wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
        b.fuse(sched)
        torch.cuda.synchronize()
        for wl, fu, r in zip(wls, fus, ref):
            st = to_linear(dict(H.state_of(fu, torch.zeros(fu.n_cells if fu.dense else fu.n_active,
                                                           device="cuda")),
                                score=np.zeros(fu.n_active, np.float32)), wl.grid.g)
            rl = to_linear(dict(r, score=np.zeros(len(r["W"]), np.float32)), wl.grid.g)
            for k in ("active", "W", "Z", "bits"):
                assert np.array_equal(st[k], rl[k]), (wl.name, k)
            fu.close()
        b.close()


def test_culled_step_in_a_cuda_graph():
    """The brick-ordered one-call step with view culling (its culling kernels on
    the context's helper stream, forked and joined by events) captured in a CUDA
    graph and replayed: the eager step's results, bitwise."""
    wl = _small3()
    d = H.upload(wl)
    fe, ref = _step(wl, d, brick=True)
    prm = H.to_params(P0)
    prm.brick_order = True
    fu = VoxelFusion(wl.grid, coords=d["coords"], params=prm)
    score = torch.empty(fu.n_active, dtype=torch.float32, device="cuda")
    labels = torch.empty(len(d["points"]), dtype=torch.uint8, device="cuda")
    views = PreparedViews(wl.cams, d["depth"], d["mask"], wl.mask_type)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fu.step(views, coords=d["coords"], score=score, xyz=d["points"], labels=labels, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fu.step(views, coords=d["coords"], score=score, xyz=d["points"], labels=labels, stream=s)
    score.fill_(7.0)
    labels.fill_(9)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    st = H.state_of(fu, score, labels)
    for k in ("active", "W", "Z", "bits", "vmask", "score", "labels"):
        assert np.array_equal(st[k], ref[k]), k
    fu.close()
    fe.close()


@pytest.mark.parametrize("brick", [False, True])
def test_scatter_unaligned_and_ragged_coordinates(brick):
    """Coordinates at a 4-byte (not 16-byte) aligned address, a count that is
    not a multiple of four and repeated coordinates take the scatter's scalar
    loads and merge: the occupied set of an aligned, de-duplicated copy."""
    wl = _plain_sparse()
    coords = torch.from_numpy(wl.coords).cuda()
    n = coords.shape[0] - 3
    buf = torch.empty(n * 3 + 3 + 1, dtype=torch.int32, device="cuda")
    buf[1:1 + 3 * n].copy_(coords[:n].reshape(-1))
    buf[1 + 3 * n:].copy_(coords[n // 2])  # one repeated coordinate
    unaligned = buf[1:].view(n + 1, 3)
    assert unaligned.data_ptr() % 16 != 0
    prm = H.to_params(P0)
    prm.brick_order = brick
    fa = VoxelFusion(wl.grid, coords=unaligned, params=prm)
    fb = VoxelFusion(wl.grid, coords=coords[:n].clone(), params=prm)
    assert fa.n_active == fb.n_active == n
    assert torch.equal(fa.active_coords(), fb.active_coords())
    fa.set_occupancy(coords=unaligned)
    fa.sync()
    assert torch.equal(fa.active_coords(), fb.active_coords())
    fa.close()
    fb.close()
