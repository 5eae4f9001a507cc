"""Batched sessions: one persistent launch over uneven sessions gives every
session the result it gets alone, bitwise (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import Autotuner, Batch, Schedule, VoxelFusion, seg_bits_to_bool
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

P0 = oracle.Params()


def _sessions():
    recipes = synth.session_mix(n_sessions=10, scale=0.25)
    out = []
    for r in recipes:
        wl = synth.session_workload(r)
        out.append((wl, H.upload(wl)))
    return out


def _alone(wl, d):
    fu = VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=H.to_params(P0))
    fu.add_views(wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
    out = fu.finalize(score=True, seg_bits=True)
    lab = fu.label_points(d["points"])
    st = fu.export_state()
    res = {"score": out["score"].cpu().numpy(), "W": st["W"].cpu().numpy(),
           "Z": st["Z"].cpu().numpy(), "bits": st["bits"].cpu().numpy(),
           "labels": lab.cpu().numpy()}
    fu.close()
    return res


@pytest.mark.parametrize("sched", [Schedule(256, 1, 8, 4096), Schedule(128, 2, 4, 1024),
                                   Schedule(64, 4, 16, 256)])
def test_batch_matches_sessions_alone(sched):
    sess = _sessions()
    ref = [_alone(wl, d) for wl, d in sess]
    fus = [VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=H.to_params(P0))
           for wl, d in sess]
    b = Batch(max_sessions=16, max_views=256)
    # two passes: views split in two batches (accumulation across batches)
    for lo, hi in ((0, 1), (1, None)):
        for (wl, d), fu in zip(sess, fus):
            h = max(1, wl.n_views // 2)
            sl = slice(0, h) if lo == 0 else slice(h, None)
            if len(wl.cams[sl]) == 0:
                continue
            b.queue(fu, wl.cams[sl], d["depth"][sl], d["mask"][sl], mask_type=wl.mask_type)
        queued = list(b.sessions)
        b.fuse(sched, dry_run=True)     # a dry run leaves the sessions untouched
        b.fuse(sched)
        scores = [torch.empty(f.n_cells if f.dense else f.n_active, device="cuda")
                  for f in queued]
        labs = []
        pts = []
        for f in queued:
            i = fus.index(f)
            pts.append(sess[i][1]["points"])
            labs.append(torch.empty(len(sess[i][1]["points"]), dtype=torch.uint8, device="cuda"))
        b.finalize(scores=scores, points=pts, labels=labs)
    torch.cuda.synchronize()
    for (wl, d), fu, r in zip(sess, fus, ref):
        st = fu.export_state()
        assert np.array_equal(st["W"].cpu().numpy(), r["W"])
        assert np.array_equal(st["Z"].cpu().numpy(), r["Z"])
        assert np.array_equal(st["bits"].cpu().numpy(), r["bits"])
    # the last finalize covered every session with views in the second pass
    for f, sc, lab in zip(queued, scores, labs):
        i = fus.index(f)
        assert np.array_equal(sc.cpu().numpy(), ref[i]["score"])
        assert np.array_equal(lab.cpu().numpy(), ref[i]["labels"])
    for f in fus:
        f.close()
    b.close()


def test_autotuner_picks_a_schedule_and_results_hold():
    sess = _sessions()[:6]
    fus = [VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=H.to_params(P0))
           for wl, d in sess]
    b = Batch()
    for (wl, d), fu in zip(sess, fus):
        b.queue(fu, wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
    tuner = Autotuner(reps=1)
    cands = [Schedule(256, 1, 8, 4096), Schedule(128, 2, 8, 1024), Schedule(256, 4, 4, 4096)]
    sch = tuner.pick(b, 12, candidates=cands)
    assert sch in cands
    b.fuse(sch)
    b.finalize()
    torch.cuda.synchronize()
    for (wl, d), fu in zip(sess, fus):
        r = _alone(wl, d)
        assert np.array_equal(fu.export_state()["W"].cpu().numpy(), r["W"])
        fu.close()


# the config-5 session mix at full size: the largest dense grid (384^3), two
# sparse contracted sets, small and mid dense grids; 2-6 views per session at
# 640x480 .. 1297x840
FULL_MIX = (3, 21, 49, 56, 9, 0)


def test_batched_sessions_match_oracle():
    """Every session folded by the batched persistent launch (and finalized
    and labelled by the batched finalize) against the FP64 oracle on sampled
    voxels: Eq. compact-fusion per session, whatever the mix around it."""
    mix = synth.session_mix(n_sessions=64, scale=1.0)
    sess = []
    for i in FULL_MIX:
        wl = synth.session_workload(mix[i])
        sess.append((wl, H.upload(wl)))
    assert any(wl.grid.contracted for wl, _ in sess) and max(wl.grid.g for wl, _ in sess) == 384
    fus = [VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=H.to_params(P0))
           for wl, d in sess]
    b = Batch(max_sessions=16, max_views=256)
    for (wl, d), fu in zip(sess, fus):
        b.queue(fu, wl.cams, d["depth"], d["mask"], mask_type=wl.mask_type)
    b.fuse(Schedule(256, 1, 8, 4096))
    scores = [torch.empty(f.n_cells if f.dense else f.n_active, device="cuda") for f in fus]
    labs = [torch.empty(len(d["points"]), dtype=torch.uint8, device="cuda") for _, d in sess]
    b.finalize(scores=scores, points=[d["points"] for _, d in sess], labels=labs)
    torch.cuda.synchronize()
    for (wl, d), fu, sc, lab in zip(sess, fus, scores, labs):
        gpu = H.state_of(fu, sc, lab)
        s = H.compare(wl, gpu, P0, sample=H.sample_of(fu.n_active, 20_000),
                      name=f"{H.current_test()} {wl.name} g={wl.grid.g}"
                           f"{' contracted' if wl.grid.contracted else ''}",
                      max_flagged=0.06)
        assert s["voted"] > 0
        fu.close()
    b.close()
