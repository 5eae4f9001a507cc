"""Serving loop: every session's result is the same alone and in the mix (GPU),
with and without memory pressure, and for the plain baselines."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import VoxelFusion, seg_bits_to_bool
from paper_2601_04860_b300.serve import (
    Server,
    Session,
    latency_summary,
    poisson_requests,
    serve_plain,
    session_data_from,
)

from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _workloads(n=8, scale=0.25):
    return [synth.session_workload(r) for r in synth.session_mix(n_sessions=n, scale=scale)]


def _data(n=8, scale=0.25, wls=None):
    wls = wls if wls is not None else _workloads(n, scale)
    return [session_data_from(wl, i) for i, wl in enumerate(wls)]


def _check_oracle(wl, got, n_req):
    """A served session's state against the FP64 oracle on the views it was
    sent, in order (views cycle when the requests outnumber them)."""
    seq = H.with_views(wl, [i % wl.n_views for i in range(n_req)])
    gpu = {"n_active": len(got["W"]), "active": got["active"], "score": got["score"],
           "seg_dense": got["seg_dense"], "vmask": got["vmask"], "n_seg": got["n_seg"],
           "W": got["W"], "Z": got["Z"], "bits": got["bits"].view(np.uint32),
           "labels": got["labels"]}
    return H.compare(seq, gpu, oracle.Params(), sample=H.sample_of(len(got["W"]), 20_000),
                     name=f"{H.current_test()} {wl.name} g={wl.grid.g}"
                          f"{' contracted' if wl.grid.contracted else ''} requests={n_req}",
                     max_flagged=0.06)


def _alone(d, n_req):
    """The session served alone: its n_req views in order (cycling)."""
    s = Session(d, torch.device("cuda"))
    for i in range(n_req):
        k = i % d.n_views
        s.fusion.add_view(d.cams[k], s.depth[k], s.mask[k], mask_type=d.mask_type)
    s.fusion.finalize(score=s.score)
    s.fusion.label_points(s.points, out=s.labels)
    st = s.fusion.export_state()
    out = {"W": st["W"].cpu().numpy(), "Z": st["Z"].cpu().numpy(),
           "bits": st["bits"].cpu().numpy(), "score": s.score.cpu().numpy(),
           "labels": s.labels.cpu().numpy()}
    s.close()
    return out


def _final(server, sid):
    """The session's state after the run: W, Z, bits, and the score and labels
    the server's last batch left in the session's buffers; an evicted session
    is re-admitted from its exported state and finalized again."""
    if sid not in server.resident:
        server._admit(sid, set())
        s = server.resident[sid]
        s.fusion.finalize(score=s.score)
        s.fusion.label_points(s.points, out=s.labels)
    s = server.resident[sid]
    torch.cuda.synchronize()
    st = s.fusion.export_state()
    fin = s.fusion.finalize(score=False, seg_bits=True, vmask=True, count=True)
    return {"W": st["W"].cpu().numpy(), "Z": st["Z"].cpu().numpy(),
            "bits": st["bits"].cpu().numpy(), "score": s.score.cpu().numpy(),
            "labels": s.labels.cpu().numpy(), "active": s.fusion.active_coords().cpu().numpy(),
            "seg_dense": seg_bits_to_bool(fin["seg_bits"], s.fusion.n_cells).cpu().numpy(),
            "vmask": fin["vmask"].cpu().numpy().view(np.uint32), "n_seg": fin["n_seg"]}


@pytest.mark.parametrize("budget_sessions", [None, 3])
def test_served_results_equal_sessions_alone(budget_sessions):
    wls = _workloads()
    data = _data(wls=wls)
    foot = [Session.footprint(d) for d in data]
    budget = sum(foot) + 1 if budget_sessions is None else sorted(foot)[-budget_sessions:]
    budget = budget if isinstance(budget, int) else sum(budget)
    reqs = poisson_requests(80, 3000.0, [d.sid for d in data])
    srv = Server(data, memory_budget=budget, max_batch=8)
    srv.run(reqs)
    assert all(r.done >= r.arrival for r in reqs)
    summ = latency_summary(reqs)
    assert summ["requests"] == 80 and summ["mean_batch"] > 1.0
    if budget_sessions is not None:
        assert srv.stats["evictions"] > 0
    n_req = {d.sid: sum(r.sid == d.sid for r in reqs) for d in data}
    for d in data:
        if n_req[d.sid] == 0:
            continue
        got = _final(srv, d.sid)
        ref = _alone(d, n_req[d.sid])
        for k in ("W", "Z", "bits", "score", "labels"):
            assert np.array_equal(got[k], ref[k]), (d.sid, k)
        _check_oracle(wls[d.sid], got, n_req[d.sid])
    srv.close()


def test_served_full_size_sessions_match_oracle():
    """The server on config-5 sessions at full size (the largest dense grid,
    384^3; sparse contracted sets; 2-6 views, 640x480 .. 1297x840): every
    session's served state against the FP64 oracle on sampled voxels."""
    mix = synth.session_mix(n_sessions=64, scale=1.0)
    wls = [synth.session_workload(mix[i]) for i in (3, 21, 49, 56, 9, 0)]
    data = _data(wls=wls)
    reqs = poisson_requests(30, 2000.0, [d.sid for d in data], seed=11)
    srv = Server(data, memory_budget=sum(Session.footprint(d) for d in data) + 1, max_batch=8)
    srv.run(reqs)
    n_req = {d.sid: sum(r.sid == d.sid for r in reqs) for d in data}
    checked = 0
    for d in data:
        if n_req[d.sid] == 0:
            continue
        _check_oracle(wls[d.sid], _final(srv, d.sid), n_req[d.sid])
        checked += 1
    assert checked >= 4
    srv.close()


def test_plain_baselines_agree_with_the_server():
    data = _data(n=4)
    reqs = poisson_requests(24, 5000.0, [d.sid for d in data], seed=7)
    n_req = {d.sid: sum(r.sid == d.sid for r in reqs) for d in data}
    for mode in ("refuse", "incremental"):
        rs = poisson_requests(24, 5000.0, [d.sid for d in data], seed=7)
        serve_plain(data, rs, mode)
        assert latency_summary(rs)["requests"] == 24
    # plain runs keep no state; check the re-fusion path against incremental alone
    for d in data[:2]:
        if n_req[d.sid] == 0:
            continue
        s = Session(d, torch.device("cuda"))
        idx = [i % d.n_views for i in range(n_req[d.sid])]
        s.fusion.add_views([d.cams[i] for i in idx], [s.depth[i] for i in idx],
                           [s.mask[i] for i in idx], mask_type=d.mask_type)
        s.fusion.finalize(score=s.score)
        ref = _alone(d, n_req[d.sid])
        assert np.array_equal(s.score.cpu().numpy(), ref["score"])
        s.close()
