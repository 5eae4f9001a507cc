"""Serving loop: every session's result is the same alone and in the mix (GPU),
with and without memory pressure, and for the plain baselines."""
import numpy as np
import pytest
import torch

import synth
from paper_2601_04860_b300 import VoxelFusion
from paper_2601_04860_b300.serve import (
    Server,
    Session,
    latency_summary,
    poisson_requests,
    serve_plain,
    session_data_from,
)

pytestmark = pytest.mark.gpu


def _data(n=8, scale=0.25):
    return [session_data_from(synth.session_workload(r), i)
            for i, r in enumerate(synth.session_mix(n_sessions=n, scale=scale))]


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
    """The session's state after the run, and its outputs recomputed from that
    state (an evicted session is re-admitted from its exported state)."""
    if sid not in server.resident:
        server._admit(sid, set())
    s = server.resident[sid]
    s.fusion.finalize(score=s.score)
    s.fusion.label_points(s.points, out=s.labels)
    torch.cuda.synchronize()
    st = s.fusion.export_state()
    return {"W": st["W"].cpu().numpy(), "Z": st["Z"].cpu().numpy(),
            "bits": st["bits"].cpu().numpy(), "score": s.score.cpu().numpy(),
            "labels": s.labels.cpu().numpy()}


@pytest.mark.parametrize("budget_sessions", [None, 3])
def test_served_results_equal_sessions_alone(budget_sessions):
    data = _data()
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
