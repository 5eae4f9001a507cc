"""Interactive serving of many fusion sessions with continuous batching.

A *session* is one scene being segmented (Sec. 3.7: after each centroid view
the user's new mask is fused and the 3D mask is shown again).  A *request*
adds the session's next view and asks for the updated scores and point
labels.  The server

* keeps every admitted session's accumulators (W, Z, view bits), its active
  list and its inputs resident on the device, and folds each new view in
  incrementally (no re-fusion of earlier views);
* admits sessions while their device footprint fits a memory budget; when a
  session cannot fit, idle sessions are evicted (their state is exported to
  host memory and re-imported when they are needed again, bit-exactly);
* batches continuously: every time the GPU has room (at most ``max_inflight``
  batches in flight, each on its own stream), all requests that have arrived
  for sessions that are admitted and not already in flight form one batch --
  one persistent fuse launch plus one finalize and one label launch -- so
  requests arriving while others run join the next batch and their work
  overlaps on the device.

Latency is measured from a request's arrival (host clock) to the moment the
host observes the completion event of the batch that served it.  Two plain
baselines serve the same request stream one request at a time: ``refuse``
(one launch per request that re-fuses all of the session's views so far, as
the paper's interactive update does) and ``incremental`` (one add_view +
finalize + labels per request, no batching).
"""
from __future__ import annotations

import ctypes
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L
from .batch import Autotuner, Batch, Schedule
from .fusion import FusionParams, PreparedViews, VoxelFusion, view_c


@dataclass
class SessionData:
    """Host-side description of one session's scene and views."""

    sid: int
    grid: object
    occ: np.ndarray | None
    coords: np.ndarray | None
    cams: list
    depth: list            # numpy float32 (H, W)
    mask: list             # numpy (binary16 bits as float16 view, or float32)
    mask_type: int
    points: np.ndarray
    params: FusionParams = field(default_factory=FusionParams)

    @property
    def n_views(self) -> int:
        return len(self.cams)


def _tensor(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


class Session:
    """A session admitted on the device."""

    def __init__(self, data: SessionData, dev):
        self.data = data
        self.occ = None if data.occ is None else _tensor(data.occ, dev)
        self.coords = None if data.coords is None else _tensor(data.coords, dev)
        self.depth = [_tensor(d, dev) for d in data.depth]
        if data.mask_type == 1:
            self.mask = [_tensor(m.view(np.float16), dev) for m in data.mask]
        else:
            self.mask = [_tensor(m, dev) for m in data.mask]
        self.points = _tensor(data.points, dev)
        self.fusion = VoxelFusion(data.grid, occ=self.occ, coords=self.coords, params=data.params)
        # one marshalled view struct per view, reused by every request
        self.view_c = [view_c(data.cams[k], self.depth[k], self.mask[k], data.mask_type)
                       for k in range(data.n_views)]
        n_score = self.fusion.n_cells if self.fusion.dense else self.fusion.n_active
        # zero-initialised and only ever written by this session: its unoccupied
        # cells stay 0, so updates write the active voxels' scores only
        self.score = torch.zeros(n_score, dtype=torch.float32, device=dev)
        self.labels = torch.empty(len(data.points), dtype=torch.uint8, device=dev)
        self.views_done = 0
        # the C-ABI arguments of a request, marshalled once
        self.c_score = ctypes.c_void_p(self.score.data_ptr())
        self.c_points = ctypes.c_void_p(self.points.data_ptr())
        self.c_labels = ctypes.c_void_p(self.labels.data_ptr())
        self.n_points = int(self.points.shape[0])
        self.c_views = [ctypes.pointer(v) for v in self.view_c]

    @staticmethod
    def footprint(data: SessionData) -> int:
        """Device bytes a session holds while admitted (inputs, state, outputs)."""
        g3 = int(data.grid.g) ** 3
        n_act = int(np.count_nonzero(data.occ)) if data.occ is not None else len(data.coords)
        inputs = sum(d.nbytes + m.nbytes for d, m in zip(data.depth, data.mask))
        inputs += data.points.nbytes + (data.occ.nbytes if data.occ is not None else
                                        data.coords.nbytes)
        state = 16 * n_act + 3 * (g3 // 8) + 64
        out = (4 * g3 if data.occ is not None else 4 * n_act) + len(data.points)
        return inputs + state + out

    def export(self):
        st = self.fusion.export_state()
        return {k: (v.cpu() if isinstance(v, torch.Tensor) else v) for k, v in st.items()}

    def close(self):
        self.fusion.close()


@dataclass
class Request:
    rid: int
    sid: int
    arrival: float          # seconds from the start of the run (host clock)
    done: float = -1.0
    batch_size: int = 0


class Server:
    """Continuous-batching server over resident sessions."""

    def __init__(self, sessions: list[SessionData], memory_budget: int, device=None,
                 max_batch: int = 64, max_inflight: int = 2, autotune: bool = False,
                 schedule: Schedule | None = None, session_factory=None, footprint=None):
        self.dev = torch.device(device or "cuda")
        # how sessions are created and sized (replaceable for host-side tests)
        self.session_factory = session_factory or Session
        self.footprint = footprint or Session.footprint
        self.data = {s.sid: s for s in sessions}
        self.budget = int(memory_budget)
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.resident: dict[int, Session] = {}
        self.evicted: dict[int, dict] = {}
        self.views_done: dict[int, int] = {s.sid: 0 for s in sessions}
        self.used = 0
        self.last_use: dict[int, float] = {}
        self.streams, self.batches = [], []
        if session_factory is None:  # a real server launches batches on its own streams
            self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(max_inflight)]
            self.batches = [Batch(max_sessions=max_batch, max_views=max_batch)
                            for _ in range(max_inflight)]
            # per stream slot: its raw handle and one completion event, reused
            # (a slot is only reused after its event completed)
            self.c_streams = [ctypes.c_void_p(st.cuda_stream) for st in self.streams]
            self.events = [torch.cuda.Event() for _ in range(max_inflight)]
            self.lib = L.load()
        self.tuner = Autotuner() if autotune else None
        self.schedule = schedule or Schedule()
        self.c_schedule = self.schedule.c()
        self.stats = {"batches": 0, "evictions": 0, "admissions": 0, "batch_sizes": []}

    # -- memory admission ---------------------------------------------------
    def _admit(self, sid: int, busy: set) -> bool:
        if sid in self.resident:
            return True
        need = self.footprint(self.data[sid])
        if need > self.budget:
            raise ValueError(f"session {sid} needs {need} bytes, above the whole budget")
        # evict idle sessions, least recently used first
        while self.used + need > self.budget:
            idle = [s for s in self.resident if s not in busy]
            if not idle:
                return False
            victim = min(idle, key=lambda s: self.last_use.get(s, -1.0))
            self._evict(victim)
        sess = self.session_factory(self.data[sid], self.dev)
        if sid in self.evicted:
            st = self.evicted.pop(sid)
            sess.fusion.import_state({k: (v.to(self.dev) if isinstance(v, torch.Tensor) else v)
                                      for k, v in st.items()})
        sess.views_done = self.views_done[sid]
        self.resident[sid] = sess
        self.used += need
        self.stats["admissions"] += 1
        return True

    def _evict(self, sid: int):
        sess = self.resident.pop(sid)
        if self.dev.type == "cuda" and torch.cuda.is_available():
            torch.cuda.synchronize(self.dev)
        self.evicted[sid] = sess.export()
        sess.close()
        self.used -= self.footprint(self.data[sid])
        self.stats["evictions"] += 1

    def admit_all(self) -> int:
        """Admit sessions up front while the budget allows; returns how many."""
        for sid in self.data:
            if sid in self.resident:
                continue
            if self.used + self.footprint(self.data[sid]) > self.budget:
                break
            self._admit(sid, set())
        if self.dev.type == "cuda" and torch.cuda.is_available():
            torch.cuda.synchronize(self.dev)
        return len(self.resident)

    # -- the loop -------------------------------------------------------------
    def run(self, requests: list[Request], t0: float | None = None) -> list[Request]:
        """Serve requests (sorted by arrival, seconds from t0) in real time."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque[Request] = deque()
        inflight = []   # (event, batch, requests, stream index)
        free = list(range(self.max_inflight))
        t0 = time.perf_counter() if t0 is None else t0
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # completions
            still = []
            for ev, b, reqs, si in inflight:
                if ev.query():
                    t = time.perf_counter() - t0
                    for r in reqs:
                        r.done = t
                    free.append(si)
                else:
                    still.append((ev, b, reqs, si))
            inflight = still
            busy = {r.sid for _, _, reqs, _ in inflight for r in reqs}
            if waiting and free:
                picked, seen, rest = [], set(), deque()
                while waiting:
                    r = waiting.popleft()
                    if (r.sid in busy or r.sid in seen or len(picked) >= self.max_batch
                            or not self._admit(r.sid, busy | seen)):
                        rest.append(r)
                    else:
                        picked.append(r)
                        seen.add(r.sid)
                waiting = rest
                if picked:
                    si = free.pop()
                    inflight.append(self._launch(picked, si))
                    continue
            if not waiting and not inflight and pending:
                # sleep until shortly before the next arrival, then poll (the
                # scheduler's wake-up overshoots short sleeps by tens of us)
                gap = pending[0].arrival - now
                if gap > 3e-4:
                    time.sleep(min(1e-3, gap - 2e-4))
        return requests

    def _launch(self, picked: list[Request], si: int):
        b = self.batches[si]
        st = self.streams[si]
        sess, views = [], []
        for r in picked:
            s = self.resident[r.sid]
            views.append(s.view_c[s.views_done % s.data.n_views])  # sessions cycle their views
            s.views_done += 1
            self.views_done[r.sid] = s.views_done
            self.last_use[r.sid] = time.perf_counter()
            sess.append(s)
        cs = self.c_streams[si]
        lib = self.lib
        if len(sess) == 1:
            # a lone request: the session's own launches (fold + finalize,
            # labels) cost less than staging a batch; bitwise the same result.
            # The C ABI is called with the session's pre-marshalled arguments.
            s = sess[0]
            h = s.fusion.handle
            k = (s.views_done - 1) % s.data.n_views
            L.check(lib.divas_fuse_update(h, s.c_views[k], 1, s.c_score, None, L.KEEP_ZEROS, cs),
                    h)
            L.check(lib.divas_label_points(h, s.c_points, s.n_points, s.c_labels, cs), h)
        elif self.tuner is not None:
            with torch.cuda.stream(st):
                for s, v in zip(sess, views):
                    b.queue_prepared(s.fusion, v)
                sch = self.tuner.pick(b, 1, candidates=[Schedule(256, 1, 8, 4096),
                                                        Schedule(256, 2, 8, 8192),
                                                        Schedule(128, 1, 16, 2048)])
                b.fuse(sch)
                b.finalize(scores=[s.score for s in sess], points=[s.points for s in sess],
                           labels=[s.labels for s in sess], keep_zeros=True)
        else:
            # the batch through the C ABI with the sessions' pre-marshalled
            # arguments: queue, one persistent fuse launch, one finalize
            bh = b._h
            for s in sess:
                k = (s.views_done - 1) % s.data.n_views
                b._check(lib.divas_batch_queue(bh, s.fusion.handle, s.c_views[k], 1))
            b._check(lib.divas_batch_fuse(bh, ctypes.byref(self.c_schedule), 0, cs))
            n = len(sess)
            sc = (ctypes.c_void_p * n)(*[s.c_score.value for s in sess])
            pts = (ctypes.c_void_p * n)(*[s.c_points.value for s in sess])
            npts = (ctypes.c_int64 * n)(*[s.n_points for s in sess])
            lab = (ctypes.c_void_p * n)(*[s.c_labels.value for s in sess])
            b._check(lib.divas_batch_finalize(bh, sc, pts, npts, lab, L.KEEP_ZEROS, cs))
        ev = self.events[si]
        ev.record(st)
        self.stats["batches"] += 1
        self.stats["batch_sizes"].append(len(picked))
        for r in picked:
            r.batch_size = len(picked)
        return ev, b, picked, si

    def close(self):
        if self.dev.type == "cuda" and torch.cuda.is_available():
            torch.cuda.synchronize(self.dev)
        for s in self.resident.values():
            s.close()
        self.resident.clear()
        for b in self.batches:
            b.close()


def poisson_requests(n: int, rate: float, sessions: list[int], seed: int = 1009) -> list[Request]:
    """n requests with exponential inter-arrival times (rate per second), each for
    a session drawn uniformly from ``sessions``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    sids = rng.choice(np.asarray(sessions), size=n)
    return [Request(i, int(s), float(a)) for i, (s, a) in enumerate(zip(sids, t))]


def serve_plain(sessions: list[SessionData], requests: list[Request], mode: str,
                device=None) -> list[Request]:
    """Baselines, one request at a time in arrival order: ``refuse`` re-fuses all
    of the session's views so far in one launch per request; ``incremental``
    folds the new view in (one add_view + finalize + labels per request)."""
    dev = torch.device(device or "cuda")
    res = {s.sid: Session(s, dev) for s in sessions}
    prepared = {}
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        s = res[r.sid]
        nv = s.data.n_views
        k = s.views_done % nv
        if mode == "refuse":
            s.fusion.reset()
            upto = s.views_done + 1
            idx = [(i % nv) for i in range(upto)]
            for c0 in range(0, upto, 32):
                part = idx[c0:c0 + 32]
                key = (r.sid, tuple(part))
                if key not in prepared:
                    prepared[key] = PreparedViews([s.data.cams[i] for i in part],
                                                  [s.depth[i] for i in part],
                                                  [s.mask[i] for i in part], s.data.mask_type)
                s.fusion.add_views(prepared[key])
        else:
            s.fusion.add_view(s.data.cams[k], s.depth[k], s.mask[k], mask_type=s.data.mask_type)
        s.views_done += 1
        s.fusion.finalize(score=s.score)
        s.fusion.label_points(s.points, out=s.labels)
        torch.cuda.current_stream().synchronize()
        r.done = time.perf_counter() - t0
        r.batch_size = 1
    torch.cuda.synchronize(dev)
    for s in res.values():
        s.close()
    return requests


def latency_summary(requests: list[Request]) -> dict:
    lat = np.array([(r.done - r.arrival) * 1e3 for r in requests if r.done >= 0])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "throughput_rps": len(lat) / span if span > 0 else float("nan"),
            "mean_batch": float(np.mean([r.batch_size for r in requests]))}


def session_data_from(wl, sid: int, params: FusionParams | None = None) -> SessionData:
    """SessionData of a synthetic workload (any object with the Workload fields)."""
    return SessionData(sid, wl.grid, wl.occ, wl.coords, list(wl.cams), list(wl.depth),
                       list(wl.mask), wl.mask_type, wl.points, params or FusionParams())
