#!/usr/bin/env python
"""Benchmark of the depth-weighted multi-view voxel fusion hot path.

One step = one pass of the whole hot path over one synthetic scene shaped
like the paper's forward-facing workload (LLFF-like, Sec. 4.1): 256^3 dense
grid over [-1, 1]^3 (16.8M voxels), 8 anchor views of 1008x756 (FP32 planar
depth, FP16 soft masks) ray-cast from 200 seeded ellipsoids and a back
plane, a ~5 % surface-shell occupancy prior and 1M points to label:

  A1  occupancy prior -> active list             (4 kernels)
  A2-A6 project / gate / depth-weight / accumulate, 8 views in one launch
  A7  normalise + consensus -> dense 256^3 score grid + seg bitfield
  A8  Pass 1 labels of 1M points

``value`` = nominal voxel-view updates/s = g^3 x views / step time, all
inputs resident in HBM, L2 flushed between timed steps.  ``e2e`` = the same
metric through the public API with pinned host buffers: every step copies all
of its inputs in and its outputs (V_seg bitfield, point labels) out inside the
timed region, copies of one step overlapping the kernels of the next.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload.  Under torchrun every rank runs an
independent replica (the path has no exchange step): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("voxel-view updates/s and per-update fusion ms p50/p99 vs plain launch; "
          "% HBM roofline")
UNIT = "voxel-view updates/s"
WORKLOADS = {
    "forward-dense-256": "256^3 dense grid, 8 views 1008x756 FP32 depth + FP16 masks, "
                         "200 ellipsoids + back plane, 1M points",
    "unbounded-sparse-512": "contracted 512^3 grid, 12M sparse occupied voxels, 16 views "
                            "1297x840, 1000 ellipsoids on a ground plane, 3M points",
}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# DRAM traffic per launch of the one-call step's kernels, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only while the sources
# those kernels are compiled from are byte-identical to the ones profiled.  The
# other modes' kernels live in their own files (included after the step
# kernels, in their own functions), and the header declares host types only,
# so they are not part of the hash.
STEP_SOURCES = ("paper_2601_04860_b300/csrc/divas_fuse.cu",
                "paper_2601_04860_b300/csrc/fuse_math.cuh")
TRAFFIC_CAPTURE = {
    "source_sha1": "f85cc2b98d0769c4b02d830db8d3249398a36aa3",
    "forward-dense-256": {"k_fuse_fin": 28_112_384 + 18_184_448,
                          "k_tile_count": 16_800_256 + 2_048, "k_tile_emit": 2_369_280,
                          "k_label": 13_339_904},
}


def source_sha1() -> str:
    """sha1 over 'sha1  path' lines of the step kernels' sources (as sha1sum
    would print them)."""
    import hashlib
    lines = []
    for f in STEP_SOURCES:
        h = hashlib.sha1(open(os.path.join(ROOT, f), "rb").read()).hexdigest()
        lines.append(f"{h}  {f}\n")
    return hashlib.sha1("".join(lines).encode()).hexdigest()


def traffic_for(workload, kernel):
    if source_sha1() != TRAFFIC_CAPTURE["source_sha1"]:
        return None  # the kernel changed since the counters were taken
    return TRAFFIC_CAPTURE.get(workload, {}).get(kernel)


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks (the slowest rank times the job)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job rate: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


# warp instructions per voxel-view of the contracted fusion kernel on the
# unbounded-sparse workload (ncu smsp__inst_executed.sum of one launch divided
# by its 12M active voxels x 16 views), per active-list order: brick order runs
# k_fuse_fin_cull (316,070,407 per launch), linear order k_fuse_fin (435,256,325)
SPARSE_FUSE_INSTS_PER_VOXEL_VIEW = {"brick": 316_070_407 / 192e6, "linear": 435_256_325 / 192e6}


ACTIVE_ORDER = "auto"  # --active-order


def fusion_params(wl):
    """Fusion constants for a workload: the active list brick-major (warp-level
    view culling; per-voxel results unchanged) for --active-order brick, and
    for auto on sparse priors; grids need a multiple of 8 voxels per side.
    Auto keeps dense priors linear: on the 256^3 scene the culled step
    measured no faster (62.2 vs 61.8 us)."""
    from paper_2601_04860_b300 import FusionParams
    brick = ACTIVE_ORDER == "brick" or (ACTIVE_ORDER == "auto" and wl.coords is not None)
    return FusionParams(brick_order=brick and wl.grid.g % 8 == 0)


def linear_state(fu, st: dict, score, dense: bool) -> dict:
    """W, Z, view bits (and a sparse score) of a context in ascending linear
    order of their voxels, whatever the context's active order."""
    out = {"W": st["W"].cpu().numpy(), "Z": st["Z"].cpu().numpy(),
           "bits": st["bits"].cpu().numpy().view(np.uint32), "score": score.cpu().numpy()}
    act = fu.active_coords().cpu().numpy().astype(np.int64)
    g = fu.g
    o = np.argsort((act[:, 2] * g + act[:, 1]) * g + act[:, 0], kind="stable")
    for k in ("W", "Z", "bits"):
        out[k] = out[k][o]
    if not dense:
        out["score"] = out["score"][o]
    return out


def make_workload(name):
    import synth
    if name == "forward-dense-256":
        return synth.config2()
    if name == "unbounded-sparse-512":
        return synth.config3()
    raise SystemExit(f"unknown workload {name}")


class L2Flush:
    """Between timed iterations: writes a 256 MB buffer (twice the 126 MB L2),
    then reads another 256 MB buffer, so that no line of the step's data is left
    in L2 and the flush's own dirty lines are written back before the next
    timed region rather than inside it."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.r = torch.ones(64 << 20, dtype=torch.float32, device=dev)

    def zero_(self):
        self.w.zero_()
        self.r.sum()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "100"], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# --------------------------------------------------------------------------
def oracle_rate(wl, seconds: float, seed: int = 0, repeats: int = 3):
    """Time the FP64 oracle on a random sample of the active voxels (all views)
    and of the points; returns the extrapolated full-step seconds (the median
    of `repeats` timed runs of the same sample) and details with the spread."""
    import oracle
    cores = oracle.set_threads(0)
    lin = wl.active_linear()
    rng = np.random.Generator(np.random.PCG64(seed))
    prm = oracle.Params()
    pilot = rng.choice(len(lin), size=min(len(lin), 20000), replace=False)
    t0 = time.perf_counter()
    oracle.fuse(wl.grid, lin[pilot], wl.cams, wl.depth, wl.mask, wl.mask_type, prm)
    t_pilot = time.perf_counter() - t0
    per_run = seconds / max(1, repeats)
    n = int(min(len(lin), max(1000, len(pilot) * 0.8 * per_run / max(t_pilot, 1e-6))))
    sample = np.sort(rng.choice(len(lin), size=n, replace=False))
    npts = min(len(wl.points), 300_000)
    fulls, fuse_s, label_s = [], [], []
    for _ in range(max(1, repeats)):
        t0 = time.perf_counter()
        out = oracle.fuse(wl.grid, lin[sample], wl.cams, wl.depth, wl.mask, wl.mask_type, prm)
        t_fuse = time.perf_counter() - t0
        seg = oracle.dense_seg(wl.grid, lin[sample], out["seg"])
        t0 = time.perf_counter()
        oracle.label(wl.grid, seg, wl.points[:npts])
        t_lab = time.perf_counter() - t0
        fulls.append(t_fuse * len(lin) / n + t_lab * len(wl.points) / npts)
        fuse_s.append(t_fuse)
        label_s.append(t_lab)
    full = float(np.median(fulls))
    return full, {"cores": cores, "sample_voxels": n, "active_voxels": int(len(lin)),
                  "sample_points": npts, "fuse_s": float(np.median(fuse_s)),
                  "label_s": float(np.median(label_s)), "repeats": len(fulls),
                  "full_s_min": float(min(fulls)), "full_s_max": float(max(fulls)),
                  "sample_index": sample, "sample_out": out}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
KERNEL_OF = {"compaction": "k_tile_count+k_tile_emit", "fuse": "k_fuse",
             "finalize": "k_finalize", "label": "k_label", "fuse_finalize": "k_fuse_fin"}


def algorithmic_bytes(wl, n_active):
    """Bytes the method must move per step, per kernel (first touch only)."""
    g3 = wl.n_voxels if wl.occ is not None else None
    S = wl.n_views
    view_bytes = sum(d.nbytes + m.nbytes for d, m in zip(wl.depth, wl.mask))
    npts = len(wl.points)
    cells = int(wl.grid.g) ** 3
    zeros = 0
    if wl.occ is not None:
        comp = cells + cells // 8 + 4 * n_active          # occ read, bits, active list
        fin = cells // 8 + 8 * n_active + 4 * cells + cells // 8  # bits, W+Z, P, seg
        zeros = 4 * (cells - n_active) + cells // 8       # unoccupied score cells, bits read
    else:
        comp = 12 * len(wl.coords) + cells // 8 + 4 * n_active
        fin = 8 * n_active + 4 * n_active + cells // 8
    fuse = 4 * n_active + 12 * n_active + view_bytes        # index, W+Z+bits, rasters
    lab = 13 * npts + cells // 8
    algo = {"compaction": comp + cells // 8,                # + the seg clear (step)
            "fuse": fuse, "finalize": fin, "label": lab,
            # + P of the active voxels, seg bits, zeros of the unoccupied cells
            "fuse_finalize": fuse + 4 * n_active + cells // 8 + zeros}
    return algo, view_bytes, S, g3


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2601_04860_b300 import FusionParams, PreparedViews, VoxelFusion

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = make_workload(args.workload)
    occ = None if wl.occ is None else torch.from_numpy(wl.occ).to(dev)
    coords = None if wl.coords is None else torch.from_numpy(wl.coords).to(dev)
    depth = [torch.from_numpy(d).to(dev) for d in wl.depth]
    if wl.mask_type == 1:
        mask = [torch.from_numpy(m.view(np.float16)).to(dev) for m in wl.mask]
    else:
        mask = [torch.from_numpy(m).to(dev) for m in wl.mask]
    pts = torch.from_numpy(np.ascontiguousarray(wl.points)).to(dev)
    fu = VoxelFusion(wl.grid, occ=occ, coords=coords, params=fusion_params(wl))
    n_active = fu.n_active
    dense = wl.occ is not None
    score = torch.empty(fu.n_cells if dense else n_active, dtype=torch.float32, device=dev)
    labels = torch.empty(len(wl.points), dtype=torch.uint8, device=dev)
    flush = L2Flush(dev)
    S = wl.n_views
    N = fu.n_cells if dense else n_active
    pv = PreparedViews(wl.cams, depth, mask, wl.mask_type)
    phases = ["compaction", "fuse", "finalize", "label"]
    kernels_per_phase = {"compaction": 2 if dense else 3, "fuse": math.ceil(S / 32),
                         "finalize": 1, "label": 1}
    # the one-call step: compaction (2 or 3 kernels), fusion + finalize (1, which on a
    # dense grid also writes the zeros of the unoccupied score cells), labels (1)
    step_phases = ["compaction", "fuse_finalize", "label"]
    step_kernels = {"compaction": 2 if dense else 3, "fuse_finalize": 1, "label": 1}

    def step(ev=None):
        if ev:
            ev[0].record()
        fu.set_occupancy(occ=occ, coords=coords)
        if ev:
            ev[1].record()
        fu.add_views(pv)
        if ev:
            ev[2].record()
        fu.finalize(score=score)
        if ev:
            ev[3].record()
        fu.label_points(pts, out=labels)
        if ev:
            ev[4].record()

    # eager warm-up on a side stream, then capture one step in a CUDA graph whose
    # event-record nodes time each phase on the device
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(5)]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(ev)
    for _ in range(args.warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    # the headline step: the same work through the one-call entry point (four
    # launches); its stage events become event-record nodes of the graph
    pv_all = pv if len(pv.chunks) == 1 else None
    fast = None
    if pv_all is not None:
        with torch.cuda.stream(side):
            for _ in range(3):
                fu.step(pv_all, occ=occ, coords=coords, score=score, xyz=pts, labels=labels)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        fev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(4)]
        sev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(4)]
        for e in fev + sev:
            e.record()  # creates the events (torch creates them on first record)
        torch.cuda.synchronize()
        # the timed graph has events around the step only; a second graph of the
        # same step also marks the stage boundaries
        fast = torch.cuda.CUDAGraph()
        with torch.cuda.graph(fast):
            fu.step(pv_all, occ=occ, coords=coords, score=score, xyz=pts, labels=labels,
                    stage_events=[fev[0], None, None, fev[3]])
        staged = torch.cuda.CUDAGraph()
        with torch.cuda.graph(staged):
            fu.step(pv_all, occ=occ, coords=coords, score=score, xyz=pts, labels=labels,
                    stage_events=sev)
        for _ in range(args.warmup):
            flush.zero_()
            fast.replay()
            flush.zero_()
            staged.replay()
        torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    step_ms, phase, sep_ms = [], {k: [] for k in phases}, []
    sphase = {k: [] for k in step_phases}
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (not inside the graph's events)
        if fast is not None:
            fast.replay()
            torch.cuda.synchronize()
            step_ms.append(fev[0].elapsed_time(fev[3]))
            flush.zero_()
            staged.replay()
            torch.cuda.synchronize()
            for i, name in enumerate(step_phases):
                sphase[name].append(sev[i].elapsed_time(sev[i + 1]))
            flush.zero_()
        graph.replay()
        torch.cuda.synchronize()
        sep_ms.append(ev[0].elapsed_time(ev[4]))
        if fast is None:
            step_ms.append(sep_ms[-1])
        for i, name in enumerate(phases):
            phase[name].append(ev[i].elapsed_time(ev[i + 1]))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = np.array(step_ms)
    ms = max_over_ranks(float(step_ms.mean()), world, dev)

    if args.quick:  # timed graph steps only (profiling runs)
        res = {"metric": METRIC, "value": job_throughput(N * S, world, ms), "unit": UNIT,
               "ms_per_step": ms,
               "step_phase_ms": {k: float(np.mean(v)) for k, v in sphase.items() if v},
               "phase_ms": {k: float(np.mean(v)) for k, v in phase.items()},
               "quick": True}
        fu.close()
        return res, wl

    # the same step launched eagerly through the Python API (host launch cost included)
    eager = []
    for _ in range(max(5, args.steps // 2)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        torch.cuda.synchronize()
        eager.append(a.elapsed_time(b))

    # per-update latency: one more view folded into a session holding S-1 views
    # and finalized, through divas_fuse_update (one fusion launch; the score
    # buffer holds this context's earlier result, so only active voxels are
    # written) -- eager API calls, and the same update replayed as a graph; the
    # separate add_views + finalize calls as a graph for reference
    upd, upd_g, upd_sep = [], [], []
    pv_last = PreparedViews(wl.cams[-1:], depth[-1:], mask[-1:], wl.mask_type)
    pv_first = PreparedViews(wl.cams[:-1], depth[:-1], mask[:-1], wl.mask_type)
    n_upd = max(20, args.steps)
    for k in range(n_upd):
        fu.set_occupancy(occ=occ, coords=coords)
        fu.add_views(pv_first)
        flush.zero_()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fu.update(pv_last, score=score, keep_zeros=True)
        b.record()
        torch.cuda.synchronize()
        upd.append(a.elapsed_time(b))
    graphs = {}
    for name in ("update", "separate"):
        fu.set_occupancy(occ=occ, coords=coords)
        fu.add_views(pv_first)
        torch.cuda.synchronize()
        ue = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        ug = torch.cuda.CUDAGraph()
        with torch.cuda.graph(ug):
            ue[0].record()
            if name == "update":
                fu.update(pv_last, score=score, keep_zeros=True)
            else:
                fu.add_views(pv_last)
                fu.finalize(score=score)
            ue[1].record()
        graphs[name] = (ug, ue)
    for k in range(n_upd):
        for name, out in (("update", upd_g), ("separate", upd_sep)):
            ug, ue = graphs[name]
            fu.set_occupancy(occ=occ, coords=coords)
            fu.add_views(pv_first)
            flush.zero_()
            torch.cuda.synchronize()
            ug.replay()
            torch.cuda.synchronize()
            out.append(ue[0].elapsed_time(ue[1]))
    upd = np.array(upd)
    upd_g = np.array(upd_g)
    upd_sep = np.array(upd_sep)

    # end to end through the public API: every step copies all of its inputs
    # (occupancy prior, rasters, points) from pinned host memory and its
    # outputs (the seg bitfield V_seg and the point labels) back to pinned host
    # memory; the probability grid stays on the device.  The inputs of a step
    # sit in one pinned host arena and move in one copy, its outputs in
    # another (paper_2601_04860_b300.staging.Arena: a producer writes a step's
    # inputs straight into the arena's host views).  Three streams (copy-in,
    # kernels, copy-out) on one arena set pipeline the steps without a host
    # synchronisation: step k + 1's copy-in starts once step k's kernels have
    # read their inputs, step k's copy-out overlaps it.  (Two arena sets, so
    # that step k + 1's copy could also overlap step k's kernels, moved the
    # copies at a lower rate on this machine: 1.76-1.80 ms per step against
    # 1.27 ms.)  The serial figure (one stream, a synchronisation per step) is
    # reported beside it, and so is the pipelined run with one copy per buffer
    # (`per_buffer_ms_per_step`).
    from paper_2601_04860_b300.staging import Arena
    n_seg_words = (fu.n_cells + 31) // 32
    in_specs = []
    if occ is not None:
        in_specs.append(("occ", tuple(occ.shape), occ.dtype))
    if coords is not None:
        in_specs.append(("coords", tuple(coords.shape), coords.dtype))
    in_specs += [(f"depth{k}", tuple(d.shape), d.dtype) for k, d in enumerate(depth)]
    in_specs += [(f"mask{k}", tuple(m.shape), m.dtype) for k, m in enumerate(mask)]
    in_specs.append(("pts", tuple(pts.shape), pts.dtype))
    out_specs = [("seg", (n_seg_words,), torch.int32), ("labels", tuple(labels.shape), labels.dtype)]
    sets = []
    for _ in range(1):
        ai, ao = Arena(in_specs, dev), Arena(out_specs, dev)
        if occ is not None:
            ai.host["occ"].copy_(torch.from_numpy(wl.occ))
        if coords is not None:
            ai.host["coords"].copy_(torch.from_numpy(wl.coords))
        for k, d in enumerate(depth):
            ai.host[f"depth{k}"].copy_(d.cpu())
        for k, m in enumerate(mask):
            ai.host[f"mask{k}"].copy_(m.cpu())
        ai.host["pts"].copy_(pts.cpu())
        st = {"in": ai, "out": ao,
              "pv": PreparedViews(wl.cams, [ai.device[f"depth{k}"] for k in range(len(depth))],
                                  [ai.device[f"mask{k}"] for k in range(len(mask))], wl.mask_type)}
        sets.append(st)
    h2d = sets[0]["in"].payload_bytes()
    d2h = sets[0]["out"].payload_bytes()
    s_in, s_k, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_run(n_steps: int, overlap: bool, per_buffer: bool = False) -> float:
        """n_steps end-to-end steps; returns ms per step (device events from
        the first copy-in to the last copy-out)."""
        in_free = [None]   # kernels of the step that last read the set's inputs
        out_free = [None]  # copy-out of the step that last wrote the set's outputs
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(s_in)
        for k in range(n_steps):
            st = sets[0]
            j = 0
            ai, ao = st["in"], st["out"]
            with torch.cuda.stream(s_in):
                if in_free[j] is not None:
                    s_in.wait_event(in_free[j])
                if per_buffer:
                    for name in ai.host:
                        ai.device[name].copy_(ai.host[name], non_blocking=True)
                else:
                    ai.upload(s_in)
                e_in = torch.cuda.Event()
                e_in.record(s_in)
            s_k.wait_event(e_in)
            if out_free[j] is not None:
                s_k.wait_event(out_free[j])
            d_occ = ai.device.get("occ")
            d_coords = ai.device.get("coords")
            if len(st["pv"].chunks) == 1:
                fu.step(st["pv"], occ=d_occ, coords=d_coords, score=score,
                        seg_bits=ao.device["seg"], xyz=ai.device["pts"],
                        labels=ao.device["labels"], stream=s_k)
            else:
                fu.set_occupancy(occ=d_occ, coords=d_coords, stream=s_k)
                fu.add_views(st["pv"], stream=s_k)
                fu.finalize(score=score, seg_bits=ao.device["seg"], stream=s_k)
                fu.label_points(ai.device["pts"], out=ao.device["labels"], stream=s_k)
            e_k = torch.cuda.Event()
            e_k.record(s_k)
            in_free[j] = e_k
            s_out.wait_event(e_k)
            with torch.cuda.stream(s_out):
                if per_buffer:
                    for name in ao.host:
                        ao.host[name].copy_(ao.device[name], non_blocking=True)
                else:
                    ao.download(s_out)
                e_o = torch.cuda.Event()
                e_o.record(s_out)
                out_free[j] = e_o
            if not overlap:
                torch.cuda.synchronize()
        end.record(s_out)
        torch.cuda.synchronize()
        return start.elapsed_time(end) / n_steps

    e2e_run(4, True)
    e2e_run(2, False)
    e2e_run(2, True, per_buffer=True)
    e2e_steps = max(10, args.steps)
    e2e_ms = max_over_ranks(float(np.mean([e2e_run(e2e_steps, True) for _ in range(3)])), world, dev)
    e2e_serial_ms = float(np.mean([e2e_run(e2e_steps, False) for _ in range(2)]))
    e2e_per_buffer_ms = float(np.mean([e2e_run(e2e_steps, True, per_buffer=True) for _ in range(2)]))
    # the labels read back (same inputs every step) equal the device result
    if not torch.equal(sets[0]["out"].host["labels"], labels.cpu()):
        raise RuntimeError("end-to-end read-back differs from the device labels")

    algo, view_bytes, _, _ = algorithmic_bytes(wl, n_active)
    peak, peak_kind = peaks()
    pm = {k: float(np.mean(v)) for k, v in phase.items()}
    if fast is not None:  # the dominant single-kernel stage of the timed step
        spm = {k: float(np.mean(v)) for k, v in sphase.items()}
        cand = {k: (spm[k], algo[k]) for k in step_phases if step_kernels[k] == 1}
        launches = 2 * sum(step_kernels.values()) + sum(kernels_per_phase.values())
    else:
        spm = None
        cand = {k: (pm[k], algo[k]) for k in phases if kernels_per_phase[k] == 1}
        launches = sum(kernels_per_phase.values())
    dom = max(cand, key=lambda k: cand[k][0])
    achieved = cand[dom][1] / (cand[dom][0] * 1e-3) / 1e9
    step_bytes = sum(algo[k] for k in step_phases)
    res = {
        "metric": METRIC, "value": job_throughput(N * S, world, ms), "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ray-cast scene; no dataset)",
        "config": {**workload_config(args.workload, wl),
                   "l2": "flushed between timed steps (a 256 MB buffer written, then a 256 MB buffer read, outside the timed events)",
                   "launch": "one CUDA graph replay of divas_fuse_step per step (device time "
                             "from in-graph events around it); stage times from a second graph "
                             "of the same step with events between its launches; "
                             "separate_calls_* from a graph of the separate API calls",
                   "parallelism": f"replicas x{world}",
                   "active_order": "brick-major (warp-level view culling)"
                                   if fu.params.brick_order else "linear"},
        "roofline": {"bound": "hbm", "kernel": KERNEL_OF[dom], "achieved": achieved,
                     "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic_for(args.workload, KERNEL_OF[dom]),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": int(cand[dom][1]),
                     "ms_per_launch": cand[dom][0]},
        "step_roofline": {"algorithmic_bytes": int(step_bytes),
                          "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
                          "frac": step_bytes / (ms * 1e-3) / 1e9 / peak},
        "step_phase_ms": spm,
        "separate_calls_phase_ms": pm,
        "separate_calls_ms_per_step": float(np.mean(sep_ms)),
        "phase_bytes": {k: int(v) for k, v in algo.items()},
        "eager_ms_per_step": float(np.mean(eager)),
        "per_update_ms": {"what": "fold 1 view into a session of S-1 views + finalize "
                                  "(divas_fuse_update, one fusion launch), L2 flushed",
                          "p50": float(np.percentile(upd, 50)),
                          "p99": float(np.percentile(upd, 99)),
                          "graph_p50": float(np.percentile(upd_g, 50)),
                          "graph_p99": float(np.percentile(upd_g, 99)),
                          "separate_calls_graph_p50": float(np.percentile(upd_sep, 50)),
                          "separate_calls_graph_p99": float(np.percentile(upd_sep, 99))},
        "active_updates_per_s": world * n_active * S / (ms * 1e-3),
        "e2e": {"value": job_throughput(N * S, world, e2e_ms), "unit": UNIT,
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "what": "VoxelFusion.step per step with every input copied in from pinned host "
                        "memory and V_seg + point labels copied out, each direction one copy of "
                        "a pinned transfer arena (staging.Arena); copy-in / kernel / copy-out "
                        "streams pipelined without a host synchronisation",
                "serial_ms_per_step": e2e_serial_ms,
                "per_buffer_ms_per_step": e2e_per_buffer_ms},
        "gpu_launches": int(launches * args.steps),
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    # the timed step's outputs, for the parity check against the oracle sample
    if not args.quick:
        if fast is not None:
            fast.replay()
        else:
            graph.replay()
        torch.cuda.synchronize()
        st = fu.export_state()
        fin = fu.finalize(score=False, seg_bits=True)
        res["_parity_gpu"] = dict(linear_state(fu, st, score, dense),
                                  seg_words=fin["seg_bits"].cpu().numpy().view(np.uint32),
                                  labels=labels.cpu().numpy())
    fu.close()
    return res, wl


def bench_parity(wl, gpu: dict, sample, o: dict, npts: int) -> dict:
    """The timed step's outputs against the FP64 oracle on the CPU baseline's
    voxel sample: voxels the oracle flags as within 1e-6 of a rounding or
    threshold boundary are counted and excluded; every other sampled voxel must
    match (view bits and seg exactly, W, Z and P within 1e-5 relative), and so
    must the labels of the points that fall in sampled, unflagged voxels."""
    import oracle
    lin = wl.active_linear()[sample]
    g = int(wl.grid.g)
    dense = wl.occ is not None
    flagged = o["flags"] != 0
    ok = ~flagged
    rel = lambda a, b: np.abs(a.astype(np.float64) - b) > 1e-5 * np.abs(b)  # noqa: E731
    P = gpu["score"][lin] if dense else gpu["score"][sample]
    seg = ((gpu["seg_words"][lin >> 5] >> (lin & 31).astype(np.uint32)) & 1).astype(bool)
    bad = ok & ((gpu["bits"][sample] != o["bits"]) | rel(gpu["W"][sample], o["W"]) |
                rel(gpu["Z"][sample], o["Z"]) | rel(P, o["P"]) | (seg != o["seg"].astype(bool)))
    # labels: points whose cell is a sampled, unflagged voxel, not near a cell face
    seg_o = np.zeros(g ** 3, np.uint8)
    seg_o[lin] = o["seg"]
    pts = wl.points[:npts]
    lab_o, pfl = oracle.label(wl.grid, seg_o, pts)
    x = pts.astype(np.float64)
    if wl.grid.contracted:
        r = np.linalg.norm(x, axis=1, keepdims=True)
        with np.errstate(invalid="ignore", divide="ignore"):
            x = np.where(r > 1.0, (2.0 - 1.0 / r) * x / r, x)
    org = np.asarray(wl.grid.origin, np.float32).astype(np.float64)
    with np.errstate(invalid="ignore"):
        c = np.floor((x - org) / float(np.float32(wl.grid.h)))
        inside = np.all((c >= 0) & (c < g), axis=1)
    c = np.where(inside[:, None], c, 0).astype(np.int64)
    cell = (c[:, 2] * g + c[:, 1]) * g + c[:, 0]
    good_cell = np.zeros(g ** 3, bool)
    good_cell[lin[ok]] = True
    pok = inside & good_cell[cell] & (pfl == 0)
    lab_bad = int((gpu["labels"][:npts][pok] != lab_o[pok]).sum())
    return {"config": wl.name, "voxels_compared": int(len(sample)),
            "flagged": int(flagged.sum()), "flagged_frac": float(flagged.mean()),
            "mismatches_outside_flagged": int(bad.sum()),
            "points_compared": int(pok.sum()), "point_mismatches": lab_bad,
            "rule": "bits, seg exact; W, Z, P within 1e-5 relative; labels exact; "
                    "flagged = within 1e-6 of a rounding or threshold boundary"}


def measure_sparse(dev, steps: int, cpu_seconds: float = 8.0):
    """Config 3 (unbounded sparse): the one-call step on the contracted 512^3
    grid with ~12M occupied voxels given as int32 coordinates, 16 views
    1297x840, 3M points, replayed from a CUDA graph (events around it), L2
    flushed between steps; stage times from a second graph whose step records
    events between its launches.  The fusion is ALU-bound here (compensated
    projection of far contracted voxels): besides its HBM fraction, its
    instruction-issue fraction is reported from the warp instructions one
    launch executes (ncu, smsp__inst_executed.sum, scaled to this launch)
    against the issue peak SMs x 4 schedulers x one warp instruction per
    clock at the sampled SM clock."""
    import torch

    from paper_2601_04860_b300 import FusionParams, PreparedViews, VoxelFusion
    wl = make_workload("unbounded-sparse-512")
    coords = torch.from_numpy(wl.coords).to(dev)
    depth = [torch.from_numpy(d).to(dev) for d in wl.depth]
    mask = [torch.from_numpy(m.view(np.float16)).to(dev) for m in wl.mask]
    pts = torch.from_numpy(np.ascontiguousarray(wl.points)).to(dev)
    fu = VoxelFusion(wl.grid, coords=coords, params=fusion_params(wl))
    na = fu.n_active
    score = torch.empty(na, dtype=torch.float32, device=dev)
    labels = torch.empty(len(wl.points), dtype=torch.uint8, device=dev)
    pv = PreparedViews(wl.cams, depth, mask, wl.mask_type)
    flush = L2Flush(dev)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            fu.step(pv, coords=coords, score=score, xyz=pts, labels=labels)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(4)]
    sev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(4)]
    for e in ev + sev:
        e.record()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fu.step(pv, coords=coords, score=score, xyz=pts, labels=labels,
                stage_events=[ev[0], None, None, ev[3]])
    gs = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gs):
        fu.step(pv, coords=coords, score=score, xyz=pts, labels=labels, stage_events=sev)
    clocks = Clocks(dev.index or 0)
    clocks.start()
    ms, st = [], {"compaction": [], "fuse_finalize": [], "label": []}
    for k in range(2 + steps):
        flush.zero_()
        g.replay()
        torch.cuda.synchronize()
        flush.zero_()
        gs.replay()
        torch.cuda.synchronize()
        if k >= 2:
            ms.append(ev[0].elapsed_time(ev[3]))
            for i, name in enumerate(st):
                st[name].append(sev[i].elapsed_time(sev[i + 1]))
    clk = clocks.stop()
    m = float(np.mean(ms))
    stm = {k: float(np.mean(v)) for k, v in st.items()}
    S = wl.n_views
    algo, view_bytes, _, _ = algorithmic_bytes(wl, na)
    peak, peak_kind = peaks()
    fb = algo["fuse_finalize"]
    ach = fb / (stm["fuse_finalize"] * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk.get("sm_mhz") or 2032.0
    issue_peak = props.multi_processor_count * 4 * sm_mhz * 1e6  # warp instructions / s
    order = "brick" if fu.params.brick_order else "linear"
    ipv = SPARSE_FUSE_INSTS_PER_VOXEL_VIEW[order]
    insts = None if ipv is None else ipv * na * S
    out = {"workload": "unbounded-sparse-512 (contracted 512^3 grid, ~12M occupied voxels as "
                       "int32 coordinates, 16 views 1297x840 FP32 depth + FP16 masks, 3M points)",
           "ms_per_step": m, "updates_per_s": na * S / (m * 1e-3), "active_voxels": int(na),
           "views": S, "stage_ms": stm,
           "roofline": {"bound": "alu",
                        "kernel": "k_fuse_fin_cull (contracted)" if order == "brick"
                                  else "k_fuse_fin (contracted)",
                        "achieved": None if insts is None
                                    else insts / (stm["fuse_finalize"] * 1e-3) / 1e12,
                        "peak": issue_peak / 1e12, "unit": "warp Tinst/s",
                        "frac": None if insts is None
                                else insts / (stm["fuse_finalize"] * 1e-3) / issue_peak,
                        "insts_per_launch": insts,
                        "insts_source": "ncu smsp__inst_executed.sum per voxel-view of this "
                                        "kernel (profiles/unbounded-sparse-512_launch_list.md)",
                        "hbm_achieved_gbs": ach, "hbm_frac": ach / peak, "hbm_peak_kind": peak_kind,
                        "algorithmic_bytes_per_launch": int(fb)},
           "clocks": clk,
           "active_order": "brick-major (8^3 bricks; warp-level view culling)"
                           if fu.params.brick_order else "linear",
           "gpu_launches_per_step": 5 if fu.params.brick_order else 4}
    # the timed step's outputs, for the parity check against the oracle sample
    g.replay()
    torch.cuda.synchronize()
    fin = fu.finalize(score=False, seg_bits=True)
    pgpu = dict(linear_state(fu, fu.export_state(), score, False),
                seg_words=fin["seg_bits"].cpu().numpy().view(np.uint32),
                labels=labels.cpu().numpy())
    fu.close()
    # the oracle on a bounded sample of the same workload
    full_s, det = oracle_rate(wl, cpu_seconds, repeats=1)
    out["cpu_baseline"] = {"value": na * S / full_s, "unit": UNIT, "cores": det["cores"],
                           "kind": "oracle",
                           "sample": f"{det['sample_voxels']} of {det['active_voxels']} active "
                                     f"voxels x {S} views + {det['sample_points']} points, "
                                     f"extrapolated to the full step"}
    try:
        out["parity"] = bench_parity(wl, pgpu, det["sample_index"], det["sample_out"],
                                     det["sample_points"])
    except Exception as e:  # noqa: BLE001
        out["parity"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def _tuple_step(dev, n_abs: float | None = None):
    """Depth-tuple mode on the 256^3 forward-facing scene (8 views 1008x756 with
    d_min / d_med / d_max / n_samp rasters; paper defaults, or another n_abs):
    the context and one step = occupancy gate + the tuple views (per-view maps,
    candidate scan, heavy pass) + finalize + labels."""
    import torch

    import synth
    from paper_2601_04860_b300 import FusionParams, TupleParams, VoxelFusion
    tw = synth.with_tuple(synth.config2())
    occ = torch.from_numpy(tw.occ).to(dev)
    T = tw.tuple
    ras = {k: [torch.from_numpy(a).to(dev) for a in T[k]] for k in ("d_min", "d_med", "d_max")}
    ns = [torch.from_numpy(a.view(np.int16)).to(dev) for a in T["n_samp"]]
    mask = [torch.from_numpy(m.view(np.float16)).to(dev) for m in tw.mask]
    pts = torch.from_numpy(np.ascontiguousarray(tw.points)).to(dev)
    fu = VoxelFusion(tw.grid, occ=occ, params=FusionParams())
    score = torch.empty(fu.n_cells, dtype=torch.float32, device=dev)
    labels = torch.empty(len(tw.points), dtype=torch.uint8, device=dev)
    tp = TupleParams() if n_abs is None else TupleParams(n_abs=n_abs)

    def step(ev=None):
        fu.set_occupancy(occ=occ)
        fu.add_views_tuple(tw.cams, ras["d_min"], ras["d_med"], ras["d_max"], ns, mask,
                           T["d_cam"], tw.mask_type, tparams=tp, stage_events=ev)
        fu.finalize(score=score)
        fu.label_points(pts, out=labels)
    return fu, step, tw, tp


def _tuple_scan_bytes(tw, n_active: int) -> int:
    """Algorithmic bytes of one candidate-scan launch (first views of a
    context): the active list (4 B per voxel) and the zeroed accumulators (12
    B), plus each view's centre rasters read once (d_min and d_med FP32, the
    mask)."""
    mb = 2 if tw.mask_type == 1 else 4
    return 16 * n_active + sum(c.W * c.H * (8 + mb) for c in tw.cams)


def measure_tuple(dev, steps: int):
    """The depth-tuple step replayed from a CUDA graph (events around it only),
    L2 flushed between steps, for the paper's defaults and with the thin path
    voting (n_abs = 4); stage times from a second graph whose tuple call
    records events between its launches; the candidate scan's roofline; the
    oracle on the host as its CPU baseline."""
    import torch
    out = {"workload": "forward-dense-256-tuple (config-2 scene with a depth tuple per view: "
                       "d_min / d_med / d_max FP32, n_samp uint16; 8 views 1008x756)",
           "what": "graph replay of set_occupancy + add_views_tuple (8 views) + finalize + "
                   "label_points; L2 flushed per step"}
    flush = L2Flush(dev)
    peak, peak_kind = peaks()
    for name, n_abs in (("paper_defaults", None), ("thin_active_n_abs_4", 4.0)):
        fu, step, tw, tp = _tuple_step(dev, n_abs)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        sev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(4)]
        for e in sev:
            e.record()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ev[0].record()
            step()
            ev[1].record()
        gs = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gs):
            step(sev)
        ms, st = [], {"maps": [], "scan": [], "heavy": []}
        for k in range(3 + steps):
            flush.zero_()
            g.replay()
            torch.cuda.synchronize()
            flush.zero_()
            gs.replay()
            torch.cuda.synchronize()
            if k >= 3:
                ms.append(ev[0].elapsed_time(ev[1]))
                st["maps"].append(sev[0].elapsed_time(sev[1]))
                st["scan"].append(sev[1].elapsed_time(sev[2]))
                st["heavy"].append(sev[2].elapsed_time(sev[3]))
        n, S, na = fu.n_cells, tw.n_views, fu.n_active
        m = float(np.mean(ms))
        stm = {k: float(np.mean(v)) for k, v in st.items()}
        scan_bytes = _tuple_scan_bytes(tw, na)
        ach = scan_bytes / (stm["scan"] * 1e-3) / 1e9
        out[name] = {"n_abs": tp.n_abs, "ms_per_step": m, "updates_per_s": n * S / (m * 1e-3),
                     "active_updates_per_s": na * S / (m * 1e-3),
                     "stage_ms": stm,
                     "roofline": {"bound": "hbm", "kernel": "k_tuple_scan", "achieved": ach,
                                  "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                  "traffic": None, "peak_kind": peak_kind,
                                  "algorithmic_bytes_per_launch": scan_bytes,
                                  "ms_per_launch": stm["scan"]}}
        fu.close()
    out["cpu_baseline"] = tuple_cpu_baseline(tw)
    return out


def tuple_cpu_baseline(tw):
    """The oracle's depth-tuple fusion (paper defaults) on the host cores over
    every active voxel x 8 views of the 256^3 scene, as nominal voxel-view
    updates/s (g^3 x views / time)."""
    import oracle
    cores = oracle.set_threads(0)
    lin = tw.active_linear()
    t0 = time.perf_counter()
    oracle.fuse_tuple(tw.grid, lin, tw.cams, tw.tuple, tw.mask, tw.mask_type,
                      params=oracle.Params().f32(), tparams=oracle.TupleParams().f32())
    dt = time.perf_counter() - t0
    g = tw.grid.g
    return {"value": g ** 3 * tw.n_views / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle", "seconds": dt,
            "sample": f"all {len(lin)} active voxels x {tw.n_views} views (fusion only, no "
                      "finalize or labels)"}


def profile_tuple_steps(args):
    """Profiling target of the depth-tuple step: N eager steps (per step:
    k_tile_count, k_tile_emit, k_mask_tile_max, k_tuple_scan, k_tuple_heavy,
    k_finalize, k_label on the 256^3 scene, whose footprints are summed
    directly) and nothing else."""
    import torch
    fu, step, _, _ = _tuple_step(torch.device("cuda"))
    for _ in range(args.profile_tuple_steps):
        step()
    torch.cuda.synchronize()
    fu.sync()
    print(json.dumps({"profile_tuple_steps": args.profile_tuple_steps,
                      "workload": "forward-dense-256-tuple", "active_voxels": fu.n_active}))
    fu.close()
    return 0


def _nerf_step(dev, preset: str = "llff"):
    """The NeRF variant on the 256^3 forward-facing scene (8 views 1008x756
    with d_min / d_exp / d_max / n_samp rasters and a 256^3 FP32 density
    grid; Table kernel_hyperparams, LLFF or Mip-NeRF 360 column): the context
    and one step = density floor (rho >= 10) + occupancy gate + the NeRF views
    (mask-tile maps, scan, heavy pass) + finalize + labels."""
    import torch

    import synth
    from paper_2601_04860_b300 import FusionParams, NerfParams, VoxelFusion, density_floor
    wl = synth.config2()
    nw, rho = synth.with_nerf_tuple(wl), synth.nerf_density(wl)
    T = nw.tuple
    ras = {k: [torch.from_numpy(a).to(dev) for a in T[k]] for k in ("d_min", "d_exp", "d_max")}
    ns = [torch.from_numpy(a.view(np.int16)).to(dev) for a in T["n_samp"]]
    mask = [torch.from_numpy(m.view(np.float16)).to(dev) for m in nw.mask]
    pts = torch.from_numpy(np.ascontiguousarray(nw.points)).to(dev)
    drho = torch.from_numpy(rho).to(dev)
    occ = torch.empty(drho.numel(), dtype=torch.uint8, device=dev)
    fu = VoxelFusion(nw.grid, occ=density_floor(drho, 10.0), params=FusionParams())
    score = torch.empty(fu.n_cells, dtype=torch.float32, device=dev)
    labels = torch.empty(len(nw.points), dtype=torch.uint8, device=dev)
    npar = NerfParams() if preset == "llff" else NerfParams.mip360()

    def step(ev=None):
        density_floor(drho, 10.0, out=occ)
        fu.set_occupancy(occ=occ)
        fu.add_views_nerf(nw.cams, ras["d_min"], ras["d_exp"], ras["d_max"], ns, mask,
                          nw.mask_type, nparams=npar, density=drho, stage_events=ev)
        fu.finalize(score=score)
        fu.label_points(pts, out=labels)
    return fu, step, nw, rho, npar


def _nerf_scan_bytes(nw, n_active: int) -> int:
    """Algorithmic bytes of one NeRF scan launch (first views of a context):
    the active list (4 B per voxel), each voxel's density (4 B) and its
    written accumulators (12 B), plus each view's rasters read once (d_min,
    d_exp, d_max FP32, n_samp 2 B, the mask)."""
    mb = 2 if nw.mask_type == 1 else 4
    return 20 * n_active + sum(c.W * c.H * (14 + mb) for c in nw.cams)


def measure_nerf(dev, steps: int):
    """The NeRF-variant step replayed from a CUDA graph (events around it
    only), L2 flushed between steps, with the LLFF and the Mip-NeRF 360
    constants; stage times from a second graph whose NeRF call records events
    between its launches; the scan's roofline; the oracle on the host."""
    import torch
    out = {"workload": "forward-dense-256-nerf (config-2 scene with a NeRF depth tuple per view: "
                       "d_min / d_exp / d_max FP32, n_samp uint16; 256^3 FP32 density; 8 views "
                       "1008x756)",
           "what": "graph replay of density_floor + set_occupancy + add_views_nerf (8 views) + "
                   "finalize + label_points; L2 flushed per step"}
    flush = L2Flush(dev)
    peak, peak_kind = peaks()
    for preset in ("llff", "mip360"):
        fu, step, nw, rho, npar = _nerf_step(dev, preset)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        sev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(4)]
        for e in sev:
            e.record()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ev[0].record()
            step()
            ev[1].record()
        gs = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gs):
            step(sev)
        ms, st = [], {"maps": [], "scan": [], "heavy": []}
        for k in range(3 + steps):
            flush.zero_()
            g.replay()
            torch.cuda.synchronize()
            flush.zero_()
            gs.replay()
            torch.cuda.synchronize()
            if k >= 3:
                ms.append(ev[0].elapsed_time(ev[1]))
                st["maps"].append(sev[0].elapsed_time(sev[1]))
                st["scan"].append(sev[1].elapsed_time(sev[2]))
                st["heavy"].append(sev[2].elapsed_time(sev[3]))
        n, S, na = fu.n_cells, nw.n_views, fu.n_active
        m = float(np.mean(ms))
        stm = {k: float(np.mean(v)) for k, v in st.items()}
        scan_bytes = _nerf_scan_bytes(nw, na)
        ach = scan_bytes / (stm["scan"] * 1e-3) / 1e9
        out[preset] = {"ms_per_step": m, "updates_per_s": n * S / (m * 1e-3),
                       "active_updates_per_s": na * S / (m * 1e-3), "stage_ms": stm,
                       "roofline": {"bound": "hbm", "kernel": "k_nerf_scan", "achieved": ach,
                                    "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                    "traffic": None, "peak_kind": peak_kind,
                                    "algorithmic_bytes_per_launch": scan_bytes,
                                    "ms_per_launch": stm["scan"]}}
        fu.close()
    out["cpu_baseline"] = nerf_cpu_baseline(nw, rho)
    return out


def nerf_cpu_baseline(nw, rho):
    """The oracle's NeRF-variant fusion (LLFF constants) on the host cores over
    every active voxel x 8 views of the 256^3 scene, as nominal voxel-view
    updates/s (g^3 x views / time)."""
    import oracle
    cores = oracle.set_threads(0)
    lin = nw.active_linear()
    t0 = time.perf_counter()
    oracle.fuse_nerf(nw.grid, lin, nw.cams, nw.tuple, nw.mask, nw.mask_type,
                     params=oracle.Params().f32(), nparams=oracle.NerfParams().f32(),
                     rho=rho[lin].astype(np.float64))
    dt = time.perf_counter() - t0
    g = nw.grid.g
    return {"value": g ** 3 * nw.n_views / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle", "seconds": dt,
            "sample": f"all {len(lin)} active voxels x {nw.n_views} views (fusion only, no "
                      "finalize or labels)"}


def profile_nerf_steps(args):
    """Profiling target of the NeRF-variant step: N eager steps (per step:
    k_density_floor, k_tile_count, k_tile_emit, k_mask_tiles, k_nerf_scan,
    k_nerf_heavy, k_finalize, k_label on the 256^3 scene) and nothing else."""
    import torch
    fu, step, _, _, _ = _nerf_step(torch.device("cuda"))
    for _ in range(args.profile_nerf_steps):
        step()
    torch.cuda.synchronize()
    fu.sync()
    print(json.dumps({"profile_nerf_steps": args.profile_nerf_steps,
                      "workload": "forward-dense-256-nerf", "active_voxels": fu.n_active}))
    fu.close()
    return 0


def _weight_step(dev, mode: str):
    """Depth-weighted masks on the 256^3 forward-facing scene (8 views
    1008x756, FP16 masks, 3 positive prompts per view on the target): the
    context and one step = depth_weight (8 views) + occupancy gate + the
    weighted views + finalize + labels."""
    import torch

    import synth
    from paper_2601_04860_b300 import MASK_F32, FusionParams, VoxelFusion
    wl = synth.config2()
    pr = synth.prompts(wl)
    occ = torch.from_numpy(wl.occ).to(dev)
    depth = [torch.from_numpy(x).to(dev) for x in wl.depth]
    mask = [torch.from_numpy(m.view(np.int16)).to(dev) for m in wl.mask]
    wbuf = [torch.empty(x.shape, dtype=torch.float32, device=dev) for x in depth]
    pts = torch.from_numpy(np.ascontiguousarray(wl.points)).to(dev)
    fu = VoxelFusion(wl.grid, occ=occ, params=FusionParams())
    score = torch.empty(fu.n_cells, dtype=torch.float32, device=dev)
    labels = torch.empty(len(wl.points), dtype=torch.uint8, device=dev)

    def step(ev=None):
        if ev:
            ev[0].record()
        fu.depth_weight(depth, mask, wl.mask_type, mode=mode, prompts=pr, out=wbuf)
        if ev:
            ev[1].record()
        fu.set_occupancy(occ=occ)
        fu.add_views(wl.cams, depth, wbuf, mask_type=MASK_F32)
        fu.finalize(score=score)
        fu.label_points(pts, out=labels)

    def fused_step(ev=None):
        # the weight applied where each vote reads the mask: no weighted rasters
        fu.set_occupancy(occ=occ)
        fu.add_views_weighted(wl.cams, depth, mask, mask_type=wl.mask_type, mode=mode,
                              prompts=pr)
        fu.finalize(score=score)
        fu.label_points(pts, out=labels)

    def plain_step(ev=None):
        fu.set_occupancy(occ=occ)
        fu.add_views(wl.cams, depth, mask, mask_type=wl.mask_type)
        fu.finalize(score=score)
        fu.label_points(pts, out=labels)
    step.fused = fused_step
    step.plain = plain_step
    return fu, step, wl, pr


def measure_weighting(dev, steps: int):
    """The depth-weighted step replayed from a CUDA graph (events around it),
    L2 flushed between steps, for the band-pass (with P98 selection) and the
    min-max weighting; the weighting stage's time from events inside a
    second graph, its roofline, and the oracle on the host."""
    import torch
    out = {"workload": "forward-dense-256-weighted (config-2 scene; 8 views 1008x756, FP16 "
                       "masks, 3 positive prompts per view; weighted masks FP32)",
           "what": "graph replay of depth_weight (8 views) + set_occupancy + add_views "
                   "(weighted masks) + finalize + label_points; fused: set_occupancy + "
                   "add_views_weighted (selection passes + one fusion launch, no weighted "
                   "rasters) + finalize + label_points; plain: the unweighted step; L2 "
                   "flushed per step"}
    flush = L2Flush(dev)
    peak, peak_kind = peaks()
    for mode in ("band", "nerf"):
        fu, step, wl, pr = _weight_step(dev, mode)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        sev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ev[0].record()
            step()
            ev[1].record()
        gs = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gs):
            step(sev)
        ms, wms = [], []
        for k in range(3 + steps):
            flush.zero_()
            g.replay()
            torch.cuda.synchronize()
            flush.zero_()
            gs.replay()
            torch.cuda.synchronize()
            if k >= 3:
                ms.append(ev[0].elapsed_time(ev[1]))
                wms.append(sev[0].elapsed_time(sev[1]))
        # the one-pass fused step and the plain (unweighted) step, same graph setup
        extra = {}
        for name, fn in (("fused", step.fused), ("plain", step.plain)):
            with torch.cuda.stream(side):
                for _ in range(3):
                    fn()
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            fe = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
            gf = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gf):
                fe[0].record()
                fn()
                fe[1].record()
            t = []
            for k in range(3 + steps):
                flush.zero_()
                gf.replay()
                torch.cuda.synchronize()
                if k >= 3:
                    t.append(fe[0].elapsed_time(fe[1]))
            extra[name] = float(np.mean(t))
        m, w = float(np.mean(ms)), float(np.mean(wms))
        algo = sum(c.W * c.H * (4 + 2 + 4) for c in wl.cams)  # depth, FP16 mask, FP32 out
        ach = algo / (w * 1e-3) / 1e9
        out[mode] = {"ms_per_step": m, "updates_per_s": fu.n_cells * wl.n_views / (m * 1e-3),
                     "weighting_ms": w,
                     "fused_ms_per_step": extra["fused"],
                     "plain_ms_per_step": extra["plain"],
                     "fused_vs_plain_plus_weighting": extra["fused"] / (extra["plain"] + w),
                     "roofline": {"bound": "hbm", "kernel": "depth_weight (all passes)",
                                  "achieved": ach, "peak": peak, "unit": "GB/s",
                                  "frac": ach / peak, "traffic": None, "peak_kind": peak_kind,
                                  "algorithmic_bytes_per_launch": algo, "ms_per_launch": w}}
        fu.close()
    out["cpu_baseline"] = weighting_cpu_baseline(wl, pr)
    return out


def weighting_cpu_baseline(wl, pr):
    """The oracle's band-pass weighting (FP64 NumPy, one host thread) of the
    8 views, as weighted pixels/s."""
    import oracle.weighting as OW
    t0 = time.perf_counter()
    for k in range(wl.n_views):
        OW.gs_band(wl.depth[k], wl.mask[k], wl.mask_type, pr[k])
    dt = time.perf_counter() - t0
    px = sum(c.W * c.H for c in wl.cams)
    return {"value": px / dt, "unit": "weighted pixels/s", "cores": 1, "kind": "oracle",
            "seconds": dt, "sample": f"all {wl.n_views} views (band-pass, with P98)"}


def profile_weight_steps(args):
    """Profiling target of the depth-weighted step (band-pass): N eager steps
    (per step: k_weight_init, k_weight_pass1, k_weight_digit x2,
    k_weight_final, k_weight_apply, then k_tile_count, k_tile_emit, k_fuse,
    k_finalize, k_label) and nothing else."""
    import torch
    fu, step, _, _ = _weight_step(torch.device("cuda"), "band")
    for _ in range(args.profile_weight_steps):
        step()
    torch.cuda.synchronize()
    fu.sync()
    print(json.dumps({"profile_weight_steps": args.profile_weight_steps,
                      "workload": "forward-dense-256-weighted"}))
    fu.close()
    return 0


def measure_occupancy(dev, steps: int):
    """Occupancy construction from a surfel cloud of the 256^3 scene (its 1M
    surface points as centres, 0.5% floaters, two scales and a dyadic opacity
    each): the frame call (two exact selection rounds; synchronises) timed
    with events around it; the occupancy call (density zeroed, opacity
    scatter-add, tau_TF floor) replayed from a CUDA graph, with its roofline;
    the fusion step on the constructed occupancy (8 views); the oracle on the
    host."""
    import torch

    import synth
    from paper_2601_04860_b300 import (FusionParams, PreparedViews, VoxelFusion, occupancy,
                                       scene_frame)
    wl = synth.config2()
    mu, sc, al = synth.gaussians(wl)
    dmu, dsc, dal = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (mu, sc, al))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    fms = []
    for k in range(3 + steps):
        ev[0].record()
        f = scene_frame(dmu, dsc)
        ev[1].record()
        torch.cuda.synchronize()
        if k >= 3:
            fms.append(ev[0].elapsed_time(ev[1]))
    n = f.g ** 3
    density = torch.empty(n, dtype=torch.float32, device=dev)
    occ = torch.empty(n, dtype=torch.uint8, device=dev)
    for _ in range(3):
        occupancy(dmu, dal, f, density=density, occ=occ)
    torch.cuda.synchronize()
    ge = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ge[0].record()
        occupancy(dmu, dal, f, density=density, occ=occ)
        ge[1].record()
    oms = []
    for k in range(3 + steps):
        g.replay()
        torch.cuda.synchronize()
        if k >= 3:
            oms.append(ge[0].elapsed_time(ge[1]))
    om = float(np.mean(oms))
    algo = len(mu) * 16 + n * (4 + 4 + 1)  # surfels read; density zeroed, read; occupancy written
    peak, peak_kind = peaks()
    ach = algo / (om * 1e-3) / 1e9
    n_active = int(occ.sum().item())
    # the fusion step on the constructed occupancy
    grid = f.grid()
    fu = VoxelFusion(grid, occ=occ, params=FusionParams())
    depth = [torch.from_numpy(x).to(dev) for x in wl.depth]
    mask = [torch.from_numpy(m.view(np.int16)).to(dev) for m in wl.mask]
    pv = PreparedViews(wl.cams, depth, mask, wl.mask_type)
    pts = torch.from_numpy(np.ascontiguousarray(wl.points)).to(dev)
    score = torch.empty(n, dtype=torch.float32, device=dev)
    labels = torch.empty(len(wl.points), dtype=torch.uint8, device=dev)
    flush = L2Flush(dev)
    for _ in range(3):
        fu.step(pv, occ=occ, score=score, xyz=pts, labels=labels)
    torch.cuda.synchronize()
    se = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
    gs = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gs):
        se[0].record()
        fu.step(pv, occ=occ, score=score, xyz=pts, labels=labels)
        se[1].record()
    sms = []
    for k in range(3 + steps):
        flush.zero_()
        gs.replay()
        torch.cuda.synchronize()
        if k >= 3:
            sms.append(se[0].elapsed_time(se[1]))
    sm = float(np.mean(sms))
    fu.close()
    out = {"workload": f"gaussians-from-forward-dense-256 ({len(mu)} surfels; frame -> g = {f.g}, "
                       f"h = {f.h:.6g}, b = {f.b:g}; {n_active} occupied voxels)",
           "frame_ms": float(np.mean(fms)), "occupancy_ms": om,
           "surfels_per_s": len(mu) / ((float(np.mean(fms)) + om) * 1e-3),
           "roofline": {"bound": "hbm", "kernel": "occupancy (memset + k_gauss_scatter + "
                                                  "k_density_floor)",
                        "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "traffic": None, "peak_kind": peak_kind,
                        "algorithmic_bytes_per_launch": algo, "ms_per_launch": om},
           "fusion_step_ms": sm,
           "fusion_updates_per_s": n * wl.n_views / (sm * 1e-3)}
    out["cpu_baseline"] = occupancy_cpu_baseline(mu, sc, al)
    return out


def occupancy_cpu_baseline(mu, sc, al):
    """The oracle's frame and occupancy (FP64 NumPy, one host thread) on the
    same cloud, as surfels/s."""
    import oracle.occupancy as O
    t0 = time.perf_counter()
    f = O.scene_frame(mu, sc)
    O.occupancy(mu, al, f)
    dt = time.perf_counter() - t0
    return {"value": len(mu) / dt, "unit": "surfels/s", "cores": 1, "kind": "oracle",
            "seconds": dt, "sample": f"all {len(mu)} surfels (frame + occupancy, g = {f['g']})"}


def profile_occupancy_steps(args):
    """Profiling target of the occupancy construction: N frame + occupancy
    calls on the 256^3 scene's surfel cloud (per call: k_gauss_smax, the
    selection launches, k_gauss_dist, again the selection, k_gauss_frame,
    then k_gauss_scatter and k_density_floor) and nothing else."""
    import torch

    import synth
    from paper_2601_04860_b300 import occupancy, scene_frame
    wl = synth.config2()
    mu, sc, al = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in synth.gaussians(wl))
    for _ in range(args.profile_occupancy_steps):
        f = scene_frame(mu, sc)
        occ, _ = occupancy(mu, al, f)
    torch.cuda.synchronize()
    print(json.dumps({"profile_occupancy_steps": args.profile_occupancy_steps, "g": f.g,
                      "occupied": int(occ.sum().item())}))
    return 0


def _surfel_setup(dev):
    """The surfel leg's inputs on the 256^3 scene: its 1M surface points as
    surfel centres (two scales, a random orientation, 2% needles of aspect
    100-1000) and a context holding the finalized fusion of its 8 views."""
    import torch

    import synth
    from paper_2601_04860_b300 import FusionParams, VoxelFusion
    wl = synth.config2()
    mu, sc, _ = synth.gaussians(wl, floaters=0.0)
    q = synth.quaternions(len(mu))
    rng = np.random.Generator(np.random.PCG64(21))
    k = rng.choice(len(mu), len(mu) // 50, replace=False)
    sc[k, 0] *= rng.uniform(100, 1000, size=len(k)).astype(np.float32)
    occ = torch.from_numpy(wl.occ).to(dev)
    depth = [torch.from_numpy(x).to(dev) for x in wl.depth]
    mask = [torch.from_numpy(m.view(np.int16)).to(dev) for m in wl.mask]
    fu = VoxelFusion(wl.grid, occ=occ, params=FusionParams())
    fu.add_views(wl.cams, depth, mask, mask_type=wl.mask_type)
    fu.finalize(score=True)
    dm, ds, dq = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (mu, sc, q))
    return wl, fu, mask, (mu, sc, q), (dm, ds, dq)


def profile_surfel_steps(args):
    """Profiling target of the voxel-to-surfel mapping: the fusion set-up,
    then N surfel_labels calls (k_surfel_aspect, the selection launches,
    k_surfel_pass, k_surfel_big, k_surfel_big_out) and nothing else."""
    import torch
    dev = torch.device("cuda")
    wl, fu, mask, _, (dm, ds, dq) = _surfel_setup(dev)
    for _ in range(args.profile_surfel_steps):
        fu.surfel_labels(dm, ds, dq, wl.cams, mask, wl.mask_type)
    torch.cuda.synchronize()
    print(json.dumps({"profile_surfel_steps": args.profile_surfel_steps,
                      "workload": "surfels-on-forward-dense-256", "surfels": int(dm.shape[0])}))
    fu.close()
    return 0


def measure_surfels(dev, steps: int):
    """Voxel-to-surfel mapping on the 256^3 scene: its 1M surface points as
    surfel centres (two scales, a random orientation, 2% needles) against the
    finalized fusion of its 8 views; the call (aspects, the P99 selection,
    the per-surfel pass) replayed from a CUDA graph, L2 flushed; its roofline
    (surfel inputs and outputs once); the oracle on a sample on the host."""
    import torch
    wl, fu, mask, (mu, sc, q), (dm, ds, dq) = _surfel_setup(dev)
    for _ in range(3):
        r = fu.surfel_labels(dm, ds, dq, wl.cams, mask, wl.mask_type)
    torch.cuda.synchronize()
    flush = L2Flush(dev)
    ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ev[0].record()
        r = fu.surfel_labels(dm, ds, dq, wl.cams, mask, wl.mask_type)
        ev[1].record()
    ms = []
    for k in range(3 + steps):
        flush.zero_()
        g.replay()
        torch.cuda.synchronize()
        if k >= 3:
            ms.append(ev[0].elapsed_time(ev[1]))
    m = float(np.mean(ms))
    n = len(mu)
    f1 = int(fu.label_points(dm).sum().item())
    f2, f = int(r["f2"].sum().item()), int(r["f"].sum().item())
    fu.close()
    algo = n * (12 + 8 + 16 + 1 + 1 + 4)  # centres, scales, quaternions; f, f2, kappa
    peak, peak_kind = peaks()
    ach = algo / (m * 1e-3) / 1e9
    return {"workload": f"surfels-on-forward-dense-256 ({n} surfels, 8 views; passes kept "
                        f"{f1} / {f2} / {f})",
            "ms": m, "surfels_per_s": n / (m * 1e-3),
            "roofline": {"bound": "hbm", "kernel": "surfel_labels (k_surfel_aspect + selection + "
                                                  "k_surfel_pass)",
                         "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": None, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": algo, "ms_per_launch": m},
            "cpu_baseline": surfels_cpu_baseline(wl, mu, sc, q)}


def surfels_cpu_baseline(wl, mu, sc, q, n_sample: int = 20_000):
    """The oracle's Passes 2-3 (FP64 NumPy and Python loops, one thread) on a
    sample of the surfels, given its own Pass 1 and view masks, as surfels/s."""
    import oracle
    import oracle.surfels as S
    lin = wl.active_linear()
    o = oracle.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, wl.mask_type, oracle.Params())
    seg = oracle.dense_seg(wl.grid, lin, o["seg"])
    idx = np.arange(0, len(mu), max(1, len(mu) // n_sample))[:n_sample]
    F1, _ = oracle.label(wl.grid, seg, mu[idx])
    g, h = wl.grid.g, np.float64(np.float32(wl.grid.h))
    org = np.asarray(wl.grid.origin, np.float32).astype(np.float64)
    cell = np.floor((mu[idx].astype(np.float64) - org) / h).astype(np.int64)
    vlin = (cell[:, 2] * g + cell[:, 1]) * g + cell[:, 0]
    pos = np.clip(np.searchsorted(lin, vlin), 0, len(lin) - 1)
    vbits = np.where((lin[pos] == vlin) & (F1 > 0), o["bits"][pos], 0).astype(np.uint32)
    t0 = time.perf_counter()
    S.surfel_labels(mu[idx], sc[idx], q[idx], F1 > 0, vbits, wl.cams, wl.mask, wl.mask_type)
    dt = time.perf_counter() - t0
    return {"value": len(idx) / dt, "unit": "surfels/s", "cores": 1, "kind": "oracle",
            "seconds": dt, "sample": f"{len(idx)} of {len(mu)} surfels (every "
                                     f"{len(mu) // len(idx)}th; Passes 2-3)"}


def measure_adjoint(dev, steps: int):
    """Config 4: forward + hand-written backward through the autograd Function on
    the 256^3 forward-facing scene with FP32 logits and depth as leaves: eager,
    and the same forward + BCE + backward captured once in a CUDA graph and
    replayed (the views are marshalled at capture only).  The adjoint kernel's
    own time comes from a graph of the backward call alone."""
    import torch

    import synth
    from paper_2601_04860_b300 import MASK_LOGIT_F32, FusionParams, VoxelFusion, fuse
    wl = synth.config4()
    occ = torch.from_numpy(wl.occ).to(dev)
    logits = [torch.from_numpy(m).to(dev).requires_grad_(True) for m in wl.mask]
    depths = [torch.from_numpy(d).to(dev).requires_grad_(True) for d in wl.depth]
    fu = VoxelFusion(wl.grid, occ=occ, params=FusionParams())
    lin = torch.from_numpy(wl.active_linear()).to(dev)
    y = (torch.rand(len(lin), device=dev) < 0.1).float()  # any fixed target works for timing
    flush = L2Flush(dev)

    def fwd_bwd():
        P = fuse(fu, wl.cams, logits, depths, MASK_LOGIT_F32)
        Pc = P[lin].clamp(1e-6, 1 - 1e-6)
        loss = -(y * torch.log(Pc) + (1 - y) * torch.log(1 - Pc)).sum()
        loss.backward()
        return loss

    fwd, bwd = [], []
    for k in range(3 + steps):
        for t in logits + depths:
            t.grad = None
        flush.zero_()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        P = fuse(fu, wl.cams, logits, depths, MASK_LOGIT_F32)
        Pc = P[lin].clamp(1e-6, 1 - 1e-6)
        loss = -(y * torch.log(Pc) + (1 - y) * torch.log(1 - Pc)).sum()
        b.record()
        loss.backward()
        c.record()
        torch.cuda.synchronize()
        if k >= 3:
            fwd.append(a.elapsed_time(b))
            bwd.append(b.elapsed_time(c))
    eager_grads = [t.grad.clone() for t in logits + depths]
    # the whole step in a CUDA graph (warm-up on a side stream, then capture;
    # the gradients are written into tensors the graph owns).  Fresh leaves: the
    # eager steps' autograd nodes (and their default-stream gradient
    # accumulation) must not be reused inside the capture.
    del P, Pc, loss
    logits = [t.detach().clone().requires_grad_(True) for t in logits]
    depths = [t.detach().clone().requires_grad_(True) for t in depths]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            for t in logits + depths:
                t.grad = None
            fwd_bwd()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for t in logits + depths:
        t.grad = None
    ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ev[0].record()
        fwd_bwd()
        ev[1].record()
    gms = []
    for k in range(3 + steps):
        flush.zero_()
        g.replay()
        torch.cuda.synchronize()
        if k >= 3:
            gms.append(ev[0].elapsed_time(ev[1]))
    same = all(torch.equal(t.grad, e) for t, e in zip(logits + depths, eager_grads))
    # the adjoint kernel alone: a graph of the backward call (gradient rasters
    # zeroed outside it), for its roofline
    gP = torch.ones(fu.n_cells, device=dev)
    gm = [torch.zeros_like(t) for t in logits]
    gd = [torch.zeros_like(t) for t in depths]
    with torch.no_grad():
        fu.reset()
        fu.add_views(wl.cams, [d.detach() for d in depths], [m.detach() for m in logits],
                     mask_type=MASK_LOGIT_F32)
    torch.cuda.synchronize()
    bev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
    gb = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gb):
        bev[0].record()
        fu.backward(wl.cams, [d.detach() for d in depths], [m.detach() for m in logits], gP,
                    grad_mask=gm, grad_depth=gd, mask_type=MASK_LOGIT_F32)
        bev[1].record()
    kms = []
    for k in range(3 + steps):
        flush.zero_()
        gb.replay()
        torch.cuda.synchronize()
        if k >= 3:
            kms.append(bev[0].elapsed_time(bev[1]))
    n, na, S = fu.n_cells, fu.n_active, wl.n_views
    st = fu.export_state()
    n_voted = int((st["Z"] > 0).sum())
    n_votes = int(np.unpackbits(st["bits"].cpu().numpy().view(np.uint8)).sum())
    fu.close()
    # algorithmic bytes of one backward launch: every active voxel's index, Z
    # and cotangent; a voted voxel's W and its S gathers (depth and logit, 4 B
    # each); a vote's two gradient read-modify-writes (8 B each).  Voxels that
    # never voted (Z = 0) are skipped after their first loads.
    kb = 12 * na + n_voted * (4 + 8 * S) + 16 * n_votes
    peak, peak_kind = peaks()
    km = float(np.mean(kms))
    fb = float(np.mean(gms))
    return {"workload": "differentiable-256 (config-2 scene, FP32 logits + depth as leaves)",
            "fwd_ms": float(np.mean(fwd)), "bwd_ms": float(np.mean(bwd)),
            "graph_fwd_bwd_ms": fb,
            "graph_fwd_bwd_updates_per_s": n * S / (fb * 1e-3),
            "graph_grads_equal_eager": bool(same),
            "fwd_bwd_updates_per_s": n * S / ((np.mean(fwd) + np.mean(bwd)) * 1e-3),
            "backward_kernel_ms": km, "voted_voxels": n_voted, "votes": n_votes,
            "roofline": {"bound": "hbm", "kernel": "k_backward", "algorithmic_bytes_per_launch":
                         int(kb), "achieved": kb / (km * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": kb / (km * 1e-3) / 1e9 / peak,
                         "peak_kind": peak_kind},
            "what": "eager autograd: fuse() + BCE on active voxels, then loss.backward() "
                    "(adjoint kernel + gradient raster zero-fill); graph: the same captured "
                    "once and replayed; L2 flushed per step"}


def measure_sessions(dev, scale: float, n_sessions: int, rates, budget_frac: float = 1.0,
                     n_warm: int = 200, n_timed: int = 2000):
    """Config 5: many uneven sessions.  (a) Batched: every session's views in ONE
    persistent fuse launch + one finalize + one label launch, autotuned and
    replayed from a CUDA graph, vs the plain per-session launches.  (b) Served:
    Poisson requests (one new view each) through the continuous-batching server
    vs the paper-style re-fusion and the incremental one-request-at-a-time
    baselines."""
    import torch

    import synth
    from paper_2601_04860_b300 import Autotuner, Batch, Schedule
    from paper_2601_04860_b300.serve import (Server, Session, latency_summary,
                                             poisson_requests, serve_plain, session_data_from)
    t_gen = time.perf_counter()
    recipes = synth.session_mix(n_sessions=n_sessions, scale=scale)
    data = []
    for i, r in enumerate(recipes):
        wl = synth.session_workload(r)
        data.append(session_data_from(wl, i, fusion_params(wl)))
    t_gen = time.perf_counter() - t_gen
    nominal = sum((int(d.grid.g) ** 3 if d.occ is not None else len(d.coords)) * d.n_views
                  for d in data)
    out = {"sessions": n_sessions, "scale": scale, "generation_s": t_gen,
           "dense": sum(d.occ is not None for d in data),
           "views_total": sum(d.n_views for d in data),
           "voxel_views_nominal": int(nominal),
           "brick_ordered": sum(bool(d.params.brick_order) for d in data)}
    # (a) batched vs plain, all views of every session
    sess = [Session(d, dev) for d in data]
    flush = L2Flush(dev)

    def plain_pass():
        for s in sess:
            s.fusion.reset()
            s.fusion.add_views(s.data.cams, s.depth, s.mask, mask_type=s.data.mask_type)
            s.fusion.finalize(score=s.score)
            s.fusion.label_points(s.points, out=s.labels)
    for _ in range(2):
        plain_pass()
    torch.cuda.synchronize()
    ms = []
    for _ in range(5):
        flush.zero_()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plain_pass()
        b_.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b_))
    out["plain_ms"] = float(np.mean(ms))
    batch = Batch(max_sessions=n_sessions, max_views=sum(d.n_views for d in data))
    for s in sess:
        s.fusion.reset()
        batch.queue(s.fusion, s.data.cams, s.depth, s.mask, mask_type=s.data.mask_type)
    tuner = Autotuner(reps=2)
    cands = [Schedule(t, v, c, tile) for t in (128, 256) for v in (1, 2) for c in (4, 8)
             for tile in (t * v * 16, t * v * 64)]
    sch = tuner.pick(batch, max(d.n_views for d in data), candidates=cands)
    out["schedule"] = {"threads": sch.threads, "voxels_per_thread": sch.voxels_per_thread,
                       "ctas_per_sm": sch.ctas_per_sm, "tile": sch.tile}
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(3)]
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        ev[0].record()
        batch.fuse(sch)
        ev[1].record()
        batch.finalize(scores=[s.score for s in sess], points=[s.points for s in sess],
                       labels=[s.labels for s in sess])
        ev[2].record()
    fuse_ms, all_ms = [], []
    for k in range(8):
        flush.zero_()
        graph.replay()
        torch.cuda.synchronize()
        if k >= 2:
            fuse_ms.append(ev[0].elapsed_time(ev[1]))
            all_ms.append(ev[0].elapsed_time(ev[2]))
    out["batched_graph_ms"] = float(np.mean(all_ms))
    out["batched_fuse_ms"] = float(np.mean(fuse_ms))
    # algorithmic bytes of the batched fold (first touch only): per session the
    # active list, W / Z / bits read and written, its rasters once; and of the
    # finalize + labels: scores (dense: the g^3 grid), seg bits, points, labels
    fuse_b = fin_b = 0
    for s in sess:
        na = s.fusion.n_active
        g3 = s.fusion.n_cells
        fuse_b += 4 * na + 24 * na + sum(d.nbytes + m.nbytes for d, m in
                                         zip(s.data.depth, s.data.mask))
        fin_b += (4 * g3 if s.fusion.dense else 4 * na) + 12 * na + g3 // 8 + \
            13 * len(s.data.points)
    peak, peak_kind = peaks()
    fuse_s = out["batched_fuse_ms"] * 1e-3
    out["batched_roofline"] = {
        "bound": "hbm", "kernel": "k_batch_fuse", "algorithmic_bytes_per_launch": int(fuse_b),
        "achieved": fuse_b / fuse_s / 1e9, "peak": peak, "unit": "GB/s",
        "frac": fuse_b / fuse_s / 1e9 / peak, "peak_kind": peak_kind,
        "finalize_labels_bytes": int(fin_b),
        "finalize_labels_frac": fin_b / ((out["batched_graph_ms"] - out["batched_fuse_ms"]) *
                                         1e-3) / 1e9 / peak,
        "what": "all sessions of the mix in one persistent launch (dense and sparse)"}
    out["batched_updates_per_s"] = nominal / (np.mean(all_ms) * 1e-3)
    out["plain_updates_per_s"] = nominal / (out["plain_ms"] * 1e-3)
    out["launches"] = {"batched": 3 + 0, "plain": 4 * n_sessions}
    del graph
    # the dense and the sparse (contracted) sessions as separate batches: the
    # dense grids' fold against the HBM roofline, the contracted sets' fold
    # (ALU-bound: compensated projections) for reference
    for kind in ("dense", "sparse"):
        part = [s for s in sess if s.fusion.dense == (kind == "dense")]
        if not part:
            continue
        bp = Batch(max_sessions=len(part), max_views=sum(s.data.n_views for s in part))
        for s in part:
            s.fusion.reset()
            bp.queue(s.fusion, s.data.cams, s.depth, s.mask, mask_type=s.data.mask_type)
        pe = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        gp = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(gp):
            pe[0].record()
            bp.fuse(sch)
            pe[1].record()
        pms = []
        for k in range(6):
            flush.zero_()
            gp.replay()
            torch.cuda.synchronize()
            if k >= 2:
                pms.append(pe[0].elapsed_time(pe[1]))
        pb = sum(4 * s.fusion.n_active + 24 * s.fusion.n_active +
                 sum(d.nbytes + m.nbytes for d, m in zip(s.data.depth, s.data.mask))
                 for s in part)
        act = sum(s.fusion.n_active * s.data.n_views for s in part)
        t = float(np.mean(pms))
        out[f"batched_fuse_{kind}"] = {
            "sessions": len(part), "ms": t, "active_voxel_views": int(act),
            "ns_per_active_voxel_view": t * 1e6 / max(1, act),
            "roofline": {"bound": "hbm" if kind == "dense" else "alu",
                         "algorithmic_bytes_per_launch": int(pb),
                         "achieved_gbs": pb / (t * 1e-3) / 1e9,
                         "hbm_frac": pb / (t * 1e-3) / 1e9 / peak, "peak_kind": peak_kind}}
        del gp
        bp.close()
    for s in sess:
        s.close()
    batch.close()
    torch.cuda.synchronize()
    # (b) served requests: n_warm warm-up requests, then n_timed timed ones, on
    # one Poisson stream per rate (the same stream for the server and the two
    # plain baselines)
    foot = sum(Session.footprint(d) for d in data)
    served = {"warmup_requests": n_warm, "timed_requests": n_timed}
    for rate in rates:
        res = {}
        for mode in ("server", "incremental", "refuse"):
            reqs = poisson_requests(n_warm + n_timed, float(rate), [d.sid for d in data],
                                    seed=1005 + 4)
            timed = reqs[n_warm:]
            if mode == "server":
                srv = Server(data, memory_budget=int(foot * budget_frac) + 1, max_batch=64)
                srv.admit_all()
                srv.run(reqs)
                res[mode] = latency_summary(timed)
                res[mode]["evictions"] = srv.stats["evictions"]
                srv.close()
            else:
                serve_plain(data, reqs, mode)
                res[mode] = latency_summary(timed)
        served[str(rate)] = res
    out["served"] = served
    return out


def profile_steps(args):
    """Profiling target: init (3 launches: count, count, emit) then N eager
    one-call steps (4 launches each: k_tile_count, k_tile_emit, k_fuse_fin,
    k_label on a dense workload) and nothing else."""
    import torch

    from paper_2601_04860_b300 import FusionParams, PreparedViews, VoxelFusion

    dev = torch.device("cuda")
    wl = make_workload(args.workload)
    occ = None if wl.occ is None else torch.from_numpy(wl.occ).to(dev)
    coords = None if wl.coords is None else torch.from_numpy(wl.coords).to(dev)
    depth = [torch.from_numpy(d).to(dev) for d in wl.depth]
    mask = [torch.from_numpy(m.view(np.float16) if wl.mask_type == 1 else m).to(dev)
            for m in wl.mask]
    pts = torch.from_numpy(np.ascontiguousarray(wl.points)).to(dev)
    fu = VoxelFusion(wl.grid, occ=occ, coords=coords, params=fusion_params(wl))
    score = torch.empty(fu.n_cells if occ is not None else fu.n_active, dtype=torch.float32,
                        device=dev)
    labels = torch.empty(len(wl.points), dtype=torch.uint8, device=dev)
    pv = PreparedViews(wl.cams, depth, mask, wl.mask_type)
    for _ in range(args.profile_steps):
        fu.step(pv, occ=occ, coords=coords, score=score, xyz=pts, labels=labels)
    torch.cuda.synchronize()
    fu.sync()
    print(json.dumps({"profile_steps": args.profile_steps, "workload": args.workload,
                      "active_voxels": fu.n_active}))
    fu.close()
    return 0


def run(args):
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        if rank != 0:
            return 0
        return run_reference(args)
    if args.profile_steps:
        return profile_steps(args)
    if args.profile_tuple_steps:
        return profile_tuple_steps(args)
    if args.profile_weight_steps:
        return profile_weight_steps(args)
    if args.profile_nerf_steps:
        return profile_nerf_steps(args)
    if args.profile_surfel_steps:
        return profile_surfel_steps(args)
    if args.profile_occupancy_steps:
        return profile_occupancy_steps(args)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res, wl = run_ours(args, rank, world, local_rank)
    import torch
    dev = torch.device("cuda", local_rank)
    dense_ws = args.workload == "forward-dense-256"

    def leg(name, enabled, fn):
        """An additional leg; its failure is reported in its key, not fatal."""
        if not enabled or args.quick:
            return
        try:
            res[name] = fn()
        except Exception as e:  # noqa: BLE001
            import traceback
            traceback.print_exc()
            res[name] = {"error": f"{type(e).__name__}: {e}"}

    leg("sessions", not args.no_sessions,
        lambda: measure_sessions(dev, args.sessions_scale, args.sessions,
                                 [float(r) for r in args.rates.split(",")],
                                 n_warm=args.warm_requests, n_timed=args.timed_requests))
    leg("adjoint", not args.no_adjoint, lambda: measure_adjoint(dev, max(5, args.steps // 2)))
    leg("unbounded_sparse", not args.no_sparse and dense_ws,
        lambda: measure_sparse(dev, max(5, args.steps // 2)))
    leg("tuple", not args.no_tuple and dense_ws, lambda: measure_tuple(dev, max(5, args.steps // 2)))
    leg("nerf", not args.no_nerf and dense_ws, lambda: measure_nerf(dev, max(5, args.steps // 2)))
    leg("weighting", not args.no_weighting and dense_ws,
        lambda: measure_weighting(dev, max(5, args.steps // 2)))
    leg("occupancy", not args.no_occupancy and dense_ws,
        lambda: measure_occupancy(dev, max(5, args.steps // 2)))
    leg("surfels", not args.no_surfels and dense_ws,
        lambda: measure_surfels(dev, max(5, args.steps // 2)))
    pgpu = res.pop("_parity_gpu", None)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        full_s, det = oracle_rate(wl, args.cpu_seconds)
        if pgpu is not None:
            try:
                res["parity"] = bench_parity(wl, pgpu, det["sample_index"], det["sample_out"],
                                             det["sample_points"])
            except Exception as e:  # noqa: BLE001
                res["parity"] = {"error": f"{type(e).__name__}: {e}"}
            pgpu = None
        if pgpu is not None:
            res["parity"] = bench_parity(wl, pgpu, det["sample_index"], det["sample_out"],
                                         det["sample_points"])
        N = res["config"]["voxels_nominal"]
        res["cpu_baseline"] = {
            "value": N * wl.n_views / full_s, "unit": UNIT, "cores": det["cores"],
            "kind": "oracle",
            "sample": (f"{det['sample_voxels']} of {det['active_voxels']} active voxels x "
                       f"{wl.n_views} views + {det['sample_points']} points, extrapolated "
                       f"to the full step; median of {det['repeats']} timed runs"),
            "seconds": det["fuse_s"] + det["label_s"],
            "repeats": det["repeats"],
            "spread": [N * wl.n_views / det["full_s_max"], N * wl.n_views / det["full_s_min"]]}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def workload_config(name, wl):
    """The config keys both arms report for a workload."""
    return {"workload": name, "description": WORKLOADS[name], "grid": int(wl.grid.g),
            "views": int(wl.n_views), "active_voxels": int(len(wl.active_linear())),
            "voxels_nominal": int(wl.n_voxels), "points": int(len(wl.points))}


def run_reference(args):
    wl = make_workload(args.workload)
    per_step = max(1.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    times, det = [], None
    for k in range(args.warmup + args.steps):
        full_s, det = oracle_rate(wl, per_step, seed=k, repeats=1)
        if k >= args.warmup:
            times.append(full_s)
    N = wl.n_voxels
    ms = float(np.median(times)) * 1e3
    v = N * wl.n_views / (ms * 1e-3)
    sample = (f"each step: {det['sample_voxels']} of {det['active_voxels']} active voxels x "
              f"{wl.n_views} views + {det['sample_points']} points, extrapolated to the full "
              f"step; the median over the {len(times)} timed steps (spread "
              f"{1e3 * min(times):.1f}-{1e3 * max(times):.1f} ms)")
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded ray-cast scene; no dataset)",
           "config": {**workload_config(args.workload, wl),
                      "parallelism": f"oracle on {det['cores']} host cores"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": det["cores"], "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="forward-dense-256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the forward+backward leg")
    ap.add_argument("--no-sessions", action="store_true", help="skip the batched/served leg")
    ap.add_argument("--no-tuple", action="store_true", help="skip the depth-tuple-mode leg")
    ap.add_argument("--no-sparse", action="store_true",
                    help="skip the unbounded-sparse (config 3) leg")
    ap.add_argument("--no-nerf", action="store_true", help="skip the NeRF-variant leg")
    ap.add_argument("--no-weighting", action="store_true",
                    help="skip the depth-weighted-mask leg")
    ap.add_argument("--no-occupancy", action="store_true",
                    help="skip the occupancy-construction leg")
    ap.add_argument("--no-surfels", action="store_true", help="skip the voxel-to-surfel leg")
    ap.add_argument("--sessions", type=int, default=64, help="sessions in the batched/served leg")
    ap.add_argument("--sessions-scale", type=float, default=1.0,
                    help="size scale of the sessions (1.0 = the full session mix)")
    ap.add_argument("--rates", default="200,1000,5000,20000",
                    help="request rates (per second) to serve")
    ap.add_argument("--warm-requests", type=int, default=200,
                    help="served leg: untimed warm-up requests per rate")
    ap.add_argument("--timed-requests", type=int, default=2000,
                    help="served leg: timed requests per rate")
    ap.add_argument("--quick", action="store_true",
                    help="timed graph steps only: no eager, per-update, e2e or CPU legs")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="profiling target: run N eager one-call steps and exit")
    ap.add_argument("--profile-tuple-steps", type=int, default=0,
                    help="profiling target: run N eager depth-tuple steps and exit")
    ap.add_argument("--profile-nerf-steps", type=int, default=0,
                    help="profiling target: run N eager NeRF-variant steps and exit")
    ap.add_argument("--profile-surfel-steps", type=int, default=0,
                    help="profiling target: run N voxel-to-surfel calls and exit")
    ap.add_argument("--profile-weight-steps", type=int, default=0,
                    help="profiling target: run N eager depth-weighted steps and exit")
    ap.add_argument("--profile-occupancy-steps", type=int, default=0,
                    help="profiling target: run N occupancy constructions and exit")
    ap.add_argument("--active-order", choices=("auto", "brick", "linear"), default="auto",
                    help="active-list order of the fused contexts (brick: warp-level view "
                         "culling; auto: brick for sparse priors, linear for dense ones)")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    global ACTIVE_ORDER
    ACTIVE_ORDER = args.active_order
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
