"""Helpers shared by the GPU parity tests: upload a synthetic workload, run the
CUDA path through the C ABI, run the oracle on the same inputs, compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2601_04860_b300 import FusionParams, VoxelFusion, seg_bits_to_bool

EXACT_FLAGS = 0xFFFFFFFF  # any near-boundary flag excludes a voxel from exact checks
RTOL = 1e-5               # scores W, Z, P: relative tolerance in FP32

# near-boundary counts of the parity checks of this session (printed and
# written to a JSON file by the test session's terminal summary)
PARITY: list[dict] = []


def current_test() -> str:
    """The running test's id (file::name[params])."""
    import os
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0].split("/")[-1]


def record(name: str, voxels: int, flagged: int, mismatches: int = 0, **extra) -> dict:
    """Note one parity check: items compared, items the oracle flags as within
    1e-6 of a boundary (excluded from the exact checks), mismatches outside
    them (0 when the check passed)."""
    row = {"check": name, "items": int(voxels), "flagged": int(flagged),
           "flagged_frac": float(flagged) / max(1, int(voxels)), "mismatches": int(mismatches)}
    row.update({k: (int(v) if isinstance(v, (np.integer, int)) else v) for k, v in extra.items()})
    PARITY.append(row)
    return row


def to_params(p: oracle.Params) -> FusionParams:
    return FusionParams(p.tau_m, p.gamma, p.alpha1, p.tau_cons, p.eps, p.z_near)


def upload(wl):
    dev = torch.device("cuda")
    d = {}
    d["occ"] = None if wl.occ is None else torch.from_numpy(wl.occ).to(dev)
    d["coords"] = None if wl.coords is None else torch.from_numpy(wl.coords).to(dev)
    d["depth"] = [torch.from_numpy(x).to(dev) for x in wl.depth]
    if wl.mask_type == oracle.MASK_F16:
        d["mask"] = [torch.from_numpy(m.view(np.float16)).to(dev) for m in wl.mask]
    else:
        d["mask"] = [torch.from_numpy(m).to(dev) for m in wl.mask]
    d["points"] = torch.from_numpy(np.ascontiguousarray(wl.points)).to(dev)
    return d


def run_gpu(wl, params: oracle.Params, mode="oneshot", dev_inputs=None, want_pix=False,
            labels=True):
    """Fuse every view of ``wl`` on the GPU; returns numpy outputs."""
    d = dev_inputs or upload(wl)
    fu = VoxelFusion(wl.grid, occ=d["occ"], coords=d["coords"], params=to_params(params))
    mt = wl.mask_type
    if mode == "oneshot":
        fu.add_views(wl.cams, d["depth"], d["mask"], mask_type=mt)
    elif mode == "incremental":
        for c, dp, m in zip(wl.cams, d["depth"], d["mask"]):
            fu.add_view(c, dp, m, mask_type=mt)
    elif mode == "split":  # two calls of several views each
        h = max(1, wl.n_views // 2)
        fu.add_views(wl.cams[:h], d["depth"][:h], d["mask"][:h], mask_type=mt)
        if wl.n_views > h:
            fu.add_views(wl.cams[h:], d["depth"][h:], d["mask"][h:], mask_type=mt)
    else:
        raise ValueError(mode)
    out = fu.finalize(score=True, seg_bits=True, vmask=True, count=True)
    st = fu.export_state()
    res = {
        "n_active": fu.n_active,
        "active": fu.active_coords().cpu().numpy(),
        "score": out["score"].cpu().numpy(),
        "seg_dense": seg_bits_to_bool(out["seg_bits"], fu.n_cells).cpu().numpy(),
        "vmask": out["vmask"].cpu().numpy().view(np.uint32),
        "n_seg": out["n_seg"],
        "W": st["W"].cpu().numpy(),
        "Z": st["Z"].cpu().numpy(),
        "bits": st["bits"].cpu().numpy().view(np.uint32),
    }
    if labels:
        res["labels"] = fu.label_points(d["points"]).cpu().numpy()
    if want_pix:
        res["pix"] = np.stack([fu.debug_project(c).cpu().numpy() for c in wl.cams], axis=1)
    torch.cuda.synchronize()
    fu.close()
    return res


def state_of(fu, score: torch.Tensor, labels: torch.Tensor | None = None) -> dict:
    """A context's fused state in the form compare() takes: W, Z and view bits
    exported, the given score buffer and point labels (e.g. written by a
    batched finalize or the server), seg bits / view masks / the seg count from
    a finalize into scratch buffers (it reads W and Z, it does not change them)."""
    st = fu.export_state()
    out = fu.finalize(score=False, seg_bits=True, vmask=True, count=True)
    res = {"n_active": fu.n_active, "active": fu.active_coords().cpu().numpy(),
           "score": score.cpu().numpy(),
           "seg_dense": seg_bits_to_bool(out["seg_bits"], fu.n_cells).cpu().numpy(),
           "vmask": out["vmask"].cpu().numpy().view(np.uint32), "n_seg": out["n_seg"],
           "W": st["W"].cpu().numpy(), "Z": st["Z"].cpu().numpy(),
           "bits": st["bits"].cpu().numpy().view(np.uint32)}
    if labels is not None:
        res["labels"] = labels.cpu().numpy()
    return res


def with_views(wl, order):
    """A shallow copy of a workload whose views are wl's views in ``order``
    (repeats allowed: a view folded twice votes twice)."""
    import copy
    w2 = copy.copy(wl)
    w2.cams = [wl.cams[i] for i in order]
    w2.depth = [wl.depth[i] for i in order]
    w2.mask = [wl.mask[i] for i in order]
    return w2


def sample_of(n: int, k: int, seed: int = 1):
    """Sorted random sample of k of n active-list positions (all when n <= k)."""
    if n <= k:
        return None
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=k, replace=False))


def compare(wl, gpu: dict, params: oracle.Params, check_labels=True, sample=None, name=None,
            max_flagged=0.01):
    """Element-by-element comparison against the oracle; returns a summary dict.

    ``sample``: optional indices into the active list to compare (full-size runs);
    ``max_flagged``: ceiling of the fraction of near-boundary voxels (flagged by
    the oracle, excluded from the exact checks)."""
    lin = wl.active_linear()
    g = wl.grid.g
    act = gpu["active"].astype(np.int64)
    gpu_lin = (act[:, 2] * g + act[:, 1]) * g + act[:, 0]
    assert gpu["n_active"] == len(lin)
    assert (gpu_lin == lin).all(), "active list differs from the occupied set"
    idx = np.arange(len(lin)) if sample is None else np.asarray(sample)
    o = oracle.fuse(wl.grid, lin[idx], wl.cams, wl.depth, wl.mask, wl.mask_type, params,
                    want_pix="pix" in gpu)
    flagged = o["flags"] != 0
    ok = ~flagged
    summary = {"voxels": int(len(idx)), "flagged": int(flagged.sum()),
               "voted": int((o["Z"] > 0).sum())}
    assert flagged.mean() <= max_flagged, ("near-boundary fraction", flagged.mean())
    if "pix" in gpu:
        gp = gpu["pix"][idx]
        assert (gp[ok] == o["pix"][ok]).all(), "voxel-to-pixel indices differ"
    assert (gpu["bits"][idx][ok] == o["bits"][ok]).all(), "votes differ"
    for key in ("W", "Z"):
        a = gpu[key][idx][ok].astype(np.float64)
        b = o[key][ok]
        bad = np.abs(a - b) > RTOL * np.abs(b)
        assert not bad.any(), (key, a[bad][:5], b[bad][:5])
    P_gpu = gpu["score"][lin[idx]] if wl.occ is not None else gpu["score"][idx]
    a = P_gpu[ok].astype(np.float64)
    b = o["P"][ok]
    assert not (np.abs(a - b) > RTOL * np.abs(b)).any(), "scores differ"
    seg_gpu = gpu["seg_dense"][lin[idx]]
    assert (seg_gpu[ok] == o["seg"][ok].astype(bool)).all(), "consensus differs"
    assert (gpu["vmask"][idx][ok] == o["vmask"][ok]).all(), "vmask differs"
    other = np.ones(g ** 3, bool)
    other[lin] = False
    if wl.occ is not None:
        assert (gpu["score"][other] == 0).all(), "unoccupied voxels must score 0"
    assert not gpu["seg_dense"][other].any(), "unoccupied voxels must not be segmented"
    assert gpu["n_seg"] == int(gpu["seg_dense"].sum())
    if sample is None:
        assert abs(gpu["n_seg"] - int(o["seg"].sum())) <= summary["flagged"]
    if check_labels and "labels" in gpu:
        summary.update(compare_labels(wl, gpu, o, lin, idx, flagged, sample))
    record(name or current_test(), summary["voxels"], summary["flagged"],
           **{k: v for k, v in summary.items() if k in ("points", "points_excluded")})
    return summary


def compare_labels(wl, gpu, o, lin, idx, flagged, sample):
    g = wl.grid.g
    seg_o = np.zeros(g ** 3, np.uint8)
    seg_o[lin[idx]] = o["seg"]
    pts = wl.points
    lab_o, pflags = oracle.label(wl.grid, seg_o, pts)
    bad_vox = np.zeros(g ** 3, bool)
    bad_vox[lin[idx][flagged]] = True
    # points inside flagged voxels, or near a voxel face, are excluded
    vox = _point_voxels(wl, pts)
    excl = (pflags != 0) | ((vox >= 0) & bad_vox[np.maximum(vox, 0)])
    if sample is not None:
        # with a voxel sample, only points in sampled voxels are checked
        covered = np.zeros(g ** 3, bool)
        covered[lin[idx]] = True
        excl |= ~((vox >= 0) & covered[np.maximum(vox, 0)])
    ok = ~excl
    assert (gpu["labels"][ok] == lab_o[ok]).all(), "labels differ"
    return {"points": int(len(pts)), "points_excluded": int(excl.sum()),
            "labelled": int(gpu["labels"].sum())}


def _point_voxels(wl, pts):
    """Linear voxel index of each point (FP64; -1 outside / NaN), for exclusions."""
    g = wl.grid.g
    x = pts.astype(np.float64)
    if wl.grid.contracted:
        r = np.linalg.norm(x, axis=1, keepdims=True)
        with np.errstate(invalid="ignore", divide="ignore"):
            x = np.where(r > 1.0, (2.0 - 1.0 / r) * x / r, x)
    o = np.asarray(wl.grid.origin, np.float32).astype(np.float64)
    with np.errstate(invalid="ignore"):
        s = np.floor((x - o) / float(np.float32(wl.grid.h)))
        inside = np.all((s >= 0) & (s < g), axis=1)
    s = np.where(inside[:, None], s, 0).astype(np.int64)
    v = (s[:, 2] * g + s[:, 1]) * g + s[:, 0]
    return np.where(inside, v, -1)
