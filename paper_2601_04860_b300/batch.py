"""Batched fusion of many sessions in one persistent launch, and its autotuner.

``Batch`` wraps the ``divas_batch_*`` C ABI: queue (session, views) pairs --
contexts of any size, kind and view count -- then ``fuse`` folds all of them
in ONE persistent kernel (work items = (session, tile of its active list),
taken dynamically by the CTAs) and ``finalize`` normalises, thresholds and
labels all of them in one launch each.  Every session's result is bitwise the
one it would get alone.

``Autotuner`` picks the launch schedule (threads per CTA, voxels per thread,
CTAs per SM, tile size) by timing dry runs -- which write to batch scratch and
leave the sessions untouched -- with CUDA events, and caches the winner per
workload class.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
from dataclasses import asdict, dataclass

import torch

from . import _lib as L
from .fusion import VoxelFusion, _ptr, _stream, view_c


class DivasSchedule(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("voxels_per_thread", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("tile", ctypes.c_int32)]


_P = ctypes.c_void_p
_BATCH_SIGS = {
    "divas_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32]),
    "divas_batch_queue": (ctypes.c_int, [_P, _P, ctypes.POINTER(L.DivasView), ctypes.c_int32]),
    "divas_batch_fuse": (ctypes.c_int, [_P, ctypes.POINTER(DivasSchedule), ctypes.c_int32, _P]),
    "divas_batch_finalize": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_P),
                                            ctypes.c_uint32, _P]),
    "divas_batch_clear": (ctypes.c_int, [_P]),
    "divas_batch_size": (ctypes.c_int32, [_P]),
    "divas_batch_last_error": (ctypes.c_char_p, [_P]),
    "divas_batch_destroy": (None, [_P]),
}


def _lib():
    lib = L.load()
    if not getattr(lib, "_batch_ready", False):
        for name, (res, args) in _BATCH_SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        lib._batch_ready = True
    return lib


@dataclass(frozen=True)
class Schedule:
    threads: int = 256
    voxels_per_thread: int = 1
    ctas_per_sm: int = 8
    tile: int = 4096

    def c(self) -> DivasSchedule:
        return DivasSchedule(self.threads, self.voxels_per_thread, self.ctas_per_sm, self.tile)


class Batch:
    """A reusable batch of (session, views) pairs."""

    def __init__(self, max_sessions: int = 256, max_views: int = 2048):
        self.lib = _lib()
        self._h = ctypes.c_void_p()
        st = self.lib.divas_batch_create(ctypes.byref(self._h), int(max_sessions), int(max_views))
        L.check(st, None)
        self.sessions: list[VoxelFusion] = []
        self._keep = []

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.divas_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != L.DIVAS_OK:
            msg = self.lib.divas_batch_last_error(self._h)
            raise L.DivasError(st, msg.decode() if msg else "")

    def __len__(self) -> int:
        return int(self.lib.divas_batch_size(self._h))

    def queue(self, fusion: VoxelFusion, cams, depths, masks, mask_type: int | None = None):
        """Queue 1..32 views of one session (a session appears once per batch)."""
        n = len(cams)
        arr = (L.DivasView * n)()
        for k in range(n):
            arr[k] = view_c(cams[k], depths[k], masks[k], mask_type)
        self._keep.append((depths, masks))
        self._check(self.lib.divas_batch_queue(self._h, fusion.handle, arr, n))
        self.sessions.append(fusion)

    def queue_prepared(self, fusion: VoxelFusion, view: L.DivasView):
        """Queue one already marshalled view of one session."""
        self._check(self.lib.divas_batch_queue(self._h, fusion.handle, ctypes.byref(view), 1))
        self.sessions.append(fusion)

    def fuse(self, schedule: Schedule | None = None, dry_run: bool = False, stream=None):
        sch = (schedule or Schedule()).c()
        self._check(self.lib.divas_batch_fuse(self._h, ctypes.byref(sch), 1 if dry_run else 0,
                                              _stream(stream)))

    def finalize(self, scores=None, points=None, labels=None, keep_zeros=False, stream=None):
        """scores / points / labels: per queued session, tensors or None.
        ``keep_zeros``: the dense score tensors already hold zeros for their
        unoccupied voxels (e.g. zero-initialised and only ever written by this
        session), so only the active voxels' scores are written."""
        n = len(self.sessions)
        sc = (_P * n)(*[(_ptr(t).value if t is not None else None)
                        for t in (scores or [None] * n)])
        pts = (_P * n)(*[(_ptr(t).value if t is not None else None)
                         for t in (points or [None] * n)])
        npts = (ctypes.c_int64 * n)(*[(t.shape[0] if t is not None else 0)
                                      for t in (points or [None] * n)])
        lab = (_P * n)(*[(_ptr(t).value if t is not None else None)
                         for t in (labels or [None] * n)])
        self._check(self.lib.divas_batch_finalize(self._h, sc, pts, npts, lab,
                                                  L.KEEP_ZEROS if keep_zeros else 0,
                                                  _stream(stream)))
        self.sessions = []
        self._keep = []

    def clear(self):
        self._check(self.lib.divas_batch_clear(self._h))
        self.sessions = []
        self._keep = []


class Autotuner:
    """Times dry runs of every candidate schedule on the queued batch and keeps
    the fastest per workload class (sessions, active voxels, views), in memory
    and optionally in a JSON file."""

    CANDIDATES = [Schedule(t, v, c, tile)
                  for t in (128, 256) for v in (1, 2, 4) for c in (4, 8, 16)
                  for tile in (t * v * 4, t * v * 16, t * v * 64)]

    def __init__(self, cache_path: str | None = None, reps: int = 3):
        self.cache_path = cache_path
        self.reps = reps
        self.cache: dict[str, Schedule] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = {k: Schedule(**v) for k, v in json.load(f).items()}

    @staticmethod
    def key(batch: Batch, n_views: int) -> str:
        vox = sum(s.n_active for s in batch.sessions)
        return (f"s{2 ** math.ceil(math.log2(max(1, len(batch.sessions))))}"
                f"-v{2 ** math.ceil(math.log2(max(1, vox)))}"
                f"-k{2 ** math.ceil(math.log2(max(1, n_views)))}")

    def pick(self, batch: Batch, n_views: int, candidates=None) -> Schedule:
        k = self.key(batch, n_views)
        if k in self.cache:
            return self.cache[k]
        best, best_ms = None, float("inf")
        for sch in candidates or self.CANDIDATES:
            batch.fuse(sch, dry_run=True)  # warm (allocates the scratch once)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(self.reps):
                batch.fuse(sch, dry_run=True)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / self.reps
            if ms < best_ms:
                best, best_ms = sch, ms
        self.cache[k] = best
        if self.cache_path:
            with open(self.cache_path, "w") as f:
                json.dump({kk: asdict(v) for kk, v in self.cache.items()}, f)
        return best
