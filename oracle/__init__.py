"""FP64 CPU oracle of depth-weighted multi-view voxel fusion (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The library
(``paper_2601_04860_b300``) never imports, links or runs anything here, and
this package imports nothing from the library: the two share no code.

``oracle.c`` is the plain definition of the fusion rule (Sec. 3.5, Eq.
compact-fusion, Eq. gs-depthweight, Eq. vmask, the thick-path algorithms of
Appendices A.2 and B.5), of the depth-tuple modes (the 2DGS thick and thin
paths of Sec. 3.5 and the NeRF variant of the appendix "NeRF-Backbone 3D
Fusion Details") and of the Pass 1 label lookup (Eq. pass1); ``brute.py`` is
an independent NumPy restatement that re-casts every pixel ray analytically
instead of reading the stored depth map, and states the tuple modes with
explicit ray vectors.

Parity status: every function here is pinned by tests against closed forms,
invariants, an independent brute force or finite differences (see the tests
named ``test_oracle_*``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")

MASK_F32 = 0
MASK_F16 = 1
MASK_LOGIT_F32 = 2

FLAG_PIX = 1
FLAG_DEPTH = 2
FLAG_ZNEAR = 4
FLAG_CONS = 8
FLAG_CONTRACT = 16


def build() -> str:
    """Compile ``oracle.c`` (gcc, -O2, OpenMP, no fast-math, no FP contraction)."""
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                    _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


class _View(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("depth", ctypes.c_void_p),
                ("mask", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("tau_m", "gamma", "alpha1", "tau_cons", "eps", "z_near", "logit_tau")]


class _TView(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("d_min", ctypes.c_void_p),
                ("d_med", ctypes.c_void_p), ("d_max", ctypes.c_void_p),
                ("n_samp", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("d_cam", ctypes.c_double)]


class _TParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("beta", "gamma_st", "tau_thin", "rho_cover", "rho_occ", "n_abs", "dist_gate",
                 "behind_margin", "k_dg", "rho_thin")]


class _NParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("gamma", "beta", "b_max", "lambda_range", "rho_thin", "rho_cover", "tau_thin",
                 "m_thin", "k_dg")]


def _configure(lib):
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    L = ctypes.c_int64
    lib.oracle_fuse.argtypes = [I, P, D, I, L, P, I, P, I, P, P, P, P, P, P, P, P, P]
    lib.oracle_fuse.restype = None
    lib.oracle_fuse_grad.argtypes = [I, P, D, I, L, P, I, P, I, P, P, P, P]
    lib.oracle_fuse_grad.restype = None
    lib.oracle_label.argtypes = [I, P, D, I, P, L, P, P, P]
    lib.oracle_label.restype = None
    lib.oracle_project.argtypes = [I, P, D, I, L, P, P, D, P, P]
    lib.oracle_project.restype = None
    lib.oracle_set_threads.argtypes = [I]
    lib.oracle_set_threads.restype = I
    lib.oracle_fuse_tuple.argtypes = [I, P, D, I, L, P, P, I, P, I, P, P, P, P, P, P, P, P, P, P]
    lib.oracle_fuse_tuple.restype = None
    lib.oracle_fuse_nerf.argtypes = [I, P, D, I, L, P, P, I, P, I, P, P, P, P, P, P, P, P, P, P]
    lib.oracle_fuse_nerf.restype = None
    return lib


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = _configure(ctypes.CDLL(build()))
    return _lib_handle


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Params:
    """Fusion constants.  Defaults: tau_m = 0.5, the thick-path mask gate
    (Algorithms A.2 / B.5); gamma = 1.0 and tau_cons = 0.5 (Table
    gs-hyperparams); alpha1 = 0.5, eps = 1e-12 and z_near = 1e-6 are readings
    (the paper gives no value for alpha1 or eps)."""

    tau_m: float = 0.5
    gamma: float = 1.0
    alpha1: float = 0.5
    tau_cons: float = 0.5
    eps: float = 1e-12
    z_near: float = 1e-6

    def f32(self) -> "Params":
        """The same constants rounded to float32 (what an FP32 caller passes)."""
        return Params(*[float(np.float32(v)) for v in
                        (self.tau_m, self.gamma, self.alpha1, self.tau_cons, self.eps,
                         self.z_near)])

    def logit_tau(self) -> float:
        """Logit-mask gate threshold: float32 rounding of log(tau_m / (1 - tau_m))."""
        t = self.tau_m
        if t <= 0.0:
            return -math.inf
        if t >= 1.0:
            return math.inf
        return float(np.float32(math.log(t / (1.0 - t))))

    def _c(self) -> _Params:
        return _Params(self.tau_m, self.gamma, self.alpha1, self.tau_cons, self.eps, self.z_near,
                       self.logit_tau())


@dataclass
class TupleParams:
    """Depth-tuple-mode constants (Table gs-hyperparams: beta 0.05, gamma_st
    1.5, tau_thin 0.6, rho_cover 0.5, rho_occ 0.1, n_abs 25, the 1.5 h_v
    distance gate and the 2 h_v behind margin).  k_dg (the depth-gradient
    factor's decay, App. D, "k > 0" without a value) and rho_thin (the thin
    path's density floor, no 2DGS value) are readings: k_dg = 0 (pi_dg = 1)
    and rho_thin = 1 (every voxel of a binary prior is eligible)."""

    beta: float = 0.05
    gamma_st: float = 1.5
    tau_thin: float = 0.6
    rho_cover: float = 0.5
    rho_occ: float = 0.1
    n_abs: float = 25.0
    dist_gate: float = 1.5
    behind_margin: float = 2.0
    k_dg: float = 0.0
    rho_thin: float = 1.0

    def f32(self) -> "TupleParams":
        return TupleParams(*[float(np.float32(getattr(self, f))) for f in
                             self.__dataclass_fields__])

    def _c(self) -> _TParams:
        return _TParams(*[float(getattr(self, f)) for f in self.__dataclass_fields__])


@dataclass
class NerfParams:
    """NeRF-variant constants (Table kernel_hyperparams, LLFF column: gamma
    4.0, beta 0.2, b_max 10, lambda_range 0.05, rho_thin_thresh 50,
    rho_cover 0.20, tau_thin 0.6; the thin path's eligibility m > 0.1 from
    its three-criterion rule).  ``mip360()`` gives the Mip-NeRF 360 column.
    k_dg (the depth-gradient decay, App. D gives no value) is a reading:
    0, so pi_dg = 1."""

    gamma: float = 4.0
    beta: float = 0.2
    b_max: float = 10.0
    lambda_range: float = 0.05
    rho_thin: float = 50.0
    rho_cover: float = 0.2
    tau_thin: float = 0.6
    m_thin: float = 0.1
    k_dg: float = 0.0

    @staticmethod
    def mip360() -> "NerfParams":
        return NerfParams(gamma=0.5, b_max=1.0, lambda_range=5.0, rho_thin=30.0, rho_cover=0.3)

    def f32(self) -> "NerfParams":
        return NerfParams(*[float(np.float32(getattr(self, f))) for f in
                            self.__dataclass_fields__])

    def _c(self) -> _NParams:
        return _NParams(*[float(getattr(self, f)) for f in self.__dataclass_fields__])


def _tviews(cams, tup, masks):
    arr = (_TView * len(cams))()
    keep = []
    for i, cam in enumerate(cams):
        ras = [np.ascontiguousarray(tup[k][i], np.float32) for k in ("d_min", "d_med", "d_max")]
        n = np.ascontiguousarray(tup["n_samp"][i], np.uint16)
        m = np.ascontiguousarray(masks[i])
        keep += ras + [n, m]
        v = arr[i]
        R = np.asarray(cam.R, np.float32).reshape(-1)
        for k in range(9):
            v.R[k] = float(R[k])
        for k in range(3):
            v.t[k] = float(np.asarray(cam.t, np.float32)[k])
        v.fx, v.fy, v.cx, v.cy = cam.fx, cam.fy, cam.cx, cam.cy
        v.W, v.H = cam.W, cam.H
        for r in ras + [n, m]:
            assert r.shape == (cam.H, cam.W)
        v.d_min, v.d_med, v.d_max = (r.ctypes.data for r in ras)
        v.n_samp = n.ctypes.data
        v.mask = m.ctypes.data
        v.d_cam = float(np.float32(tup["d_cam"][i])) if "d_cam" in tup else 0.0
    return arr, keep


def _views(cams, depths, masks):
    arr = (_View * len(cams))()
    keep = []
    for i, (cam, d, m) in enumerate(zip(cams, depths, masks)):
        d = np.ascontiguousarray(d, np.float32)
        m = np.ascontiguousarray(m)
        keep += [d, m]
        v = arr[i]
        R = np.asarray(cam.R, np.float32).reshape(-1)
        for k in range(9):
            v.R[k] = float(R[k])
        for k in range(3):
            v.t[k] = float(np.asarray(cam.t, np.float32)[k])
        v.fx, v.fy, v.cx, v.cy = cam.fx, cam.fy, cam.cx, cam.cy
        v.W, v.H = cam.W, cam.H
        assert d.shape == (cam.H, cam.W) and m.shape == (cam.H, cam.W)
        v.depth = d.ctypes.data
        v.mask = m.ctypes.data
    return arr, keep


def _grid_args(grid):
    origin = np.ascontiguousarray(np.asarray(grid.origin, np.float32).astype(np.float64))
    return int(grid.g), origin, float(np.float32(grid.h)), int(bool(grid.contracted))


class OracleApi:
    """The oracle's entry points bound to one compiled copy of ``oracle.c``."""

    def __init__(self, lib):
        self.lib = lib

    def fuse(self, grid, lin, cams, depths, masks, mask_type, params: Params | None = None,
             want_pix: bool = False) -> dict:
        """Fuse views into the voxels with ascending-or-not linear indices ``lin``.

        Returns float64 W, Z, P; uint8 seg; uint32 bits, vmask, flags; and, with
        ``want_pix``, int32 pix (n_vox x n_views)."""
        params = params or Params()
        lin = np.ascontiguousarray(lin, np.int64)
        n = len(lin)
        g, origin, h, contracted = _grid_args(grid)
        views, keep = _views(cams, depths, masks)
        out = dict(W=np.empty(n), Z=np.empty(n), P=np.empty(n), seg=np.empty(n, np.uint8),
                   bits=np.empty(n, np.uint32), vmask=np.empty(n, np.uint32),
                   flags=np.empty(n, np.uint32))
        pix = np.empty((n, len(cams)), np.int32) if want_pix else None
        pr = params._c()
        self.lib.oracle_fuse(g, _p(origin), h, contracted, n, _p(lin), len(cams), views,
                             int(mask_type), ctypes.byref(pr), _p(out["W"]), _p(out["Z"]),
                             _p(out["P"]), _p(out["seg"]), _p(out["bits"]), _p(out["vmask"]),
                             _p(out["flags"]), _p(pix))
        del keep
        if want_pix:
            out["pix"] = pix
        return out

    def fuse_tuple(self, grid, lin, cams, tup, masks, mask_type, params: Params | None = None,
                   tparams: TupleParams | None = None, rho=None) -> dict:
        """Depth-tuple-mode fusion (thick path with the tuple gates + thin path)
        of views with rasters ``tup`` (dict of per-view lists d_min, d_med,
        d_max, n_samp and per-view d_cam) into the voxels ``lin``.  Returns
        float64 W, Z, P; uint8 seg; uint32 bits, flags; uint8 kind (n_vox x
        n_views: 0 no vote, 1 thick, 2 thin); float64 thin (thin score t)."""
        params = params or Params()
        tparams = tparams or TupleParams()
        lin = np.ascontiguousarray(lin, np.int64)
        n = len(lin)
        g, origin, h, contracted = _grid_args(grid)
        views, keep = _tviews(cams, tup, masks)
        rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
        out = dict(W=np.empty(n), Z=np.empty(n), P=np.empty(n), seg=np.empty(n, np.uint8),
                   bits=np.empty(n, np.uint32), flags=np.empty(n, np.uint32),
                   kind=np.empty((n, len(cams)), np.uint8), thin=np.empty((n, len(cams))))
        pr = params._c()
        tp = tparams._c()
        self.lib.oracle_fuse_tuple(g, _p(origin), h, contracted, n, _p(lin), _p(rho), len(cams),
                                   views, int(mask_type), ctypes.byref(pr), ctypes.byref(tp),
                                   _p(out["W"]), _p(out["Z"]), _p(out["P"]), _p(out["seg"]),
                                   _p(out["bits"]), _p(out["flags"]), _p(out["kind"]),
                                   _p(out["thin"]))
        del keep
        return out

    def fuse_nerf(self, grid, lin, cams, tup, masks, mask_type, params: Params | None = None,
                  nparams: NerfParams | None = None, rho=None) -> dict:
        """NeRF-variant fusion (thick path: ray-voxel alignment, distance and
        depth tolerances, Gaussian band weight; thin path: footprint support
        count and peak mask) of views with rasters ``tup`` (dict of per-view
        lists d_min, d_exp, d_max, n_samp: planar depths and the sample
        count) into the voxels ``lin`` with densities ``rho`` (None: 1 each).
        Returns float64 W, Z, P; uint8 seg; uint32 bits, flags; uint8 kind
        (n_vox x n_views: 0 no vote, 1 thick, 2 thin); float64 thin (t)."""
        params = params or Params()
        nparams = nparams or NerfParams()
        lin = np.ascontiguousarray(lin, np.int64)
        n = len(lin)
        g, origin, h, contracted = _grid_args(grid)
        views, keep = _tviews(cams, {"d_min": tup["d_min"], "d_med": tup["d_exp"],
                                     "d_max": tup["d_max"], "n_samp": tup["n_samp"]}, masks)
        rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
        out = dict(W=np.empty(n), Z=np.empty(n), P=np.empty(n), seg=np.empty(n, np.uint8),
                   bits=np.empty(n, np.uint32), flags=np.empty(n, np.uint32),
                   kind=np.empty((n, len(cams)), np.uint8), thin=np.empty((n, len(cams))))
        pr = params._c()
        npr = nparams._c()
        self.lib.oracle_fuse_nerf(g, _p(origin), h, contracted, n, _p(lin), _p(rho), len(cams),
                                  views, int(mask_type), ctypes.byref(pr), ctypes.byref(npr),
                                  _p(out["W"]), _p(out["Z"]), _p(out["P"]), _p(out["seg"]),
                                  _p(out["bits"]), _p(out["flags"]), _p(out["kind"]),
                                  _p(out["thin"]))
        del keep
        return out

    def fuse_grad(self, grid, lin, cams, depths, masks, mask_type, gP, params: Params | None = None):
        """Adjoint of ``fuse``: per-view float64 rasters (gM, gD) for a cotangent gP on P."""
        params = params or Params()
        lin = np.ascontiguousarray(lin, np.int64)
        g, origin, h, contracted = _grid_args(grid)
        views, keep = _views(cams, depths, masks)
        gP = np.ascontiguousarray(gP, np.float64)
        gM = [np.zeros((c.H, c.W)) for c in cams]
        gD = [np.zeros((c.H, c.W)) for c in cams]
        pM = (ctypes.c_void_p * len(cams))(*[a.ctypes.data for a in gM])
        pD = (ctypes.c_void_p * len(cams))(*[a.ctypes.data for a in gD])
        pr = params._c()
        self.lib.oracle_fuse_grad(g, _p(origin), h, contracted, len(lin), _p(lin), len(cams), views,
                                int(mask_type), ctypes.byref(pr), _p(gP), pM, pD)
        del keep
        return gM, gD

    def label(self, grid, seg_dense: np.ndarray, xyz: np.ndarray):
        """Pass 1 labels (uint8) and near-boundary flags (uint32) of points ``xyz``."""
        g, origin, h, contracted = _grid_args(grid)
        seg_dense = np.ascontiguousarray(seg_dense, np.uint8)
        assert seg_dense.size == g ** 3
        xyz = np.ascontiguousarray(xyz, np.float32)
        n = len(xyz)
        labels = np.empty(n, np.uint8)
        flags = np.empty(n, np.uint32)
        self.lib.oracle_label(g, _p(origin), h, contracted, _p(seg_dense), n, _p(xyz), _p(labels),
                            _p(flags))
        return labels, flags

    def project(self, grid, lin, cam, z_near: float = 1e-6):
        """Pixel index (iy * W + ix, -1 = skipped) of every voxel in one view, and flags."""
        lin = np.ascontiguousarray(lin, np.int64)
        g, origin, h, contracted = _grid_args(grid)
        dummy_d = np.zeros((cam.H, cam.W), np.float32)
        views, keep = _views([cam], [dummy_d], [dummy_d])
        pix = np.empty(len(lin), np.int32)
        flags = np.empty(len(lin), np.uint32)
        self.lib.oracle_project(g, _p(origin), h, contracted, len(lin), _p(lin), views, float(z_near),
                              _p(pix), _p(flags))
        del keep
        return pix, flags

    def set_threads(self, n: int = 0) -> int:
        """Set the OpenMP thread count (n <= 0 keeps it); returns the count in use."""
        return int(self.lib.oracle_set_threads(int(n)))


_default = None


def _api() -> OracleApi:
    global _default
    if _default is None:
        _default = OracleApi(_lib())
    return _default


def variant(so_path: str) -> OracleApi:
    """Entry points of another compiled copy of the oracle (used by the tests
    that plant a mistake in the oracle and check that a pin catches it)."""
    return OracleApi(_configure(ctypes.CDLL(so_path)))


def fuse(*a, **k):
    return _api().fuse(*a, **k)


def fuse_grad(*a, **k):
    return _api().fuse_grad(*a, **k)


def fuse_tuple(*a, **k):
    return _api().fuse_tuple(*a, **k)


def fuse_nerf(*a, **k):
    return _api().fuse_nerf(*a, **k)


def label(*a, **k):
    return _api().label(*a, **k)


def project(*a, **k):
    return _api().project(*a, **k)


def set_threads(n: int = 0) -> int:
    return _api().set_threads(n)


def dense_seg(grid, lin, seg) -> np.ndarray:
    """Scatter per-voxel seg values into a dense g^3 uint8 volume (0 elsewhere)."""
    out = np.zeros(int(grid.g) ** 3, np.uint8)
    out[np.asarray(lin, np.int64)] = seg
    return out


def bce_loss_grad(P: np.ndarray, y: np.ndarray, clamp: float = 1e-6):
    """Voxel-space BCE, L = sum -[y log Pc + (1 - y) log(1 - Pc)], Pc = clamp(P,
    clamp, 1 - clamp); returns (L, dL/dP) with zero gradient where the clamp
    is active."""
    P = np.asarray(P, np.float64)
    y = np.asarray(y, np.float64)
    Pc = np.clip(P, clamp, 1.0 - clamp)
    L = float(-(y * np.log(Pc) + (1.0 - y) * np.log(1.0 - Pc)).sum())
    g = -(y / Pc - (1.0 - y) / (1.0 - Pc))
    g = np.where((P > clamp) & (P < 1.0 - clamp), g, 0.0)
    return L, g
