"""Occupancy construction from 2DGS surfels: the scene frame (Eqs. scene-norm
and voxel-size) and the opacity scatter-add with the tau_TF floor (Sec. 3.5
"Occupancy by Morton-scattered opacity"), binding
``divas_scene_frame_from_gaussians`` and ``divas_occupancy_from_gaussians``."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib as L
from .fusion import _ptr, _stream


@dataclass
class OccupancyParams:
    alpha_v: float = 3.0
    beta_v: float = 1.0
    pad: float = 1.05
    g0: int = 256
    g_max: int = 512
    tau_tf: float = 0.5

    def c(self) -> L.DivasOccupancyParams:
        return L.DivasOccupancyParams(self.alpha_v, self.beta_v, self.pad, self.g0, self.g_max,
                                      self.tau_tf, 0)


@dataclass
class FrameGrid:
    """The fusion's plain grid of a frame (origin c - b, edge h, side g)."""
    g: int
    origin: tuple
    h: float
    contracted: bool = False


@dataclass
class SceneFrame:
    c: tuple
    r_fg: float
    b: float
    s_bar: float
    h: float
    origin: tuple
    g: int

    def grid(self) -> FrameGrid:
        return FrameGrid(self.g, tuple(float(x) for x in self.origin), float(self.h))

    def c_struct(self) -> L.DivasSceneFrame:
        f = L.DivasSceneFrame()
        for k in range(3):
            f.c[k], f.origin[k] = self.c[k], self.origin[k]
        f.r_fg, f.b, f.s_bar, f.h, f.g = self.r_fg, self.b, self.s_bar, self.h, self.g
        return f


def _check_pts(mu: torch.Tensor, cols: int, name: str):
    if mu.dtype != torch.float32 or mu.dim() != 2 or mu.shape[1] != cols or not mu.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (m, {cols}) float32 tensor")


def scene_frame(mu: torch.Tensor, scales: torch.Tensor, params: OccupancyParams | None = None,
                stream=None) -> SceneFrame:
    """The frame of m surfels (centres (m, 3), scales (m, 2), FP32 CUDA);
    synchronises."""
    _check_pts(mu, 3, "mu")
    _check_pts(scales, 2, "scales")
    if scales.shape[0] != mu.shape[0]:
        raise ValueError("one scale pair per centre")
    p = (params or OccupancyParams()).c()
    f = L.DivasSceneFrame()
    L.check(L.load().divas_scene_frame_from_gaussians(_ptr(mu), _ptr(scales), mu.shape[0],
                                                      ctypes.byref(p), ctypes.byref(f),
                                                      _stream(stream)))
    return SceneFrame(tuple(f.c), f.r_fg, f.b, f.s_bar, f.h, tuple(f.origin), f.g)


def occupancy(mu: torch.Tensor, alpha: torch.Tensor, frame: SceneFrame, tau_tf: float = 0.5,
              density: torch.Tensor | None = None, occ: torch.Tensor | None = None, stream=None):
    """The dense occupancy prior (g^3 uint8, x fastest) and the density (g^3
    float32) of the surfels in ``frame``."""
    _check_pts(mu, 3, "mu")
    if alpha.dtype != torch.float32 or alpha.shape != (mu.shape[0],) or not alpha.is_contiguous():
        raise ValueError("alpha must be a contiguous (m,) float32 tensor")
    n = frame.g ** 3
    if density is None:
        density = torch.empty(n, dtype=torch.float32, device=mu.device)
    if occ is None:
        occ = torch.empty(n, dtype=torch.uint8, device=mu.device)
    if density.numel() != n or occ.numel() != n:
        raise ValueError("density and occ hold g^3 cells")
    f = frame.c_struct()
    L.check(L.load().divas_occupancy_from_gaussians(_ptr(mu), _ptr(alpha), mu.shape[0],
                                                    ctypes.byref(f), tau_tf, _ptr(density),
                                                    _ptr(occ), _stream(stream)))
    return occ, density
