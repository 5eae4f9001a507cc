"""Python face of the fusion library: one ``VoxelFusion`` per occupied set.

Argument marshalling only -- every step runs in the CUDA kernels of
``libdivas_fuse.so`` (the C ABI in ``include/divas_fuse.h``).  PyTorch
supplies device memory and the current stream.

Notation follows the paper: W and Z are the weighted-vote and weight
accumulators of Eq. vmask, P = W / Z the fused probability of Eq.
compact-fusion, seg the consensus set {P >= tau_cons}, vmask the per-voxel
view-coverage bitmask.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib as L


@dataclass
class FusionParams:
    """Thick-path constants (defaults: tau_mask 0.5 = the thick-path entry gate of
    Algorithms A.2 / B.5; gamma 1.0 and tau_cons 0.5 from Table gs-hyperparams;
    alpha1 0.5 and eps 1e-12, for which the paper gives no value)."""

    tau_mask: float = 0.5
    gamma: float = 1.0
    alpha1: float = 0.5
    tau_cons: float = 0.5
    eps: float = 1e-12
    z_near: float = 1e-6
    # sparse priors (g a multiple of 8): keep the active list in brick-major
    # order (8^3 bricks), so that the fusion can skip whole warps' views that no
    # voxel of the warp can vote in; per-voxel results are unchanged
    brick_order: bool = False

    def c(self) -> L.DivasParams:
        return L.DivasParams(self.tau_mask, self.gamma, self.alpha1, self.tau_cons, self.eps,
                             self.z_near, L.ORDER_BRICKS if self.brick_order else 0)


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def camera_c(cam) -> L.DivasCamera:
    """Any object with R (3x3), t (3), fx, fy, cx, cy, W, H -> divas_camera."""
    c = L.DivasCamera()
    c.W, c.H = int(cam.W), int(cam.H)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = [float(v) for row in _rows(cam.R) for v in row]
    for k in range(9):
        c.R[k] = R[k]
    t = [float(v) for v in _flat(cam.t)]
    for k in range(3):
        c.t[k] = t[k]
    return c


def _rows(R):
    try:
        return [list(r) for r in R]
    except TypeError:
        return [list(R[3 * i:3 * i + 3]) for i in range(3)]


def _flat(x):
    try:
        return [float(v) for v in x.reshape(-1)]
    except AttributeError:
        return [float(v) for v in x]


def mask_type_of(mask: torch.Tensor, logits: bool = False) -> int:
    if mask.dtype == torch.float16:
        return L.MASK_F16
    if mask.dtype == torch.float32:
        return L.MASK_LOGIT_F32 if logits else L.MASK_F32
    raise ValueError(f"unsupported mask dtype {mask.dtype}")


def view_c(cam, depth: torch.Tensor, mask: torch.Tensor, mask_type: int | None = None,
           logits: bool = False) -> L.DivasView:
    if depth.dtype != torch.float32:
        raise ValueError("depth must be float32")
    if tuple(depth.shape[-2:]) != (int(cam.H), int(cam.W)) or mask.shape != depth.shape:
        raise ValueError("depth and mask must be H x W")
    v = L.DivasView()
    v.cam = camera_c(cam)
    v.depth = _ptr(depth)
    v.mask = _ptr(mask)
    v.mask_type = mask_type if mask_type is not None else mask_type_of(mask, logits)
    return v


@dataclass
class TupleParams:
    """Depth-tuple-mode constants (``divas_tuple_params``; defaults of Table
    gs-hyperparams, k_dg = 0 and rho_thin = 1)."""
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

    def c(self) -> L.DivasTupleParams:
        return L.DivasTupleParams(*[float(getattr(self, f)) for f in self.__dataclass_fields__])


@dataclass
class NerfParams:
    """NeRF-variant constants (``divas_nerf_params``; Table
    kernel_hyperparams, LLFF column by default, ``mip360()`` for the other;
    m_thin = 0.1, k_dg = 0)."""
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

    def c(self) -> L.DivasNerfParams:
        return L.DivasNerfParams(*[float(getattr(self, f)) for f in self.__dataclass_fields__], 0)


def density_floor(density: torch.Tensor, rho_thresh: float, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """The occupancy prior of a NeRF density grid (``divas_density_floor``):
    uint8 ``density >= rho_thresh`` of a contiguous float32 tensor (16-byte
    aligned; ``out`` 4-byte aligned)."""
    if density.dtype != torch.float32 or not density.is_contiguous() or not density.is_cuda:
        raise ValueError("density must be a contiguous float32 CUDA tensor")
    if out is None:
        out = torch.empty(density.shape, dtype=torch.uint8, device=density.device)
    elif out.dtype != torch.uint8 or out.numel() != density.numel() or not out.is_contiguous():
        raise ValueError("out must be a contiguous uint8 tensor of the density's size")
    lib = L.load()
    st = lib.divas_density_floor(_ptr(density), density.numel(), float(rho_thresh), _ptr(out),
                                 _stream(stream))
    if st != 0:
        raise L.DivasError(f"divas_density_floor failed ({st}): check alignment and arguments")
    return out


def tuple_views_c(cams, d_min, d_med, d_max, n_samp, masks, d_cams, mask_type: int):
    """Marshal tuple views (device tensors: float32 depths, uint16-compatible
    n_samp as torch.int16 / uint16 storage, masks as for ``view_c``)."""
    arr = (L.DivasTupleView * len(cams))()
    for k, cam in enumerate(cams):
        for nm, ten in (("d_min", d_min[k]), ("d_med", d_med[k]), ("d_max", d_max[k])):
            if ten.dtype != torch.float32 or tuple(ten.shape) != (int(cam.H), int(cam.W)):
                raise ValueError(f"{nm} must be float32 H x W")
        if n_samp[k].element_size() != 2 or tuple(n_samp[k].shape) != (int(cam.H), int(cam.W)):
            raise ValueError("n_samp must be 16-bit H x W")
        v = arr[k]
        v.cam = camera_c(cam)
        v.d_min, v.d_med, v.d_max = _ptr(d_min[k]), _ptr(d_med[k]), _ptr(d_max[k])
        v.n_samp = _ptr(n_samp[k])
        v.mask = _ptr(masks[k])
        v.mask_type = int(mask_type)
        v.d_cam = float(d_cams[k])
    return arr


class PreparedViews:
    """Views marshalled once into ``divas_view`` structs (chunks of up to 32), so
    that repeated launches skip the per-call Python marshalling.  Keeps the
    rasters alive."""

    def __init__(self, cams, depths, masks, mask_type: int | None = None, logits=False):
        self.n = len(cams)
        self._keep = (list(depths), list(masks))
        self.chunks = []
        for s0 in range(0, self.n, L.MAX_VIEWS_PER_CALL):
            s1 = min(self.n, s0 + L.MAX_VIEWS_PER_CALL)
            arr = (L.DivasView * (s1 - s0))()
            for k in range(s0, s1):
                arr[k - s0] = view_c(cams[k], depths[k], masks[k], mask_type, logits)
            self.chunks.append((arr, s1 - s0))


class VoxelFusion:
    """Device-resident fusion state for one occupied set (dense prior or sparse set).

    ``grid``: object with g, origin (3), h, contracted.  Exactly one of
    ``occ`` (uint8 g^3, x fastest) and ``coords`` ((n, 3) int32) is given,
    both CUDA tensors."""

    def __init__(self, grid, occ: torch.Tensor | None = None,
                 coords: torch.Tensor | None = None, params: FusionParams | None = None,
                 stream=None):
        self.lib = L.load()
        self.params = params or FusionParams()
        g = L.DivasGrid()
        g.kind = 0 if occ is not None else 1
        g.g = int(grid.g)
        for k in range(3):
            g.origin[k] = float(grid.origin[k])
        g.h = float(grid.h)
        g.contracted = 1 if getattr(grid, "contracted", False) else 0
        self.grid_c = g
        self.g = int(grid.g)
        self.dense = occ is not None
        if occ is not None:
            occ = occ.contiguous()
            if occ.dtype != torch.uint8 or occ.numel() != self.g ** 3:
                raise ValueError("occ must be uint8 with g^3 elements")
        if coords is not None:
            coords = coords.contiguous()
            if coords.dtype != torch.int32 or coords.dim() != 2 or coords.shape[1] != 3:
                raise ValueError("coords must be (n, 3) int32")
        self._h = ctypes.c_void_p()
        n = 0 if coords is None else coords.shape[0]
        st = self.lib.divas_fuse_init(ctypes.byref(self._h), ctypes.byref(g), _ptr(occ),
                                      _ptr(coords), n, ctypes.byref(self.params.c()),
                                      _stream(stream))
        L.check(st, None)

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.divas_fuse_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        L.check(st, self._h)

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def n_active(self) -> int:
        return int(self.lib.divas_fuse_n_active(self._h))

    @property
    def n_views(self) -> int:
        return int(self.lib.divas_fuse_n_views(self._h))

    @property
    def n_cells(self) -> int:
        return self.g ** 3

    # -- the hot path ------------------------------------------------------
    def set_occupancy(self, occ=None, coords=None, stream=None):
        n = 0 if coords is None else coords.shape[0]
        self._check(self.lib.divas_fuse_set_occupancy(self._h, _ptr(occ), _ptr(coords), n,
                                                      _stream(stream)))

    def add_view(self, cam, depth, mask, mask_type: int | None = None, logits=False,
                 stream=None):
        mt = mask_type if mask_type is not None else mask_type_of(mask, logits)
        c = camera_c(cam)
        self._check(self.lib.divas_fuse_add_view(self._h, ctypes.byref(c), _ptr(depth),
                                                 _ptr(mask), mt, _stream(stream)))

    def add_views(self, cams, depths=None, masks=None, mask_type: int | None = None,
                  logits=False, stream=None):
        """Fold views in index order, up to 32 per launch.  ``cams`` may be a
        ``PreparedViews`` (then depths / masks are not given)."""
        pv = cams if isinstance(cams, PreparedViews) else PreparedViews(
            cams, depths, masks, mask_type, logits)
        s = _stream(stream)
        for arr, n in pv.chunks:
            self._check(self.lib.divas_fuse_add_views(self._h, arr, n, s))

    def add_views_tuple(self, cams, d_min, d_med, d_max, n_samp, masks, d_cams, mask_type: int,
                        tparams: "TupleParams | None" = None, stage_events=None, stream=None):
        """Fold depth-tuple views (``divas_fuse_add_views_tuple``), up to 32.
        ``stage_events``: optional four ``torch.cuda.Event`` (timing enabled)
        marking before the per-view maps / after them / after the candidate
        scan / after the heavy pass (``divas_fuse_add_views_tuple_profiled``)."""
        if len(cams) > L.MAX_VIEWS_PER_CALL:
            raise ValueError("add_views_tuple() takes up to 32 views")
        arr = tuple_views_c(cams, d_min, d_med, d_max, n_samp, masks, d_cams, mask_type)
        tp = (tparams or TupleParams()).c()
        if stage_events is None:
            self._check(self.lib.divas_fuse_add_views_tuple(self._h, arr, len(cams),
                                                            ctypes.byref(tp), _stream(stream)))
            return
        if len(stage_events) != 4:
            raise ValueError("stage_events takes four events")
        evs = (ctypes.c_void_p * 4)(*[(e.cuda_event if e is not None else None)
                                      for e in stage_events])
        self._check(self.lib.divas_fuse_add_views_tuple_profiled(
            self._h, arr, len(cams), ctypes.byref(tp), evs, _stream(stream)))

    def add_views_nerf(self, cams, d_min, d_exp, d_max, n_samp, masks, mask_type: int,
                       nparams: "NerfParams | None" = None, density: torch.Tensor | None = None,
                       stage_events=None, stream=None):
        """Fold NeRF depth-tuple views (``divas_fuse_add_views_nerf``), up to
        32; ``density`` None (density 1 everywhere) or the g^3 float32 grid.
        ``stage_events``: optional four ``torch.cuda.Event`` (before the
        mask-tile maps / after them / after the scan / after the heavy pass)."""
        if len(cams) > L.MAX_VIEWS_PER_CALL:
            raise ValueError("add_views_nerf() takes up to 32 views")
        if density is not None and (density.dtype != torch.float32 or not density.is_contiguous()
                                    or density.numel() != self.n_cells):
            raise ValueError("density must be a contiguous float32 tensor of g^3 cells")
        arr = tuple_views_c(cams, d_min, d_exp, d_max, n_samp, masks, [0.0] * len(cams), mask_type)
        npr = (nparams or NerfParams()).c()
        if stage_events is None:
            self._check(self.lib.divas_fuse_add_views_nerf(self._h, arr, len(cams),
                                                           ctypes.byref(npr), _ptr(density),
                                                           _stream(stream)))
            return
        if len(stage_events) != 4:
            raise ValueError("stage_events takes four events")
        evs = (ctypes.c_void_p * 4)(*[(e.cuda_event if e is not None else None)
                                      for e in stage_events])
        self._check(self.lib.divas_fuse_add_views_nerf_profiled(
            self._h, arr, len(cams), ctypes.byref(npr), _ptr(density), evs, _stream(stream)))

    def depth_weight(self, depths, masks, mask_type: int, mode: str = "band", prompts=None,
                     out=None, stats: bool = False, stream=None):
        """Depth-weighted masks (``divas_depth_weight``) of up to 32 views:
        ``mode`` "nerf" (Eq. nerf-depthweight: min-max-normalised depth) or
        "band" (Eqs. depthband, gs-bandpass: the depth band of ``prompts``,
        per view a list of (x, y) pixels, and the view centre, with the
        98th-percentile far depth).  Returns the FP32 weighted masks (``out``
        or new tensors) and, with ``stats``, an (n, 4) float32 tensor of the
        per-view constants."""
        n = len(depths)
        if n < 1 or n > L.MAX_VIEWS_PER_CALL or len(masks) != n:
            raise ValueError("depth_weight() takes 1..32 views with one mask each")
        m = {"nerf": L.WEIGHT_NERF_MINMAX, "band": L.WEIGHT_GS_BAND}[mode]
        prompts = prompts if prompts is not None else [[] for _ in range(n)]
        if out is None:
            out = [torch.empty(d.shape, dtype=torch.float32, device=d.device) for d in depths]
        arr = (L.DivasWeightView * n)()
        for k in range(n):
            d, mk, o = depths[k], masks[k], out[k]
            if d.dtype != torch.float32 or d.dim() != 2 or not d.is_contiguous():
                raise ValueError("depth rasters must be contiguous (H, W) float32")
            if o.shape != d.shape or o.dtype != torch.float32 or not o.is_contiguous():
                raise ValueError("out rasters must be contiguous (H, W) float32")
            if mk.shape != d.shape or not mk.is_contiguous():
                raise ValueError("masks must be contiguous (H, W)")
            pk = list(prompts[k])
            if len(pk) > L.MAX_PROMPTS:
                raise ValueError("at most 15 prompts per view")
            arr[k].depth, arr[k].mask, arr[k].out = d.data_ptr(), mk.data_ptr(), o.data_ptr()
            arr[k].mask_type, arr[k].H, arr[k].W = mask_type, d.shape[0], d.shape[1]
            arr[k].n_prompts = len(pk)
            for q, (x, y) in enumerate(pk):
                arr[k].prompt_xy[2 * q], arr[k].prompt_xy[2 * q + 1] = int(x), int(y)
        st = torch.empty((n, 4), dtype=torch.float32, device=depths[0].device) if stats else None
        self._check(self.lib.divas_depth_weight(self._h, arr, n, m, _ptr(st), _stream(stream)))
        return (out, st) if stats else out

    def add_views_weighted(self, cams, depths=None, masks=None, mask_type: int | None = None,
                           mode: str = "band", prompts=None, logits=False, stats: bool = False,
                           stream=None):
        """Fold views with the depth weight of ``depth_weight`` applied where
        each vote reads the mask (``divas_fuse_add_views_weighted``: no
        weighted raster is written).  ``cams``: cameras with ``depths`` and
        ``masks``, or a PreparedViews of at most 32 views; ``mode`` "nerf" or
        "band"; ``prompts``: per view a list of (x, y) pixels (band).  With
        ``stats``, returns the (n, 4) float32 tensor of per-view constants."""
        if isinstance(cams, PreparedViews):
            if len(cams.chunks) != 1:
                raise ValueError("add_views_weighted() takes up to 32 views")
            arr, n = cams.chunks[0]
            dev = cams._keep[0][0].device
        else:
            n = len(cams)
            if n < 1 or n > L.MAX_VIEWS_PER_CALL:
                raise ValueError("add_views_weighted() takes 1..32 views")
            arr = (L.DivasView * n)()
            for k in range(n):
                arr[k] = view_c(cams[k], depths[k], masks[k], mask_type, logits)
            dev = depths[0].device
        m = {"nerf": L.WEIGHT_NERF_MINMAX, "band": L.WEIGHT_GS_BAND}[mode]
        pr = (L.DivasWeightView * n)()
        prompts = prompts if prompts is not None else [[] for _ in range(n)]
        for k in range(n):
            pk = list(prompts[k])
            if len(pk) > L.MAX_PROMPTS:
                raise ValueError("at most 15 prompts per view")
            pr[k].n_prompts = len(pk)
            for q, (x, y) in enumerate(pk):
                pr[k].prompt_xy[2 * q], pr[k].prompt_xy[2 * q + 1] = int(x), int(y)
        st = torch.empty((n, 4), dtype=torch.float32, device=dev) if stats else None
        self._check(self.lib.divas_fuse_add_views_weighted(self._h, arr, pr, n, m, _ptr(st),
                                                           _stream(stream)))
        return st

    def overlay(self, cam, depth: torch.Tensor, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        """The back-projected overlay of a view (``divas_overlay``): uint8 (H,
        W), the seg bit of the cell under each pixel's rendered surface point."""
        if depth.dtype != torch.float32 or depth.dim() != 2 or not depth.is_contiguous():
            raise ValueError("depth must be a contiguous (H, W) float32 tensor")
        if tuple(depth.shape) != (int(cam.H), int(cam.W)):
            raise ValueError(f"depth is {tuple(depth.shape)}, the camera is {cam.H} x {cam.W}")
        if out is None:
            out = torch.empty(depth.shape, dtype=torch.uint8, device=depth.device)
        elif out.dtype != torch.uint8 or out.shape != depth.shape or not out.is_contiguous():
            raise ValueError("out must be a contiguous uint8 tensor shaped like depth")
        c = camera_c(cam)
        self._check(self.lib.divas_overlay(self._h, ctypes.byref(c), _ptr(depth), _ptr(out),
                                           _stream(stream)))
        return out

    def surfel_labels(self, mu: torch.Tensor, scales: torch.Tensor, quats: torch.Tensor, cams,
                      masks, mask_type: int, tau_m: float = 0.5, tau_kappa: float = 0.5,
                      eps_aspect: float = 1e-8, stream=None) -> dict:
        """Voxel-to-surfel mapping, Passes 1-3 (``divas_surfel_labels``) of
        m surfels (centres (m, 3), scales (m, 2), quaternions (m, 4) (w, x, y,
        z), FP32 CUDA) against this context's last finalize; ``cams`` /
        ``masks``: the views folded into it, in order.  Returns uint8 ``f``
        (final) and ``f2`` (after the needle cull) and FP32 ``kappa``."""
        m = mu.shape[0]
        for x, c in ((mu, 3), (scales, 2), (quats, 4)):
            if x.dtype != torch.float32 or x.shape != (m, c) or not x.is_contiguous():
                raise ValueError("mu / scales / quats: contiguous float32 (m, 3) / (m, 2) / (m, 4)")
        n = len(cams)
        if n > L.MAX_VIEWS_PER_CALL or len(masks) != n:
            raise ValueError("up to 32 views, one mask each")
        cam_arr = (L.DivasCamera * max(n, 1))(*[camera_c(c) for c in cams])
        mask_arr = (ctypes.c_void_p * max(n, 1))(*[mk.data_ptr() for mk in masks])
        p = L.DivasSurfelParams(tau_m, tau_kappa, eps_aspect, 0)
        f = torch.empty(m, dtype=torch.uint8, device=mu.device)
        f2 = torch.empty(m, dtype=torch.uint8, device=mu.device)
        kappa = torch.empty(m, dtype=torch.float32, device=mu.device)
        self._check(self.lib.divas_surfel_labels(
            self._h, _ptr(mu), _ptr(scales), _ptr(quats), m, cam_arr, mask_arr, mask_type, n,
            ctypes.byref(p), _ptr(f), _ptr(f2), _ptr(kappa), _stream(stream)))
        return {"f": f, "f2": f2, "kappa": kappa}

    def update(self, views, score: torch.Tensor | None = None,
               seg_bits: torch.Tensor | None = None, keep_zeros: bool = False, stream=None):
        """Incremental update: fold ``views`` (a ``PreparedViews`` or one
        ``DivasView``) onto the stored accumulators and finalize in one fusion
        launch (``divas_fuse_update``).  ``keep_zeros``: ``score`` /
        ``seg_bits`` already hold zeros for every unoccupied voxel (e.g. an
        earlier result of this context for the same occupied set), so only the
        active entries are written."""
        flags = L.KEEP_ZEROS if keep_zeros else 0
        s = _stream(stream)
        if isinstance(views, L.DivasView):
            chunks = [(ctypes.pointer(views), 1)]
        else:
            chunks = views.chunks
        if len(chunks) != 1:
            raise ValueError("update() takes up to 32 views")
        arr, n = chunks[0]
        self._check(self.lib.divas_fuse_update(self._h, arr, n, _ptr(score), _ptr(seg_bits), flags,
                                               s))

    def finalize(self, score: bool | torch.Tensor = True, seg_bits: bool | torch.Tensor = False,
                 vmask: bool | torch.Tensor = False, count: bool = False, stream=None) -> dict:
        """Outputs as CUDA tensors: score (float32, g^3 dense or n_active sparse),
        seg_bits (int32 view of ceil(g^3/32) uint32 words), vmask (int32 view of
        n_active uint32), and n_seg (int, synchronises) when ``count``."""
        dev = torch.device("cuda")
        out = {}

        def _buf(flag, n, dtype):
            if isinstance(flag, torch.Tensor):
                return flag
            if flag:
                return torch.empty(n, dtype=dtype, device=dev)
            return None
        n_score = self.n_cells if self.dense else self.n_active
        out["score"] = _buf(score, n_score, torch.float32)
        out["seg_bits"] = _buf(seg_bits, (self.n_cells + 31) // 32, torch.int32)
        out["vmask"] = _buf(vmask, self.n_active, torch.int32)
        nseg = ctypes.c_int64(0)
        self._check(self.lib.divas_fuse_finalize(
            self._h, _ptr(out["score"]), _ptr(out["seg_bits"]), _ptr(out["vmask"]),
            ctypes.byref(nseg) if count else None, _stream(stream)))
        if count:
            out["n_seg"] = int(nseg.value)
        return {k: v for k, v in out.items() if v is not None}

    def step(self, views: "PreparedViews", occ=None, coords=None, score=None, seg_bits=None,
             xyz=None, labels=None, stage_events=None, stream=None):
        """The whole hot path in one call (occupancy gate, views, finalize,
        labels): four launches for a dense prior in linear order (a sparse
        prior adds the coordinate scatter, view culling two launches on the
        context's helper stream, joined back).  ``stage_events``: optional four
        ``torch.cuda.Event`` (timing enabled, already recorded once) marking
        before compaction / after compaction / after fusion / after labels."""
        if len(views.chunks) != 1:
            raise ValueError("step() takes up to 32 views")
        arr, n = views.chunks[0]
        n_c = 0 if coords is None else coords.shape[0]
        n_p = 0 if xyz is None else xyz.shape[0]
        if stage_events is None:
            self._check(self.lib.divas_fuse_step(self._h, _ptr(occ), _ptr(coords), n_c, arr, n,
                                                 _ptr(score), _ptr(seg_bits), _ptr(xyz), n_p,
                                                 _ptr(labels), _stream(stream)))
            return
        if len(stage_events) != 4:
            raise ValueError("stage_events takes four events")
        evs = (ctypes.c_void_p * 4)(*[(e.cuda_event if e is not None else None)
                                      for e in stage_events])
        self._check(self.lib.divas_fuse_step_profiled(self._h, _ptr(occ), _ptr(coords), n_c, arr,
                                                      n, _ptr(score), _ptr(seg_bits), _ptr(xyz),
                                                      n_p, _ptr(labels), evs, _stream(stream)))

    def label_points(self, xyz: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        """Pass 1 labels (uint8) of (n, 3) float32 points."""
        xyz = xyz.contiguous()
        if xyz.dtype != torch.float32 or xyz.dim() != 2 or xyz.shape[1] != 3:
            raise ValueError("xyz must be (n, 3) float32")
        n = xyz.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, device=xyz.device)
        self._check(self.lib.divas_label_points(self._h, _ptr(xyz), n, _ptr(out),
                                                _stream(stream)))
        return out

    # -- state -------------------------------------------------------------
    def reset(self, stream=None):
        self._check(self.lib.divas_fuse_reset(self._h, _stream(stream)))

    def sync(self, stream=None):
        self._check(self.lib.divas_fuse_sync(self._h, _stream(stream)))

    def active_coords(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.n_active, 3), dtype=torch.int32, device="cuda")
        if out.numel() == 0:
            return out
        self._check(self.lib.divas_fuse_active_coords(self._h, _ptr(out), _stream(stream)))
        return out

    def export_state(self, stream=None) -> dict:
        n = self.n_active
        W = torch.empty(n, dtype=torch.float32, device="cuda")
        Z = torch.empty(n, dtype=torch.float32, device="cuda")
        b = torch.empty(n, dtype=torch.int32, device="cuda")
        if n == 0:
            return {"W": W, "Z": Z, "bits": b, "n_views": self.n_views}
        self._check(self.lib.divas_fuse_export_state(self._h, _ptr(W), _ptr(Z), _ptr(b),
                                                     _stream(stream)))
        return {"W": W, "Z": Z, "bits": b, "n_views": self.n_views}

    def import_state(self, state: dict, stream=None):
        if state["W"].numel() == 0:
            return
        self._check(self.lib.divas_fuse_import_state(
            self._h, _ptr(state["W"]), _ptr(state["Z"]), _ptr(state["bits"]),
            int(state["n_views"]), _stream(stream)))

    # -- adjoint and test hooks ---------------------------------------------
    def backward(self, cams, depths, masks, grad_score: torch.Tensor, grad_mask=None,
                 grad_depth=None, mask_type: int | None = None, logits=False, stream=None):
        """Accumulate dL/dmask and dL/ddepth rasters for the cotangent grad_score."""
        n = len(cams)
        if n > L.MAX_VIEWS_PER_CALL:
            raise ValueError("backward supports up to 32 views per call")
        arr = (L.DivasView * n)()
        for k in range(n):
            arr[k] = view_c(cams[k], depths[k], masks[k], mask_type, logits)
        for name, grads in (("grad_mask", grad_mask), ("grad_depth", grad_depth)):
            for k, t in enumerate(grads or []):
                if t is not None and (t.dtype != torch.float32 or t.shape != depths[k].shape):
                    raise ValueError(f"{name}[{k}] must be a float32 H x W raster")
        gm = (ctypes.c_void_p * n)(*[(_ptr(t).value if t is not None else None)
                                     for t in (grad_mask or [None] * n)])
        gd = (ctypes.c_void_p * n)(*[(_ptr(t).value if t is not None else None)
                                     for t in (grad_depth or [None] * n)])
        self._check(self.lib.divas_fuse_backward(self._h, arr, n, _ptr(grad_score.contiguous()),
                                                 gm, gd, _stream(stream)))

    def debug_project(self, cam, stream=None) -> torch.Tensor:
        out = torch.empty(self.n_active, dtype=torch.int32, device="cuda")
        if out.numel() == 0:
            return out
        c = camera_c(cam)
        self._check(self.lib.divas_debug_project(self._h, ctypes.byref(c), _ptr(out),
                                                 _stream(stream)))
        return out


def seg_bits_to_bool(seg_bits: torch.Tensor, n_cells: int) -> torch.Tensor:
    """Unpack an int32 view of the uint32 seg words into a bool tensor of n_cells."""
    w = seg_bits.to(torch.int64) & 0xFFFFFFFF
    shifts = torch.arange(32, device=w.device, dtype=torch.int64)
    bits = (w[:, None] >> shifts[None, :]) & 1
    return bits.reshape(-1)[:n_cells].to(torch.bool)
