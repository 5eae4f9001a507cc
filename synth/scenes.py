"""Scene recipes, cameras and the ctypes binding of ``synth.c``.

Every array here is input data for the fusion: nothing in this module
projects voxels, gates votes or accumulates weights.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "_synth.so")

MASK_F32 = 0
MASK_F16 = 1
MASK_LOGIT_F32 = 2


def build() -> str:
    """Compile ``synth.c`` into ``_synth.so`` (gcc, OpenMP) if it is stale."""
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.synth_render.argtypes = [I, P, P, P, P, I, P, P, P, P, P, P, D, D, D, D, I, I, P, P]
        lib.synth_render.restype = None
        lib.synth_render_tuple.argtypes = [I, P, P, P, P, I, P, P, P, P, P, P, D, D, D, D, I, I,
                                           P, P, P, P]
        lib.synth_render_tuple.restype = None
        lib.synth_occ_sphere_band.argtypes = [I, P, P, D, I, P, D, P]
        lib.synth_occ_sphere_band.restype = None
        lib.synth_occ_corner_sign.argtypes = [I, P, P, P, I, P, P, I, P, D, P]
        lib.synth_occ_corner_sign.restype = None
        lib.synth_soft_mask.argtypes = [P, I, I, D, I, P, P]
        lib.synth_soft_mask.restype = None
        lib.synth_contracted_distance.argtypes = [I, P, P, P, D, I, D, P]
        lib.synth_contracted_distance.restype = None
        _lib_handle = lib
    return _lib_handle


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# data types
# --------------------------------------------------------------------------
@dataclass
class Camera:
    """Pinhole camera, OpenCV world->camera (x right, y down, z forward).

    ``R`` row-major 3x3 and ``t`` are float32; the intrinsics are float32
    values held as Python floats.  Pixel (i, j) has its centre at
    (i + 1/2, j + 1/2).
    """

    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int

    @property
    def centre(self) -> np.ndarray:
        R = self.R.astype(np.float64)
        return -R.T @ self.t.astype(np.float64)


@dataclass
class Grid:
    """Voxel grid: voxel (i, j, k) centre = origin + (idx + 1/2) h.

    ``contracted``: the grid lives in contracted space [-2, 2]^3.
    """

    g: int
    origin: tuple
    h: float
    contracted: bool = False


@dataclass
class Scene:
    ell_c: np.ndarray      # (n, 3) centres
    ell_axes: np.ndarray   # (n, 3) semi-axes
    ell_rot: np.ndarray    # (n, 3, 3) axes as columns
    ell_id: np.ndarray     # (n,) int32 ids
    pl_n: np.ndarray       # (m, 3) plane normals
    pl_d: np.ndarray       # (m,) offsets: n.x = d
    pl_rad: np.ndarray     # (m,) disc radius (<= 0: unbounded)
    pl_id: np.ndarray      # (m,) int32 ids
    target_ids: np.ndarray  # ids that the mask calls "object"

    @property
    def ell_M(self) -> np.ndarray:
        """M = A^-1 R^T so that the surface is |M (x - c)| = 1."""
        inv_a = 1.0 / self.ell_axes
        return np.ascontiguousarray(
            (inv_a[:, :, None] * np.transpose(self.ell_rot, (0, 2, 1))).reshape(-1, 9))

    @property
    def ell_brad(self) -> np.ndarray:
        return self.ell_axes.max(axis=1).copy()


@dataclass
class Workload:
    name: str
    grid: Grid
    occ: np.ndarray | None        # dense prior: g^3 uint8, x fastest
    coords: np.ndarray | None     # sparse prior: (n, 3) int32 (i, j, k), ascending linear index
    cams: list
    depth: list                   # per view float32 (H, W), planar camera-Z, +inf = miss
    mask: list                    # per view: float32 (F32/LOGIT) or uint16 binary16 bits (F16)
    mask_type: int
    hit: list                     # per view int32 (H, W) primitive id, -1 = miss
    points: np.ndarray            # (n, 3) float32
    scene: Scene
    meta: dict = field(default_factory=dict)
    # depth-tuple mode (per view): d_min / d_med / d_max float32 (H, W) planar,
    # +inf = miss; n_samp uint16 (H, W); d_cam float (camera-target distance)
    tuple: dict | None = None

    @property
    def n_views(self) -> int:
        return len(self.cams)

    @property
    def n_voxels(self) -> int:
        """Voxels the fusion iterates: g^3 for a dense prior, n_occ for a sparse one."""
        if self.occ is not None:
            return int(self.grid.g) ** 3
        return int(self.coords.shape[0])

    def active_linear(self) -> np.ndarray:
        """Ascending linear indices (x fastest) of the occupied voxels."""
        g = self.grid.g
        if self.occ is not None:
            return np.flatnonzero(self.occ).astype(np.int64)
        c = self.coords.astype(np.int64)
        return np.unique((c[:, 2] * g + c[:, 1]) * g + c[:, 0])


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------
def look_at(centre, target, up, fx, fy, cx, cy, W, H) -> Camera:
    """OpenCV look-at camera: z = normalize(target - centre), x = normalize(z x up),
    y = z x x, R = [x; y; z], t = -R centre (all rounded to float32)."""
    c = np.asarray(centre, np.float64)
    z = np.asarray(target, np.float64) - c
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z]).astype(np.float32)
    t = (-(R.astype(np.float64) @ c)).astype(np.float32)
    return Camera(R, t, float(np.float32(fx)), float(np.float32(fy)), float(np.float32(cx)),
                  float(np.float32(cy)), int(W), int(H))


def _random_rotations(rng, n) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _yaw_rotations(angles) -> np.ndarray:
    c, s = np.cos(angles), np.sin(angles)
    R = np.zeros((len(angles), 3, 3))
    R[:, 0, 0] = c
    R[:, 0, 1] = -s
    R[:, 1, 0] = s
    R[:, 1, 1] = c
    R[:, 2, 2] = 1.0
    return R


def render(scene: Scene, cam: Camera):
    """Planar depth (float32, +inf = miss) and hit id (int32, -1 = miss)."""
    lib = _lib()
    depth = np.empty((cam.H, cam.W), np.float32)
    hit = np.empty((cam.H, cam.W), np.int32)
    ell_c = np.ascontiguousarray(scene.ell_c, np.float64)
    ell_M = scene.ell_M
    brad = np.ascontiguousarray(scene.ell_brad, np.float64)
    ell_id = np.ascontiguousarray(scene.ell_id, np.int32)
    pl_n = np.ascontiguousarray(scene.pl_n, np.float64).reshape(-1)
    pl_d = np.ascontiguousarray(scene.pl_d, np.float64)
    pl_rad = np.ascontiguousarray(scene.pl_rad, np.float64)
    pl_id = np.ascontiguousarray(scene.pl_id, np.int32)
    R = np.ascontiguousarray(cam.R, np.float64).reshape(-1)
    t = np.ascontiguousarray(cam.t, np.float64)
    lib.synth_render(len(ell_c), _p(ell_c), _p(ell_M), _p(brad), _p(ell_id), len(pl_d),
                     _p(pl_n), _p(pl_d), _p(pl_rad), _p(pl_id), _p(R), _p(t), cam.fx, cam.fy,
                     cam.cx, cam.cy, cam.W, cam.H, _p(depth), _p(hit))
    return depth, hit


def render_tuple(scene: Scene, cam: Camera):
    """Front-hit depth, exit depth of that primitive, surface crossings along
    the whole ray, and hit id (float32, float32, int32, int32; (H, W))."""
    lib = _lib()
    front = np.empty((cam.H, cam.W), np.float32)
    back = np.empty((cam.H, cam.W), np.float32)
    cross = np.empty((cam.H, cam.W), np.int32)
    hit = np.empty((cam.H, cam.W), np.int32)
    ell_c = np.ascontiguousarray(scene.ell_c, np.float64)
    brad = np.ascontiguousarray(scene.ell_brad, np.float64)
    ell_id = np.ascontiguousarray(scene.ell_id, np.int32)
    pl_n = np.ascontiguousarray(scene.pl_n, np.float64).reshape(-1)
    pl_d = np.ascontiguousarray(scene.pl_d, np.float64)
    pl_rad = np.ascontiguousarray(scene.pl_rad, np.float64)
    pl_id = np.ascontiguousarray(scene.pl_id, np.int32)
    R = np.ascontiguousarray(cam.R, np.float64).reshape(-1)
    t = np.ascontiguousarray(cam.t, np.float64)
    lib.synth_render_tuple(len(ell_c), _p(ell_c), _p(scene.ell_M), _p(brad), _p(ell_id),
                           len(pl_d), _p(pl_n), _p(pl_d), _p(pl_rad), _p(pl_id), _p(R), _p(t),
                           cam.fx, cam.fy, cam.cx, cam.cy, cam.W, cam.H, _p(front), _p(back),
                           _p(cross), _p(hit))
    return front, back, cross, hit


def with_tuple(wl: "Workload", seed: int = 1100, band: float = 2.0, untrusted: float = 0.03,
               d_cam_scale: float = 0.8, target=(0.0, 0.0, 0.0)) -> "Workload":
    """The workload plus depth-tuple rasters for its cameras (depth-tuple mode,
    Sec. 3.5), the way a 2DGS renderer would report them for opaque surfaces:
    d_min = front hit; d_max = d_min + band h (1 + U[0, 1/2]) (the splat band,
    h the grid's voxel edge); d_med = d_min + U[0, 1/2] (d_max - d_min), except
    for a fraction ``untrusted`` of hit pixels where d_med = d_min - U[0.1, 1] h
    (a tilted-surfel anomaly, d_min > d_med); n_samp = 3 x (surfaces the ray
    crosses) + U{0, 1, 2}; misses are +inf.  d_cam = d_cam_scale x the camera
    centre's distance to ``target``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = float(wl.grid.h)
    t = {"d_min": [], "d_med": [], "d_max": [], "n_samp": [], "d_cam": []}
    for cam in wl.cams:
        front, _back, cross, _hit = render_tuple(wl.scene, cam)
        hitm = np.isfinite(front)
        d_max = front.astype(np.float64) + band * h * (1.0 + 0.5 * rng.uniform(0, 1, front.shape))
        with np.errstate(invalid="ignore"):  # misses: inf - inf, replaced by +inf below
            d_med = front + 0.5 * rng.uniform(0, 1, front.shape) * (d_max - front)
        anom = hitm & (rng.uniform(0, 1, front.shape) < untrusted)
        d_med = np.where(anom, front - rng.uniform(0.1, 1.0, front.shape) * h, d_med)
        inf = np.float32(np.inf)
        t["d_min"].append(np.where(hitm, front, inf).astype(np.float32))
        t["d_med"].append(np.where(hitm, d_med, inf).astype(np.float32))
        t["d_max"].append(np.where(hitm, d_max, inf).astype(np.float32))
        t["n_samp"].append((3 * cross + rng.integers(0, 3, cross.shape)).astype(np.uint16))
        C = -np.asarray(cam.R, np.float64).T @ np.asarray(cam.t, np.float64)
        t["d_cam"].append(float(d_cam_scale * np.linalg.norm(C - np.asarray(target))))
    out = Workload(**{k: getattr(wl, k) for k in wl.__dataclass_fields__ if k != "tuple"})
    out.tuple = t
    out.name = wl.name + "-tuple"
    return out


def with_nerf_tuple(wl: "Workload", seed: int = 1500, noisy: float = 0.05) -> "Workload":
    """The workload plus the depth tuple a NeRF renderer reports (the NeRF
    variant of the fusion): planar depths d_min = front hit - U[0, 1] h (the
    first significant sample), d_exp = front hit + U[-1/4, 3/4] h (the
    expected depth), d_max = min(exit of the hit primitive, front hit + U[1,
    6] h) but at least d_exp (the cumulative-weight cut-off inside the
    object's volume), n_samp = 4 + U{0..23} + 4 x (surfaces crossed) ray
    samples; on a fraction ``noisy`` of hit pixels d_exp is off by U[-8, 8] h
    (a depth outlier).  Misses are +inf with n_samp = 0.  Stored as
    ``tuple`` with keys d_min, d_exp, d_max, n_samp."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = float(wl.grid.h)
    t = {"d_min": [], "d_exp": [], "d_max": [], "n_samp": []}
    for cam in wl.cams:
        front, back, cross, _hit = render_tuple(wl.scene, cam)
        hitm = np.isfinite(front)
        f = np.where(hitm, front, 0.0).astype(np.float64)
        shape = front.shape
        d_min = f - rng.uniform(0.0, 1.0, shape) * h
        d_exp = f + rng.uniform(-0.25, 0.75, shape) * h
        out = hitm & (rng.uniform(0, 1, shape) < noisy)
        d_exp = np.where(out, f + rng.uniform(-8.0, 8.0, shape) * h, d_exp)
        cut = f + rng.uniform(1.0, 6.0, shape) * h
        bk = np.where(np.isfinite(back) & (back > front), back, cut).astype(np.float64)
        d_max = np.maximum(np.minimum(bk, cut), d_exp)
        d_min = np.minimum(d_min, d_exp)
        inf = np.float32(np.inf)
        t["d_min"].append(np.where(hitm, d_min, inf).astype(np.float32))
        t["d_exp"].append(np.where(hitm, d_exp, inf).astype(np.float32))
        t["d_max"].append(np.where(hitm, d_max, inf).astype(np.float32))
        ns = 4 + rng.integers(0, 24, shape) + 4 * cross
        t["n_samp"].append(np.where(hitm, ns, 0).astype(np.uint16))
    out_wl = Workload(**{k: getattr(wl, k) for k in wl.__dataclass_fields__ if k != "tuple"})
    out_wl.tuple = t
    out_wl.name = wl.name + "-nerf"
    return out_wl


def nerf_density(wl: "Workload", seed: int = 1600, haze: float = 0.01,
                 lo: float = 10.0, hi: float = 200.0) -> np.ndarray:
    """A dense g^3 FP32 density grid (x fastest) for the workload's occupied
    voxels, the way a NeRF's density field sampled at voxel centres looks:
    log-uniform in [lo, hi) on the occupied prior, U[0, lo) haze on a fraction
    ``haze`` of the other cells, 0 elsewhere.  density >= lo gives back the
    prior."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = int(wl.grid.g)
    if wl.occ is not None:
        occ = np.asarray(wl.occ, np.uint8).reshape(-1) != 0
    else:
        occ = np.zeros(g ** 3, bool)
        occ[wl.active_linear()] = True
    rho = np.zeros(g ** 3, np.float32)
    k = int(occ.sum())
    rho[occ] = np.exp(rng.uniform(np.log(lo), np.log(hi), k)).astype(np.float32)
    rho[occ] = np.maximum(rho[occ], np.float32(lo))
    free = np.nonzero(~occ)[0]
    pick = rng.choice(len(free), size=int(haze * len(free)), replace=False)
    rho[free[pick]] = np.minimum(rng.uniform(0.0, lo, len(pick)), np.nextafter(np.float32(lo), np.float32(0)))
    return rho


def gaussians(wl: "Workload", seed: int = 1300, floaters: float = 0.005, dyadic: bool = True):
    """A 2DGS surfel cloud for the workload's scene (the input of the
    occupancy construction, Sec. 3.5): centres = the workload's surface points
    plus a fraction ``floaters`` scattered uniformly in a box 20x the scene's
    (the outlier tail the P99 radius ignores); two scales per surfel U[0.5,
    1.5] x h / 3 (h the workload's voxel edge, so that 3 s_bar is about h);
    opacities U[0.05, 0.6], rounded to multiples of 1/64 when ``dyadic`` (FP32
    sums of them are exact in any order).  Returns (mu (m, 3), scales (m, 2),
    alpha (m,)), FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = np.asarray(wl.points, np.float32).copy()
    m = len(mu)
    nf = int(round(floaters * m))
    lo, hi = mu.min(0), mu.max(0)
    ctr, ext = 0.5 * (lo + hi), 10.0 * (hi - lo)
    idx = rng.choice(m, size=nf, replace=False)
    mu[idx] = (ctr + rng.uniform(-1.0, 1.0, size=(nf, 3)) * ext).astype(np.float32)
    h = float(wl.grid.h)
    scales = (rng.uniform(0.5, 1.5, size=(m, 2)) * h / 3.0).astype(np.float32)
    alpha = rng.uniform(0.05, 0.6, size=m)
    if dyadic:
        alpha = np.round(alpha * 64.0) / 64.0
    return mu, scales, alpha.astype(np.float32)


def quaternions(m: int, seed: int = 1400) -> np.ndarray:
    """m seeded uniform random unit quaternions (w, x, y, z), FP32 (the
    surfels' orientations)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.normal(size=(m, 4))
    return (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)


def prompts(wl: "Workload", n: int = 3, seed: int = 1200, thresh: float = 0.9) -> list:
    """Positive prompts per view, the clicks a user would place on the target:
    up to n pixels (x, y) drawn (seeded, without replacement) from those whose
    mask probability exceeds thresh."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in wl.mask:
        if wl.mask_type == 1:
            p = np.asarray(m).view(np.float16).astype(np.float64)
        elif wl.mask_type == 2:
            p = 1.0 / (1.0 + np.exp(-np.asarray(m, np.float64)))
        else:
            p = np.asarray(m, np.float64)
        ys, xs = np.nonzero(p > thresh)
        pick = rng.choice(len(xs), size=min(n, len(xs)), replace=False) if len(xs) else []
        out.append([(int(xs[i]), int(ys[i])) for i in pick])
    return out


def soft_mask_f16(indicator: np.ndarray, rng, sigma=2.0, radius=6, noise_std=0.05) -> np.ndarray:
    """Indicator -> Gaussian blur (sigma px, clamp-to-edge) -> + N(0, noise_std)
    -> clamp [0, 1] -> binary16 bits (uint16)."""
    H, W = indicator.shape
    ind = np.ascontiguousarray(indicator, np.uint8)
    noise = rng.normal(0.0, noise_std, size=(H, W)).astype(np.float32)
    out = np.empty((H, W), np.uint16)
    _lib().synth_soft_mask(_p(ind), W, H, float(sigma), int(radius), _p(noise), _p(out))
    return out


def _sample_ellipsoid_surface(rng, scene: Scene, idx: np.ndarray, count: int) -> np.ndarray:
    """Area-uniform samples on the union of ellipsoids ``idx`` (rejection)."""
    axes = scene.ell_axes[idx]
    bound = 4 * np.pi * axes.prod(axis=1) / axes.min(axis=1)
    prob = bound / bound.sum()
    out = []
    got = 0
    while got < count:
        m = int((count - got) * 1.6) + 64
        e = rng.choice(len(idx), size=m, p=prob)
        u = rng.normal(size=(m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        a = axes[e]
        acc = a.min(axis=1) * np.linalg.norm(u / a, axis=1)
        keep = rng.random(m) < acc
        e, u, a = e[keep], u[keep], a[keep]
        local = a * u
        world = np.einsum("nij,nj->ni", scene.ell_rot[idx][e], local) + scene.ell_c[idx][e]
        out.append(world)
        got += len(world)
    return np.concatenate(out)[:count]


def _finish_workload(name, grid, occ, coords, cams, scene, rng_mask, rng_flip, mask_mode,
                     flips, points, meta) -> Workload:
    depth, hit, mask = [], [], []
    targets = np.asarray(scene.target_ids)
    for cam in cams:
        d, hid = render(scene, cam)
        ind = np.isin(hid, targets)
        depth.append(d)
        hit.append(hid)
        if mask_mode == "binary":
            m = ind.astype(np.float32)
            if flips > 0:
                f = rng_flip.random(m.shape) < flips
                m = np.where(f, 1.0 - m, m).astype(np.float32)
            mask.append(m)
        else:
            mask.append(soft_mask_f16(ind, rng_mask))
    mask_type = MASK_F32 if mask_mode == "binary" else MASK_F16
    return Workload(name, grid, occ, coords, cams, depth, mask, mask_type, hit,
                    points.astype(np.float32), scene, meta)


# --------------------------------------------------------------------------
# config 1: tiny sphere scene
# --------------------------------------------------------------------------
def config1(seed: int = 1001, g: int = 64, n_views: int = 4, W: int = 256, H: int = 192,
            f: float = 220.0, flips: float = 0.02, n_points: int = 20000,
            band: float = 0.03, ring_phase: float = 0.1, ring_height: float = 0.25) -> Workload:
    """64^3 over [-1,1]^3, 3 spheres (centres U[-0.5,0.5]^3, radii U[0.2,0.35],
    redrawn until pairwise gaps are >= 0.05), 4 cameras on a ring of radius 3
    (azimuth 2 pi k/4 + ring_phase, height ring_height, so that the cameras are
    not aligned with the grid axes) looking at the origin (up +z),
    256x192, f = 220, binary FP32 mask of sphere 0 with Bernoulli(flips)
    flips, occupancy = within ``band`` of a sphere surface, points uniform on
    the sphere surfaces (area-weighted)."""
    rs = np.random.Generator(np.random.PCG64(seed + 0))
    centres = np.empty((3, 3))
    radii = np.empty(3)
    for k in range(3):  # redraw until separated from the earlier spheres by 0.05
        while True:
            centres[k] = rs.uniform(-0.5, 0.5, size=3)
            radii[k] = rs.uniform(0.2, 0.35)
            gap = [np.linalg.norm(centres[k] - centres[q]) - radii[k] - radii[q] for q in range(k)]
            if all(d >= 0.05 for d in gap):
                break
    scene = Scene(centres, np.repeat(radii[:, None], 3, 1), np.tile(np.eye(3), (3, 1, 1)),
                  np.arange(3, dtype=np.int32), np.zeros((0, 3)), np.zeros(0), np.zeros(0),
                  np.zeros(0, np.int32), np.array([0], np.int32))
    cams = []
    for k in range(n_views):
        a = 2 * np.pi * k / n_views + ring_phase
        cams.append(look_at((3 * np.cos(a), 3 * np.sin(a), ring_height), (0, 0, 0), (0, 0, 1),
                            f, f, W / 2, H / 2, W, H))
    h = np.float32(2.0 / g)
    grid = Grid(g, (-1.0, -1.0, -1.0), float(h), False)
    occ = np.empty(g ** 3, np.uint8)
    o = np.array(grid.origin, np.float64)
    _lib().synth_occ_sphere_band(3, _p(np.ascontiguousarray(centres)),
                                 _p(np.ascontiguousarray(radii)), band, g, _p(o), float(h),
                                 _p(occ))
    rp = np.random.Generator(np.random.PCG64(seed + 3))
    pts = _sample_ellipsoid_surface(rp, scene, np.arange(3), n_points)
    return _finish_workload("config1", grid, occ, None, cams, scene,
                            np.random.Generator(np.random.PCG64(seed + 1)),
                            np.random.Generator(np.random.PCG64(seed + 2)), "binary", flips, pts,
                            {"seed": seed})


# --------------------------------------------------------------------------
# config 2: forward-facing dense
# --------------------------------------------------------------------------
def _config2_scene(seed, n_ell):
    rs = np.random.Generator(np.random.PCG64(seed + 0))
    c = np.empty((n_ell, 3))
    c[:, :2] = rs.uniform(-0.8, 0.8, size=(n_ell, 2))
    c[:, 2] = rs.uniform(-0.6, 0.6, size=n_ell)
    # keep the line of sight to the target clear: clutter centres inside the
    # cylinder |xy| < 0.4 in front of the target (z < 0.25) are redrawn
    for i in range(1, n_ell):
        while np.hypot(c[i, 0], c[i, 1]) < 0.4 and c[i, 2] < 0.25:
            c[i, :2] = rs.uniform(-0.8, 0.8, size=2)
            c[i, 2] = rs.uniform(-0.6, 0.6)
    rot = _random_rotations(rs, n_ell)
    axes = rs.uniform(0.02, 0.2, size=(n_ell, 3))
    c[0] = 0.0
    axes[0] = rs.uniform(0.15, 0.2, size=3)
    return Scene(c, axes, rot, np.arange(n_ell, dtype=np.int32),
                 np.array([[0.0, 0.0, 1.0]]), np.array([0.9]), np.array([0.0]),
                 np.array([n_ell], np.int32), np.array([0], np.int32))


def config2(seed: int = 1002, g: int = 256, n_views: int = 8, W: int = 1008, H: int = 756,
            f: float = 800.0, n_ell: int = 200, n_points: int = 1_000_000) -> Workload:
    """256^3 over [-1,1]^3; 200 ellipsoids (centres U[-0.8,0.8]^2 x U[-0.6,0.6],
    redrawn while inside the cylinder |xy| < 0.4, z < 0.25 in front of the
    target, uniform rotations, semi-axes U[0.02,0.2]; ellipsoid 0 = target at the
    origin with semi-axes U[0.15,0.2]) + back plane z = 0.9; 8 cameras on a
    4x2 grid (x in +-0.05, +-0.15; y in +-0.05; z = -2.5; each position
    jittered by U[-0.01, 0.01]^3) looking along +z;
    1008x756, f = 800; FP16 soft masks of ellipsoid 0; occupancy = voxels whose
    corners straddle a surface; points = surface samples + N(0, (h/2)^2).

    Smaller ``W``/``H`` scale ``f`` and the principal point with the image."""
    scene = _config2_scene(seed, n_ell)
    scale = W / 1008.0
    fs = f * scale
    xs = (-0.15, -0.05, 0.05, 0.15)
    ys = (-0.05, 0.05)
    # rig positions plus a seeded U[-0.01, 0.01]^3 jitter, so that the rig is not
    # commensurate with the voxel lattice (no systematic pixel-boundary ties)
    rj = np.random.Generator(np.random.PCG64(seed + 5))
    pos = [np.array((x, y, -2.5)) + rj.uniform(-0.01, 0.01, 3) for y in ys for x in xs][:n_views]
    cams = []
    for p in pos:
        R = np.eye(3, dtype=np.float32)
        t = (-np.asarray(p)).astype(np.float32)
        cams.append(Camera(R, t, float(np.float32(fs)), float(np.float32(fs)),
                           float(np.float32(W / 2)), float(np.float32(H / 2)), W, H))
    h = np.float32(2.0 / g)
    grid = Grid(g, (-1.0, -1.0, -1.0), float(h), False)
    occ = np.empty(g ** 3, np.uint8)
    o = np.array(grid.origin, np.float64)
    pl_n = np.ascontiguousarray(scene.pl_n.reshape(-1))
    _lib().synth_occ_corner_sign(len(scene.ell_c), _p(np.ascontiguousarray(scene.ell_c)),
                                 _p(scene.ell_M), _p(np.ascontiguousarray(scene.ell_brad)),
                                 len(scene.pl_d), _p(pl_n), _p(np.ascontiguousarray(scene.pl_d)),
                                 g, _p(o), float(h), _p(occ))
    rp = np.random.Generator(np.random.PCG64(seed + 3))
    n_ell_pts = int(round(0.85 * n_points))
    pe = _sample_ellipsoid_surface(rp, scene, np.arange(len(scene.ell_c)), n_ell_pts)
    pp = np.column_stack([rp.uniform(-1, 1, n_points - n_ell_pts),
                          rp.uniform(-1, 1, n_points - n_ell_pts),
                          np.full(n_points - n_ell_pts, 0.9)])
    pts = np.concatenate([pe, pp])
    pts = pts + rp.normal(0.0, float(h) / 2, size=pts.shape)
    pts = pts[rp.permutation(len(pts))]
    return _finish_workload("config2", grid, occ, None, cams, scene,
                            np.random.Generator(np.random.PCG64(seed + 1)), None, "soft", 0.0,
                            pts, {"seed": seed})


def config4(seed: int = 1004, **kw) -> Workload:
    """Config 2's scene with FP32 mask logits: l = logit(clamp(m, 1e-4, 1 - 1e-4))
    of the soft mask (decoded from binary16), as a differentiable leaf."""
    wl = config2(seed=seed, **kw)
    logits = []
    for m in wl.mask:
        p = m.view(np.float16).astype(np.float64)
        p = np.clip(p, 1e-4, 1 - 1e-4)
        logits.append(np.log(p / (1 - p)).astype(np.float32))
    wl.mask = logits
    wl.mask_type = MASK_LOGIT_F32
    wl.name = "config4"
    return wl


# --------------------------------------------------------------------------
# config 3: unbounded sparse, contracted grid
# --------------------------------------------------------------------------
def contract_np(x: np.ndarray) -> np.ndarray:
    r = np.linalg.norm(x, axis=-1, keepdims=True)
    safe = np.maximum(r, 1e-300)
    return np.where(r <= 1.0, x, (2.0 - 1.0 / safe) * x / safe)


def _config3_scene(seed, n_ell, cams_pos):
    rs = np.random.Generator(np.random.PCG64(seed + 0))
    c = np.empty((n_ell, 3))
    axes = np.empty((n_ell, 3))
    yaw = rs.uniform(0, 2 * np.pi, size=n_ell)
    for i in range(n_ell):
        while True:
            r = np.exp(rs.uniform(np.log(0.3), np.log(50.0)))
            a = rs.uniform(0, 2 * np.pi)
            ax = rs.uniform(0.05, 0.6, size=3)
            ci = np.array([r * np.cos(a), r * np.sin(a), ax[2]])
            if len(cams_pos) == 0:  # cameras unknown: keep clear of the whole orbit annulus
                if abs(r - 4.0) > ax.max() + 0.1:
                    break
            elif np.min(np.linalg.norm(cams_pos - ci, axis=1)) > ax.max() + 0.1:
                break
        c[i] = ci
        axes[i] = ax
    rot = _yaw_rotations(yaw)
    ids = np.arange(n_ell, dtype=np.int32)
    return Scene(c, axes, rot, ids, np.array([[0.0, 0.0, 1.0]]), np.array([0.0]),
                 np.array([50.0]), np.array([n_ell], np.int32), ids[ids % 5 == 0])


_ND_CACHE: dict = {}


def config3(seed: int = 1003, g: int = 512, n_views: int = 16, W: int = 1297, H: int = 840,
            f: float = 1100.0, n_ell: int = 1000, n_occ: int | None = 12_000_000,
            n_points: int = 3_000_000, s_max: float = 6.0,
            view_seed: int | None = None) -> Workload:
    """Contracted 512^3 grid over [-2,2]^3 stored as a sparse occupied set;
    1,000 ellipsoids resting on the ground z = 0 (radial distance
    log-uniform [0.3, 50], semi-axes U[0.05, 0.6], group = id mod 5, target
    group 0), ground disc of radius 50, sky = inf; 16 cameras on an orbit of
    radius 4 (azimuth 2 pi k/16 + U[-0.1, 0.1], height U[0.5, 2]) looking at
    (0, 0, 0.5); 1297x840, f = 1100; FP16 soft masks of group 0.

    Occupancy: the ``n_occ`` voxels nearest (in contracted-space distance, in
    units of the contracted voxel edge) to a contracted surface; ``n_occ``
    defaults to 12M at g = 512 and scales with g^3 otherwise."""
    rc = np.random.Generator(np.random.PCG64((seed if view_seed is None else view_seed) + 5))
    az = 2 * np.pi * np.arange(n_views) / n_views + rc.uniform(-0.1, 0.1, n_views)
    hts = rc.uniform(0.5, 2.0, n_views)
    cams_pos = np.column_stack([4 * np.cos(az), 4 * np.sin(az), hts])
    scene = _config3_scene(seed, n_ell, np.zeros((0, 3)) if view_seed is not None else cams_pos)
    scale = W / 1297.0
    cams = [look_at(p, (0, 0, 0.5), (0, 0, 1), f * scale, f * scale, W / 2, H / 2, W, H)
            for p in cams_pos]
    if n_occ is None:
        n_occ = int(round(12_000_000 * (g / 512) ** 3))
    key = (seed, g, n_ell, float(s_max))
    nd = _ND_CACHE.get(key)
    if nd is None:
        nd = np.empty(g ** 3, np.float32)
        _lib().synth_contracted_distance(len(scene.ell_c), _p(np.ascontiguousarray(scene.ell_c)),
                                         _p(scene.ell_M), _p(np.ascontiguousarray(scene.ell_brad)),
                                         2.0 - 1.0 / 50.0, g, float(s_max), _p(nd))
        _ND_CACHE.clear()  # keep one field (they are large)
        _ND_CACHE[key] = nd
    finite = np.flatnonzero(np.isfinite(nd))
    if len(finite) > n_occ:
        vals = nd[finite]
        kth = np.partition(vals, n_occ - 1)[n_occ - 1]
        sel = finite[vals <= kth]
    else:
        kth = np.float32(s_max)
        sel = finite
    sel = np.sort(sel)
    coords = np.column_stack([sel % g, (sel // g) % g, sel // (g * g)]).astype(np.int32)
    h = np.float32(4.0 / g)
    grid = Grid(g, (-2.0, -2.0, -2.0), float(h), True)
    rp = np.random.Generator(np.random.PCG64(seed + 3))
    n_e = int(round(0.7 * n_points))
    pe = _sample_ellipsoid_surface(rp, scene, np.arange(len(scene.ell_c)), n_e)
    n_g = n_points - n_e
    rr = np.exp(rp.uniform(np.log(0.3), np.log(50.0), n_g))
    aa = rp.uniform(0, 2 * np.pi, n_g)
    pg = np.column_stack([rr * np.cos(aa), rr * np.sin(aa), np.zeros(n_g)])
    pts = np.concatenate([pe, pg])
    pts = pts + rp.normal(0.0, 0.01, size=pts.shape)
    pts = pts[rp.permutation(len(pts))]
    return _finish_workload("config3", grid, None, coords, cams, scene,
                            np.random.Generator(np.random.PCG64(seed + 1)), None, "soft", 0.0,
                            pts, {"seed": seed, "s_threshold": float(kth)})


# --------------------------------------------------------------------------
# config 5: many uneven sessions
# --------------------------------------------------------------------------
def session_mix(seed: int = 1005, n_sessions: int = 64, scale: float = 1.0) -> list:
    """Per-session recipes (not yet generated): dense grid from {64,128,256,384}^3
    or a sparse contracted set of U[0.5, 8]M voxels (50/50), views U{2..12},
    resolution from {640x480, 1008x756, 1297x840}, 200k points.

    ``scale`` < 1 shrinks grids, sets, resolutions and point counts for tests."""
    rng = np.random.Generator(np.random.PCG64(seed + 4))
    out = []
    res = [(640, 480), (1008, 756), (1297, 840)]
    for s in range(n_sessions):
        dense = bool(rng.random() < 0.5)
        g = int(rng.choice([64, 128, 256, 384]))
        n_sparse = int(rng.uniform(0.5e6, 8e6))
        views = int(rng.integers(2, 13))
        W, H = res[int(rng.integers(0, 3))]
        out.append(dict(session=s, dense=dense, g=g, n_sparse=n_sparse, views=views, W=W, H=H,
                        n_points=200_000, scene_seed=int(seed * 100 + s),
                        sparse_seed=int(seed * 100), scale=scale))
    return out


def session_workload(recipe: dict) -> Workload:
    """Generate one session of ``session_mix``: dense sessions use the
    forward-facing scene, sparse ones the unbounded contracted scene."""
    sc = recipe.get("scale", 1.0)
    W = max(16, int(round(recipe["W"] * sc)))
    H = max(16, int(round(recipe["H"] * sc)))
    npts = max(256, int(round(recipe["n_points"] * sc)))
    if recipe["dense"]:
        g = max(16, int(round(recipe["g"] * sc)))
        wl = config2(seed=recipe["scene_seed"], g=g, n_views=min(8, recipe["views"]), W=W, H=H,
                     n_points=npts)
        if recipe["views"] > 8:  # extra views: same rig, pulled back along z
            extra = []
            for k in range(recipe["views"] - 8):
                c0 = wl.cams[k % 8]
                t = c0.t.copy()
                t[2] = np.float32(t[2] + 0.25 * (1 + k // 8))
                extra.append(Camera(c0.R.copy(), t, c0.fx, c0.fy, c0.cx, c0.cy, c0.W, c0.H))
            rm = np.random.Generator(np.random.PCG64(recipe["scene_seed"] + 7))
            for cam in extra:
                d, hid = render(wl.scene, cam)
                wl.cams.append(cam)
                wl.depth.append(d)
                wl.hit.append(hid)
                wl.mask.append(soft_mask_f16(np.isin(hid, wl.scene.target_ids), rm))
    else:
        # sparse sessions share one unbounded scene (its contracted distance field
        # is computed once) and differ in views, resolution and occupied-set size
        g = max(32, int(round(384 * sc)))
        n_occ = max(1000, int(round(recipe["n_sparse"] * sc ** 3)))
        n_occ = min(n_occ, int(0.12 * g ** 3))
        wl = config3(seed=recipe["sparse_seed"], g=g, n_views=recipe["views"], W=W, H=H,
                     n_occ=n_occ, n_points=npts, n_ell=200,
                     view_seed=recipe["scene_seed"])
    wl.name = f"session{recipe['session']}"
    wl.meta.update(recipe)
    return wl


def digest(wl: Workload) -> str:
    """Short content hash of a workload's inputs (for logs)."""
    h = hashlib.sha1()
    for d in wl.depth:
        h.update(d.tobytes())
    for m in wl.mask:
        h.update(m.tobytes())
    if wl.occ is not None:
        h.update(wl.occ.tobytes())
    if wl.coords is not None:
        h.update(wl.coords.tobytes())
    return h.hexdigest()[:12]
