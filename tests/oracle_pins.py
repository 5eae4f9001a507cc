"""Pins of the FP64 oracle against the paper and the mathematics.

Each ``pin_*`` function takes an oracle API object (``oracle`` itself, or a
deliberately broken copy built by the mutation test) and raises
AssertionError when the oracle disagrees with what the paper and the
mathematics fix.  None of them calls the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth
from oracle import brute

P_DEFAULT = oracle.Params()


# --------------------------------------------------------------------------
# small fixtures
# --------------------------------------------------------------------------
def _probe_setup(t_z=2.0):
    """Grid 8^3 over [-1,1]^3 (h = 1/4) and one camera R = I looking along +z
    that sees voxel (3, 4, 5) at pixel (16, 12), u = 16.25, v = 12.75."""
    grid = synth.Grid(8, (-1.0, -1.0, -1.0), 0.25, False)
    ijk = (3, 4, 5)
    x = [-1.0 + (c + 0.5) * 0.25 for c in ijk]
    cam = synth.Camera(np.eye(3, dtype=np.float32),
                       np.array([-x[0], -x[1], t_z], np.float32), 20.0, 20.0, 16.25, 12.75, 32,
                       24)
    lin = np.array([(ijk[2] * 8 + ijk[1]) * 8 + ijk[0]], np.int64)
    p_z = x[2] + t_z
    return grid, cam, lin, p_z


def _raster(cam, value, at=None, fill=np.inf):
    a = np.full((cam.H, cam.W), fill, np.float32)
    if at is not None:
        a[at] = value
    return a


def small_sphere_workload(g=16, flips=0.02, **kw):
    return synth.config1(g=g, flips=flips, n_points=2000, **kw)


def small_forward_workload(g=32, n_views=3, n_ell=30, W=252, H=189):
    wl = synth.config2(g=g, n_views=8, W=W, H=H, n_ell=n_ell, n_points=4000)
    keep = [0, 3, 7][:n_views]
    wl.cams = [wl.cams[i] for i in keep]
    wl.depth = [wl.depth[i] for i in keep]
    wl.mask = [wl.mask[i] for i in keep]
    wl.hit = [wl.hit[i] for i in keep]
    return wl


def small_unbounded_workload(g=32, n_views=4, W=162, H=105, n_ell=60):
    return synth.config3(g=g, n_views=n_views, W=W, H=H, n_ell=n_ell, n_occ=None,
                         n_points=4000)


# --------------------------------------------------------------------------
# P1: single view, closed form (Eq. gs-depthweight, Eq. vmask, Eq. compact-fusion)
# --------------------------------------------------------------------------
def pin_single_view_closed_form(orc):
    grid, cam, lin, p_z = _probe_setup()
    Delta = 0.25  # gamma = 1 times h
    at = (12, 16)
    for r, m, votes in [(0.0, 0.8, True), (0.5, 0.8, True), (-0.75, 0.625, True),
                        (1.0, 0.9, True), (-1.0, 0.75, True),
                        (1.0 + 2.0 ** -18, 0.9, False), (-1.0 - 2.0 ** -18, 0.9, False),
                        (0.25, 0.5, True), (0.25, float(np.nextafter(np.float32(0.5),
                                                                     np.float32(0))), False)]:
        m = float(np.float32(m))
        D = np.float32(p_z - r * Delta)
        assert float(D) == p_z - r * Delta or not votes
        out = orc.fuse(grid, lin, [cam], [_raster(cam, D, at)], [_raster(cam, m, at, 0.0)],
                       oracle.MASK_F32, P_DEFAULT, want_pix=True)
        assert out["pix"][0, 0] == 12 * 32 + 16, out["pix"]
        if votes:
            w = math.exp(-0.5 * r * r)
            assert abs(out["Z"][0] - w) <= 1e-15, (r, out["Z"][0], w)
            assert abs(out["W"][0] - m * w) <= 1e-15
            assert abs(out["P"][0] - m) <= 1e-15
            assert out["bits"][0] == 1
            assert out["seg"][0] == (1 if m >= 0.5 else 0)
        else:
            assert out["Z"][0] == 0.0 and out["W"][0] == 0.0 and out["P"][0] == 0.0
            assert out["bits"][0] == 0 and out["seg"][0] == 0
    # e = 0 gives w = 1; |e| = Delta gives w = exp(-alpha1)
    for alpha1 in (0.0, 0.5, 2.0):
        prm = oracle.Params(alpha1=alpha1)
        out = orc.fuse(grid, lin, [cam], [_raster(cam, np.float32(p_z - Delta), at)],
                       [_raster(cam, 1.0, at, 0.0)], oracle.MASK_F32, prm)
        assert abs(out["Z"][0] - math.exp(-alpha1)) <= 1e-15
    # two views (same camera, two rasters): P = (m0 w0 + m1 w1) / (w0 + w1)
    r0, r1, m0, m1 = 0.5, -0.25, 0.75, 0.5625
    out = orc.fuse(grid, lin, [cam, cam],
                   [_raster(cam, np.float32(p_z - r0 * Delta), at),
                    _raster(cam, np.float32(p_z - r1 * Delta), at)],
                   [_raster(cam, m0, at, 0.0), _raster(cam, m1, at, 0.0)], oracle.MASK_F32,
                   P_DEFAULT)
    w0, w1 = math.exp(-0.5 * r0 * r0), math.exp(-0.5 * r1 * r1)
    assert abs(out["P"][0] - (m0 * w0 + m1 * w1) / (w0 + w1)) <= 1e-15
    assert out["bits"][0] == 3
    # gamma scales the tolerance: r = 0.75 of gamma*h with gamma = 2
    out = orc.fuse(grid, lin, [cam], [_raster(cam, np.float32(p_z - 0.375), at)],
                   [_raster(cam, 1.0, at, 0.0)], oracle.MASK_F32, oracle.Params(gamma=2.0))
    assert abs(out["Z"][0] - math.exp(-0.5 * 0.75 ** 2)) <= 1e-15
    # a non-finite or non-positive depth never votes; a voxel behind the camera never votes
    for Dbad in (np.inf, np.nan, 0.0, -1.0):
        out = orc.fuse(grid, lin, [cam], [_raster(cam, Dbad, at)], [_raster(cam, 1.0, at, 0.0)],
                       oracle.MASK_F32, P_DEFAULT)
        assert out["Z"][0] == 0.0
    grid2, cam2, lin2, _ = _probe_setup(t_z=-5.0)
    out = orc.fuse(grid2, lin2, [cam2], [_raster(cam2, 1.0, at)], [_raster(cam2, 1.0, at, 0.0)],
                   oracle.MASK_F32, P_DEFAULT, want_pix=True)
    assert out["Z"][0] == 0.0 and out["pix"][0, 0] == -1
    # binary16 and logit masks read the same probability
    half = np.full((cam.H, cam.W), np.float16(0.0)).view(np.uint16)
    half[at] = np.float16(0.75).view(np.uint16)
    out = orc.fuse(grid, lin, [cam], [_raster(cam, np.float32(p_z), at)], [half],
                   oracle.MASK_F16, P_DEFAULT)
    assert out["P"][0] == 0.75
    lg = _raster(cam, math.log(3.0), at, -10.0)
    out = orc.fuse(grid, lin, [cam], [_raster(cam, np.float32(p_z), at)], [lg],
                   oracle.MASK_LOGIT_F32, P_DEFAULT)
    assert abs(out["P"][0] - 1.0 / (1.0 + math.exp(-float(np.float32(math.log(3.0)))))) < 1e-15


# --------------------------------------------------------------------------
# pixel convention: pixel (i, j) covers [i, i+1) x [j, j+1); floor; half-open frame
# --------------------------------------------------------------------------
def pin_pixel_convention(orc):
    grid, cam, lin, p_z = _probe_setup()
    cases = [((16.25, 12.75), 12 * 32 + 16), ((0.0, 0.0), 0), ((31.5, 23.5), 23 * 32 + 31),
             ((32.0, 5.0), -1), ((5.0, 24.0), -1), ((-0.25, 5.0), -1), ((3.0, 7.0), 7 * 32 + 3)]
    for (cx, cy), want in cases:
        c = synth.Camera(cam.R, cam.t, cam.fx, cam.fy, cx, cy, cam.W, cam.H)
        pix, _ = orc.project(grid, lin, c)
        assert pix[0] == want, ((cx, cy), pix[0], want)
    # off-axis: u = fx * p_x / p_z + cx with p_x = 0.5, p_z = p_z
    c = synth.Camera(cam.R, np.array([cam.t[0] + 0.5, cam.t[1] - 0.25, cam.t[2]], np.float32),
                     cam.fx, cam.fy, 10.0, 10.0, cam.W, cam.H)
    u = 20.0 * 0.5 / p_z + 10.0
    v = 20.0 * -0.25 / p_z + 10.0
    pix, _ = orc.project(grid, lin, c)
    assert pix[0] == int(math.floor(v)) * 32 + int(math.floor(u))
    # anisotropic focal lengths: u uses fx and v uses fy
    c = synth.Camera(cam.R, np.array([cam.t[0] + 0.5, cam.t[1] - 0.25, cam.t[2]], np.float32),
                     12.0, 28.0, 10.0, 10.0, cam.W, cam.H)
    u = 12.0 * 0.5 / p_z + 10.0
    v = 28.0 * -0.25 / p_z + 10.0
    pix, _ = orc.project(grid, lin, c)
    assert pix[0] == int(math.floor(v)) * 32 + int(math.floor(u)), (pix[0], u, v)
    # a rotated camera: R maps world x to camera y and world y to camera -x
    R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], np.float32)
    x = np.array([-1.0 + 3.5 * 0.25, -1.0 + 4.5 * 0.25, -1.0 + 5.5 * 0.25])
    t = np.array([0.3, -0.2, 2.0], np.float32)
    c = synth.Camera(R, t, 16.0, 16.0, 16.0, 12.0, cam.W, cam.H)
    p = R.astype(np.float64) @ x + t
    u = 16.0 * p[0] / p[2] + 16.0
    v = 16.0 * p[1] / p[2] + 12.0
    pix, _ = orc.project(grid, lin, c)
    assert pix[0] == int(math.floor(v)) * 32 + int(math.floor(u)), (pix[0], u, v)


# --------------------------------------------------------------------------
# P2: alpha1 = 0 makes P the arithmetic mean of the accepting views' masks
# --------------------------------------------------------------------------
def pin_alpha0_mean(orc):
    wl = small_sphere_workload(g=16, flips=0.0)
    rng = np.random.Generator(np.random.PCG64(7))
    masks = [rng.random(m.shape).astype(np.float32) for m in wl.mask]
    lin = wl.active_linear()
    prm = oracle.Params(alpha1=0.0, tau_m=0.0)
    out = orc.fuse(wl.grid, lin, wl.cams, wl.depth, masks, oracle.MASK_F32, prm, want_pix=True)
    voted = 0
    for a in range(len(lin)):
        ms = [masks[i].reshape(-1)[out["pix"][a, i]] for i in range(wl.n_views)
              if (out["bits"][a] >> i) & 1]
        if ms:
            voted += 1
            assert abs(out["P"][a] - float(np.mean(np.asarray(ms, np.float64)))) <= 1e-12
            assert out["Z"][a] == float(len(ms))
        else:
            assert out["P"][a] == 0.0 and out["Z"][a] == 0.0
    assert voted > 50


# --------------------------------------------------------------------------
# P3: invariants
# --------------------------------------------------------------------------
def pin_invariants(orc):
    for wl, prm in [(small_sphere_workload(g=32), P_DEFAULT),
                    (small_sphere_workload(g=32), oracle.Params(tau_m=0.0)),
                    (small_forward_workload(), P_DEFAULT),
                    (small_forward_workload(), oracle.Params(tau_m=0.0, alpha1=1.5))]:
        lin = wl.active_linear()
        out = orc.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, wl.mask_type, prm)
        W, Z, P = out["W"], out["Z"], out["P"]
        assert (W >= 0).all() and (W <= Z * (1 + 1e-15)).all()
        voted = Z > 0
        assert voted.sum() > 20
        assert (Z[voted] >= math.exp(-prm.alpha1) * (1 - 1e-15)).all()
        assert (P[voted] >= prm.tau_m - 1e-15).all() and (P <= 1 + 1e-15).all()
        assert (P[~voted] == 0).all()
        assert (out["seg"] == (P >= prm.tau_cons)).all()
        assert (out["vmask"] == np.where(out["seg"] == 1, out["bits"], 0)).all()
        # every vote sets its view bit; a voxel with no bit has no weight
        assert ((out["bits"] != 0) == voted).all()
        # reversing the view order leaves P and seg unchanged and reverses the bits
        rev = orc.fuse(wl.grid, lin, wl.cams[::-1], wl.depth[::-1], wl.mask[::-1],
                       wl.mask_type, prm)
        assert np.allclose(rev["P"], P, rtol=0, atol=1e-12)
        assert (rev["seg"] == out["seg"]).all()
        S = wl.n_views
        rb = np.zeros_like(out["bits"])
        for i in range(S):
            rb |= ((out["bits"] >> i) & 1) << (S - 1 - i)
        assert (rev["bits"] == rb).all()
        # voxels order does not matter
        perm = np.random.Generator(np.random.PCG64(3)).permutation(len(lin))
        sh = orc.fuse(wl.grid, lin[perm], wl.cams, wl.depth, wl.mask, wl.mask_type, prm)
        assert (sh["P"] == P[perm]).all()


def pin_scale_invariance(orc):
    wl = small_forward_workload()
    lin = wl.active_linear()
    base = orc.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, wl.mask_type, P_DEFAULT,
                    want_pix=True)
    s = 2.0  # a power of two keeps every float32 input exact
    grid = synth.Grid(wl.grid.g, tuple(s * o for o in wl.grid.origin), s * wl.grid.h)
    cams = [synth.Camera(c.R, (c.t * np.float32(s)).astype(np.float32), c.fx, c.fy, c.cx, c.cy,
                         c.W, c.H) for c in wl.cams]
    depth = [(d * np.float32(s)).astype(np.float32) for d in wl.depth]
    sc = orc.fuse(grid, lin, cams, depth, wl.mask, wl.mask_type, P_DEFAULT, want_pix=True)
    assert (sc["pix"] == base["pix"]).all()
    assert (sc["bits"] == base["bits"]).all()
    assert np.allclose(sc["P"], base["P"], rtol=0, atol=1e-15)
    assert np.allclose(sc["Z"], base["Z"], rtol=1e-15, atol=0)


# --------------------------------------------------------------------------
# P4: analytic sphere scene (Sec. 3.5: voxels on the visible object surface)
# --------------------------------------------------------------------------
def pin_sphere_scene(orc):
    wl = small_sphere_workload(g=32, flips=0.0)
    lin = wl.active_linear()
    x, hv, _ = brute.voxel_centres(wl.grid, lin)
    sc = wl.scene
    dist = np.abs(np.linalg.norm(x[:, None, :] - sc.ell_c[None], axis=2) - sc.ell_axes[None, :, 0])
    Delta = float(wl.grid.h)
    # tau_m = 0.5 with a binary mask: every vote carries m = 1, so voted voxels score 1
    out = orc.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, wl.mask_type, P_DEFAULT)
    voted = out["Z"] > 0
    assert voted.sum() > 100
    assert (out["P"][voted] == 1.0).all()
    dmax = max(float(np.max(d[np.isfinite(d)])) for d in wl.depth)
    bound = Delta * 1.05 + 0.75 * dmax / wl.cams[0].fx + 1e-9
    assert (dist[voted, 0] <= bound).all(), dist[voted, 0].max()
    # tau_m = 0: every depth-consistent view votes; voxels on sphere 0's surface
    # and away from the other spheres see only m = 1 votes
    out0 = orc.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, wl.mask_type,
                    oracle.Params(tau_m=0.0))
    near0 = (dist[:, 0] <= Delta / 4) & (np.min(dist[:, 1:], axis=1) > 3 * Delta) & (out0["Z"] > 0)
    assert near0.sum() > 20
    assert (out0["P"][near0] == 1.0).all()
    # and voxels on the other spheres, far from sphere 0, never reach consensus
    far = (np.min(dist[:, 1:], axis=1) <= Delta / 4) & (dist[:, 0] > 3 * Delta) & (out0["Z"] > 0)
    assert far.sum() > 20
    assert (out0["P"][far] == 0.0).all()


# --------------------------------------------------------------------------
# P5: independent brute force with analytic depth
# --------------------------------------------------------------------------
def _compare_brute(orc, wl, prm, mask_kind):
    lin = wl.active_linear()
    o = orc.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, wl.mask_type, prm, want_pix=True)
    b = brute.fuse(wl.grid, lin, wl.cams, wl.mask, wl.scene, tau_m=prm.tau_m, gamma=prm.gamma,
                   alpha1=prm.alpha1, tau_cons=prm.tau_cons, eps=prm.eps, z_near=prm.z_near,
                   mask_kind=mask_kind)
    skip = (o["flags"] != 0) | b["ambiguous"]
    ok = ~skip
    assert ok.sum() >= 0.98 * len(lin), (skip.sum(), len(lin))
    assert (o["pix"][ok] == b["pix"][ok]).all()
    assert (o["bits"][ok] == b["bits"][ok]).all(), np.flatnonzero(o["bits"][ok] != b["bits"][ok])
    # the stored FP32 depth differs from the analytic one by half an ulp; the
    # weight moves by at most 2 alpha1 |r| |dD| / Delta per view
    assert np.allclose(o["Z"][ok], b["Z"][ok], rtol=1e-5, atol=0)
    assert np.allclose(o["W"][ok], b["W"][ok], rtol=1e-5, atol=0)
    assert np.allclose(o["P"][ok], b["P"][ok], rtol=0, atol=1e-5)
    sure = ok & (np.abs(b["P"] - prm.tau_cons) > 1e-5)
    assert (o["seg"][sure] == b["seg"][sure]).all()
    assert (o["Z"] > 0).sum() > 20
    return int(skip.sum())


def pin_bruteforce(orc):
    _compare_brute(orc, small_sphere_workload(g=16), P_DEFAULT, "f32")
    _compare_brute(orc, small_sphere_workload(g=32), oracle.Params(tau_m=0.0), "f32")
    _compare_brute(orc, small_forward_workload(), P_DEFAULT, "f16")
    _compare_brute(orc, small_forward_workload(), oracle.Params(tau_m=0.0, alpha1=1.0), "f16")
    _compare_brute(orc, small_unbounded_workload(), P_DEFAULT, "f16")
    _compare_brute(orc, small_unbounded_workload(), oracle.Params(tau_m=0.0, gamma=2.0), "f16")


# --------------------------------------------------------------------------
# P6: Pass 1 labels (Eq. pass1)
# --------------------------------------------------------------------------
def pin_labels(orc):
    rng = np.random.Generator(np.random.PCG64(11))
    for contracted in (False, True):
        g = 16
        if contracted:
            grid = synth.Grid(g, (-2.0, -2.0, -2.0), 0.25, True)
            d = rng.normal(size=(3000, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            pts = d * np.exp(rng.uniform(np.log(0.05), np.log(200.0), size=(3000, 1)))
        else:
            grid = synth.Grid(g, (-1.0, -1.0, -1.0), 0.125, False)
            pts = rng.uniform(-1.3, 1.3, size=(3000, 3))
        pts = pts.astype(np.float32)
        pts[0] = np.nan
        pts[1] = [-1.0, -1.0, -1.0]
        pts[2] = [1.0, 0.0, 0.0]
        pts[3] = [0.0, 0.0, 0.0]
        seg = rng.integers(0, 2, size=g ** 3).astype(np.uint8)
        lab, flags = orc.label(grid, seg, pts)
        ref = brute.label(grid, seg, pts)
        assert (lab == ref).all()
        assert lab[0] == 0
        if not contracted:
            assert lab[1] == seg[0]                          # -1 lies in voxel 0
            assert lab[2] == 0                               # +1 is outside (strict)
            assert lab[3] == seg[(8 * g + 8) * g + 8]        # a face goes to the higher index
        # with every voxel segmented, only the inside of the half-open box
        # [origin, origin + g h) labels 1
        ones = np.ones(g ** 3, np.uint8)
        hi = float(grid.origin[0]) + g * float(grid.h)
        lo = float(grid.origin[0])
        if contracted:  # contract(x) reaches the box face only at infinity; probe |x| large
            edge = np.array([[1e3, 0, 0], [0, -1e3, 0], [0.5, 0.25, -0.5]], np.float32)
            lab, _ = orc.label(grid, ones, edge)
            assert list(lab) == [1, 1, 1]
        else:
            edge = np.array([[hi, 0, 0], [0, hi, 0], [0, 0, hi], [lo, lo, lo],
                             [np.nextafter(np.float32(hi), np.float32(0)), 0, 0],
                             [np.nextafter(np.float32(lo), np.float32(-2)), 0, 0]], np.float32)
            lab, _ = orc.label(grid, ones, edge)
            assert list(lab) == [0, 0, 0, 1, 1, 0], lab
        # points at voxel centres pick that voxel
        ijk = rng.integers(0, g, size=(200, 3))
        o = np.asarray(grid.origin)
        cen = (o + (ijk + 0.5) * grid.h).astype(np.float32)
        if contracted:
            keep = np.linalg.norm(cen, axis=1) < 1.0
            ijk, cen = ijk[keep], cen[keep]
        lab, _ = orc.label(grid, seg, cen)
        assert (lab == seg[(ijk[:, 2] * g + ijk[:, 1]) * g + ijk[:, 0]]).all()


# --------------------------------------------------------------------------
# P7: adjoint vs central finite differences of the FP64 forward
# --------------------------------------------------------------------------
def target_truth(wl, lin):
    """y_v = 1 iff the target ellipsoid's implicit function changes sign over the
    voxel's 8 corners or is <= 0 at its centre."""
    sc = wl.scene
    M = sc.ell_M[0].reshape(3, 3)
    c0 = sc.ell_c[0]
    g = wl.grid.g
    o = np.asarray(wl.grid.origin, np.float64)
    h = float(wl.grid.h)
    lin = np.asarray(lin, np.int64)
    idx = np.stack([lin % g, (lin // g) % g, lin // (g * g)], axis=1).astype(np.float64)

    def f(p):
        y = (p - c0) @ M.T
        return np.einsum("ij,ij->i", y, y) - 1.0
    vals = np.stack([f(o + (idx + np.array([a & 1, (a >> 1) & 1, (a >> 2) & 1])) * h)
                     for a in range(8)], axis=1)
    straddle = (vals > 0).any(axis=1) & (vals <= 0).any(axis=1)
    inside = f(o + (idx + 0.5) * h) <= 0
    return (straddle | inside).astype(np.float64)


def fd_check(orc, wl, mask_type, n_per_view=60, n_random=20, eps_mask=1e-3, eps_depth=1e-4,
             seed=5):
    lin = wl.active_linear()
    y = target_truth(wl, lin)
    prm = P_DEFAULT
    base = orc.fuse(wl.grid, lin, wl.cams, wl.depth, wl.mask, mask_type, prm, want_pix=True)
    _, gP = oracle.bce_loss_grad(base["P"], y)
    gM, gD = orc.fuse_grad(wl.grid, lin, wl.cams, wl.depth, wl.mask, mask_type, gP, prm)
    rng = np.random.Generator(np.random.PCG64(seed))
    gmax = max(max(np.abs(a).max() for a in gM), max(np.abs(a).max() for a in gD))
    assert gmax > 0
    checked = excluded = 0
    for which, grads, leaves in (("mask", gM, wl.mask), ("depth", gD, wl.depth)):
        for i in range(wl.n_views):
            nz = np.flatnonzero(grads[i].reshape(-1))
            pick = rng.choice(nz, size=min(n_per_view, len(nz)), replace=False) if len(nz) else []
            pick = np.concatenate([np.asarray(pick, np.int64),
                                   rng.integers(0, grads[i].size, n_random)])
            aff = np.flatnonzero(np.isin(base["pix"][:, i], pick))
            for p in pick:
                sel = aff[base["pix"][aff, i] == p]
                vals = []
                eps = eps_mask if which == "mask" else eps_depth
                flat = np.ascontiguousarray(leaves[i]).reshape(-1)
                old = flat[p]
                for sgn in (+1, -1):
                    # perturb one pixel of a copy of the leaf list (the raster
                    # itself is changed in place and restored)
                    flat[p] = np.float32(float(old) + sgn * eps)
                    arrs = list(leaves)
                    arrs[i] = flat.reshape(leaves[i].shape)
                    if which == "mask":
                        o2 = orc.fuse(wl.grid, lin[sel], wl.cams, wl.depth, arrs, mask_type, prm)
                    else:
                        o2 = orc.fuse(wl.grid, lin[sel], wl.cams, arrs, wl.mask, mask_type, prm)
                    vals.append((o2, float(flat[p])))
                flat[p] = old
                (op, xp), (om, xm) = vals
                if len(sel) and ((op["bits"] != base["bits"][sel]).any()
                                 or (om["bits"] != base["bits"][sel]).any()):
                    excluded += 1  # a gate flips inside the stencil
                    continue
                lim = 10 * eps + 1e-6  # the loss's clamp acts as a gate too
                Ps = np.concatenate([base["P"][sel], op["P"], om["P"]])
                if ((Ps > 0) & ((Ps < lim) | (Ps > 1 - lim))).any():
                    excluded += 1
                    continue
                Lp, _ = oracle.bce_loss_grad(op["P"], y[sel])
                Lm, _ = oracle.bce_loss_grad(om["P"], y[sel])
                fd = (Lp - Lm) / (xp - xm)
                an = grads[i].reshape(-1)[p]
                assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-3 * gmax), (which, i, p, fd, an)
                checked += 1
    assert checked > 100, checked
    return checked, excluded


def gradient_fd_config4_size(orc):
    """Config 4's stated check: central differences (eps = 1e-3) of the FP64
    forward on a 32^3 grid with 3 views (0, 3, 7) at 1008 x 756, 600 pixels
    per view with a nonzero analytic gradient plus 100 random ones, for the
    logits and the depths, against the oracle's analytic adjoint."""
    wl = synth.config4(g=32, n_views=8, W=1008, H=756, n_ell=30, n_points=1000)
    keep = [0, 3, 7]
    wl.cams = [wl.cams[i] for i in keep]
    wl.depth = [np.ascontiguousarray(wl.depth[i]) for i in keep]
    wl.mask = [np.ascontiguousarray(wl.mask[i]) for i in keep]
    return fd_check(orc, wl, oracle.MASK_LOGIT_F32, n_per_view=600, n_random=100,
                    eps_mask=1e-3, eps_depth=1e-3)


def pin_gradient_fd(orc):
    wl = synth.config4(g=32, n_views=8, W=252, H=189, n_ell=30, n_points=1000)
    keep = [0, 3, 7]
    wl.cams = [wl.cams[i] for i in keep]
    wl.depth = [wl.depth[i] for i in keep]
    wl.mask = [wl.mask[i] for i in keep]
    fd_check(orc, wl, oracle.MASK_LOGIT_F32)
    # probability masks: gradient with respect to m itself
    probs = [(1.0 / (1.0 + np.exp(-m.astype(np.float64)))).astype(np.float32) for m in wl.mask]
    wl.mask = probs
    fd_check(orc, wl, oracle.MASK_F32, n_per_view=30, n_random=10)


# --------------------------------------------------------------------------
# depth-tuple mode (Sec. 3.5 "Footprint statistics" .. "Thin-structure path";
# Algorithms "Thick-/Thin-Structure Segmentation for 2DGS", App. B.5)
# --------------------------------------------------------------------------
def _tuple_setup():
    """Grid 8^3 over [-1,1]^3 (h = 1/4), voxel (3, 4, 5) at x = (-1/8, 1/8, 3/8)
    seen on-axis (the ray through its projection is the optical axis, so
    t* = x_d = 2.375 and the planar-to-ray factor is 1) by a camera R = I,
    f = 100, principal point (50.25, 40.75), 100 x 80: the voxel projects to
    pixel (50, 40) and its corners to u in [44.69, 55.81], v in [35.19, 46.31]
    -> footprint pixels 44..55 x 35..46 (A = 144), clipped box area 123.5."""
    grid = synth.Grid(8, (-1.0, -1.0, -1.0), 0.25, False)
    cam = synth.Camera(np.eye(3, dtype=np.float32), np.array([0.125, -0.125, 2.0], np.float32),
                       100.0, 100.0, 50.25, 40.75, 100, 80)
    lin = np.array([(5 * 8 + 4) * 8 + 3], np.int64)
    return grid, cam, lin, 2.375


def _tuple_run(orc, d_min, d_med, d_max, n=5, mask=1.0, d_cam=3.0, tparams=None, params=None):
    grid, cam, lin, xd = _tuple_setup()

    def ras(v, dtype=np.float32):
        return np.broadcast_to(np.asarray(v, dtype), (cam.H, cam.W)).copy()
    tup = {"d_min": [ras(d_min)], "d_med": [ras(d_med)], "d_max": [ras(d_max)],
           "n_samp": [ras(n, np.uint16)], "d_cam": [d_cam]}
    r = orc.fuse_tuple(grid, lin, [cam], tup, [ras(mask)], oracle.MASK_F32,
                       params=params or P_DEFAULT, tparams=tparams or oracle.TupleParams())
    return r, tup


def _w(lo, hi, t_hat, alpha1=0.5):
    lo, hi = float(np.float32(lo)), float(np.float32(hi))
    return math.exp(-alpha1 * ((t_hat - 0.5 * (lo + hi)) / (0.5 * (hi - lo))) ** 2)


def pin_tuple_closed_form(orc):
    xd = 2.375
    # base: d_med at the voxel, median reference, t_hat = t* -> w at the band offset
    r, _ = _tuple_run(orc, 2.275, 2.375, 2.575)
    assert r["kind"][0, 0] == 1
    assert math.isclose(r["W"][0], _w(2.275, 2.575, xd), rel_tol=1e-12)
    assert math.isclose(r["Z"][0], r["W"][0], rel_tol=1e-15) and r["P"][0] == 1.0
    # see-through (d_med > gamma_st d_cam): front surface reference, one-sided gate,
    # t_hat clamped to d_min
    r, _ = _tuple_run(orc, 2.275, 2.375, 2.575, d_cam=1.0)
    assert r["kind"][0, 0] == 1
    assert math.isclose(r["W"][0], _w(2.275, 2.575, float(np.float32(2.275))), rel_tol=1e-12)
    # layered centre pixel: front reference and a tightened tolerance
    # 0.25 / (1 + 0.05 E), E = 60 - 775/144, rejects x_d - d_min = 0.1; the
    # thin path then certifies the footprint: t = m_max = 1, W = Z = 1
    n = np.full((80, 100), 5, np.uint16)
    n[40, 50] = 60
    r, _ = _tuple_run(orc, 2.275, 2.375, 2.575, n=n)
    assert r["kind"][0, 0] == 2 and r["W"][0] == 1.0 and r["Z"][0] == 1.0
    # the same with the centre count just below mean + sigma is not layered
    # (but still tightened): median reference, thick vote
    n[40, 50] = 6
    r, _ = _tuple_run(orc, 2.275, 2.375, 2.575, n=n)
    assert r["kind"][0, 0] == 1
    # one-sided gate: voxel 0.2 in front of d_min (see-through), tolerance
    # tightened to 0.25 / 1.3 < 0.2 by a centre count 16 over a 0/20 checkerboard
    # (mean 10, sigma 10: not layered): x_d - d_min = -0.2 passes, |.| would not
    n = np.where((np.add.outer(np.arange(80), np.arange(100)) % 2) == 0, 0, 20).astype(np.uint16)
    n[40, 50] = 16
    r, _ = _tuple_run(orc, 2.575, 2.675, 2.775, n=n, d_cam=1.0)
    assert r["kind"][0, 0] == 1
    assert math.isclose(r["W"][0], _w(2.575, 2.775, float(np.float32(2.575))), rel_tol=1e-12)
    # untrusted (d_min > d_med) everywhere: no thick vote, the thin path
    # (median reference per pixel) votes
    r, _ = _tuple_run(orc, 2.475, 2.375, 2.575)
    assert r["kind"][0, 0] == 2 and r["W"][0] == 1.0
    # behind the surface by 0.6 > 2 h_v: neither path
    r, _ = _tuple_run(orc, 1.775, 1.775, 1.975)
    assert r["kind"][0, 0] == 0 and r["Z"][0] == 0.0
    # 0.1 behind the median with a centre mask below tau_m: the behind gate lets
    # it through (0.1 <= 2 h_v) and the footprint certifies it (thin vote)
    m = np.ones((80, 100), np.float32)
    m[40, 50] = 0.3
    r, _ = _tuple_run(orc, 2.175, 2.275, 2.475, mask=m)
    assert r["kind"][0, 0] == 2 and r["W"][0] == 1.0
    # depth-gradient factor: a step of 0.05 in (d_min + d_max)/2 across the
    # centre pixel's neighbours; see-through reference (|t* - t_hat| = 0.1):
    # k = 1000 -> pi = exp(-2.5) -> 0.25 pi < 0.1 rejects; k = 0 accepts
    lo = np.full((80, 100), 2.275, np.float32)
    lo[:, 51:] += np.float32(0.05)
    hi = lo + np.float32(0.3)
    r, _ = _tuple_run(orc, lo, 2.375, hi, d_cam=1.0, tparams=oracle.TupleParams(k_dg=1000.0))
    assert r["kind"][0, 0] != 1
    r, _ = _tuple_run(orc, lo, 2.375, hi, d_cam=1.0, tparams=oracle.TupleParams(k_dg=0.0))
    assert r["kind"][0, 0] == 1
    # thin floors: support below n_min, coverage below rho_cover
    r, _ = _tuple_run(orc, 2.475, 2.375, 2.575, tparams=oracle.TupleParams(n_abs=145.0))
    assert r["kind"][0, 0] == 0
    m = np.zeros((80, 100), np.float32)
    m[35:40, 44:56] = 1.0  # 60 of 144 depth-valid pixels mask-positive: 0.42 < 0.5
    r, _ = _tuple_run(orc, 2.475, 2.375, 2.575, mask=m)
    assert r["kind"][0, 0] == 0
    m[40, 44:56] = 1.0     # 72 of 144: exactly 0.5 (inclusive)
    r, _ = _tuple_run(orc, 2.475, 2.375, 2.575, mask=m)
    assert r["kind"][0, 0] == 2
    # distance gate (1.5 h_v): with an 8 x 8 mask hole around the centre (80 of
    # 144 pixels positive) the nearest mask-positive unprojection lies 0.101
    # from the centre: inside 1.5 h_v = 0.375, outside 0.3 h_v = 0.075
    m = np.ones((80, 100), np.float32)
    m[37:45, 46:54] = 0.0
    r, _ = _tuple_run(orc, 2.475, 2.375, 2.575, mask=m)
    assert r["kind"][0, 0] == 2
    r, _ = _tuple_run(orc, 2.475, 2.375, 2.575, mask=m,
                      tparams=oracle.TupleParams(dist_gate=0.3))
    assert r["kind"][0, 0] == 0


def pin_tuple_bruteforce(orc):
    wl = synth.config2(g=40, W=140, H=105, n_ell=40, n_points=500)
    tw = synth.with_tuple(wl)
    lin = wl.active_linear()
    for tp, prm in [(oracle.TupleParams(n_abs=4.0, k_dg=30.0), P_DEFAULT),
                    (oracle.TupleParams(n_abs=2.0, rho_cover=0.3, tau_thin=0.3),
                     oracle.Params(tau_m=0.3, alpha1=1.0))]:
        r = orc.fuse_tuple(wl.grid, lin, wl.cams, tw.tuple, wl.mask, wl.mask_type, params=prm,
                           tparams=tp)
        b = brute.fuse_tuple(wl.grid, lin, wl.cams, tw.tuple, wl.mask, wl.mask_type,
                             tau_m=prm.tau_m, alpha1=prm.alpha1, **{
                                 k: getattr(tp, k) for k in tp.__dataclass_fields__})
        ok = r["flags"] == 0
        assert ok.mean() > 0.95
        assert (b["kind"] == 1).sum() > 50 and (b["kind"] == 2).sum() > 50
        assert np.array_equal(r["kind"][ok], b["kind"][ok])
        assert np.array_equal(r["bits"][ok], b["bits"][ok])
        assert np.allclose(r["W"][ok], b["W"][ok], rtol=1e-12, atol=1e-300)
        assert np.allclose(r["Z"][ok], b["Z"][ok], rtol=1e-12, atol=1e-300)


# --------------------------------------------------------------------------
# NeRF variant (appendix "NeRF-Backbone 3D Fusion Details"; Algorithms
# "Thick-Structure Segmentation via Depth-Weighted Voxel Aggregation" and
# "Thin-Structure Segmentation via Footprint-Based Coverage Analysis")
# --------------------------------------------------------------------------
def _nerf_run(orc, d_min, d_exp, d_max, n=5, mask=1.0, rho=None, nparams=None):
    """The single-voxel setup of the 2DGS pins (x_d = 2.375, centre pixel
    (50, 40) whose centre ray is k = (0.0025, -0.0025, 1), h_v = 1/4,
    footprint pixels 44..55 x 35..46, N = 144)."""
    grid, cam, lin, xd = _tuple_setup()

    def ras(v, dtype=np.float32):
        return np.broadcast_to(np.asarray(v, dtype), (cam.H, cam.W)).copy()
    tup = {"d_min": [ras(d_min)], "d_exp": [ras(d_exp)], "d_max": [ras(d_max)],
           "n_samp": [ras(n, np.uint16)]}
    return orc.fuse_nerf(grid, lin, [cam], tup, [ras(mask)], oracle.MASK_F32, params=P_DEFAULT,
                         nparams=nparams or oracle.NerfParams(),
                         rho=None if rho is None else np.array([rho], np.float64))


def pin_nerf_closed_form(orc):
    f = lambda v: float(np.float32(v))  # noqa: E731  (raster values are FP32)
    k = np.array([0.0025, -0.0025, 1.0])
    p = np.array([0.0, 0.0, 2.375])
    # base: the band contains the projection onto the centre ray, z_c =
    # <p, k> / |k|^2; weight from |z_c - mid| / half-width
    r = _nerf_run(orc, 2.275, 2.375, 2.575)
    zc = p @ k / (k @ k)
    w = math.exp(-0.5 * (abs(zc - 0.5 * (f(2.275) + f(2.575))) / (0.5 * (f(2.575) - f(2.275)))) ** 2)
    assert r["kind"][0, 0] == 1 and math.isclose(r["W"][0], w, rel_tol=1e-12)
    assert math.isclose(r["Z"][0], w, rel_tol=1e-12)
    # a thick vote leaves no thin vote, density or not
    r = _nerf_run(orc, 2.275, 2.375, 2.575, rho=100.0)
    assert r["kind"][0, 0] == 1 and r["Z"][0] == r["W"][0]
    # band beyond the voxel: z_c = d_min, delta = |p - k d_min| ~ 0.3 > tau_spatial =
    # h_v + 0.05 |k| 0.1 (rejected); lambda_range = 1 widens it by |k| 0.1 (accepted,
    # r = 1 exactly: w = exp(-1/2))
    r = _nerf_run(orc, 2.675, 2.375, 2.775)
    assert r["kind"][0, 0] == 0 and r["Z"][0] == 0.0
    delta = np.linalg.norm(p - k * f(2.675))
    assert 0.25 + 0.05 * np.linalg.norm(k) * 0.1 < delta < 0.25 + np.linalg.norm(k) * 0.1
    r = _nerf_run(orc, 2.675, 2.375, 2.775, nparams=oracle.NerfParams(lambda_range=1.0))
    assert r["kind"][0, 0] == 1 and math.isclose(r["W"][0], math.exp(-0.5), rel_tol=1e-9)
    # depth tolerance (gamma + min(beta n, b_max)) h_v against |x_d - d_exp| = 1.2:
    # n = 5 -> 1.25 (accepted), n = 3 -> 1.15, b_max = 0.5 -> 1.125 (rejected)
    assert abs(2.375 - f(3.575)) > 1.15 + 1e-6 and abs(2.375 - f(3.575)) < 1.25 - 1e-6
    assert _nerf_run(orc, 2.275, 3.575, 3.675)["kind"][0, 0] == 1
    assert _nerf_run(orc, 2.275, 3.575, 3.675, n=3)["kind"][0, 0] == 0
    assert _nerf_run(orc, 2.275, 3.575, 3.675,
                     nparams=oracle.NerfParams(b_max=0.5))["kind"][0, 0] == 0
    # thin path: centre mask 0.3 (no thick entry, > m_thin), density 100 >= 50,
    # d_exp at the voxel everywhere; s supportive pixels (m = 1) of N = 144:
    # vote iff s >= 0.2 N = 28.8
    for s, want in ((28, 0), (29, 2)):
        m = np.zeros((80, 100), np.float32)
        m.reshape(-1)[np.ravel_multi_index((np.arange(35, 47).repeat(12)[:s],
                                            np.tile(np.arange(44, 56), 12)[:s]), (80, 100))] = 1.0
        m[40, 50] = 0.3
        r = _nerf_run(orc, 2.275, 2.375, 2.575, mask=m, rho=100.0)
        assert r["kind"][0, 0] == want, (s, r["kind"])
        if want:
            assert r["W"][0] == 1.0 and r["Z"][0] == 1.0
    # coverage is inclusive: rho_cover = 1/4 of N = 144 is exactly 36
    m = np.zeros((80, 100), np.float32)
    m[35:38, 44:56] = 1.0
    m[40, 50] = 0.3
    r = _nerf_run(orc, 2.275, 2.375, 2.575, mask=m, rho=100.0,
                  nparams=oracle.NerfParams(rho_cover=0.25))
    assert r["kind"][0, 0] == 2
    # m_max over the whole box: supportive pixels at 0.7, one unsupported
    # pixel at 0.95 (its d_exp far off) -> t = 0.95
    m = np.full((80, 100), 0.7, np.float32)
    m[40, 50] = 0.3
    m[36, 45] = 0.95
    e = np.full((80, 100), 2.375, np.float32)
    e[36, 45] = 9.0
    r = _nerf_run(orc, 2.275, e, 9.5, mask=m, rho=100.0)
    assert r["kind"][0, 0] == 2 and r["W"][0] == f(0.95) and r["thin"][0, 0] == f(0.95)
    # the thin depth tolerance doubles gamma: (2 gamma + 1) h_v = 2.25 admits
    # |x_d - d_exp| = 2.2; gamma h_v + 0.25 = 1.25 would not
    m = np.ones((80, 100), np.float32)
    m[40, 50] = 0.3
    r = _nerf_run(orc, 2.275, 2.375 + 2.2, 5.0, mask=m, rho=100.0)
    assert r["kind"][0, 0] == 2
    r = _nerf_run(orc, 2.275, 2.375 + 2.3, 5.0, mask=m, rho=100.0)
    assert r["kind"][0, 0] == 0
    # thin eligibility: density below rho_thin, centre mask not above 0.1
    assert _nerf_run(orc, 2.275, 2.375, 2.575, mask=m, rho=49.0)["kind"][0, 0] == 0
    m[40, 50] = np.float32(0.1)
    assert _nerf_run(orc, 2.275, 2.375, 2.575, mask=m, rho=100.0,
                     nparams=oracle.NerfParams(m_thin=float(np.float32(0.1))))["kind"][0, 0] == 0
    # clipped footprint: the camera shifted so the voxel projects to pixel
    # (1, 40): its box covers pixels 0..6 (7 of 12 columns), N = 84; 17 of
    # them supportive is enough (17 >= 16.8), 16 is not
    grid, cam, lin, xd = _tuple_setup()
    cam2 = synth.Camera(cam.R, cam.t, cam.fx, cam.fy, 1.25, cam.cy, cam.W, cam.H)
    for s, want in ((16, 0), (17, 2)):
        m = np.zeros((80, 100), np.float32)
        rows = np.arange(35, 47).repeat(7)[:s]
        cols = np.tile(np.arange(0, 7), 12)[:s]
        m[rows, cols] = 1.0
        m[40, 1] = 0.3  # (rows 35..37 hold the supportive pixels)
        ras = lambda v, dt=np.float32: np.broadcast_to(np.asarray(v, dt), (80, 100)).copy()  # noqa: E731
        tup = {"d_min": [ras(2.275)], "d_exp": [ras(2.375)], "d_max": [ras(2.575)],
               "n_samp": [ras(5, np.uint16)]}
        r = orc.fuse_nerf(grid, lin, [cam2], tup, [m], oracle.MASK_F32, params=P_DEFAULT,
                          nparams=oracle.NerfParams(), rho=np.array([100.0]))
        assert r["kind"][0, 0] == want, (s, r["kind"])


def pin_nerf_bruteforce(orc):
    wl = synth.config2(g=40, W=140, H=105, n_ell=40, n_points=500)
    nw = synth.with_nerf_tuple(wl)
    rho = synth.nerf_density(wl)
    lin = wl.active_linear()
    masks32 = [m.view(np.float16).astype(np.float32) if m.dtype == np.uint16 else m
               for m in wl.mask]
    mt = oracle.MASK_F32 if wl.mask_type == oracle.MASK_F16 else wl.mask_type
    for npar, prm, masks, mtype in [
            (oracle.NerfParams(), P_DEFAULT, wl.mask, wl.mask_type),
            (oracle.NerfParams.mip360(), oracle.Params(tau_m=0.4, alpha1=1.0), masks32, mt),
            (oracle.NerfParams(k_dg=30.0, rho_cover=0.4, tau_thin=0.3), P_DEFAULT,
             [np.log(np.clip(m, 1e-6, 1 - 1e-6) / (1 - np.clip(m, 1e-6, 1 - 1e-6))).astype(np.float32)
              for m in masks32], oracle.MASK_LOGIT_F32)]:
        r = orc.fuse_nerf(wl.grid, lin, wl.cams, nw.tuple, masks, mtype, params=prm,
                          nparams=npar, rho=rho[lin].astype(np.float64))
        b = brute.fuse_nerf(wl.grid, lin, wl.cams, nw.tuple, masks, mtype, rho=rho[lin],
                            tau_m=prm.tau_m, alpha1=prm.alpha1,
                            **{k: getattr(npar, k) for k in npar.__dataclass_fields__})
        ok = r["flags"] == 0
        assert ok.mean() > 0.95
        assert (b["kind"] == 1).sum() > 50 and (b["kind"] == 2).sum() > 20
        assert np.array_equal(r["kind"][ok], b["kind"][ok])
        assert np.array_equal(r["bits"][ok], b["bits"][ok])
        assert np.allclose(r["W"][ok], b["W"][ok], rtol=1e-12, atol=1e-300)
        assert np.allclose(r["Z"][ok], b["Z"][ok], rtol=1e-12, atol=1e-300)


ALL_PINS = [pin_nerf_closed_form, pin_single_view_closed_form, pin_pixel_convention,
            pin_alpha0_mean, pin_invariants, pin_scale_invariance, pin_sphere_scene,
            pin_bruteforce, pin_labels, pin_gradient_fd, pin_tuple_closed_form,
            pin_tuple_bruteforce, pin_nerf_bruteforce]


# --------------------------------------------------------------------------
# near-boundary flags: a decision within 1e-6 (relative to its own scale) of
# flipping is flagged, one farther away is not
# --------------------------------------------------------------------------
FLAG_TUPLE = 32
NEAR, FAR = 0.5e-6, 2e-6


def _flag_probe(orc, cx=16.25, depth=None, mask=1.0):
    grid, cam, lin, p_z = _probe_setup()
    cam = synth.Camera(cam.R, cam.t, cam.fx, cam.fy, float(np.float32(cx)), cam.cy, cam.W, cam.H)
    at = (12, int(math.floor(cx)))
    D = _raster(cam, p_z if depth is None else depth, at)
    M = _raster(cam, mask, at, fill=0.0)
    return orc.fuse(grid, lin, [cam], [D], [M], oracle.MASK_F32, P_DEFAULT), p_z


def pin_near_boundary_flags(orc):
    # pixel: the voxel sits on the optical axis (p_x = 0), so u = cx; a
    # principal point 16 + m (1 + |cx|) above the integer 16 puts u there
    for m, want in ((NEAR, True), (FAR, False)):
        cx = float(np.float32(16.0 + m * 17.0))
        margin = (cx - 16.0) / (1.0 + cx)
        assert (margin < 1e-6) == want
        r, _ = _flag_probe(orc, cx=cx)
        assert bool(r["flags"][0] & oracle.FLAG_PIX) == want, (m, r["flags"])
        assert r["bits"][0] == 1  # the vote itself is unaffected
    # depth gate |e| <= Delta = 1/4, margin ||e| - Delta| / max(p_z, D): the
    # depth just inside and just outside the band, near and far from its edge
    for side in (+1, -1):
        for m, want in ((NEAR, True), (FAR, False)):
            _, p_z = _flag_probe(orc)
            D = float(np.float32(p_z - 0.25 + side * m * p_z))
            margin = abs(abs(p_z - D) - 0.25) / max(p_z, D)
            assert (margin < 1e-6) == want
            r, _ = _flag_probe(orc, depth=D)
            assert bool(r["flags"][0] & oracle.FLAG_DEPTH) == want, (side, m, r["flags"])
            assert r["bits"][0] == (1 if side > 0 else 0)
    # consensus P >= tau_cons: one view votes, so P = m exactly
    for m, want in ((NEAR, True), (FAR, False)):
        mk = float(np.float32(0.5 + m))
        r, _ = _flag_probe(orc, mask=mk)
        assert r["P"][0] == mk and bool(r["flags"][0] & oracle.FLAG_CONS) == want
    # 2DGS thin path, distance gate dist_gate h_v against the nearest
    # mask-positive unprojection (the 8 x 8 mask hole of pin_tuple_closed_form:
    # untrusted everywhere, so every pixel unprojects at d_med = 2.375 and the
    # distance is 2.375 |((x + 1/2 - cx) / fx, (y + 1/2 - cy) / fy)|)
    grid, cam, lin, xd = _tuple_setup()
    mk = np.ones((80, 100), np.float32)
    mk[37:45, 46:54] = 0.0
    d_med = float(np.float32(2.375))
    best = min(d_med * math.hypot((x + 0.5 - 50.25) / 100.0, (y + 0.5 - 40.75) / 100.0)
               for y in range(35, 47) for x in range(44, 56) if mk[y, x] > 0.5)
    for m, want in ((NEAR, True), (FAR, False)):
        for side, vote in ((+1, 2), (-1, 0)):
            gate = best * (1.0 + side * m)
            r, _ = _tuple_run(orc, 2.475, 2.375, 2.575, mask=mk,
                              tparams=oracle.TupleParams(dist_gate=gate / 0.25))
            assert bool(r["flags"][0] & FLAG_TUPLE) == want, (m, side, r["flags"])
            assert r["kind"][0, 0] == vote
    # NeRF thick path, spatial gate delta = |p - k d_min| (the band lies
    # beyond the voxel, z_c = d_min) against tau = h_v + lambda |k| (d_max - d_min)
    f = lambda v: float(np.float32(v))  # noqa: E731
    k = np.array([0.0025, -0.0025, 1.0])
    p = np.array([0.0, 0.0, 2.375])
    delta = float(np.linalg.norm(p - k * f(2.675)))
    band = f(2.775) - f(2.675)
    for m, want in ((NEAR, True), (FAR, False)):
        for side, vote in ((+1, 1), (-1, 0)):
            lam = (delta * (1.0 + side * m) - 0.25) / (np.linalg.norm(k) * band)
            r = _nerf_run(orc, 2.675, 2.375, 2.775, nparams=oracle.NerfParams(lambda_range=lam))
            assert bool(r["flags"][0] & FLAG_TUPLE) == want, (m, side, r["flags"])
            assert r["kind"][0, 0] == vote


ALL_PINS.append(pin_near_boundary_flags)
