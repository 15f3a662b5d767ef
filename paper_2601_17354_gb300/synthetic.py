"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module only draws numbers: it holds none of the rasterizer's arithmetic (no projection,
no spherical-harmonic evaluation, no compositing).  Every array is numpy float32 in the planar
structure-of-arrays layout the library takes:

    means          [3][N]       world position
    log_scales     [3][N]       per-axis log standard deviation
    quats          [4][N]       unnormalised rotation quaternion (w, x, y, z)
    opacity_logits [N]          logit of the opacity
    sh             [3][K][N]    colour coefficients, channel-major, K = (degree + 1)^2

Cameras are pinhole with OpenCV axes (x right, y down, z forward); ``viewmat`` is the row-major
3x4 world-to-camera matrix [R | t].

The workloads stand in for the paper's captured scenes (LLFF, Mip-NeRF 360 and the authors'
phone captures, 18k-168k Gaussians per scene in Table I), which are not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# The degree-0 spherical-harmonic basis function is the constant 1/sqrt(4*pi); a DC coefficient
# drawn from this symmetric range therefore gives a degree-0 colour (coefficient * basis + 0.5)
# uniform in [0, 1].
_DC_HALF_RANGE = 0.5 * math.sqrt(4.0 * math.pi)


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray  # float32 [3, 4] world -> camera
    near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """The same camera restricted to the pixel window [x0, x0+w) x [y0, y0+h).

        Shifting the principal point by the window origin keeps every pixel centre at the same
        ray, so with x0, y0 multiples of the tile size the tile membership is unchanged.
        """
        return Camera(w, h, self.fx, self.fy, self.cx - x0, self.cy - y0,
                      self.viewmat.copy(), self.near, self.bg)


@dataclass
class Gaussians:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def arrays(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logits, self.sh]

    def copy(self) -> "Gaussians":
        return Gaussians(*[a.copy() for a in self.arrays()], self.sh_degree, dict(self.extra))

    def subset(self, idx) -> "Gaussians":
        idx = np.asarray(idx)
        return Gaussians(np.ascontiguousarray(self.means[:, idx]),
                         np.ascontiguousarray(self.log_scales[:, idx]),
                         np.ascontiguousarray(self.quats[:, idx]),
                         np.ascontiguousarray(self.opacity_logits[idx]),
                         np.ascontiguousarray(self.sh[:, :, idx]), self.sh_degree)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def lookat_viewmat(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World-to-camera [R | t] for a camera at ``eye`` looking at ``target`` (OpenCV axes)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    return _f32(np.concatenate([R, t[:, None]], axis=1))


def random_params(rng: np.random.Generator, means: np.ndarray, sh_degree: int,
                  log_scale_mean: float, log_scale_std: float,
                  logit_mean: float, logit_std: float, rest_std: float) -> Gaussians:
    """Gaussian attributes drawn around given centres [3][N]."""
    n = means.shape[1]
    k = (sh_degree + 1) ** 2
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(3, n))
    quats = rng.normal(size=(4, n))
    logits = rng.normal(logit_mean, logit_std, size=n)
    sh = np.zeros((3, k, n))
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, size=(3, n))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, size=(3, k - 1, n))
    return Gaussians(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), sh_degree)


# ----------------------------------------------------------------------------------------------
# Tiny workload: 2,000 Gaussians, SH degree 0, 128x128, fx = fy = 150
# ----------------------------------------------------------------------------------------------

def tiny_scene(seed: int = 0, n: int = 2000, width: int = 128, height: int = 128,
               focal: float = 150.0):
    """Uniform cloud in [-1,1]^3 seen from distance 3, with a random-uniform target image.

    Means U[-1,1]^3; log-scales N(-3, 0.3); quaternions N(0, I4) (unnormalised); opacity
    logits N(0, 1); degree-0 colour uniform in [0, 1]; black background.
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(3, n))
    g = random_params(rng, means, 0, -3.0, 0.3, 0.0, 1.0, 0.0)
    view = np.zeros((3, 4), np.float32)
    view[0, 0] = view[1, 1] = view[2, 2] = 1.0
    view[2, 3] = 3.0  # camera centre at (0, 0, -3), looking along +z at the origin
    cam = Camera(width, height, focal, focal, width / 2.0, height / 2.0, view)
    target = _f32(rng.uniform(0.0, 1.0, size=(3, height, width)))
    return g, cam, target


# ----------------------------------------------------------------------------------------------
# Surface scenes: points on 8 random spheres and 4 random square planes inside [-2, 2]^3
# ----------------------------------------------------------------------------------------------

@dataclass
class Surfaces:
    sphere_c: np.ndarray  # [8, 3]
    sphere_r: np.ndarray  # [8]
    plane_c: np.ndarray   # [4, 3]
    plane_u: np.ndarray   # [4, 3] in-plane unit axis
    plane_v: np.ndarray   # [4, 3] in-plane unit axis
    plane_side: np.ndarray  # [4]

    def areas(self) -> np.ndarray:
        return np.concatenate([4.0 * np.pi * self.sphere_r ** 2, self.plane_side ** 2])


def random_surfaces(rng: np.random.Generator, n_spheres: int = 8, n_planes: int = 4) -> Surfaces:
    sc = rng.uniform(-1.5, 1.5, size=(n_spheres, 3))
    sr = rng.uniform(0.2, 0.8, size=n_spheres)
    pc = rng.uniform(-1.5, 1.5, size=(n_planes, 3))
    normal = rng.normal(size=(n_planes, 3))
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    helper = rng.normal(size=(n_planes, 3))
    u = np.cross(normal, helper)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(normal, u)
    side = rng.uniform(0.5, 2.0, size=n_planes)
    return Surfaces(sc, sr, pc, u, v, side)


def sample_surface_points(rng: np.random.Generator, surf: Surfaces, n: int) -> np.ndarray:
    """n points on the surfaces, allocated in proportion to area, all inside [-2, 2]^3; [3][n]."""
    areas = surf.areas()
    prob = areas / areas.sum()
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 1.3) + 64
        which = rng.choice(len(prob), size=m, p=prob)
        pts = np.empty((m, 3))
        ns = len(surf.sphere_r)
        is_sphere = which < ns
        k = int(is_sphere.sum())
        if k:
            d = rng.normal(size=(k, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            idx = which[is_sphere]
            pts[is_sphere] = surf.sphere_c[idx] + surf.sphere_r[idx, None] * d
        if m - k:
            idx = which[~is_sphere] - ns
            a = rng.uniform(-0.5, 0.5, size=(m - k, 1)) * surf.plane_side[idx, None]
            b = rng.uniform(-0.5, 0.5, size=(m - k, 1)) * surf.plane_side[idx, None]
            pts[~is_sphere] = surf.plane_c[idx] + a * surf.plane_u[idx] + b * surf.plane_v[idx]
        inside = np.all(np.abs(pts) <= 2.0, axis=1)
        out = np.concatenate([out, pts[inside]], axis=0)
    return np.ascontiguousarray(out[:n].T)


def ring_cameras(rng: np.random.Generator, count: int, width: int, height: int, focal: float,
                 radius: float = 4.0, max_elev_deg: float = 10.0):
    """``count`` cameras evenly spaced in azimuth on a ring of ``radius`` in the world xy-plane,
    elevation jittered uniformly in +-max_elev_deg, z up, all looking at the origin."""
    cams = []
    elev = np.deg2rad(rng.uniform(-max_elev_deg, max_elev_deg, size=count))
    for i in range(count):
        az = 2.0 * np.pi * i / count
        eye = radius * np.array([np.cos(az) * np.cos(elev[i]), np.sin(az) * np.cos(elev[i]),
                                 np.sin(elev[i])])
        cams.append(Camera(width, height, focal, focal, width / 2.0, height / 2.0,
                           lookat_viewmat(eye)))
    return cams


@dataclass
class SurfaceScene:
    gt: Gaussians          # hidden ground-truth Gaussians
    init: Gaussians        # trainable starting point (noisy resampled surface points)
    cameras: list          # ring cameras
    surfaces: Surfaces

    def train_views(self):
        return [i for i in range(len(self.cameras)) if i % 8 != 0]

    def test_views(self):
        return [i for i in range(len(self.cameras)) if i % 8 == 0]


def surface_scene(seed: int, n: int, sh_degree: int = 3, width: int = 1280, height: int = 720,
                  focal: float = 1000.0, n_cameras: int = 64, n_init: int | None = None,
                  position_noise: float = 0.01) -> SurfaceScene:
    """Ground-truth Gaussians on 8 spheres + 4 planes, ring cameras, and a trainable start.

    GT attributes: log-scales N(-4, 0.3), random rotations, opacity logits N(1, 0.5), DC colour
    uniform in [0, 1], higher bands N(0, 0.05).  The trainable set starts from freshly sampled
    points on the same surfaces with N(0, position_noise) noise and the same attribute laws
    (an initializer may overwrite scales, rotations and opacities).
    """
    rng = np.random.default_rng(seed)
    surf = random_surfaces(rng)
    gt_pts = sample_surface_points(rng, surf, n)
    gt = random_params(rng, gt_pts, sh_degree, -4.0, 0.3, 1.0, 0.5, 0.05)
    ni = n if n_init is None else n_init
    init_pts = sample_surface_points(rng, surf, ni) + rng.normal(0.0, position_noise, size=(3, ni))
    init = random_params(rng, init_pts, sh_degree, -4.0, 0.3, 1.0, 0.5, 0.05)
    cams = ring_cameras(rng, n_cameras, width, height, focal)
    return SurfaceScene(gt, init, cams, surf)


def random_image(seed: int, width: int, height: int, low: float = -1.0, high: float = 1.0):
    """A seeded [3][H][W] float32 field, e.g. an upstream gradient dL/dimage."""
    rng = np.random.default_rng(seed)
    return _f32(rng.uniform(low, high, size=(3, height, width)))


def batched_scenes(seed: int, n_scenes: int = 16, views_per_scene: int = 4,
                   n_range=(20_000, 300_000), resolutions=((640, 480), (960, 720), (1280, 720)),
                   sh_degree: int = 3):
    """Uneven batch: per scene a log-uniform Gaussian count and a resolution drawn from the list;
    focal length scaled with the width so the field of view matches the 1280x720, fx=1000 scene."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scenes):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        focal = 1000.0 * w / 1280.0
        sc = surface_scene(int(rng.integers(1 << 31)), n, sh_degree, w, h, focal,
                           n_cameras=views_per_scene)
        out.append(sc)
    return out


@dataclass
class BAProblem:
    """Bundle-adjustment inputs drawn for the geometry prior (Sec. III-A): ground-truth ring cameras
    and surface points, their perturbed starting values, per (camera, point) pixel noise, and per
    point a feature track over consecutive cameras (start, length), as a tracker following a
    feature through a keyframe sequence would give.  Which pairs are observed and where (the
    projection) is left to the caller."""
    K: tuple                 # (fx, fy, cx, cy)
    width: int
    height: int
    R_gt: np.ndarray         # [C][3][3] world -> camera rotations
    t_gt: np.ndarray         # [C][3]
    P_gt: np.ndarray         # [n][3]
    R_init: np.ndarray       # [C][3][3] = small random rotation @ R_gt (camera 0 exact)
    t_init: np.ndarray       # [C][3]
    P_init: np.ndarray       # [n][3]
    noise: np.ndarray        # [C][n][2] pixel noise, sigma `pixel_sigma`
    pixel_sigma: float
    track_start: np.ndarray  # [n] first camera of the point's feature track
    track_len: np.ndarray    # [n] track length in consecutive cameras (2..12)


def _small_rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    """Rotation matrix of a random unit quaternion within about max_deg of the identity."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    half = 0.5 * np.deg2rad(rng.uniform(0.0, max_deg))
    w, (x, y, z) = np.cos(half), np.sin(half) * axis
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def ba_problem(seed: int, n_cams: int = 32, n_points: int = 20000, width: int = 1280, height: int = 720,
               focal: float = 1000.0, rot_deg: float = 0.5, trans: float = 0.02, point: float = 0.01,
               pixel_sigma: float = 0.5) -> BAProblem:
    rng = np.random.default_rng(seed)
    cams = ring_cameras(rng, n_cams, width, height, focal)
    R = np.array([c.viewmat[:, :3] for c in cams], np.float64)
    t = np.array([c.viewmat[:, 3] for c in cams], np.float64)
    P = sample_surface_points(rng, random_surfaces(rng), n_points).T.astype(np.float64)
    Rp = np.array([R[i] if i == 0 else _small_rotation(rng, rot_deg) @ R[i] for i in range(n_cams)])
    tp = t + np.vstack([np.zeros(3), rng.normal(0.0, trans, (n_cams - 1, 3))])
    Pp = P + rng.normal(0.0, point, P.shape)
    noise = rng.normal(0.0, pixel_sigma, (n_cams, n_points, 2))
    track_start = rng.integers(0, n_cams, n_points)
    track_len = rng.integers(2, 13, n_points)
    return BAProblem((focal, focal, width / 2.0, height / 2.0), width, height, R, t, P, Rp, tp, Pp,
                     noise, pixel_sigma, track_start, track_len)


# ------------------------------------------------------------------------------------------------
# Multi-view stereo inputs: textured analytic surfaces seen by ring keyframes
# ------------------------------------------------------------------------------------------------
@dataclass
class MVSScene:
    """Keyframe images of textured spheres and squares, their exact depth maps, and sparse surface
    points standing in for the bundle-adjusted points (Sec. III-A).  The images come from ray
    casting the analytic surfaces (pixel-centre rays, nearest hit), so they are exact data for
    both the CUDA path and the oracle and the depth maps are the ground truth."""
    surfaces: Surfaces
    cameras: list            # ring keyframes
    images: list             # [3][H][W] float32 per camera (None where not rendered)
    depths: list             # [H][W] float64 camera-z of the visible surface, inf on background
    sparse: np.ndarray       # [n][3] float64 surface points with N(0, 0.005) noise


def _hash_cells(ix, iy, iz, salt):
    """Deterministic pseudo-random values in [0, 1) of integer lattice cells (a multiply-xorshift
    mix of the three cell indices)."""
    h = (ix.astype(np.int64) * 73856093) ^ (iy.astype(np.int64) * 19349663) ^ (iz.astype(np.int64) * 83492791)
    h = (h ^ salt) & 0xFFFFFFFF
    h = (h * 0x45D9F3B) & 0xFFFFFFFF
    h = ((h >> 16) ^ h) * 0x45D9F3B & 0xFFFFFFFF
    h = (h >> 16) ^ h
    return (h & 0xFFFFFF) / float(1 << 24)


def surface_texture(points: np.ndarray, surface_id: np.ndarray, tints: np.ndarray) -> np.ndarray:
    """RGB [n][3] of surface points: a per-surface tint times two octaves of cell noise (cells of
    0.02 and 0.05 world units), in [0.15, 1]."""
    fine = _hash_cells(*np.floor(points / 0.02).T.astype(np.int64), 17)
    coarse = _hash_cells(*np.floor(points / 0.05).T.astype(np.int64), 29)
    lum = 0.15 + 0.85 * (0.6 * fine + 0.4 * coarse)
    return lum[:, None] * tints[surface_id]


def cast_surfaces(surf: Surfaces, cam: Camera):
    """Ray-cast the surfaces through every pixel centre of ``cam``: (hit points [H*W][3], camera-z
    depth [H*W] (inf on background), surface index [H*W] (-1 on background))."""
    H, W = cam.height, cam.width
    R = cam.viewmat[:, :3].astype(np.float64)
    t = cam.viewmat[:, 3].astype(np.float64)
    eye = -R.T @ t
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dirs_c = np.stack([(xs - cam.cx) / cam.fx, (ys - cam.cy) / cam.fy, np.ones_like(xs)], axis=-1).reshape(-1, 3)
    dirs = dirs_c @ R                      # world directions with camera-z component 1
    best = np.full(H * W, np.inf)
    sid = np.full(H * W, -1)
    for k in range(len(surf.sphere_r)):
        oc = eye - surf.sphere_c[k]
        a = np.einsum("ij,ij->i", dirs, dirs)
        b = 2.0 * dirs @ oc
        c = oc @ oc - surf.sphere_r[k] ** 2
        disc = b * b - 4 * a * c
        ok = disc > 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t0 = (-b - sq) / (2 * a)
        t1 = (-b + sq) / (2 * a)
        tt = np.where(t0 > 1e-6, t0, t1)
        hit = ok & (tt > 1e-6) & (tt < best)
        best = np.where(hit, tt, best)
        sid = np.where(hit, k, sid)
    ns = len(surf.sphere_r)
    for k in range(len(surf.plane_side)):
        n = np.cross(surf.plane_u[k], surf.plane_v[k])
        den = dirs @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            tt = ((surf.plane_c[k] - eye) @ n) / den
        p = eye + tt[:, None] * dirs
        du = (p - surf.plane_c[k]) @ surf.plane_u[k]
        dv = (p - surf.plane_c[k]) @ surf.plane_v[k]
        half = 0.5 * surf.plane_side[k]
        hit = (np.abs(den) > 1e-12) & (tt > 1e-6) & (np.abs(du) <= half) & (np.abs(dv) <= half) & (tt < best)
        best = np.where(hit, tt, best)
        sid = np.where(hit, ns + k, sid)
    pts = eye + np.where(np.isfinite(best), best, 0.0)[:, None] * dirs
    return pts, best, sid   # dirs have camera-z 1, so the ray parameter is the camera-z depth


def mvs_scene(seed: int, n_cameras: int = 64, width: int = 640, height: int = 360, focal: float = 500.0,
              n_sparse: int = 20000, views=None) -> MVSScene:
    """Ring keyframes (as the surface scene, 640 x 360 at fx = 500: the 1280 x 720 keyframes at half
    resolution) of 8 textured spheres and 4 textured squares; images and depth maps for ``views``
    (all cameras by default)."""
    rng = np.random.default_rng(seed)
    surf = random_surfaces(rng)
    tints = rng.uniform(0.4, 1.0, size=(len(surf.sphere_r) + len(surf.plane_side), 3))
    cams = ring_cameras(rng, n_cameras, width, height, focal)
    sparse = sample_surface_points(rng, surf, n_sparse).T + rng.normal(0.0, 0.005, size=(n_sparse, 3))
    images, depths = [None] * n_cameras, [None] * n_cameras
    for i in (range(n_cameras) if views is None else views):
        pts, depth, sid = cast_surfaces(surf, cams[i])
        rgb = np.zeros((height * width, 3))
        hit = sid >= 0
        rgb[hit] = surface_texture(pts[hit], sid[hit], tints)
        images[i] = _f32(rgb.reshape(height, width, 3).transpose(2, 0, 1))
        depths[i] = depth.reshape(height, width)
    return MVSScene(surf, cams, images, depths, sparse)
