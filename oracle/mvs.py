"""CPU oracle of the single-reference cost-volume MVS of the geometry prior (Sec. III-A: depth
range from the projected sparse points, reference view by Eq. 4, census matching cost, plane
sweep, SGM aggregation, confidence filter, fusion into points) -- TEST INFRASTRUCTURE ONLY
(imported by the tests and the benchmark's CPU-baseline leg, never by the product path).

The paper names the ingredients and two numbers (the range rule [0.5 q.05, 1.5 q.95] and the
confidence threshold 0.4); everything else is a reading, shared with the CUDA path:

  luma        Y = 0.299 R + 0.587 G + 0.114 B (Rec. 601), FP32, each product and sum rounded;
  census      7 x 7 window, 48 bits in raster order of the neighbours (centre skipped), bit set
              when the neighbour is darker than the centre; neighbours outside the image leave
              their bit clear;
  hypotheses  D fronto-parallel planes of the target camera, uniform in inverse depth from
              1/d_max (k = 0) to 1/d_min (k = D - 1);
  plane map   H_k = K_r (R + t n^T / d_k) K_t^-1 with n = e3 and (R, t) the target-to-reference
              motion, built in FP64 in the order written below and rounded to FP32; a target pixel
              centre (x + 0.5, y + 0.5) maps through H_k in FP32 (products and sums rounded, no
              fusion, IEEE division) and takes the reference pixel whose [i, i + 1) square holds the
              result;
  cost        Hamming distance of the two census codes (0..48); 24 when the point is behind the
              reference camera or outside its image;
  SGM         4 paths (left to right, right to left, top down, bottom up), P1 = 8, P2 = 32,
              L(p, k) = C(p, k) + min(L(q, k), L(q, k -+ 1) + P1, min_i L(q, i) + P2) - min_i L(q, i)
              for the previous pixel q on the path (L = C at the path's first pixel); S = sum of the
              four L (integers throughout);
  depth       k* = first minimiser of S; S2 = the smallest S over |k - k*| >= 2; kept when
              0 < k* < D - 1 and 1 - S(k*) / S2 >= 0.4, decided as 5 (S2 - S1) >= 2 S2 in integers;
              sub-plane refinement by the parabola through k* - 1, k*, k* + 1 in inverse depth
              (offset in FP32, depth in FP64);
  fusion      kept pixels back-projected to world points (FP64, rounded to FP32), all targets
              concatenated;
  range       camera-z of the sparse points in front (z > 0.2) and inside the target image,
              quantiles with linear interpolation between order statistics; [0.5 q.05, 1.5 q.95];
  reference   Eq. 4 with b the distance between camera centres, b_target = 0.1 x the median
              sparse depth of the target, sigma_b = 0.5 b_target, alpha the angle between the two
              optical axes and alpha_min = 5 degrees; the best other keyframe (ties: lowest index).

Parity status: pinned by census invariance to increasing intensity maps and its closed form on a
single bright pixel, the plane map against direct projection of points on each plane, zero cost
for a view paired with itself, SGM against brute-force minimisation over label sequences on tiny
rows and its P1 = P2 = 0 special case, the parabola's exactness on quadratic costs, the range
quantiles against numpy.quantile, and the fused depths against the ray-cast ground truth of the
synthetic scene.
"""
from __future__ import annotations

import math

import numpy as np

RADIUS = 3
INVALID = 24
P1 = 8
P2 = 32
NEAR = 0.2
B_TARGET_FRACTION = 0.1
SIGMA_B_FRACTION = 0.5
ALPHA_MIN = math.radians(5.0)
CONF = 0.4

f32 = np.float32


def luma(rgb: np.ndarray) -> np.ndarray:
    r, g, b = (np.asarray(rgb[c], f32) for c in range(3))
    return (f32(0.299) * r + f32(0.587) * g) + f32(0.114) * b


def census(Y: np.ndarray) -> np.ndarray:
    """uint64 codes [H][W]."""
    H, W = Y.shape
    pad = np.full((H + 2 * RADIUS, W + 2 * RADIUS), np.inf, f32)   # outside: never darker
    pad[RADIUS:RADIUS + H, RADIUS:RADIUS + W] = Y
    code = np.zeros((H, W), np.uint64)
    bit = 0
    for dy in range(-RADIUS, RADIUS + 1):
        for dx in range(-RADIUS, RADIUS + 1):
            if dy == 0 and dx == 0:
                continue
            nb = pad[RADIUS + dy:RADIUS + dy + H, RADIUS + dx:RADIUS + dx + W]
            code |= (nb < Y).astype(np.uint64) << np.uint64(bit)
            bit += 1
    return code


def inverse_depths(d_min: float, d_max: float, D: int):
    """(inv_far, step): inverse depth of plane k is inv_far + k step."""
    inv_far = 1.0 / d_max
    inv_near = 1.0 / d_min
    return inv_far, (inv_near - inv_far) / (D - 1)


def relative_pose(view_t: np.ndarray, view_r: np.ndarray):
    """Target-camera to reference-camera motion from two world-to-camera [R | t] (FP32 inputs),
    in FP64 with left-to-right sums: R = R_r R_t^T, t = t_r - R t_t."""
    Rt = [[float(view_t[i][j]) for j in range(3)] for i in range(3)]
    tt = [float(view_t[i][3]) for i in range(3)]
    Rr = [[float(view_r[i][j]) for j in range(3)] for i in range(3)]
    tr = [float(view_r[i][3]) for i in range(3)]
    R = [[(Rr[i][0] * Rt[j][0] + Rr[i][1] * Rt[j][1]) + Rr[i][2] * Rt[j][2] for j in range(3)] for i in range(3)]
    t = [tr[i] - ((R[i][0] * tt[0] + R[i][1] * tt[1]) + R[i][2] * tt[2]) for i in range(3)]
    return R, t


def plane_maps(cam_t, cam_r, inv_far: float, step: float, D: int) -> np.ndarray:
    """H_k [D][9] FP32 (row-major) for the D planes."""
    R, t = relative_pose(cam_t.viewmat, cam_r.viewmat)
    fxt, fyt, cxt, cyt = (float(f32(v)) for v in (cam_t.fx, cam_t.fy, cam_t.cx, cam_t.cy))
    fxr, fyr, cxr, cyr = (float(f32(v)) for v in (cam_r.fx, cam_r.fy, cam_r.cx, cam_r.cy))
    ax, ay = cxt / fxt, cyt / fyt
    out = np.zeros((D, 9), f32)
    for k in range(D):
        inv = inv_far + k * step
        g = []
        for i in range(3):
            m0, m1, m2 = R[i][0], R[i][1], R[i][2] + t[i] * inv
            g.append((m0 / fxt, m1 / fyt, (m2 - m0 * ax) - m1 * ay))
        h = [[fxr * g[0][j] + cxr * g[2][j] for j in range(3)],
             [fyr * g[1][j] + cyr * g[2][j] for j in range(3)],
             [g[2][j] for j in range(3)]]
        out[k] = np.array(h, np.float64).reshape(9).astype(f32)
    return out


def _popcount64(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64)
    c = np.zeros(x.shape, np.int64)
    for s in range(0, 64, 8):
        c += np.array([bin(v).count("1") for v in range(256)], np.int64)[((x >> np.uint64(s)) & np.uint64(255)).astype(np.int64)]
    return c


def map_pixels(Hk: np.ndarray, W_t: int, H_t: int, W_r: int, H_r: int):
    """The reference pixel (iu, iv) of every target pixel centre under one FP32 plane map, and
    whether it is valid (in front, inside the reference image)."""
    h = [f32(v) for v in Hk]
    xc = (np.arange(W_t, dtype=f32) + f32(0.5))[None, :].repeat(H_t, 0)
    yc = (np.arange(H_t, dtype=f32) + f32(0.5))[:, None].repeat(W_t, 1)
    a = (h[0] * xc + h[1] * yc) + h[2]
    b = (h[3] * xc + h[4] * yc) + h[5]
    c = (h[6] * xc + h[7] * yc) + h[8]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        u = a / c
        v = b / c
        ok = (c > 0) & (u >= 0) & (u < f32(W_r)) & (v >= 0) & (v < f32(H_r))
    iu = np.where(ok, np.floor(np.where(ok, u, 0)), 0).astype(np.int64)
    iv = np.where(ok, np.floor(np.where(ok, v, 0)), 0).astype(np.int64)
    return iu, iv, ok


def cost_volume(cen_t: np.ndarray, cen_r: np.ndarray, maps: np.ndarray) -> np.ndarray:
    """uint8 [H][W][D]."""
    H, W = cen_t.shape
    Hr, Wr = cen_r.shape
    D = maps.shape[0]
    C = np.empty((H, W, D), np.uint8)
    for k in range(D):
        iu, iv, ok = map_pixels(maps[k], W, H, Wr, Hr)
        ham = _popcount64(cen_t ^ cen_r[iv, iu])
        C[:, :, k] = np.where(ok, ham, INVALID)
    return C


def sgm_path(C: np.ndarray, p1: int = P1, p2: int = P2) -> np.ndarray:
    """One left-to-right path over every row of C [H][W][D] (int64 L)."""
    H, W, D = C.shape
    L = np.zeros((H, W, D), np.int64)
    L[:, 0] = C[:, 0]
    big = np.iinfo(np.int64).max // 4
    for x in range(1, W):
        prev = L[:, x - 1]
        m = prev.min(axis=1, keepdims=True)
        up = np.concatenate([prev[:, 1:], np.full((H, 1), big)], axis=1) + p1
        dn = np.concatenate([np.full((H, 1), big), prev[:, :-1]], axis=1) + p1
        best = np.minimum(np.minimum(prev, np.minimum(up, dn)), m + p2)
        L[:, x] = C[:, x].astype(np.int64) + best - m
    return L


def sgm(C: np.ndarray, p1: int = P1, p2: int = P2) -> np.ndarray:
    """S = sum of the four paths, uint16 [H][W][D]."""
    S = sgm_path(C, p1, p2)                                                  # left to right
    S += sgm_path(C[:, ::-1], p1, p2)[:, ::-1]                               # right to left
    S += sgm_path(C.transpose(1, 0, 2), p1, p2).transpose(1, 0, 2)           # top down
    S += sgm_path(C[::-1].transpose(1, 0, 2), p1, p2).transpose(1, 0, 2)[::-1]   # bottom up
    return S.astype(np.uint16)


def select_depth(S: np.ndarray, inv_far: float, step: float):
    """(k* [H][W], kept [H][W] bool, depth [H][W] float32 (nan where not kept))."""
    H, W, D = S.shape
    Si = S.astype(np.int64)
    k1 = Si.argmin(axis=2)
    s1 = np.take_along_axis(Si, k1[:, :, None], axis=2)[:, :, 0]
    ks = np.arange(D)[None, None, :]
    far = np.abs(ks - k1[:, :, None]) >= 2
    s2 = np.where(far, Si, np.iinfo(np.int64).max).min(axis=2)
    s2 = np.where(s2 == np.iinfo(np.int64).max, s1, s2)
    kept = (k1 > 0) & (k1 < D - 1) & (s2 > 0) & (5 * (s2 - s1) >= 2 * s2)
    depth = np.full((H, W), np.nan, f32)
    km = np.clip(k1 - 1, 0, D - 1)
    kp = np.clip(k1 + 1, 0, D - 1)
    sm = np.take_along_axis(Si, km[:, :, None], axis=2)[:, :, 0]
    sp = np.take_along_axis(Si, kp[:, :, None], axis=2)[:, :, 0]
    den = sm - 2 * s1 + sp
    with np.errstate(divide="ignore", invalid="ignore"):
        delta = np.where(den > 0, f32(1) * (sm - sp).astype(f32) / (f32(2) * den.astype(f32)), f32(0)).astype(f32)
    inv = inv_far + (k1.astype(np.float64) + delta.astype(np.float64)) * step
    depth[kept] = (1.0 / inv[kept]).astype(f32)
    return k1, kept, depth


def back_project(depth: np.ndarray, cam) -> tuple[np.ndarray, np.ndarray]:
    """World points [n][3] float32 of the finite depths, and their pixel indices (row-major)."""
    H, W = depth.shape
    idx = np.nonzero(np.isfinite(depth).ravel())[0]
    y, x = idx // W, idx % W
    d = depth.ravel()[idx].astype(np.float64)
    fx, fy, cx, cy = (float(f32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    R = [[float(cam.viewmat[i][j]) for j in range(3)] for i in range(3)]
    t = [float(cam.viewmat[i][3]) for i in range(3)]
    X = [d * (((x + 0.5) - cx) / fx) - t[0], d * (((y + 0.5) - cy) / fy) - t[1], d - t[2]]
    P = np.stack([(R[0][j] * X[0] + R[1][j] * X[1]) + R[2][j] * X[2] for j in range(3)], axis=1)
    return P.astype(f32), idx


def sparse_depths(points: np.ndarray, cam) -> np.ndarray:
    """Camera-z (FP64) of the FP32 sparse points in front of the camera (z > 0.2) whose projection
    falls inside the image, in point order."""
    P = np.asarray(points, f32).astype(np.float64)
    R = [[float(cam.viewmat[i][j]) for j in range(3)] for i in range(3)]
    t = [float(cam.viewmat[i][3]) for i in range(3)]
    Xc = [((R[i][0] * P[:, 0] + R[i][1] * P[:, 1]) + R[i][2] * P[:, 2]) + t[i] for i in range(3)]
    fx, fy, cx, cy = (float(f32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    z = Xc[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * (Xc[0] / z) + cx
        v = fy * (Xc[1] / z) + cy
    ok = (z > NEAR) & (u >= 0) & (u < cam.width) & (v >= 0) & (v < cam.height)
    return z[ok]


def quantile(values: np.ndarray, p: float) -> float:
    """Linear interpolation between the order statistics at floor(h) and floor(h) + 1,
    h = (n - 1) p."""
    s = np.sort(values)
    h = (len(s) - 1) * p
    lo = int(math.floor(h))
    hi = min(lo + 1, len(s) - 1)
    return float(s[lo] + (h - lo) * (s[hi] - s[lo]))


def depth_range(points: np.ndarray, cam):
    """(d_min, d_max, median) of the target from the sparse points."""
    z = sparse_depths(points, cam)
    return 0.5 * quantile(z, 0.05), 1.5 * quantile(z, 0.95), quantile(z, 0.5)


def reference_scores(cams, target: int, median_depth: float) -> np.ndarray:
    """Eq. 4 score of every keyframe as the reference of `target` (-inf for the target)."""
    def centre_axis(c):
        R = [[float(c.viewmat[i][j]) for j in range(3)] for i in range(3)]
        t = [float(c.viewmat[i][3]) for i in range(3)]
        ctr = [-((R[0][j] * t[0] + R[1][j] * t[1]) + R[2][j] * t[2]) for j in range(3)]
        return ctr, R[2]
    ct, at = centre_axis(cams[target])
    bt = B_TARGET_FRACTION * median_depth
    sb = SIGMA_B_FRACTION * bt
    out = np.full(len(cams), -np.inf)
    for j, c in enumerate(cams):
        if j == target:
            continue
        cj, aj = centre_axis(c)
        b = math.sqrt(((cj[0] - ct[0]) ** 2 + (cj[1] - ct[1]) ** 2) + (cj[2] - ct[2]) ** 2)
        cosang = (aj[0] * at[0] + aj[1] * at[1]) + aj[2] * at[2]
        alpha = math.acos(max(-1.0, min(1.0, cosang)))
        out[j] = math.exp(-((b - bt) ** 2) / (2.0 * sb * sb)) * max(alpha / ALPHA_MIN, 1.0)
    return out


def reconstruct_view(images, cams, points, target: int, D: int = 64):
    """The whole single-reference MVS of one target keyframe: (reference index, (d_min, d_max),
    S [H][W][D], k*, kept, depth, world points, pixel indices)."""
    d_min, d_max, med = depth_range(points, cams[target])
    ref = int(np.argmax(reference_scores(cams, target, med)))
    inv_far, step = inverse_depths(d_min, d_max, D)
    maps = plane_maps(cams[target], cams[ref], inv_far, step, D)
    C = cost_volume(census(luma(images[target])), census(luma(images[ref])), maps)
    S = sgm(C)
    k1, kept, depth = select_depth(S, inv_far, step)
    P, idx = back_project(depth, cams[target])
    return ref, (d_min, d_max), C, S, k1, kept, depth, P, idx
