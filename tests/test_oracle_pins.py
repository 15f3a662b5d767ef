"""Pins of the CPU oracle against things other than itself: closed forms, invariants, library
routines (scipy rotations, torch.optim.Adam), quadrature, brute force and finite differences.

CPU only.  Each test names the passage of the paper (or the numerics reading) it pins.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2601_17354_gb300 import synthetic as S

Y0 = 1.0 / (2.0 * math.sqrt(math.pi))  # degree-0 real SH, textbook value


def make_gaussians(means, log_scales, quats, logits, sh, degree):
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    return S.Gaussians(f(means), f(log_scales), f(quats), f(logits), f(sh), degree)


def axis_camera(W=64, H=64, f=100.0, bg=(0.0, 0.0, 0.0)):
    view = np.zeros((3, 4), np.float32)
    view[0, 0] = view[1, 1] = view[2, 2] = 1.0
    return S.Camera(W, H, f, f, W / 2.0, H / 2.0, view, 0.2, bg)


def dc_for(colour):
    """Degree-0 coefficient whose colour (coef * Y0 + 0.5) is `colour`."""
    return (np.asarray(colour, np.float64) - 0.5) / Y0


# ------------------------------------------------------------------------------------------------
# the deterministic fp32 exp of the decision path
# ------------------------------------------------------------------------------------------------

def test_det_expf_within_two_ulp():
    x = np.linspace(-20.0, 6.0, 20001).astype(np.float32)
    got = oracle.det_expf(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(got - ref) / ulp) <= 2.0
    assert oracle.det_expf([0.0])[0] == 1.0


# ------------------------------------------------------------------------------------------------
# spherical harmonics (colour c of the canonical buffer, Fig. 2)
# ------------------------------------------------------------------------------------------------

def _sphere_quadrature(n_theta=12, n_phi=24):
    # Gauss-Legendre in cos(theta) x uniform phi: exact for polynomials of degree < 2 n_theta
    # in z and < n_phi in the azimuth.
    zs, wz = np.polynomial.legendre.leggauss(n_theta)
    phis = 2 * np.pi * np.arange(n_phi) / n_phi
    pts, wts = [], []
    for z, w in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for p in phis:
            pts.append((r * math.cos(p), r * math.sin(p), z))
            wts.append(w * 2 * np.pi / n_phi)
    return np.array(pts), np.array(wts)


def test_sh_orthonormal_by_quadrature():
    pts, wts = _sphere_quadrature()
    Y = np.stack([oracle.sh_basis(p)[0] for p in pts])  # [P, 16]
    gram = (Y * wts[:, None]).T @ Y
    assert np.max(np.abs(gram - np.eye(16))) < 1e-12


def test_sh_addition_theorem_and_zonal_values():
    rng = np.random.default_rng(3)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y = oracle.sh_basis(d)[0]
        for l in range(4):
            band = Y[l * l:(l + 1) * (l + 1)]
            assert abs(np.sum(band ** 2) - (2 * l + 1) / (4 * np.pi)) < 1e-13
    Y = oracle.sh_basis(np.array([0.0, 0.0, 1.0]))[0]
    for l in range(4):
        for m in range(-l, l + 1):
            want = math.sqrt((2 * l + 1) / (4 * np.pi)) if m == 0 else 0.0
            assert abs(Y[l * l + l + m] - want) < 1e-14
    # degree 1 is the linear form sqrt(3/4pi) (y, z, x)
    d = np.array([0.48, -0.6, 0.64])
    Y = oracle.sh_basis(d)[0]
    assert np.allclose(Y[1:4], math.sqrt(3 / (4 * np.pi)) * np.array([d[1], d[2], d[0]]), atol=1e-15)


def test_sh_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    d = rng.normal(size=3)
    _, dY = oracle.sh_basis(d)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd = (oracle.sh_basis(d + e)[0] - oracle.sh_basis(d - e)[0]) / (2 * h)
        assert np.max(np.abs(fd - dY[:, c])) < 1e-8


# ------------------------------------------------------------------------------------------------
# projection and compositing: closed forms (Eq. 7 and its front-to-back form)
# ------------------------------------------------------------------------------------------------

def test_anisotropic_footprint_rectangle():
    """An axis-aligned elongated Gaussian facing the camera: the 2-D covariance is
    diag((f s_x / z)^2 + 0.3, (f s_y / z)^2 + 0.3), the radii are the 3-sigma extents of each axis
    and the tile rectangle follows from them (a box, not the circle of the largest axis)."""
    cam = axis_camera()
    sx, sy, z = 0.12, 0.02, 4.0
    g = make_gaussians([[0.0], [0.0], [z]], [[math.log(sx)], [math.log(sy)], [math.log(0.01)]],
                       [[1.0], [0.0], [0.0], [0.0]], [1.0], np.zeros((3, 1, 1)), 0)
    fx = float(np.float32(cam.fx))
    sxx = (fx * math.exp(float(np.float32(math.log(sx)))) / z) ** 2 + 0.3
    syy = (fx * math.exp(float(np.float32(math.log(sy)))) / z) ** 2 + 0.3
    p = oracle.project(g, cam)
    rx, ry = (math.ceil(3 * math.sqrt(v)) for v in (sxx, syy))
    assert list(p["radius"][0]) == [rx, ry] and rx > ry
    assert list(p["rect"][0]) == [max((32 - rx) // 16, 0), max((32 - ry) // 16, 0),
                                  min((32 + rx) // 16 + 1, 4), min((32 + ry) // 16 + 1, 4)]


def test_single_isotropic_gaussian_closed_form():
    cam = axis_camera()
    sigma, z, o_logit, colour = 0.05, 4.0, 1.5, np.array([0.9, 0.4, 0.2])
    g = make_gaussians([[0.0], [0.0], [z]], [[math.log(sigma)]] * 3, [[1.0], [0.0], [0.0], [0.0]],
                       [o_logit], dc_for(colour).reshape(3, 1, 1), 0)
    s = math.exp(float(np.float32(math.log(sigma))))
    o = 1.0 / (1.0 + math.exp(-float(np.float32(o_logit))))
    c = Y0 * dc_for(colour).astype(np.float32).astype(np.float64) + 0.5
    s2 = (cam.fx * s / z) ** 2 + 0.3
    p = oracle.project(g, cam)
    assert p["visible"][0] == 1
    # per-axis 3-sigma extents of the isotropic footprint: ceil(3 sqrt(s2)) on both axes
    assert list(p["radius"][0]) == [math.ceil(3 * math.sqrt(s2))] * 2
    r = p["radius"][0][0]
    assert list(p["rect"][0]) == [(32 - r) // 16, (32 - r) // 16, (32 + r) // 16 + 1, (32 + r) // 16 + 1]
    assert np.allclose(p["conic"][0], [1 / s2, 0.0, 1 / s2], rtol=1e-13, atol=1e-15)
    out = oracle.render(g, cam)
    x0, y0, x1, y1 = [16 * v for v in p["rect"][0]]
    for py in range(cam.height):
        for px in range(cam.width):
            d2 = (px + 0.5 - 32) ** 2 + (py + 0.5 - 32) ** 2
            a = min(0.99, o * math.exp(-0.5 * d2 / s2))
            inside = x0 <= px < x1 and y0 <= py < y1
            if not inside or a < 1 / 255:
                want, wantT = np.zeros(3), 1.0
            else:
                want, wantT = a * c, 1 - a
            assert np.allclose(out["image"][:, py, px], want, atol=1e-13)
            assert abs(out["T"][py, px] - wantT) < 1e-13


def test_stacked_gaussians_order_clamp_skip_and_stop():
    """Four Gaussians on the axis, canonical order shuffled against depth; front-to-back
    transmittance, the 0.99 clamp, and the stop rule (T(1-a) < 1e-4 ends before compositing)."""
    cam = axis_camera(bg=(0.1, 0.2, 0.3))
    depths = [5.0, 3.0, 4.5, 4.0]            # canonical order; depth order is 1, 3, 2, 0
    sig = [0.025 * z for z in depths]  # 2.5 px standard deviation each
    cols = np.array([[0.2, 0.3, 0.4], [0.9, 0.1, 0.5], [0.3, 0.8, 0.6], [0.7, 0.7, 0.1]])
    logit = math.log(0.96 / 0.04)
    g = make_gaussians([[0.0] * 4, [0.0] * 4, depths], [[math.log(s) for s in sig]] * 3,
                       [[1.0] * 4, [0.0] * 4, [0.0] * 4, [0.0] * 4], [logit] * 4,
                       dc_for(cols).T.reshape(3, 1, 4), 0)
    out = oracle.render(g, cam)
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    order = np.argsort(depths)
    px = py = 31  # centre (31.5, 31.5): offset 0.5 in x and y from the projected mean
    alphas, cs = [], []
    for i in order:
        s = math.exp(float(np.float32(math.log(sig[i]))))
        s2 = (cam.fx * s / depths[i]) ** 2 + 0.3
        alphas.append(min(0.99, o * math.exp(-0.5 * 0.5 / s2)))
        cs.append(Y0 * dc_for(cols[i]).astype(np.float32).astype(np.float64) + 0.5)
    # with alpha ~ 0.92 the transmittance after three entries is ~4e-4 and the fourth entry
    # would take it below 1e-4: three entries are composited
    T = 1.0
    want = np.zeros(3)
    for k in range(3):
        want += cs[k] * alphas[k] * T
        T *= 1 - alphas[k]
    assert T * (1 - alphas[3]) < 1e-4 <= T
    want += T * np.array(cam.bg)
    assert out["last"][py, px] == 3
    assert np.allclose(out["image"][:, py, px], want, atol=1e-13)
    assert abs(out["T"][py, px] - T) < 1e-15


def test_equal_depths_composite_in_canonical_order():
    """Two Gaussians at exactly the same depth: the lower canonical index is in front."""
    cam = axis_camera()
    cols = np.array([[0.9, 0.1, 0.1], [0.1, 0.1, 0.9]])
    lg = math.log(0.6 / 0.4)

    def img(order):
        g = make_gaussians([[0.0, 0.0], [0.0, 0.0], [4.0, 4.0]], [[math.log(0.06)] * 2] * 3,
                           [[1.0] * 2, [0.0] * 2, [0.0] * 2, [0.0] * 2], [lg, lg],
                           dc_for(cols[order]).T.reshape(3, 1, 2), 0)
        return oracle.render(g, cam)["image"][:, 31, 31]

    o = 1.0 / (1.0 + math.exp(-float(np.float32(lg))))
    s = math.exp(float(np.float32(math.log(0.06))))
    a = o * math.exp(-0.5 * 0.5 / ((cam.fx * s / 4.0) ** 2 + 0.3))
    c = Y0 * dc_for(cols).astype(np.float32).astype(np.float64) + 0.5
    assert np.allclose(img([0, 1]), a * c[0] + a * (1 - a) * c[1], atol=1e-13)
    assert np.allclose(img([1, 0]), a * c[1] + a * (1 - a) * c[0], atol=1e-13)


def test_alpha_clamp_at_099():
    cam = axis_camera()
    g = make_gaussians([[0.0], [0.0], [4.0]], [[math.log(0.5)]] * 3, [[1.0], [0], [0], [0]], [8.0],
                       dc_for([0.6, 0.6, 0.6]).reshape(3, 1, 1), 0)
    out = oracle.render(g, cam)
    c = Y0 * dc_for([0.6]).astype(np.float32).astype(np.float64)[0] + 0.5
    assert abs(out["image"][0, 31, 31] - 0.99 * c) < 1e-13
    assert abs(out["T"][31, 31] - 0.01) < 1e-13


def test_rotation_convention_matches_scipy():
    """Sigma = R diag(s^2) R^T with R from the (w, x, y, z) quaternion (library routine), seen
    through the on-axis Jacobian diag(f/z, f/z): Sigma2D = (f/z)^2 Sigma[:2,:2] + 0.3 I."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    cam = axis_camera(W=128, H=128, f=200.0)
    rng = np.random.default_rng(7)
    n = 16
    q = rng.normal(size=(4, n))
    ls = rng.normal(-2.5, 0.4, size=(3, n))
    g = make_gaussians(np.stack([np.zeros(n), np.zeros(n), np.full(n, 5.0)]), ls, q,
                       np.zeros(n), np.zeros((3, 1, n)), 0)
    p = oracle.project(g, cam)
    q32 = g.quats.astype(np.float64)
    s = np.exp(g.log_scales.astype(np.float64))
    for i in range(n):
        R = Rot.from_quat([q32[1, i], q32[2, i], q32[3, i], q32[0, i]]).as_matrix()
        Sig = R @ np.diag(s[:, i] ** 2) @ R.T
        S2 = (cam.fx / 5.0) ** 2 * Sig[:2, :2] + 0.3 * np.eye(2)
        Q = np.linalg.inv(S2)
        assert np.allclose(p["conic"][i], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-10)
        assert np.allclose(p["cov2d"][i], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=2e-5, atol=1e-5)


def test_off_axis_jacobian_matches_numerical_derivative():
    """Away from the axis the 2-D covariance is J W Sigma W^T J^T + 0.3 I with J the derivative
    of the pinhole map; J is taken here by central differences of (fx x/z + cx, fy y/z + cy)."""
    rng = np.random.default_rng(8)
    eye = np.array([0.5, -3.5, 1.0])
    view = S.lookat_viewmat(eye)
    cam = S.Camera(96, 80, 90.0, 95.0, 48.0, 40.0, view)
    n = 24
    mu = rng.uniform(-0.8, 0.8, size=(3, n))
    g = make_gaussians(mu, rng.normal(-2.5, 0.3, size=(3, n)), rng.normal(size=(4, n)),
                       np.zeros(n), np.zeros((3, 1, n)), 0)
    p = oracle.project(g, cam)
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    W = view[:, :3].astype(np.float64)
    t = view[:, 3].astype(np.float64)

    def pix(pc):
        return np.array([cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy])

    for i in range(n):
        if not p["visible"][i]:
            continue
        pc = W @ g.means[:, i].astype(np.float64) + t
        assert abs(pc[0] / pc[2]) < 1.3 * 0.5 * cam.width / cam.fx  # inside the clamp
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            J[:, k] = (pix(pc + e) - pix(pc - e)) / 2e-6
        qq = g.quats[:, i].astype(np.float64)
        R = Rot.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        Sig = R @ np.diag(np.exp(2 * g.log_scales[:, i].astype(np.float64))) @ R.T
        S2 = J @ W @ Sig @ W.T @ J.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S2)
        assert np.allclose(p["conic"][i], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-6)
        assert np.allclose(p["mean2d"][i], pix(pc), rtol=1e-12)
        assert np.allclose(p["uv"][i], pix(pc), rtol=1e-5)


def test_view_direction_sign_of_colour():
    """Degree-1 z coefficient only: colour = 0.5 + sqrt(3/4pi) * coef * d_z, d = unit vector
    from the camera centre to the mean."""
    cam = axis_camera()
    sh = np.zeros((3, 4, 1))
    sh[:, 2, 0] = [0.3, -0.2, 0.1]
    g = make_gaussians([[0.3], [-0.2], [4.0]], [[-3.0]] * 3, [[1.0], [0], [0], [0]], [0.0], sh, 1)
    p = oracle.project(g, cam)
    d = np.array([0.3, -0.2, 4.0])
    d = g.means[:, 0].astype(np.float64) / np.linalg.norm(g.means[:, 0].astype(np.float64))
    want = 0.5 + math.sqrt(3 / (4 * np.pi)) * sh[:, 2, 0].astype(np.float32) * d[2]
    assert np.allclose(p["rgb"][0], want, atol=1e-12)


def test_rigid_motion_invariance():
    """Moving the scene and the camera by the same rigid motion leaves the projection unchanged."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    g, cam, _ = S.tiny_scene(11, n=200)
    Q = Rot.from_euler("xyz", [0.3, -0.5, 1.1])
    d = np.array([0.4, -0.2, 0.7])
    Qm = Q.as_matrix()
    means2 = Qm @ g.means.astype(np.float64) + d[:, None]
    qs = g.quats.astype(np.float64)
    rq = Q * Rot.from_quat(np.stack([qs[1], qs[2], qs[3], qs[0]], axis=1))
    xyzw = rq.as_quat()
    quats2 = np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]])
    W = cam.viewmat[:, :3].astype(np.float64)
    t = cam.viewmat[:, 3].astype(np.float64)
    W2 = W @ Qm.T
    t2 = t - W2 @ d
    cam2 = S.Camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                    np.concatenate([W2, t2[:, None]], 1).astype(np.float32))
    g2 = make_gaussians(means2, g.log_scales, quats2, g.opacity_logits, g.sh, 0)
    p1, p2 = oracle.project(g, cam), oracle.project(g2, cam2)
    vis = (p1["visible"] == 1) & (p2["visible"] == 1)
    assert vis.sum() > 150
    assert np.allclose(p1["mean2d"][vis], p2["mean2d"][vis], rtol=1e-5, atol=1e-4)
    assert np.allclose(p1["conic"][vis], p2["conic"][vis], rtol=1e-4, atol=1e-6)


def test_decision_path_agrees_with_fp64_path():
    """The fp32 decision quantities (prescribed order) and the FP64 value path are written
    independently; on a random scene they agree to fp32 accuracy."""
    sc = S.surface_scene(5, 3000, sh_degree=1, width=320, height=240, focal=250.0, n_cameras=2)
    p = oracle.project(sc.gt, sc.cameras[0])
    v = p["visible"] == 1
    assert v.sum() > 1000
    assert np.allclose(p["uv"][v], p["mean2d"][v], rtol=1e-5, atol=1e-3)
    Q = p["conic"][v]
    det = Q[:, 0] * Q[:, 2] - Q[:, 1] ** 2
    cov = np.stack([Q[:, 2] / det, -Q[:, 1] / det, Q[:, 0] / det], 1)
    assert np.allclose(p["cov2d"][v], cov, rtol=1e-4, atol=1e-4)


# ------------------------------------------------------------------------------------------------
# compositing invariants (Eq. 7)
# ------------------------------------------------------------------------------------------------

def test_weights_and_final_transmittance_sum_to_one():
    """With every colour 0.5 and a black background, C = 0.5 sum_i w_i, so 2C + T_final = 1."""
    g, cam, _ = S.tiny_scene(1)
    g.sh[:] = 0.0
    out = oracle.render(g, cam)
    assert out["last"].max() > 10
    err = np.abs(2 * out["image"] + out["T"][None] - 1.0)
    assert err.max() < 1e-12


def test_eq7_back_to_front_equals_front_to_back():
    g, cam, _ = S.tiny_scene(2)
    cam.bg = (0.2, 0.5, 0.9)
    a = oracle.render(g, cam)["image"]
    b = oracle.render_eq7(g, cam)
    assert np.max(np.abs(a - b)) < 1e-12


def test_canonical_permutation_equivariance():
    """Eq. 10: rendering depends on the sorted view only; permuting the canonical buffer
    leaves the image unchanged and permutes the gradients the same way."""
    g, cam, _ = S.tiny_scene(3, n=500)
    perm = np.random.default_rng(0).permutation(g.n)
    gp = g.subset(perm)
    dL = S.random_image(9, cam.width, cam.height)
    a, b = oracle.render(g, cam), oracle.render(gp, cam)
    assert np.max(np.abs(a["image"] - b["image"])) < 1e-15
    g2a, ga = oracle.backward(g, cam, dL)
    g2b, gb = oracle.backward(gp, cam, dL)
    assert np.allclose(g2a[perm], g2b, rtol=1e-12, atol=1e-18)
    for k in ga:
        assert np.allclose(ga[k][..., perm], gb[k], rtol=1e-12, atol=1e-18)


# ------------------------------------------------------------------------------------------------
# keys, sort and tile ranges (the permutation pi of Eq. 10), against brute force
# ------------------------------------------------------------------------------------------------

def _tile_hit(uv, cov, tx, ty, T=16):
    """The 3-sigma ellipse / tile rule in numpy float32 (products and sums rounded one by one):
    the minimum of Q over the tile's pixel-centre box, at the clamped centre or an edge's clamped
    line minimum, is at most 9."""
    f = np.float32
    u, v = f(uv[0]), f(uv[1])
    a_, b_, c_ = f(cov[0]), f(cov[1]), f(cov[2])
    det = f(f(a_ * c_) - f(b_ * b_))
    inv = f(f(1) / det)
    ca, cb, cc = f(c_ * inv), f(f(-b_) * inv), f(a_ * inv)
    xl, xh = f(f(tx * T) + f(0.5)), f(f(tx * T + T) - f(0.5))
    yl, yh = f(f(ty * T) + f(0.5)), f(f(ty * T + T) - f(0.5))
    clamp = lambda x, lo, hi: min(max(x, lo), hi)

    def Q(X, Y):
        dx, dy = f(X - u), f(Y - v)
        return f(f(f(f(ca * dx) * dx) + f(f(f(cb + cb) * dx) * dy)) + f(f(cc * dy) * dy))
    sy, sx = f(cb / cc), f(cb / ca)
    best = Q(clamp(u, xl, xh), clamp(v, yl, yh))
    for X in (xl, xh):
        best = min(best, Q(X, clamp(f(v - f(sy * f(X - u))), yl, yh)))
    for Y in (yl, yh):
        best = min(best, Q(clamp(f(u - f(sx * f(Y - v))), xl, xh), Y))
    return bool(best <= f(9))


def test_tile_membership_is_the_three_sigma_ellipse():
    """An isotropic footprint (Q = d^2 / s2): a tile of the rectangle is listed exactly when the
    distance from the centre to its pixel-centre box is at most 3 sqrt(s2) (closed form, cases
    away from the boundary)."""
    cam = axis_camera(160, 160, 100.0)
    dropped = 0
    for sigma, x in ((0.3, 0.31), (0.25, -0.2), (0.4, 0.02)):
        g = make_gaussians([[x], [0.13], [4.0]], [[math.log(sigma)]] * 3, [[1.0], [0.0], [0.0], [0.0]],
                           [1.0], np.zeros((3, 1, 1)), 0)
        p = oracle.project(g, cam)
        keys, vals, ranges = oracle.keys(g, cam)
        TX, TY = oracle.tiles(cam)
        u, v = p["uv"][0]
        s2 = float(p["cov2d"][0][0])
        x0, y0, x1, y1 = p["rect"][0]
        listed = {int(k >> np.uint64(32)) for k in keys}
        checked = 0
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                bx = min(max(u, 16 * tx + 0.5), 16 * tx + 15.5)
                by = min(max(v, 16 * ty + 0.5), 16 * ty + 15.5)
                q = ((bx - u) ** 2 + (by - v) ** 2) / s2
                if abs(q - 9) < 1e-3:
                    continue
                assert ((ty * TX + tx) in listed) == (q <= 9), (tx, ty, q)
                checked += 1
        assert checked >= 4
        dropped += (x1 - x0) * (y1 - y0) - len(listed)
    assert dropped > 0   # rectangle corners the ellipse does not reach


@pytest.mark.parametrize("dims", [(128, 128), (100, 75)])
def test_keys_and_ranges_match_brute_force(dims):
    g, cam, _ = S.tiny_scene(4, n=1500, width=dims[0], height=dims[1])
    g.means[2, 1::7] = g.means[2, 0:-1:7][: len(g.means[2, 1::7])]  # exact depth ties
    keys, vals, ranges = oracle.keys(g, cam)
    p = oracle.project(g, cam)
    TX, TY = oracle.tiles(cam)
    depth_bits = p["depth"].view(np.uint32).astype(np.uint64)
    r = p["rect"]
    hit = {}
    for i in range(g.n):
        if p["visible"][i]:
            for ty in range(r[i, 1], r[i, 3]):
                for tx in range(r[i, 0], r[i, 2]):
                    if _tile_hit(p["uv"][i], p["cov2d"][i], tx, ty):
                        hit.setdefault(ty * TX + tx, []).append(i)
    assert len(keys) == sum(len(v) for v in hit.values())
    for t in range(TX * TY):
        ids = np.array(hit.get(t, []), np.int64)
        ids = ids[np.lexsort((ids, depth_bits[ids]))]
        s, e = ranges[t]
        assert np.array_equal(vals[s:e], ids.astype(np.uint32))
        want = (np.uint64(t) << np.uint64(32)) | depth_bits[ids]
        assert np.array_equal(keys[s:e], want)
        if len(ids) == 0:
            assert s == 0 and e == 0
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])


# ------------------------------------------------------------------------------------------------
# gradients: two derivations (Eq. 8 and direct) and FP64 central finite differences
# ------------------------------------------------------------------------------------------------

def test_eq8_and_direct_derivation_agree():
    g, cam, _ = S.tiny_scene(5)
    cam.bg = (0.3, 0.1, 0.7)
    dL = S.random_image(6, cam.width, cam.height)
    a2, a = oracle.backward(g, cam, dL, mode=0)
    b2, b = oracle.backward(g, cam, dL, mode=1)
    assert np.max(np.abs(a2 - b2)) <= 1e-12 * np.max(np.abs(a2))
    for k in a:
        assert np.max(np.abs(a[k] - b[k])) <= 1e-12 * max(np.max(np.abs(a[k])), 1e-30)


def _fd_scene():
    """Six Gaussians at SH degree 3 on a ragged 40x36 image, including one with its alpha
    clamped at 0.99 near its centre and one beyond the Jacobian clamp."""
    rng = np.random.default_rng(12)
    view = S.lookat_viewmat([0.6, -3.8, 0.9])
    cam = S.Camera(40, 36, 40.0, 42.0, 20.0, 18.0, view, 0.2, (0.2, 0.3, 0.1))
    W, t = view[:, :3].astype(np.float64), view[:, 3].astype(np.float64)
    # camera-space targets, mapped back to world space
    pcs = [(0.0, 0.0, 4.0), (0.3, -0.2, 3.6), (-0.4, 0.25, 4.4), (0.1, 0.35, 3.9), (-0.2, -0.3, 4.1),
           (2.9, 0.1, 4.0)]  # last one: x/z = 0.725 > 1.3 * 20/40 = 0.65
    means = np.stack([W.T @ (np.array(pc) - t) for pc in pcs], 1)
    n = len(pcs)
    ls = rng.normal(-2.3, 0.25, size=(3, n))
    ls[:, 5] = -1.2
    logits = rng.normal(0.5, 0.5, size=n)
    logits[0] = 7.0  # alpha clamps at 0.99 near the centre of Gaussian 0
    sh = np.zeros((3, 16, n))
    sh[:, 0] = dc_for(rng.uniform(0.2, 0.8, size=(3, n)))
    sh[:, 1:] = rng.normal(0, 0.08, size=(3, 15, n))
    sh[0, 0, 2] = dc_for(-0.3)  # red of Gaussian 2 is clamped at 0: zero gradient through it
    return make_gaussians(means, ls, rng.normal(size=(4, n)), logits, sh, 3), cam


def _signature(g, cam):
    p = oracle.project(g, cam)
    r = oracle.render(g, cam)
    return (p["rect"].tobytes(), p["visible"].tobytes(), r["last"].tobytes(),
            r["ncomp"].tobytes(), r["evals"].tobytes())


def test_gradients_match_central_finite_differences():
    g, cam = _fd_scene()
    p = oracle.project(g, cam)
    assert p["visible"].all()
    pc5 = cam.viewmat[:, :3].astype(np.float64) @ g.means[:, 5] + cam.viewmat[:, 3]
    assert pc5[0] / pc5[2] > 1.3 * 0.5 * cam.width / cam.fx
    wimg = S.random_image(13, cam.width, cam.height)
    _, an = oracle.backward(g, cam, wimg)
    base = _signature(g, cam)

    def loss(gg):
        return float(np.sum(oracle.render(gg, cam)["image"] * wimg))

    checked = skipped = 0
    for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        arr = getattr(g, name)
        grad = an[name]
        scale = np.max(np.abs(grad))
        for idx in np.ndindex(arr.shape):
            x = float(arr[idx])
            h = 2.0 ** -12 * max(1.0, abs(x))
            gp, gm = g.copy(), g.copy()
            getattr(gp, name)[idx] = np.float32(x + h)
            getattr(gm, name)[idx] = np.float32(x - h)
            if _signature(gp, cam) != base or _signature(gm, cam) != base:
                skipped += 1
                continue
            dx = float(getattr(gp, name)[idx]) - float(getattr(gm, name)[idx])
            fd = (loss(gp) - loss(gm)) / dx
            assert abs(fd - grad[idx]) <= 2e-5 * scale + 1e-4 * abs(grad[idx]), (name, idx, fd, grad[idx])
            checked += 1
    assert checked > 300 and skipped <= 0.05 * (checked + skipped)


def test_subset_backward_equals_full_backward():
    g, cam, _ = S.tiny_scene(8, n=600)
    g.sh = np.ascontiguousarray(np.concatenate([g.sh, np.zeros((3, 3, g.n), np.float32)], 1))
    g.sh_degree = 1
    g.sh[:, 1:] = np.random.default_rng(1).normal(0, 0.1, size=(3, 3, g.n)).astype(np.float32)
    dL = S.random_image(2, cam.width, cam.height)
    g2, full = oracle.backward(g, cam, dL)
    sel = np.array([0, 7, 100, 333, 599])
    s2, sp = oracle.backward_subset(g, cam, dL, sel)
    assert np.allclose(s2, g2[sel], rtol=1e-12, atol=1e-20)
    K = 4
    want = np.concatenate([full["means"][:, sel].T, full["log_scales"][:, sel].T,
                           full["quats"][:, sel].T, full["opacity_logits"][sel][:, None],
                           full["sh"][:, :, sel].reshape(3 * K, -1).T], 1)
    assert np.allclose(sp, want, rtol=1e-10, atol=1e-20)


# ------------------------------------------------------------------------------------------------
# loss and optimizer
# ------------------------------------------------------------------------------------------------

def test_l1_closed_form():
    img = np.array([0.5, 0.2, 0.9, 0.4])
    gt = np.array([0.1, 0.2, 1.0, 0.9])
    loss, grad, sse = oracle.l1(img, gt)
    assert abs(loss - (0.4 + 0.0 + 0.1 + 0.5) / 4) < 1e-15
    assert np.allclose(grad, [0.25, 0.0, -0.25, -0.25])
    assert abs(sse - (0.16 + 0.01 + 0.25)) < 1e-15


def test_adam_matches_torch_optim_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=257)
    gs = [rng.normal(size=257) * 10.0 ** rng.uniform(-3, 1) for _ in range(7)]
    lr, b1, b2, eps = 3e-3, 0.9, 0.999, 1e-15
    prm = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([prm], lr=lr, betas=(b1, b2), eps=eps, foreach=False)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for t, gk in enumerate(gs, start=1):
        prm.grad = torch.tensor(gk, dtype=torch.float64)
        opt.step()
        oracle.adam(p, np.ascontiguousarray(gk), m, v, lr, t, b1, b2, eps)
    assert np.allclose(p, prm.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_first_step_is_signed_learning_rate():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.01, 1e-6])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam(p, g, m, v, 0.1, 1)
    assert np.allclose(p, [0.9, -1.9, 0.4], atol=1e-9)


def test_fd_subset_matches_analytic_backward():
    """The subset finite-difference routine (used at full scale on the GPU machine) agrees with the
    analytic gradient on a small SH-degree-1 scene."""
    sc = S.surface_scene(9, 3000, 1, 160, 120, 140.0, n_cameras=4)
    g, cam = sc.gt, sc.cameras[1]
    w = S.random_image(3, cam.width, cam.height)
    sel = np.random.default_rng(2).choice(np.nonzero(oracle.project(g, cam)["visible"])[0], 12,
                                          replace=False)
    _, an = oracle.backward_subset(g, cam, w, sel)
    scale = np.abs(an).max(axis=1, keepdims=True)
    worst = []
    for h in (2.0 ** -12, 2.0 ** -14):
        fd = oracle.fd_subset(g, cam, w, sel, h_rel=h)
        ok = np.isfinite(fd)
        assert ok.mean() > 0.9
        worst.append(np.max((np.abs(fd - an) / (scale + 1e-30))[ok]))
    # central differences: the error is the O(h^2) truncation, 16x smaller at a 4x smaller step
    assert worst[1] < 1e-4 and worst[0] > 8 * worst[1]
