"""Pins of the oracle's compositing decisions and of its tile-membership rule against things other
than itself.  CPU only.

Compositing decisions (skip alpha < 1/255, clamp at 0.99, stop when T (1 - alpha) < 1e-4; the
reading of Sec. III-C / Eq. 7 used throughout) are taken in fp32 with a stated error bound; the
replay of forced decisions must reproduce the oracle's own render when it is given the oracle's
own decisions, must count a flip outside the bound as illegal and one inside it as legal.

Tile membership (the 3-sigma ellipse reaching a tile's pixel-centre box; the paper gives no
footprint rule) is checked against bound-constrained least squares from scipy: with the conic
M = L^T L, min over the box of (p - mu)^T M (p - mu) = min ||L p - L mu||^2, which lsq_linear solves
by its own method, sharing nothing with the oracle's clamped-centre / edge-line search.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2601_17354_gb300 import synthetic as S

Y0 = 1.0 / (2.0 * math.sqrt(math.pi))


def make_gaussians(means, log_scales, quats, logits, sh, degree):
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    return S.Gaussians(f(means), f(log_scales), f(quats), f(logits), f(sh), degree)


def axis_camera(W=64, H=64, f=100.0, bg=(0.0, 0.0, 0.0)):
    view = np.zeros((3, 4), np.float32)
    view[0, 0] = view[1, 1] = view[2, 2] = 1.0
    return S.Camera(W, H, f, f, W / 2.0, H / 2.0, view, 0.2, bg)


def all_pixels(cam):
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    return np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)


def own_decisions(g, cam, pix, tile=16):
    E = 4096
    d = oracle.decisions(g, cam, pix, E, tile)
    assert np.all(d["count"] >= 0)
    off = np.concatenate([[0], np.cumsum(d["count"])])
    codes = np.concatenate([d["code"][k, :d["count"][k]] for k in range(len(pix))])
    return d, oracle.Forced(pix, off, codes)


@pytest.mark.parametrize("seed", [0, 2])
def test_replaying_the_oracles_own_decisions_reproduces_its_render(seed):
    g, cam, _ = S.tiny_scene(seed, n=1500, width=96, height=72)
    cam.bg = (0.2, 0.1, 0.3)
    pix = all_pixels(cam)
    _, forced = own_decisions(g, cam, pix)
    ora = oracle.render(g, cam)
    rep = oracle.render_forced(g, cam, forced)
    assert rep["flips"].sum() == 0 and rep["illegal"].sum() == 0
    xs, ys = pix[:, 0], pix[:, 1]
    assert np.array_equal(rep["rgb"], ora["image"][:, ys, xs].T)
    assert np.array_equal(rep["T"], ora["T"][ys, xs])
    assert np.array_equal(rep["last"], ora["last"][ys, xs])
    assert np.array_equal(rep["ncomp"], ora["ncomp"][ys, xs])


def test_a_flip_far_from_its_threshold_is_illegal():
    g, cam, _ = S.tiny_scene(1, n=800, width=64, height=64)
    pix = all_pixels(cam)
    d, forced = own_decisions(g, cam, pix)
    codes = forced.codes.copy()
    # pick composited entries whose o 2^p is far inside (0, 0.99) and mark them skipped
    og = np.concatenate([d["og"][k, :d["count"][k]] for k in range(len(pix))])
    cand = np.flatnonzero((codes == 1) & (og > 0.05) & (og < 0.9))
    assert len(cand) > 10
    codes[cand[::7]] = 0
    planted = oracle.render_forced(g, cam, oracle.Forced(pix, forced.off, codes))
    assert planted["illegal"].sum() >= len(cand[::7]) * 0.5
    # a skipped entry forced to composite far below 1/255, and a stop forced away
    codes = forced.codes.copy()
    cand = np.flatnonzero((codes == 0) & (og < 1e-3))
    codes[cand[:5]] = 1
    assert oracle.render_forced(g, cam, oracle.Forced(pix, forced.off, codes))["illegal"].sum() >= 1


def _single(cam, logit, sigma=0.05, z=4.0, colour=(0.6, 0.5, 0.4)):
    dc = ((np.asarray(colour) - 0.5) / Y0).reshape(3, 1, 1)
    return make_gaussians([[0.0], [0.0], [z]], [[math.log(sigma)]] * 3, [[1.0], [0.0], [0.0], [0.0]],
                          [logit], dc, 0)


def test_decision_side_alpha_matches_the_closed_form():
    """o 2^p of the fp32 exponent against the closed-form o exp(-d^2 / (2 s2)) of an isotropic
    Gaussian facing the camera: agreement to fp32 accuracy of the exponent."""
    cam = axis_camera()
    g = _single(cam, 0.7)
    s = math.exp(float(np.float32(math.log(0.05))))
    o = 1.0 / (1.0 + math.exp(-float(np.float32(0.7))))
    s2 = (cam.fx * s / 4.0) ** 2 + 0.3
    pix = np.array([[x, 29] for x in range(20, 44)], np.int32)
    d = oracle.decisions(g, cam, pix, 4)
    for k, (x, y) in enumerate(pix):
        power = -0.5 * ((x + 0.5 - 32) ** 2 + (y + 0.5 - 32) ** 2) / s2
        want = o * math.exp(power)
        assert d["count"][k] == 1
        # the exponent is a few fp32 roundings of terms of size |power|
        assert abs(d["og"][k, 0] / want - 1.0) < 8 * 2.0 ** -24 * (1.0 + abs(power))


def test_ambiguous_skip_is_flagged_and_either_decision_is_legal():
    """One Gaussian whose o 2^p at a pixel sits within the bound of 1/255: the pixel is flagged and
    the replay accepts the kernel taking either branch; the same flip at a clear pixel is not."""
    cam = axis_camera()
    px, py = 41, 33
    # choose the opacity logit so that o 2^p at (px, py) is 1/255 (1 + 2e-7): the fp32 logit
    # moves o by far less than the 1e-6 bound
    base = _single(cam, 0.0, sigma=0.2)
    og0 = oracle.decisions(base, cam, np.array([[px, py]], np.int32), 4)["og"][0, 0]
    o0 = 1.0 / (1.0 + math.exp(-0.0))
    target_o = o0 * (float(np.float32(1.0 / 255.0)) * (1 + 2e-7)) / og0
    g = _single(cam, math.log(target_o / (1.0 - target_o)), sigma=0.2)
    d = oracle.decisions(g, cam, np.array([[px, py]], np.int32), 4)
    rel = d["og"][0, 0] / float(np.float32(1.0 / 255.0)) - 1.0
    eps = oracle.decision_bound()
    assert abs(rel) < eps
    ora = oracle.render(g, cam)
    assert ora["flag"][py, px] & 1
    pix = np.array([[px, py]], np.int32)
    for code in (0, 1):
        rep = oracle.render_forced(g, cam, oracle.Forced(pix, [0, 1], [code]))
        assert rep["illegal"][0] == 0
        assert rep["ncomp"][0] == code
    # the centre pixel is far from every threshold: flipping its decision is illegal
    rep = oracle.render_forced(g, cam, oracle.Forced(np.array([[32, 32]], np.int32), [0, 1], [0]))
    assert rep["illegal"][0] == 1 and ora["flag"][32, 32] == 0


def test_flags_are_rare_on_the_parity_scenes():
    """With decisions in the kernel's precision only decisions inside the error bound are flagged:
    far fewer than 1e-4 of the pixels on these scenes (0.1-1.4 % with FP64 decisions and wide
    margins)."""
    for g, cam in (S.tiny_scene(0)[:2], S.tiny_scene(2, n=20000, width=64, height=64, focal=60.0)[:2]):
        ora = oracle.render(g, cam)
        assert np.count_nonzero(ora["flag"]) <= max(1, 1e-4 * ora["flag"].size)


# ------------------------------------------------------------------------------------------------
# tile membership against bound-constrained least squares
# ------------------------------------------------------------------------------------------------

def _box_min_q(mu, conic, box):
    """min over the box [xl, xh] x [yl, yh] of (p - mu)^T M (p - mu), M = [[a, b], [b, c]], by
    scipy's bounded least squares on ||L p - L mu||^2 with M = L^T L."""
    opt = pytest.importorskip("scipy.optimize")
    a, b, c = conic
    M = np.array([[a, b], [b, c]])
    Lc = np.linalg.cholesky(M).T  # M = Lc^T Lc
    xl, xh, yl, yh = box
    r = opt.lsq_linear(Lc, Lc @ mu, bounds=([xl, yl], [xh, yh]), method="bvls", tol=1e-14)
    p = r.x
    d = p - mu
    return float(d @ M @ d)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tile_membership_against_bounded_least_squares(seed):
    """Rotated, strongly anisotropic footprints (off-diagonal conic term): a tile of the rectangle
    is listed exactly when the minimum of Q over its pixel-centre box is at most 9, the minimum
    found by scipy's bounded least squares (FP64, conic inverted from the fp32 2-D covariance);
    cases within 1e-3 of the boundary are skipped."""
    rng = np.random.default_rng(100 + seed)
    cam = axis_camera(192, 160, 220.0)
    n = 60
    means = np.stack([rng.uniform(-0.7, 0.7, n), rng.uniform(-0.6, 0.6, n), rng.uniform(3.0, 5.0, n)])
    ls = np.stack([rng.uniform(-2.2, -1.6, n), rng.uniform(-4.5, -3.5, n), rng.uniform(-4.0, -3.0, n)])
    q = rng.normal(size=(4, n))
    g = make_gaussians(means, ls, q, np.zeros(n), np.zeros((3, 1, n)), 0)
    p = oracle.project(g, cam)
    keys, _, _ = oracle.keys(g, cam)
    TX, _ = oracle.tiles(cam)
    listed = {}
    _, vals, ranges = oracle.keys(g, cam)
    for t in range(len(ranges)):
        for i in vals[ranges[t, 0]:ranges[t, 1]]:
            listed.setdefault(int(i), set()).add(t)
    checked = skipped_corners = 0
    cross = 0
    for i in range(n):
        if not p["visible"][i]:
            continue
        A, B, C = (float(v) for v in p["cov2d"][i])
        det = A * C - B * B
        conic = (C / det, -B / det, A / det)
        if abs(conic[1]) > 0.05 * math.sqrt(conic[0] * conic[2]):
            cross += 1
        mu = np.array(p["uv"][i], np.float64)
        x0, y0, x1, y1 = p["rect"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                qmin = _box_min_q(mu, conic, (16 * tx + 0.5, 16 * tx + 15.5, 16 * ty + 0.5, 16 * ty + 15.5))
                if abs(qmin - 9.0) < 9e-3:
                    continue
                got = (ty * TX + tx) in listed.get(i, set())
                assert got == (qmin <= 9.0), (i, tx, ty, qmin)
                checked += 1
                skipped_corners += qmin > 9.0
    assert cross > 20          # most footprints are rotated (b != 0)
    assert checked > 300
    assert skipped_corners > 30  # rectangle tiles the ellipse does not reach
