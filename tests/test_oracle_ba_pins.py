"""Pins of the bundle-adjustment oracle (oracle/ba.py): analytic Jacobians against central
differences, a zero step at the solution, Levenberg-Marquardt recovering the cameras and points
from perturbed starts on noise-free observations, and the gauge left in place."""
import numpy as np
import pytest

from oracle import ba as O
from paper_2601_17354_gb300 import synthetic as S


def observations(p, R, t, P, noise=True):
    """All (camera, point) pairs in front of the camera and inside the image, ordered by point."""
    cams, pts, uvs = [], [], []
    for i in range(len(R)):
        uv, Xc = O.project(R[i], t[i], P, p.K)
        ok = (Xc[:, 2] > 0.2) & (uv[:, 0] >= 0) & (uv[:, 0] < p.width) & (uv[:, 1] >= 0) & (uv[:, 1] < p.height)
        for j in np.nonzero(ok)[0]:
            cams.append(i)
            pts.append(j)
            uvs.append(uv[j] + (p.noise[i, j] if noise else 0.0))
    cams, pts, uvs = np.array(cams), np.array(pts), np.array(uvs)
    keep = np.bincount(pts, minlength=len(P))[pts] >= 2   # a point needs two views
    order = np.lexsort((cams[keep], pts[keep]))
    return cams[keep][order], pts[keep][order], uvs[keep][order]


def test_jacobians_match_central_differences():
    p = S.ba_problem(1, 6, 30)
    R, t, P = p.R_init[2], p.t_init[2], p.P_init
    Jc, Jp = O.jacobians(R, t, P, p.K)
    h = 1e-6
    for d in range(6):
        e = np.zeros(6)
        e[d] = h
        Rp, tp, _ = O.apply(R[None], t[None], P, e[None], np.zeros_like(P))
        Rm, tm, _ = O.apply(R[None], t[None], P, -e[None], np.zeros_like(P))
        fd = (O.project(Rp[0], tp[0], P, p.K)[0] - O.project(Rm[0], tm[0], P, p.K)[0]) / (2 * h)
        assert np.allclose(fd, Jc[:, :, d], rtol=1e-5, atol=1e-3), d
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (O.project(R, t, P + e, p.K)[0] - O.project(R, t, P - e, p.K)[0]) / (2 * h)
        assert np.allclose(fd, Jp[:, :, d], rtol=1e-5, atol=1e-3), d


def test_step_is_zero_at_the_solution():
    p = S.ba_problem(2, 6, 60)
    obs = observations(p, p.R_gt, p.t_gt, p.P_gt, noise=False)
    axis = O.gauge_axis(p.R_gt, p.t_gt)
    dcam, dP, cost = O.lm_step(p.R_gt, p.t_gt, p.P_gt, obs, p.K, 0.5, 2.0, 1e-4, axis)
    assert cost < 1e-16 and np.abs(dcam).max() < 1e-9 and np.abs(dP).max() < 1e-9


def test_lm_recovers_noise_free_scene_and_keeps_the_gauge():
    p = S.ba_problem(3, 6, 80)
    obs = observations(p, p.R_gt, p.t_gt, p.P_gt, noise=False)
    axis = O.gauge_axis(p.R_init, p.t_init)
    R, t, P, costs = O.solve(p.R_init, p.t_init, p.P_init, obs, p.K, 0.5, 2.0, iters=30)
    assert costs[-1] < 1e-10 * costs[0] and costs[-1] < 1e-8
    assert np.array_equal(R[0], p.R_init[0]) and np.array_equal(t[0], p.t_init[0])
    assert t[1][axis] == p.t_init[1][axis]
