"""Pins of the bundle-adjustment oracle (oracle/ba.py): analytic Jacobians against central
differences, a zero step at the solution, Levenberg-Marquardt recovering the cameras and points
from perturbed starts on noise-free observations, the gauge left in place, and the matrix-free
normal-equation residual against the dense equations."""
import numpy as np
import pytest

from oracle import ba as O
from paper_2601_17354_gb300 import synthetic as S

from tests._ba import observations


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


def test_matrix_free_residual_matches_dense_equations():
    p = S.ba_problem(4, 5, 60)
    obs = observations(p, p.R_gt, p.t_gt, p.P_gt, tracks=True)
    axis = O.gauge_axis(p.R_init, p.t_init)
    lam = 1e-2
    Hd, b, diag, ci, nc, _ = O.normal_equations(p.R_init, p.t_init, p.P_init, obs, p.K, 0.5, 2.0, lam, axis)
    rng = np.random.default_rng(0)
    dcam = rng.normal(size=(5, 6)) * 1e-3
    dP = rng.normal(size=(60, 3)) * 1e-3
    x = np.zeros(len(b))
    for i in range(5):
        for d in range(6):
            if ci[i, d] >= 0:
                x[ci[i, d]] = dcam[i, d]
    x[nc:] = dP.ravel()
    dense = Hd @ x - b
    res_c, scale_c, res_p, scale_p = O.normal_residual(p.R_init, p.t_init, p.P_init, obs, p.K, 0.5, 2.0, lam, axis,
                                                       dcam, dP)
    got = np.zeros(len(b))
    for i in range(5):
        for d in range(6):
            if ci[i, d] >= 0:
                got[ci[i, d]] = res_c[i, d]
    got[nc:] = res_p.ravel()
    assert np.allclose(got, dense, rtol=1e-9, atol=1e-9 * np.abs(dense).max())
    # the scale bounds |row| and the fixed parameters report nothing
    assert np.all(np.abs(res_c) <= scale_c * (1 + 1e-12)) and np.all(np.abs(res_p) <= scale_p * (1 + 1e-12))
    assert np.all(res_c[0] == 0) and res_c[1, 3 + axis] == 0


def test_matrix_free_residual_vanishes_at_the_dense_step():
    p = S.ba_problem(5, 6, 80)
    obs = observations(p, p.R_gt, p.t_gt, p.P_gt)
    axis = O.gauge_axis(p.R_init, p.t_init)
    dcam, dP, _ = O.lm_step(p.R_init, p.t_init, p.P_init, obs, p.K, 0.5, 2.0, 1e-3, axis)
    res_c, scale_c, res_p, scale_p = O.normal_residual(p.R_init, p.t_init, p.P_init, obs, p.K, 0.5, 2.0, 1e-3, axis,
                                                       dcam, dP)
    assert np.abs(res_c).max() <= 1e-9 * scale_c.max() and np.abs(res_p).max() <= 1e-9 * scale_p.max()
