"""GPU bundle adjustment (through the C ABI) against the oracle (Sec. III-A, Eq. 2-3).

A step is judged by its backward error: the residual of the damped normal equations, which the
oracle evaluates in FP64 (densely on small problems, matrix-free at the full 32-camera size),
relative to the row scale (|H| + lam diag H)|step| + |b|.  The GPU keeps H_tp and E = H_tp H_pp^-1
in FP32 (relative rounding u = 2^-24), sums a thread's point-pair products in FP32 (K ~ 100
terms: relative error ~ K u ~ 1e-5 of the terms summed) and eliminates the Jacobi-scaled reduced
system in FP32 (componentwise backward error ~ N u with N = 6C <= 360 here, ~2e-5; diagonal
scaling leaves componentwise bounds unchanged); the tolerance 2e-4 allows a further factor ~10
for the cancellation inside the Schur complement.  The forward error is bounded by cond(H) times the normwise backward error
(first-order perturbation theory), checked against the dense solve; LM runs are compared by the
cost they reach and the points they find."""
import numpy as np
import pytest

from oracle import ba as O
from paper_2601_17354_gb300 import synthetic as S
from tests._ba import observations

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIGMA, DELTA = 0.5, 2.0
BACKWARD_TOL = 2e-4


@pytest.fixture(scope="module")
def B():
    from paper_2601_17354_gb300 import ba
    return ba


def _setup(seed, C, n, tracks, noise=True):
    p = S.ba_problem(seed, C, n)
    cams, pts, uv = observations(p, p.R_gt, p.t_gt, p.P_gt, noise=noise, tracks=tracks)
    obs = (cams, pts, uv.astype(np.float32).astype(np.float64))
    # the GPU state is FP32: the oracle works on the same rounded values in FP64
    R, t, P = (x.astype(np.float32) for x in (p.R_init, p.t_init, p.P_init))
    return p, obs, R, t, P


def _dev(R, t, P, obs):
    cams, pts, uv = obs
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    i = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    return f(R), f(t), f(P), i(cams), i(pts), f(uv)


def _backward_error(R, t, P, obs, K, lam, axis, dcam, dP):
    res_c, sc_c, res_p, sc_p = O.normal_residual(R.astype(np.float64), t.astype(np.float64), P.astype(np.float64),
                                                 obs, K, SIGMA, DELTA, lam, axis, dcam, dP)
    ratio_c = np.abs(res_c) / np.maximum(sc_c, 1e-300)
    ratio_p = np.abs(res_p) / np.maximum(sc_p, 1e-300)
    return max(ratio_c.max(), ratio_p.max())


@pytest.mark.parametrize("seed,C,n,tracks", [(11, 6, 120, False), (12, 8, 300, True), (17, 40, 500, True),
                                             (13, 60, 700, True)])
def test_step_matches_dense_normal_equations(B, seed, C, n, tracks):
    """Up to 37 cameras the reduced system is factored by blocks in shared memory; 40 cameras take
    the packed elimination in shared memory, 60 cameras the packed elimination in global memory."""
    p, obs, R, t, P = _setup(seed, C, n, tracks)
    lam = 1e-3
    ba = B.BundleAdjuster(C, n, len(obs[0]))
    Rd, td, Pd, cd, pd, uvd = _dev(R, t, P, obs)
    dcam, dP, cost = ba.step(Rd, td, Pd, cd, pd, uvd, p.K, SIGMA, DELTA, lam)
    dcam, dP = dcam.cpu().numpy().astype(np.float64), dP.cpu().numpy().astype(np.float64)
    R64, t64, P64 = (x.astype(np.float64) for x in (R, t, P))
    axis = O.gauge_axis(R64, t64)
    dc_o, dP_o, cost_o = O.lm_step(R64, t64, P64, obs, p.K, SIGMA, DELTA, lam, axis)
    assert abs(cost - cost_o) <= 1e-9 * cost_o
    # gauge: camera 0 and one translation component of camera 1 do not move; unseen points neither
    assert np.all(dcam[0] == 0.0) and dcam[1, 3 + axis] == 0.0
    unseen = np.bincount(obs[1], minlength=n) == 0
    assert np.all(dP[unseen] == 0.0)
    eta = _backward_error(R, t, P, obs, p.K, lam, axis, dcam, dP)
    assert eta <= BACKWARD_TOL, eta
    # forward error within cond(H) x the normwise backward error of the GPU step
    Hd, b, diag, ci, nc, _ = O.normal_equations(R64, t64, P64, obs, p.K, SIGMA, DELTA, lam, axis)
    un = diag == 0.0
    Hd[un, un] = 1.0
    x_o = np.concatenate([dc_o[ci >= 0], dP_o.ravel()])
    x_g = np.concatenate([dcam[ci >= 0], dP.ravel()])
    eta_n = np.linalg.norm(Hd @ x_g - b) / (np.linalg.norm(Hd, 2) * np.linalg.norm(x_g) + np.linalg.norm(b))
    fwd = np.linalg.norm(x_g - x_o) / np.linalg.norm(x_o)
    assert fwd <= 2.0 * np.linalg.cond(Hd) * eta_n + 1e-6, (fwd, eta_n)


def test_solve_reaches_the_oracle_minimum(B):
    p, obs, R, t, P = _setup(14, 6, 150, False)
    ba = B.BundleAdjuster(6, 150, len(obs[0]))
    Rd, td, Pd, cd, pd, uvd = _dev(R, t, P, obs)
    costs, acc = ba.solve(Rd, td, Pd, cd, pd, uvd, p.K, SIGMA, DELTA, iters=15, lam0=1e-4)
    R_o, t_o, P_o, costs_o = O.solve(R.astype(np.float64), t.astype(np.float64), P.astype(np.float64), obs, p.K,
                                     SIGMA, DELTA, iters=15, lam=1e-4)
    assert acc >= 5 and np.all(np.diff(costs) <= 0)
    assert abs(costs[0] - costs_o[0]) <= 1e-9 * costs_o[0]
    assert abs(costs[-1] - costs_o[-1]) <= 1e-5 * costs_o[-1], (costs[-1], costs_o[-1])
    Rg, tg, Pg = Rd.cpu().numpy(), td.cpu().numpy(), Pd.cpu().numpy()
    assert np.array_equal(Rg[0], R[0]) and np.array_equal(tg[0], t[0])
    axis = O.gauge_axis(R.astype(np.float64), t.astype(np.float64))
    assert tg[1, axis] == t[1, axis]
    seen = np.bincount(obs[1], minlength=150) > 0
    assert np.abs(Pg[seen] - P_o[seen]).max() < 1e-4
    assert np.abs(tg - t_o).max() < 1e-4


def test_full_size_step_and_solve(B):
    """32 cameras, 20k points with feature tracks of 2-12 consecutive cameras (the benchmarked
    problem): every row of the step's normal equations, checked matrix-free; LM reaches the noise
    floor."""
    C, n = 32, 20000
    p, obs, R, t, P = _setup(7, C, n, True)
    m = len(obs[0])
    ba = B.BundleAdjuster(C, n, m)
    Rd, td, Pd, cd, pd, uvd = _dev(R, t, P, obs)
    lam = 1e-4
    dcam, dP, cost = ba.step(Rd, td, Pd, cd, pd, uvd, p.K, SIGMA, DELTA, lam)
    dcam, dP = dcam.cpu().numpy().astype(np.float64), dP.cpu().numpy().astype(np.float64)
    axis = O.gauge_axis(R.astype(np.float64), t.astype(np.float64))
    eta = _backward_error(R, t, P, obs, p.K, lam, axis, dcam, dP)
    assert eta <= BACKWARD_TOL, eta
    costs, acc = ba.solve(Rd, td, Pd, cd, pd, uvd, p.K, SIGMA, DELTA, iters=10, lam0=1e-4)
    assert np.all(np.diff(costs) <= 0) and acc >= 5
    # noise floor: whitened residuals ~ chi^2 with 2 dof per observation, minus the parameters fitted
    seen = len(np.unique(obs[1]))
    dof = 2 * m - (6 * C - 7) - 3 * seen
    assert 0.5 * dof < costs[-1] < 1.05 * dof, (costs[-1], dof)


def test_bad_observation_indices_are_rejected(B):
    from paper_2601_17354_gb300 import _lib as L
    p, obs, R, t, P = _setup(15, 6, 60, False)
    cams, pts, uv = (np.array(a) for a in obs)
    ba = B.BundleAdjuster(6, 60, len(cams))
    cases = []
    c2 = cams.copy(); c2[3] = 6; cases.append((c2, pts))                     # camera out of range
    p2 = pts.copy(); p2[-1] = 60; cases.append((cams, p2))                    # point out of range
    p3 = pts.copy(); p3[[0, -1]] = p3[[-1, 0]]; cases.append((cams, p3))      # not grouped by point
    c4 = cams.copy(); c4[1] = c4[0]; cases.append((c4, pts))                  # same camera twice in a point
    for cc, pp in cases:
        Rd, td, Pd, cd, pd, uvd = _dev(R, t, P, (cc, pp, uv))
        with pytest.raises(L.PgsError) as e:
            ba.step(Rd, td, Pd, cd, pd, uvd, p.K, SIGMA, DELTA, 1e-3)
        assert e.value.code == L.PGS_ERR_INVALID_ARG


def test_projection_matches_oracle(B):
    p = S.ba_problem(16, 5, 200)
    R, t, P = (x.astype(np.float32) for x in (p.R_gt, p.t_gt, p.P_gt))
    cams = np.repeat(np.arange(5), 200).astype(np.int32)
    pts = np.tile(np.arange(200), 5).astype(np.int32)
    ba = B.BundleAdjuster(5, 200, len(cams))
    Rd, td, Pd, cd, pd, _ = _dev(R, t, P, (cams, pts, np.zeros((len(cams), 2))))
    uv, z = ba.project(Rd, td, Pd, cd, pd, p.K)
    for i in range(5):
        uo, Xo = O.project(R[i].astype(np.float64), t[i].astype(np.float64), P.astype(np.float64), p.K)
        sel = slice(200 * i, 200 * (i + 1))
        assert np.allclose(uv.cpu().numpy()[sel], uo, rtol=0, atol=1e-3)
        assert np.allclose(z.cpu().numpy()[sel], Xo[:, 2], rtol=1e-6, atol=0)
    # an index out of range gives NaN and no access
    bad = torch.tensor([5, 0], dtype=torch.int32, device="cuda"), torch.tensor([0, 200], dtype=torch.int32, device="cuda")
    uv, z = ba.project(Rd, td, Pd, bad[0], bad[1], p.K)
    assert torch.isnan(uv).all() and torch.isnan(z).all()
