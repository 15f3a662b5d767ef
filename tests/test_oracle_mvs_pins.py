"""Pins of the MVS oracle (oracle/mvs.py): census closed forms and invariance, the plane map
against direct projection, zero cost for a view paired with itself, SGM against brute force over
label sequences and its zero-penalty special case, exact parabola refinement, quantiles against
numpy, the Eq. 4 score's closed form, and depths against the ray-cast ground truth."""
import itertools
import math

import numpy as np
import pytest

from oracle import mvs as M
from paper_2601_17354_gb300 import synthetic as S


def test_census_single_bright_pixel_and_invariance():
    Y = np.zeros((12, 15), np.float32)
    Y[6, 7] = 1.0
    c = M.census(Y)
    assert c[6, 7] == (1 << 48) - 1                     # every neighbour is darker
    c[6, 7] = 0
    assert not c.any()                                  # nothing else has a darker neighbour
    rng = np.random.default_rng(0)
    Yi = rng.integers(0, 256, (20, 23)).astype(np.float32)
    assert np.array_equal(M.census(Yi), M.census(Yi * Yi + 3 * Yi))   # strictly increasing map
    # a border pixel leaves its outside neighbours' bits clear
    Z = np.ones((9, 9), np.float32)
    Z[0, 0] = 2.0
    assert bin(int(M.census(Z)[0, 0])).count("1") == 15   # the 4 x 4 - 1 inside neighbours


def test_plane_map_matches_direct_projection():
    sc = S.mvs_scene(5, n_cameras=16, width=160, height=90, focal=125.0, views=[])
    ct, cr = sc.cameras[2], sc.cameras[3]
    inv_far, step = M.inverse_depths(2.0, 6.0, 8)
    maps = M.plane_maps(ct, cr, inv_far, step, 8)
    rng = np.random.default_rng(1)
    Rt, tt = ct.viewmat[:, :3].astype(np.float64), ct.viewmat[:, 3].astype(np.float64)
    Rr, tr = cr.viewmat[:, :3].astype(np.float64), cr.viewmat[:, 3].astype(np.float64)
    for k in range(8):
        d = 1.0 / (inv_far + k * step)
        for _ in range(20):
            x, y = rng.uniform(0, 160), rng.uniform(0, 90)
            Xt = d * np.array([(x - ct.cx) / ct.fx, (y - ct.cy) / ct.fy, 1.0])
            Xr = Rr @ (Rt.T @ (Xt - tt)) + tr
            uv = np.array([cr.fx * Xr[0] / Xr[2] + cr.cx, cr.fy * Xr[1] / Xr[2] + cr.cy])
            h = maps[k].astype(np.float64).reshape(3, 3) @ np.array([x, y, 1.0])
            assert np.allclose(h[:2] / h[2], uv, atol=2e-3), (k, h[:2] / h[2], uv)


def test_view_paired_with_itself_costs_nothing():
    sc = S.mvs_scene(6, n_cameras=16, width=96, height=64, focal=75.0, views=[1])
    cen = M.census(M.luma(sc.images[1]))
    inv_far, step = M.inverse_depths(2.0, 6.0, 6)
    maps = M.plane_maps(sc.cameras[1], sc.cameras[1], inv_far, step, 6)
    C = M.cost_volume(cen, cen, maps)
    assert not C.any()


def _brute_path(C, p1, p2):
    """min over label sequences ending at k of sum C + transition penalties (0 / P1 / P2)."""
    W, D = C.shape
    out = np.zeros((W, D), np.int64)
    for x in range(W):
        for k in range(D):
            best = None
            for seq in itertools.product(range(D), repeat=x):
                labels = list(seq) + [k]
                cost = sum(int(C[i, labels[i]]) for i in range(x + 1))
                for i in range(1, x + 1):
                    dk = abs(labels[i] - labels[i - 1])
                    cost += 0 if dk == 0 else (p1 if dk == 1 else p2)
                best = cost if best is None else min(best, cost)
            out[x, k] = best
    return out


def test_sgm_path_equals_brute_force_minimisation():
    rng = np.random.default_rng(2)
    for trial in range(4):
        C = rng.integers(0, 49, (1, 5, 4)).astype(np.uint8)
        L = M.sgm_path(C)[0]
        ref = _brute_path(C[0], M.P1, M.P2)
        shift = np.concatenate([[0], np.cumsum(L.min(axis=1))[:-1]])   # the subtracted minima
        assert np.array_equal(L + shift[:, None], ref), trial


def test_sgm_without_penalties_is_four_times_the_cost():
    rng = np.random.default_rng(3)
    C = rng.integers(0, 49, (7, 9, 5)).astype(np.uint8)
    assert np.array_equal(M.sgm(C, 0, 0), 4 * C.astype(np.uint16))


def test_parabola_refinement_and_confidence():
    D = 24
    k = np.arange(D)
    Sv = (64 * k * k - 1312 * k + 6724 + 100).astype(np.uint16)   # 64 (k - 10.25)^2 + 100
    inv_far, step = 0.2, 0.01
    k1, kept, depth = M.select_depth(Sv[None, None, :], inv_far, step)
    assert k1[0, 0] == 10 and kept[0, 0]                           # 1 - 104 / 296 >= 0.4
    assert abs(1.0 / depth[0, 0] - (inv_far + 10.25 * step)) < 1e-6
    shallow = (16 * k * k - 328 * k + 1681 + 100).astype(np.uint16)  # 1 - 101 / 149 < 0.4
    _, kept1, depth1 = M.select_depth(shallow[None, None, :], inv_far, step)
    assert not kept1[0, 0] and np.isnan(depth1[0, 0])
    flat = np.full((1, 1, D), 50, np.uint16)
    flat[0, 0, 5] = 10
    _, kept2, _ = M.select_depth(flat, inv_far, step)
    assert kept2[0, 0]                                             # 1 - 10 / 50 = 0.8
    edge = np.full((1, 1, D), 50, np.uint16)
    edge[0, 0, 0] = 1
    _, kept3, _ = M.select_depth(edge, inv_far, step)
    assert not kept3[0, 0]                                         # minimum on the first plane


def test_quantiles_and_range():
    rng = np.random.default_rng(4)
    v = rng.uniform(1, 9, 1001)
    for p in (0.05, 0.5, 0.95):
        assert abs(M.quantile(v, p) - np.quantile(v, p)) < 1e-12
    assert M.quantile(np.arange(101.0), 0.05) == 5.0


def test_reference_score_closed_form():
    class Cam:
        def __init__(self, R, t):
            self.viewmat = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    I = np.eye(3)
    bt = M.B_TARGET_FRACTION * 4.0
    cams = [Cam(I, np.zeros(3)), Cam(I, np.array([-bt, 0.0, 0.0])), Cam(I, np.array([-2 * bt, 0.0, 0.0]))]
    s = M.reference_scores(cams, 0, 4.0)
    assert s[0] == -np.inf
    assert abs(s[1] - 1.0) < 1e-6                                 # b = b_target, parallel axes
    assert abs(s[2] - math.exp(-1.0 / (2 * M.SIGMA_B_FRACTION ** 2))) < 1e-5


@pytest.mark.parametrize("target", [4, 37])
def test_depths_match_ray_cast_ground_truth(target):
    sc = S.mvs_scene(3, views=[target - 1, target, target + 1])
    ref, rng_, C, Sv, k1, kept, depth, P, idx = M.reconstruct_view(sc.images, sc.cameras, sc.sparse, target)
    gt = sc.depths[target]
    fg = kept & np.isfinite(gt)
    rel = np.abs(depth[fg] - gt[fg]) / gt[fg]
    assert fg.sum() > 0.4 * np.isfinite(gt).sum()
    assert np.median(rel) < 0.01 and (rel < 0.02).mean() > 0.9
    assert abs(ref - target) in (1, len(sc.cameras) - 1)          # a neighbouring keyframe
