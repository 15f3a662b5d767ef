"""The seeded input generators (no GPU) against the recipe they state: determinism, shapes,
distributions and camera geometry."""
import math

import numpy as np
import pytest

from paper_2601_17354_gb300 import synthetic as S


def test_tiny_scene_is_seeded_and_follows_its_laws():
    g, cam, target = S.tiny_scene(5, n=20000)
    g2, cam2, target2 = S.tiny_scene(5, n=20000)
    assert np.array_equal(g.means, g2.means) and np.array_equal(target, target2)
    assert not np.array_equal(g.means, S.tiny_scene(6, n=20000)[0].means)
    assert g.means.dtype == np.float32 and g.means.shape == (3, 20000)
    assert g.means.min() >= -1.0 and g.means.max() <= 1.0
    assert abs(g.log_scales.mean() + 3.0) < 0.01 and abs(g.log_scales.std() - 0.3) < 0.01
    assert abs(g.opacity_logits.mean()) < 0.03 and abs(g.opacity_logits.std() - 1.0) < 0.02
    assert g.sh.shape == (3, 1, 20000)
    # degree-0 colour uniform in [0, 1]: 0.5 + Y0 * DC
    rgb = 0.5 + 0.28209479177387814 * g.sh[:, 0, :]
    assert rgb.min() >= 0.0 and rgb.max() <= 1.0 and abs(rgb.mean() - 0.5) < 0.01
    # camera at (0, 0, -3) looking along +z
    V = cam.viewmat
    assert np.array_equal(V[:, :3], np.eye(3, dtype=np.float32)) and V[2, 3] == 3.0
    assert (cam.width, cam.height, cam.fx, cam.cx) == (128, 128, 150.0, 64.0)
    assert target.min() >= 0.0 and target.max() <= 1.0


def test_lookat_viewmat_is_a_rigid_map_onto_the_target():
    eye = np.array([3.0, -1.0, 2.0])
    V = S.lookat_viewmat(eye).astype(np.float64)
    R, t = V[:, :3], V[:, 3]
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-6) and np.linalg.det(R) > 0
    assert np.allclose(R @ eye + t, 0.0, atol=1e-5)  # the eye is the camera centre
    origin = R @ np.zeros(3) + t
    assert abs(origin[0]) < 1e-5 and abs(origin[1]) < 1e-5 and origin[2] > 0  # target on the axis, ahead


def test_ring_cameras_and_held_out_views():
    sc = S.surface_scene(3, 4000, sh_degree=2, width=320, height=240, focal=250.0, n_cameras=16)
    assert len(sc.cameras) == 16
    centres = []
    for c in sc.cameras:
        R, t = c.viewmat[:, :3].astype(np.float64), c.viewmat[:, 3].astype(np.float64)
        centre = -R.T @ t
        centres.append(centre)
        assert abs(np.linalg.norm(centre) - 4.0) < 1e-4
        assert abs(math.degrees(math.asin(centre[2] / 4.0))) <= 10.0 + 1e-4
    az = np.unwrap([math.atan2(c[1], c[0]) for c in centres])
    assert np.allclose(np.diff(az), 2 * math.pi / 16, atol=1e-4)
    assert sc.test_views() == [0, 8] and len(sc.train_views()) == 14
    assert set(sc.test_views()).isdisjoint(sc.train_views())


def test_surface_scene_laws_and_points_on_surfaces():
    sc = S.surface_scene(7, 30000, sh_degree=3, width=320, height=240, focal=250.0, n_cameras=8)
    g = sc.gt
    assert g.sh.shape == (3, 16, 30000)
    assert abs(g.log_scales.mean() + 4.0) < 0.01 and abs(g.log_scales.std() - 0.3) < 0.01
    assert abs(g.opacity_logits.mean() - 1.0) < 0.01 and abs(g.opacity_logits.std() - 0.5) < 0.01
    assert abs(g.sh[:, 1:, :].std() - 0.05) < 0.001
    assert np.abs(g.means).max() <= 2.0 + 1e-5  # inside [-2, 2]^3
    # every GT point lies on a sphere or on a square of the scene
    P = g.means.T.astype(np.float64)
    s = sc.surfaces
    d_sphere = np.min(np.abs(np.linalg.norm(P[:, None, :] - s.sphere_c[None], axis=2) - s.sphere_r[None]), axis=1)
    n = np.cross(s.plane_u, s.plane_v)
    rel = P[:, None, :] - s.plane_c[None]
    on_plane = (np.abs(np.einsum("pqk,qk->pq", rel, n)) < 1e-4) & \
               (np.abs(np.einsum("pqk,qk->pq", rel, s.plane_u)) <= s.plane_side[None] / 2 + 1e-4) & \
               (np.abs(np.einsum("pqk,qk->pq", rel, s.plane_v)) <= s.plane_side[None] / 2 + 1e-4)
    assert np.all((d_sphere < 1e-4) | on_plane.any(axis=1))
    # the trainable start is a different, noisy sample of the same surfaces
    assert sc.init.means.shape == g.means.shape and not np.array_equal(sc.init.means, g.means)


def test_batched_scenes_are_uneven_within_the_stated_ranges():
    scenes = S.batched_scenes(11, n_scenes=6, views_per_scene=2, n_range=(2_000, 30_000), sh_degree=0)
    assert len(scenes) == 6
    for sc in scenes:
        n = sc.gt.means.shape[1]
        assert 2_000 <= n <= 30_000
        c = sc.cameras[0]
        assert (c.width, c.height) in ((640, 480), (960, 720), (1280, 720))
        assert c.fx == pytest.approx(1000.0 * c.width / 1280.0)
        assert len(sc.cameras) == 2
    assert len({sc.gt.means.shape[1] for sc in scenes}) > 1


def test_ba_problem_perturbations_and_tracks():
    p = S.ba_problem(4, n_cams=12, n_points=3000)
    assert np.array_equal(p.R_init[0], p.R_gt[0]) and np.array_equal(p.t_init[0], p.t_gt[0])
    for i in range(1, 12):
        dR = p.R_init[i] @ p.R_gt[i].T
        angle = math.degrees(math.acos(min(1.0, (np.trace(dR) - 1.0) / 2.0)))
        assert angle <= 0.5 + 1e-6
    assert abs((p.t_init[1:] - p.t_gt[1:]).std() - 0.02) < 0.006
    assert abs((p.P_init - p.P_gt).std() - 0.01) < 0.001
    assert abs(p.noise.std() - 0.5) < 0.01
    assert p.track_len.min() >= 2 and p.track_len.max() <= 12
    assert p.track_start.min() >= 0 and p.track_start.max() < 12
    assert p.K == (1000.0, 1000.0, 640.0, 360.0)


def test_random_image_is_seeded_and_bounded():
    a = S.random_image(9, 33, 17)
    assert a.shape == (3, 17, 33) and a.dtype == np.float32
    assert np.array_equal(a, S.random_image(9, 33, 17))
    assert a.min() >= -1.0 and a.max() <= 1.0
