"""The paper's replay-cache backward (Eq. 9: per-pixel record of the forward, count reset every
render) against the oracle and against the recompute backward, including the overflow fallback
and immunity to entries a previous render left in the cache."""
import numpy as np
import pytest

import oracle
from paper_2601_17354_gb300 import synthetic as S
from tests._parity import check_render, compare_grads, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2601_17354_gb300 import rasterizer
    return rasterizer


def scene(name):
    if name == "surface":
        sc = S.surface_scene(3, 20000, 3, 200, 120, 160.0, n_cameras=8)
        return sc.gt, sc.cameras[3]
    return S.tiny_scene(1, n=1500, width=100, height=75)[:2]


def backward(R, rast, g, cam, dL):
    buf = R.GaussianBuffer.from_arrays(g)
    img = rast.render(buf, cam).clone()
    grads = buf.zeros_like()
    rast.backward(torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    assert rast.status()[0] == 0
    return img.cpu().numpy(), grads.numpy()


@pytest.mark.parametrize("k_max", [256, 3])
@pytest.mark.parametrize("name", ["ragged", "surface"])
def test_replay_matches_oracle_and_recompute(R, name, k_max):
    g, cam = scene(name)
    cam.bg = (0.1, 0.3, 0.2)
    dL = S.random_image(21, cam.width, cam.height)
    rec = R.Rasterizer()
    rec.set_variant(1, 256)
    img0, g0 = backward(R, rec, g, cam, dL)
    rep = R.Rasterizer()
    rep.set_replay_cache(k_max)
    img1, g1 = backward(R, rep, g, cam, dL)
    assert np.array_equal(img1, img0)  # recording does not change the forward
    _, forced = check_render(rep, g, cam, img1)
    _, og = oracle.backward(g, cam, dL, forced=forced)
    compare_grads(g1, og, oracle.gaussian_flags(g, cam) == 0)
    for k in g0:
        assert rel_l2(g1[k], g0[k]) < 1e-4, k


def test_entries_of_a_previous_render_are_not_replayed(R):
    g_dense, cam = scene("surface")
    g_sparse = S.tiny_scene(7, n=300, width=cam.width, height=cam.height)[0]
    dL = S.random_image(22, cam.width, cam.height)
    rep = R.Rasterizer()
    rep.set_replay_cache(64)
    backward(R, rep, g_dense, cam, dL)     # fills the cache deeply
    _, after = backward(R, rep, g_sparse, cam, dL)
    fresh = R.Rasterizer()
    fresh.set_replay_cache(64)
    _, clean = backward(R, fresh, g_sparse, cam, dL)
    for k in clean:
        assert np.array_equal(after[k], clean[k]) or rel_l2(after[k], clean[k]) < 1e-6, k


def test_switching_the_cache_needs_a_new_render(R):
    g, cam = scene("ragged")
    rast = R.Rasterizer()
    buf = R.GaussianBuffer.from_arrays(g)
    rast.render(buf, cam)
    rast.set_replay_cache(16)
    with pytest.raises(RuntimeError):
        rast.backward(torch.zeros(3, cam.height, cam.width, device="cuda"), buf.zeros_like())
