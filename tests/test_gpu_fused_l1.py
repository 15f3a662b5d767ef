"""The L1 loss fused into the compositing forward (pgs_render_l1) against pgs_render followed by
pgs_loss_l1, whose arithmetic the oracle pins (test_l1_loss_matches_oracle): the image, T_final,
last and dL/dimage bit for bit, the two loss sums to rounding, for every forward strip and tile
edge, with the replay cache on, on an empty scene, on a repeated call and through the backward
that follows."""
import numpy as np
import pytest

from paper_2601_17354_gb300 import synthetic as S
from tests._parity import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-5  # float partial sums per thread, added per CTA then in double: another order


@pytest.fixture(scope="module")
def R():
    from paper_2601_17354_gb300 import rasterizer
    return rasterizer


def surface():
    sc = S.surface_scene(3, 20000, 3, 200, 120, 160.0, n_cameras=8)
    cam = sc.cameras[3]
    cam.bg = (0.1, 0.3, 0.2)
    return sc.gt, cam


def reference(R, rast, buf, cam, target):
    """render, then the loss kernel on its image: (image, T_final, last, dL, loss)."""
    from paper_2601_17354_gb300 import _lib as L
    img = rast.render(buf, cam).clone()
    torch.cuda.synchronize()
    T = rast.read_buffer(L.PGS_BUF_T_FINAL)
    last = rast.read_buffer(L.PGS_BUF_LAST)
    dl, loss = rast.loss_l1(img, target)
    torch.cuda.synchronize()
    return img, T, last, dl.clone(), loss.cpu().numpy()


def fused(R, rast, buf, cam, target):
    from paper_2601_17354_gb300 import _lib as L
    img, dl, loss = rast.render_l1(buf, cam, target)
    torch.cuda.synchronize()
    assert rast.status()[0] == 0
    T = rast.read_buffer(L.PGS_BUF_T_FINAL)
    last = rast.read_buffer(L.PGS_BUF_LAST)
    return img, T, last, dl, loss.cpu().numpy()


def assert_same(ref, got):
    img, T, last, dl, loss = ref
    gimg, gT, glast, gdl, gloss = got
    assert torch.equal(gimg, img)
    assert np.array_equal(gT, T) and np.array_equal(glast, last)
    assert torch.equal(gdl, dl)
    assert np.all(np.abs(gloss - loss) <= LOSS_RTOL * np.abs(loss)), (gloss, loss)


def target_with_ties(img, seed):
    """A seeded target that equals the image on a lattice of pixels (sign(0) = 0 there)."""
    _, h, w = img.shape
    t = torch.from_numpy(S.random_image(seed, w, h, 0.0, 1.0)).cuda()
    t[:, ::7, ::5] = img[:, ::7, ::5]
    return t.contiguous()


# (tile edge, forward strip): one pixel per thread (scalar epilogue), two and four (pairs)
CASES = [(8, (1, 64)), (8, (2, 128)), (16, (1, 256)), (16, (2, 256)), (16, (4, 64)), (32, (2, 128)),
         (32, (4, 256))]


@pytest.mark.parametrize("tile,fwd", CASES)
def test_fused_l1_equals_render_then_loss(R, tile, fwd):
    g, cam = surface()
    buf = R.GaussianBuffer.from_arrays(g)
    ra, rb = R.Rasterizer(tile=tile), R.Rasterizer(tile=tile)
    ra.set_variants(fwd, (2, 64))
    rb.set_variants(fwd, (2, 64))
    target = target_with_ties(ra.render(buf, cam), 21)
    ref = reference(R, ra, buf, cam, target)
    got = fused(R, rb, buf, cam, target)
    assert_same(ref, got)
    assert torch.count_nonzero(got[3] == 0) >= 3 * len(range(0, cam.height, 7)) * len(range(0, cam.width, 5))


def test_fused_l1_repeated_on_one_context(R):
    """The accumulators and the ticket start from zero on every render (the projection clears
    them): a second call with another target reports that target's loss."""
    g, cam = surface()
    buf = R.GaussianBuffer.from_arrays(g)
    ra, rb = R.Rasterizer(), R.Rasterizer()
    for seed in (5, 6, 7):
        target = target_with_ties(ra.render(buf, cam), seed)
        assert_same(reference(R, ra, buf, cam, target), fused(R, rb, buf, cam, target))


def test_fused_l1_with_replay_cache(R):
    g, cam = surface()
    buf = R.GaussianBuffer.from_arrays(g)
    ra, rb = R.Rasterizer(), R.Rasterizer()
    ra.set_replay_cache(256)
    rb.set_replay_cache(256)
    target = target_with_ties(ra.render(buf, cam), 8)
    assert_same(reference(R, ra, buf, cam, target), fused(R, rb, buf, cam, target))


def test_fused_l1_empty_scene(R):
    g, cam = surface()
    g = g.subset(np.arange(0))
    buf = R.GaussianBuffer.from_arrays(g)
    ra, rb = R.Rasterizer(), R.Rasterizer()
    target = torch.from_numpy(S.random_image(9, cam.width, cam.height, 0.0, 1.0)).cuda()
    ref = reference(R, ra, buf, cam, target)
    got = fused(R, rb, buf, cam, target)
    assert_same(ref, got)
    assert torch.allclose(got[0], torch.tensor(cam.bg, device="cuda").view(3, 1, 1).expand_as(got[0]))


def test_backward_after_fused_l1(R):
    """The gradients of the backward that follows the fused call are those of render + loss +
    backward (float atomics add in a scheduling-dependent order: equal to rounding)."""
    g, cam = surface()
    buf = R.GaussianBuffer.from_arrays(g)
    ra, rb = R.Rasterizer(), R.Rasterizer()
    target = target_with_ties(ra.render(buf, cam), 10)
    _, _, _, dl_ref, _ = reference(R, ra, buf, cam, target)
    ga = buf.zeros_like()
    ra.backward(dl_ref, ga)
    _, _, _, dl, _ = fused(R, rb, buf, cam, target)
    gb = buf.zeros_like()
    rb.backward(dl, gb)
    torch.cuda.synchronize()
    assert torch.count_nonzero(ga.data) > 0
    assert rel_l2(gb.data.cpu().numpy(), ga.data.cpu().numpy()) < 1e-5


def test_fused_l1_rejects_missing_buffers(R):
    from paper_2601_17354_gb300 import _lib as L
    import ctypes as C
    g, cam = surface()
    buf = R.GaussianBuffer.from_arrays(g)
    rast = R.Rasterizer()
    img = torch.empty(3, cam.height, cam.width, device="cuda")
    cs = R.camera_struct(cam)
    gs = buf.struct()
    code = L.lib().pgs_render_l1(rast._ctx, C.byref(gs), C.byref(cs), None, C.c_void_p(img.data_ptr()),
                                 C.c_void_p(img.data_ptr()), None)
    assert code == L.PGS_ERR_INVALID_ARG
