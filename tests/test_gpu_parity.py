"""GPU parity: every stage of the CUDA path, called through the C ABI, against the CPU oracle on
the same seeded inputs."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_17354_gb300 import synthetic as S
from tests._parity import compare_forward, compare_grads, rel_l2, IMAGE_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2601_17354_gb300 import rasterizer
    return rasterizer


def render_gpu(R, g, cam, rast=None):
    rast = rast or R.Rasterizer()
    buf = R.GaussianBuffer.from_arrays(g)
    img = rast.render(buf, cam)
    torch.cuda.synchronize()
    code, pairs = rast.status()
    from paper_2601_17354_gb300 import _lib as L
    T = rast.read_buffer(L.PGS_BUF_T_FINAL).reshape(cam.height, cam.width)
    last = rast.read_buffer(L.PGS_BUF_LAST).reshape(cam.height, cam.width)
    return rast, buf, img.cpu().numpy(), T, last, code, pairs


def check_keys(rast, g, cam, tile=16):
    from paper_2601_17354_gb300 import _lib as L
    k, v, r = oracle.keys(g, cam, tile)
    gk = rast.read_buffer(L.PGS_BUF_KEYS)
    gv = rast.read_buffer(L.PGS_BUF_VALUES)
    gr = rast.read_buffer(L.PGS_BUF_RANGES).reshape(-1, 2)
    assert len(gk) == len(k)
    assert np.array_equal(gk, k), f"{np.sum(gk != k)} keys differ"
    assert np.array_equal(gv, v)
    assert np.array_equal(gr, r)
    return len(k)


SCENES = {
    "tiny_2k_128": lambda: S.tiny_scene(0)[:2],
    "ragged_100x75": lambda: S.tiny_scene(1, n=1500, width=100, height=75)[:2],
    "dense_20k_64": lambda: S.tiny_scene(2, n=20000, width=64, height=64, focal=60.0)[:2],
    "surface_sh3_200x120": lambda: (lambda sc: (sc.gt, sc.cameras[3]))(
        S.surface_scene(3, 20000, 3, 200, 120, 160.0, n_cameras=8)),
}


@pytest.mark.parametrize("name", list(SCENES))
def test_forward_keys_and_image(R, name):
    g, cam = SCENES[name]()
    rast, _, img, T, last, code, pairs = render_gpu(R, g, cam)
    assert code == 0
    P = check_keys(rast, g, cam)
    assert pairs == P
    ora = oracle.render(g, cam)
    compare_forward(img, T, last, ora, (rast, g, cam, 16))


@pytest.mark.parametrize("name", ["tiny_2k_128", "dense_20k_64", "surface_sh3_200x120"])
def test_decision_trace_against_oracle_decisions(R, name):
    """The decision trace walks every pixel as the render did (T_final bit-exact, last and the
    composited count equal), the kernel's o G of every evaluated entry (above the flush-to-zero
    range of its 2^p) lies within the oracle's stated bound of its decision-side o 2^p, and on
    unflagged pixels the two take the same decision at every entry."""
    from paper_2601_17354_gb300 import _lib as L
    from tests._parity import list_lengths
    g, cam = SCENES[name]()
    rast, _, img, T, last, code, pairs = render_gpu(R, g, cam)
    ncomp = rast.read_buffer(L.PGS_BUF_NCOMP).reshape(cam.height, cam.width)
    rng = np.random.default_rng(5)
    pix = np.stack([rng.integers(0, cam.width, 2000), rng.integers(0, cam.height, 2000)], 1).astype(np.int32)
    ora = oracle.render(g, cam)
    flagged = np.argwhere(ora["flag"] != 0)[:, ::-1].astype(np.int32)
    pix = np.concatenate([pix, flagged])
    E = int(list_lengths(g, cam, pix).max())
    tr = rast.trace_pixels(pix, E)
    od = oracle.decisions(g, cam, pix, E)
    xs, ys = pix[:, 0], pix[:, 1]
    assert np.array_equal(tr["T"].view(np.uint32), T[ys, xs].view(np.uint32))
    assert np.array_equal(tr["last"], last[ys, xs])
    assert np.array_equal(tr["ncomp"], ncomp[ys, xs])
    eps = oracle.decision_bound()
    worst = 0.0
    for k in range(len(pix)):
        n = min(tr["count"][k], od["count"][k])
        # o G of an entry does not depend on the walk before it: compare every entry both evaluated
        a, b = tr["og"][k, :n].astype(np.float64), od["og"][k, :n]
        nz = b > 2.0 ** -100  # the kernel's 2^p flushes below 2^-126 to zero (skipped either way)
        if nz.any():
            worst = max(worst, float(np.max(np.abs(a[nz] / b[nz] - 1.0))))
        if ora["flag"][ys[k], xs[k]] == 0:
            assert tr["count"][k] == od["count"][k], (xs[k], ys[k])
            assert np.array_equal(tr["code"][k, :n], od["code"][k, :n]), (xs[k], ys[k])
    print(f"largest relative deviation of the kernel's o G: {worst:.3g} (bound {eps:.3g})")
    assert worst <= eps


@pytest.mark.parametrize("tile", [8, 32])
@pytest.mark.parametrize("name", ["ragged_100x75", "surface_sh3_200x120"])
def test_other_tile_edges(R, name, tile):
    """8x8 and 32x32 tiles: keys and ranges bit-exact against the oracle binned with the same
    edge, image and gradients within tolerance, every strip the edge takes renders the same."""
    from paper_2601_17354_gb300 import _lib as L
    g, cam = SCENES[name]()
    cam.bg = (0.1, 0.3, 0.2)
    rast = R.Rasterizer(tile=tile)
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam, rast)
    assert code == 0
    assert pairs == check_keys(rast, g, cam, tile)
    ora = oracle.render(g, cam, tile)
    _, forced = compare_forward(img, T, last, ora, (rast, g, cam, tile))
    dL = S.random_image(13, cam.width, cam.height)
    grads = buf.zeros_like()
    rast.backward(torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    _, og = oracle.backward(g, cam, dL, tile, forced=forced)
    compare_grads(grads.numpy(), og, oracle.gaussian_flags(g, cam, tile) == 0)
    for pix, depth in L.VARIANTS:
        if (tile == 8 and pix == 4) or (tile == 32 and pix == 1):
            with pytest.raises(RuntimeError):
                rast.set_variant(pix, depth)
            continue
        rast.set_variant(pix, depth)
        assert np.array_equal(rast.render(buf, cam).cpu().numpy(), img), (pix, depth)


@pytest.mark.parametrize("name", list(SCENES))
def test_backward_grads(R, name):
    g, cam = SCENES[name]()
    cam.bg = (0.1, 0.3, 0.2)
    rast, buf, img, T, last, code, _ = render_gpu(R, g, cam)
    ora = oracle.render(g, cam)
    _, forced = compare_forward(img, T, last, ora, (rast, g, cam, 16))
    dL = S.random_image(11, cam.width, cam.height)
    grads = buf.zeros_like()
    rast.backward(torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    o2, og = oracle.backward(g, cam, dL, forced=forced)
    keep = oracle.gaussian_flags(g, cam) == 0
    from paper_2601_17354_gb300 import _lib as L
    g2 = rast.read_buffer(L.PGS_BUF_GRAD2D).reshape(9, g.n)
    for k in range(9):
        assert rel_l2(g2[k, keep], o2[keep, k]) < 1e-3, k
    compare_grads(grads.numpy(), og, keep)


def test_separate_forward_and_backward_variants(R):
    """A forward strip and a different backward strip on one context: the image is the oracle's
    and the gradients match it as with one variant."""
    g, cam = SCENES["surface_sh3_200x120"]()
    cam.bg = (0.1, 0.3, 0.2)
    ora = oracle.render(g, cam)
    dL = S.random_image(13, cam.width, cam.height)
    keep = oracle.gaussian_flags(g, cam) == 0
    og = None
    for fwd, bwd in (((1, 64), (4, 256)), ((4, 128), (2, 64))):
        rast = R.Rasterizer()
        rast.set_variants(fwd, bwd)
        rast, buf, img, T, last, _, _ = render_gpu(R, g, cam, rast)
        _, forced = compare_forward(img, T, last, ora, (rast, g, cam, 16))
        if og is None:
            _, og = oracle.backward(g, cam, dL, forced=forced)
        grads = buf.zeros_like()
        rast.backward(torch.from_numpy(dL).cuda(), grads)
        torch.cuda.synchronize()
        compare_grads(grads.numpy(), og, keep)


def test_fused_backward_step_matches_oracle_and_separate_calls(R):
    """pgs_backward_step == pgs_backward + pgs_step; its first-step moment m = (1 - b1) g
    exposes the in-register parameter gradient, checked against the oracle."""
    from paper_2601_17354_gb300 import _lib as L
    g, cam = SCENES["surface_sh3_200x120"]()
    cam.bg = (0.1, 0.3, 0.2)
    ora = oracle.render(g, cam)
    dL = S.random_image(12, cam.width, cam.height)
    dLt = torch.from_numpy(dL).cuda()
    ra, rb = R.Rasterizer(), R.Rasterizer()
    pa, pb = R.GaussianBuffer.from_arrays(g), R.GaussianBuffer.from_arrays(g)
    ga, ma, va = pa.zeros_like(), pa.zeros_like(), pa.zeros_like()
    mb, vb = pb.zeros_like(), pb.zeros_like()
    ra.render(pa, cam)
    torch.cuda.synchronize()
    T = ra.read_buffer(L.PGS_BUF_T_FINAL).reshape(cam.height, cam.width)
    last = ra.read_buffer(L.PGS_BUF_LAST).reshape(cam.height, cam.width)
    img = ra.render(pa, cam).cpu().numpy()
    _, forced = compare_forward(img, T, last, ora, (ra, g, cam, 16))
    ra.backward(dLt, ga)
    ra.step(pa, ga, ma, va, 1)
    rb.render(pb, cam)
    rb.backward_step(dLt, pb, mb, vb, 1)
    torch.cuda.synchronize()
    assert rb.status()[0] == 0
    assert rel_l2(mb.data.cpu().numpy(), ma.data.cpu().numpy()) < 1e-5
    assert rel_l2(vb.data.cpu().numpy(), va.data.cpu().numpy()) < 1e-5
    # t = 1: the step is lr * g / (|g| + eps), so parameters agree wherever g is not at noise level
    dp = np.abs(pb.data.cpu().numpy() - pa.data.cpu().numpy())
    assert np.mean(dp > 1e-6) < 1e-3
    _, og = oracle.backward(g, cam, dL, forced=forced)
    keep = oracle.gaussian_flags(g, cam) == 0
    grads = {k: v / (1 - np.float32(0.9)) for k, v in mb.numpy().items()}
    compare_grads(grads, og, keep)


def test_backward_accumulates(R):
    """The first backward after a render reads the screen-space gradients its forward cleared;
    every later one (or one after a variant timing, which runs backwards of its own) clears them
    itself: repeated calls add the same gradient each time."""
    g, cam = SCENES["tiny_2k_128"]()
    rast, buf, *_ = render_gpu(R, g, cam)
    dL = torch.from_numpy(S.random_image(4, cam.width, cam.height)).cuda()
    g1 = buf.zeros_like()
    rast.backward(dL, g1)
    g2 = buf.zeros_like()
    rast.backward(dL, g2)
    rast.backward(dL, g2)
    rast.time_variants(dL, reps=1)
    g3 = buf.zeros_like()
    rast.backward(dL, g3)
    torch.cuda.synchronize()
    # float atomics add in a scheduling-dependent order: equal up to rounding
    assert rel_l2(g2.data.cpu().numpy(), 2 * g1.data.cpu().numpy()) < 1e-5
    assert rel_l2(g3.data.cpu().numpy(), g1.data.cpu().numpy()) < 1e-5
    assert torch.count_nonzero(g1.data) > 0


# ----------------------------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------------------------

def test_empty_scene(R):
    g, cam = SCENES["tiny_2k_128"]()
    g = g.subset(np.arange(0))
    cam.bg = (0.25, 0.5, 0.75)
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    assert code == 0 and pairs == 0
    assert np.allclose(img, np.array(cam.bg, np.float32)[:, None, None])
    assert np.all(T == 1.0) and np.all(last == 0)


def test_all_culled_behind_camera(R):
    g, cam = SCENES["tiny_2k_128"]()
    g.means[2] = -5.0
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    assert code == 0 and pairs == 0
    assert np.all(img == 0.0) and np.all(T == 1.0)
    grads = buf.zeros_like()
    rast.backward(torch.ones(3, cam.height, cam.width, device="cuda"), grads)
    torch.cuda.synchronize()
    assert torch.count_nonzero(grads.data) == 0


def test_single_gaussian_covering_every_tile(R):
    g, cam = SCENES["ragged_100x75"]()
    g = g.subset([0])
    g.means[:, 0] = [0.0, 0.0, 0.0]
    g.log_scales[:, 0] = 0.0
    g.opacity_logits[0] = 0.5
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    TX, TY = oracle.tiles(cam)
    assert pairs == TX * TY
    check_keys(rast, g, cam)
    compare_forward(img, T, last, oracle.render(g, cam), (rast, g, cam, 16))


def test_many_super_tiles_take_two_grouping_passes(R):
    """1920x1080 with 8x8 tiles: 240 x 135 = 32,400 tiles in 30 x 34 = 1,020 super-tiles of 8 x 4
    tiles, so the coarse entries are grouped by a two-pass sort over 10-bit super-tile ids, the
    super-tiles' ranges come from the sorted keys, and the heaviest-first tile order takes its
    multi-CTA form (more than 16,384 tiles): keys, values and ranges bit-exact against the oracle,
    image and `last` checked on every pixel."""
    sc = S.surface_scene(4, 20000, 1, 1920, 1080, 1500.0, n_cameras=8)
    g, cam = sc.gt, sc.cameras[2]
    TX, TY = -(-cam.width // 8), -(-cam.height // 8)
    assert -(-TX // 8) * -(-TY // 4) > 256 and TX * TY > 16384
    rast = R.Rasterizer(tile=8)
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam, rast)
    assert code == 0
    assert pairs == check_keys(rast, g, cam, 8)
    compare_forward(img, T, last, oracle.render(g, cam, 8), (rast, g, cam, 8))


def test_one_pixel_image(R):
    g, cam = SCENES["tiny_2k_128"]()
    cam1 = S.Camera(1, 1, cam.fx, cam.fy, 0.5, 0.5, cam.viewmat)
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam1)
    assert code == 0
    check_keys(rast, g, cam1)
    compare_forward(img, T, last, oracle.render(g, cam1), (rast, g, cam1, 16))


def test_equal_depth_ties_are_stable(R):
    g, cam = SCENES["tiny_2k_128"]()
    g.means[2, 1::5] = g.means[2, 0:-1:5][: len(g.means[2, 1::5])]
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    check_keys(rast, g, cam)
    compare_forward(img, T, last, oracle.render(g, cam), (rast, g, cam, 16))


def _lengths(g, cam, tile=16):
    r = oracle.keys(g, cam, tile)[2]
    return r[:, 1] - r[:, 0]


# per-tile list lengths: all short (< 1024 entries), some of 1024 .. 8191, some of 8192 and more
# (a list longer than the 4096 keys of one radix-sort CTA spans several of them)
LENGTH_SCENES = {
    "short": (2000, 128, 150.0, lambda L: L.max() < 1024),
    "long": (20000, 64, 60.0, lambda L: np.any((L >= 1024) & (L < 8192))),
    "very_long": (60000, 32, 30.0, lambda L: np.any(L >= 8192)),
}


@pytest.mark.parametrize("name", list(LENGTH_SCENES))
def test_list_length_classes(R, name):
    """Short, long and very long tile lists, distinct depths: keys, values and ranges bit-exact."""
    n, size, focal, covers = LENGTH_SCENES[name]
    g, cam, _ = S.tiny_scene(11, n=n, width=size, height=size, focal=focal)
    assert covers(_lengths(g, cam))
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    assert code == 0
    assert pairs == check_keys(rast, g, cam)


@pytest.mark.parametrize("name", list(LENGTH_SCENES))
def test_long_equal_depth_runs(R, name):
    """40 % of the Gaussians at one depth (the identity-rotation camera makes their depths equal to
    the bit): runs of far more than 32 equal keys per tile, ordered by canonical index."""
    n, size, focal, covers = LENGTH_SCENES[name]
    g, cam, _ = S.tiny_scene(12, n=n, width=size, height=size, focal=focal)
    rng = np.random.default_rng(12)
    g.means[2, rng.random(n) < 0.4] = 0.25
    k = oracle.keys(g, cam)[0]
    runs = np.diff(np.flatnonzero(np.diff(np.concatenate([[-1], k.astype(np.int64), [-1]])) != 0))
    assert runs.max() > 32
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    assert code == 0
    assert pairs == check_keys(rast, g, cam)


def test_short_equal_depth_runs(R):
    """Triples of nearby Gaussians sharing a depth: runs of 2 and 3 equal keys inside tiles."""
    g, cam, _ = S.tiny_scene(13, n=2001, width=128, height=128)
    rng = np.random.default_rng(13)
    for c in range(3):
        base = g.means[c, 0::3]
        g.means[c, 1::3] = base + (0.0 if c == 2 else rng.uniform(-0.02, 0.02, base.shape))
        g.means[c, 2::3] = base + (0.0 if c == 2 else rng.uniform(-0.02, 0.02, base.shape))
    k = oracle.keys(g, cam)[0]
    runs = np.diff(np.flatnonzero(np.diff(np.concatenate([[-1], k.astype(np.int64), [-1]])) != 0))
    assert runs.max() in (2, 3) and np.sum(runs >= 2) > 100
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    assert code == 0
    assert pairs == check_keys(rast, g, cam)
    compare_forward(img, T, last, oracle.render(g, cam), (rast, g, cam, 16))


def test_nonfinite_parameter_is_reported_and_culled(R):
    from paper_2601_17354_gb300 import _lib as L
    g, cam = SCENES["tiny_2k_128"]()
    g.means[0, 17] = np.nan
    g.log_scales[1, 99] = np.inf
    rast, buf, img, T, last, code, pairs = render_gpu(R, g, cam)
    assert code == L.PGS_ERR_NONFINITE
    assert np.all(np.isfinite(img))
    touched = rast.read_buffer(L.PGS_BUF_TILES_TOUCHED)
    assert touched[17] == 0 and touched[99] == 0
    assert rast.status()[0] == 0  # cleared by the read


def test_capacity_overflow_is_reported_then_fits(R):
    from paper_2601_17354_gb300 import _lib as L
    g, cam = SCENES["tiny_2k_128"]()
    P = len(oracle.keys(g, cam)[0])
    small = R.Rasterizer(pair_capacity=P - 1)
    small.render(R.GaussianBuffer.from_arrays(g), cam)
    code, pairs = small.status()
    assert code == L.PGS_ERR_CAPACITY and pairs == P
    exact = R.Rasterizer(pair_capacity=P)
    _, _, img, T, last, code, pairs = render_gpu(R, g, cam, exact)
    assert code == 0 and pairs == P
    compare_forward(img, T, last, oracle.render(g, cam), (exact, g, cam, 16))


def test_sort_wait_that_runs_out_is_reported_and_the_context_recovers(R):
    """The sort's look-back waits are bounded: a pass whose first tile is never published (the
    self-test withholds it) ends with PGS_ERR_TIMEOUT instead of hanging, and the same context then
    renders the tiny scene with keys, values and ranges bit-exact."""
    from paper_2601_17354_gb300 import _lib as L
    g, cam = SCENES["tiny_2k_128"]()
    rast = R.Rasterizer()
    assert rast.selftest_timeout() == L.PGS_ERR_TIMEOUT
    assert rast.status()[0] == 0  # read and cleared by the self-test
    rast, _, img, T, last, code, pairs = render_gpu(R, g, cam, rast)
    assert code == 0
    assert pairs == check_keys(rast, g, cam)
    compare_forward(img, T, last, oracle.render(g, cam), (rast, g, cam, 16))


def test_backward_without_render_is_an_error(R):
    from paper_2601_17354_gb300 import _lib as L
    rast = R.Rasterizer()
    buf = R.GaussianBuffer(10, 0)
    with pytest.raises(L.PgsError) as e:
        rast.backward(torch.zeros(3, 4, 4, device="cuda"), buf)
    assert e.value.code == L.PGS_ERR_NO_RENDER


# ----------------------------------------------------------------------------------------------
# loss and optimizer
# ----------------------------------------------------------------------------------------------

def test_l1_loss_matches_oracle(R):
    rng = np.random.default_rng(0)
    img = rng.uniform(0, 1, size=(3, 77, 131)).astype(np.float32)
    gt = rng.uniform(0, 1, size=(3, 77, 131)).astype(np.float32)
    gt[0, 3, 4] = img[0, 3, 4]  # a zero difference: sign(0) = 0
    rast = R.Rasterizer()
    grad, out = rast.loss_l1(torch.from_numpy(img).cuda(), torch.from_numpy(gt).cuda())
    loss, ograd, sse = oracle.l1(img.astype(np.float64), gt.astype(np.float64))
    out = out.cpu().numpy()
    assert abs(out[0] - loss) <= 1e-6 * loss
    assert abs(out[1] - sse) <= 1e-5 * sse
    assert np.allclose(grad.cpu().numpy(), ograd, rtol=1e-6, atol=0)


@pytest.mark.parametrize("n,degree", [(1000, 3), (1001, 1), (7, 0)])
def test_adam_matches_oracle(R, n, degree):
    rng = np.random.default_rng(n)
    rows = R.rows_of(degree)
    p0 = rng.normal(size=(rows, n)).astype(np.float32)
    rast = R.Rasterizer()
    P = R.GaussianBuffer(n, degree, data=torch.from_numpy(p0.copy()).cuda())
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    lr = np.array(R.DEFAULT_LR)
    K = (degree + 1) ** 2
    row_lr = np.concatenate([[lr[0]] * 3, [lr[1]] * 3, [lr[2]] * 4, [lr[3]],
                             [lr[4] if k % K == 0 else lr[5] for k in range(3 * K)]])
    po, mo, vo = p0.astype(np.float64), np.zeros((rows, n)), np.zeros((rows, n))
    for t in range(1, 6):
        gk = (rng.normal(size=(rows, n)) * 10.0 ** rng.uniform(-4, 0)).astype(np.float32)
        G.data.copy_(torch.from_numpy(gk))
        rast.step(P, G, M, V, t)
        for r in range(rows):
            pr, mr, vr = po[r].copy(), mo[r].copy(), vo[r].copy()
            # the library takes fp32 hyper-parameters: the oracle uses the same values
            oracle.adam(pr, gk[r].astype(np.float64), mr, vr, float(np.float32(row_lr[r])), t,
                        float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-15)))
            po[r], mo[r], vo[r] = pr, mr, vr
    torch.cuda.synchronize()
    assert torch.count_nonzero(G.data) == 0
    assert np.allclose(P.data.cpu().numpy(), po, rtol=1e-5, atol=1e-6)
    # fp32 moments against FP64: m can cancel towards zero, so the absolute floor scales with m
    mg = M.data.cpu().numpy()
    assert np.all(np.abs(mg - mo) <= 1e-5 * np.abs(mo) + 1e-6 * np.abs(mo).max())
    assert np.allclose(V.data.cpu().numpy(), vo, rtol=1e-5, atol=1e-6 * vo.max())
