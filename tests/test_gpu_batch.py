"""Batched training (many views of uneven scenes in one persistent launch, CUDA graph, autotuner)
against the single-view path, which the oracle parity tests pin."""
import numpy as np
import pytest

import oracle
from paper_2601_17354_gb300 import synthetic as S
from tests._parity import check_render, compare_grads, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2601_17354_gb300 import _lib, autotune, batch, rasterizer
    return rasterizer, batch, autotune, _lib


def small_batch(seed=0):
    """Three scenes with uneven Gaussian counts and resolutions, two views each."""
    specs = [(4000, 160, 120, 140.0), (9000, 96, 64, 80.0), (2500, 130, 100, 120.0)]
    scenes, views = [], []
    for s, (n, w, h, f) in enumerate(specs):
        sc = S.surface_scene(seed * 10 + s, n, 1, w, h, f, n_cameras=4)
        scenes.append(sc)
        for v in (0, 2):
            views.append((s, sc.cameras[v], S.random_image(100 * s + v, w, h, 0.0, 1.0)))
    return scenes, views


def make_trainer(mods, scenes, views, **kw):
    R, B, _, _ = mods
    bufs = [R.GaussianBuffer.from_arrays(sc.init) for sc in scenes]
    tv = [(s, c, torch.from_numpy(t).cuda()) for s, c, t in views]
    return B.BatchTrainer(bufs, tv, **kw), bufs


def test_batch_step_matches_single_view_calls(mods):
    R, B, _, L = mods
    scenes, views = small_batch()
    bt, bufs = make_trainer(mods, scenes, views)
    bt.step()
    torch.cuda.synchronize()
    assert bt.status()[0] == 0
    losses = bt.losses()
    # single-view reference: per scene, accumulate the gradients of its views, then one Adam step
    rast = R.Rasterizer()
    for s, sc in enumerate(scenes):
        p = R.GaussianBuffer.from_arrays(sc.init)
        g, m, v = p.zeros_like(), p.zeros_like(), p.zeros_like()
        for k, (vs, cam, tgt) in enumerate(views):
            if vs != s:
                continue
            img = rast.render(p, cam)
            assert torch.equal(img, bt.images[k]), f"render {k} differs"
            dl, loss = rast.loss_l1(img, torch.from_numpy(tgt).cuda())
            assert abs(float(loss[0]) - losses[k, 0]) <= 1e-6 * losses[k, 0]
            rast.backward(dl, g)
        rast.step(p, g, m, v, 1)
        torch.cuda.synchronize()
        assert rel_l2(bt.m[s].data.cpu().numpy(), m.data.cpu().numpy()) < 1e-5
        assert rel_l2(bt.v[s].data.cpu().numpy(), v.data.cpu().numpy()) < 1e-5
        dp = np.abs(bufs[s].data.cpu().numpy() - p.data.cpu().numpy())
        assert np.mean(dp > 1e-6) < 2e-3


def test_batch_render_matches_oracle(mods):
    R = mods[0]
    scenes, views = small_batch(1)
    bt, _ = make_trainer(mods, scenes, views)
    bt.step()
    torch.cuda.synchronize()
    s, cam, _ = views[2]
    img = bt.images[2].cpu().numpy()
    # flagged pixels are replayed through a single-view context's decision trace, whose render
    # is the batch's bit for bit
    rast = R.Rasterizer()
    assert np.array_equal(rast.render(R.GaussianBuffer.from_arrays(scenes[s].init), cam).cpu().numpy(), img)
    check_render(rast, scenes[s].init, cam, img)


def uneven_sh3_batch():
    """Three SH3 scenes with uneven Gaussian counts and resolutions (two of them with a partial
    last tile row and column), two views each."""
    specs = [(6000, 160, 120, 140.0), (12000, 100, 72, 80.0), (3000, 130, 100, 120.0)]
    scenes, views = [], []
    for s, (n, w, h, f) in enumerate(specs):
        sc = S.surface_scene(40 + s, n, 3, w, h, f, n_cameras=4)
        scenes.append(sc)
        for v in (0, 3):
            views.append((s, sc.cameras[v], S.random_image(300 + 10 * s + v, w, h, 0.0, 1.0)))
    return scenes, views


def test_batch_sh3_uneven_against_oracle(mods):
    """The batched step at SH3 over uneven scenes, against the oracle directly: every render's
    image (every pixel), each scene's gradient summed over its views (Eq. 10 scatter of every
    view into the scene's canonical buffer), and the Adam update of each scene with the
    multi-view settings (square-root learning rate, beta ** views) applied on the oracle side."""
    R, B, _, L = mods
    from paper_2601_17354_gb300 import evaluate
    scenes, views = uneven_sh3_batch()
    assert all(c.height % 16 for _, c, _ in views[2:])  # partial last tile rows
    adam = evaluate.batched_adam(2)
    bt, bufs = make_trainer(mods, scenes, views, adam=adam)
    p0 = [b.data.cpu().numpy().astype(np.float64) for b in bufs]
    bt.step()
    torch.cuda.synchronize()
    assert bt.status()[0] == 0
    b1, b2, eps = (float(np.float32(x)) for x in (adam.b1, adam.b2, adam.eps))
    lr = [float(np.float32(x)) for x in adam.lr]
    for s, sc in enumerate(scenes):
        g = sc.init
        K = (g.sh_degree + 1) ** 2
        total = None
        keep = np.ones(g.n, bool)
        rast = R.Rasterizer()
        for k, (vs, cam, tgt) in enumerate(views):
            if vs != s:
                continue
            img = bt.images[k].cpu().numpy()
            single = rast.render(R.GaussianBuffer.from_arrays(g), cam).cpu().numpy()
            assert np.array_equal(single, img), f"render {k}: batch and single view differ"
            ora, forced = check_render(rast, g, cam, img)
            _, dl, _ = oracle.l1(ora["image"], np.asarray(tgt, np.float64))
            _, og = oracle.backward(g, cam, dl, forced=forced)
            total = og if total is None else {q: total[q] + og[q] for q in og}
            keep &= oracle.gaussian_flags(g, cam) == 0
        # m after the first step is (1 - b1) g: the summed gradient of the scene's views
        got = {q: v / (1.0 - np.float32(adam.b1)) for q, v in bt.m[s].numpy().items()}
        compare_grads(got, total, keep)
        # Adam on the oracle's gradient, row by row with the group learning rates
        flat = np.concatenate([total[q].reshape(-1, g.n) for q in R.GROUPS])
        row_lr = np.array([lr[0]] * 3 + [lr[1]] * 3 + [lr[2]] * 4 + [lr[3]] +
                          [lr[4] if r % K == 0 else lr[5] for r in range(3 * K)])
        pw, mw, vw = p0[s].copy(), np.zeros_like(p0[s]), np.zeros_like(p0[s])
        for r in range(flat.shape[0]):
            pr, mr, vr = pw[r].copy(), mw[r].copy(), vw[r].copy()
            oracle.adam(pr, np.ascontiguousarray(flat[r]), mr, vr, row_lr[r], 1, b1, b2, eps)
            pw[r], mw[r], vw[r] = pr, mr, vr
        assert rel_l2(bt.m[s].data.cpu().numpy(), mw) < 1e-3
        assert rel_l2(bt.v[s].data.cpu().numpy(), vw) < 2e-3
        # the first step moves every parameter by lr g / (|g| + eps): equal wherever the
        # gradient is clear of its error
        dp_gpu = bufs[s].data.cpu().numpy() - p0[s]
        dp_ora = pw - p0[s]
        clear = np.abs(flat) > 1e-2 * np.sqrt(np.mean(flat ** 2, axis=1, keepdims=True))
        assert clear.mean() > 0.5
        assert np.all(np.abs(dp_gpu - dp_ora)[clear] <= 1e-6 + 1e-3 * np.abs(dp_ora)[clear])


def test_split_batch_calls_dssim_against_oracle(mods):
    """pgs_render_batch, the caller's L1 + D-SSIM gradient of every render (pgs_loss_dssim), and
    pgs_backward_batch at SH3 over uneven scenes: every render against the oracle (every pixel),
    each scene's gradient (summed over its views, Eq. 10's scatter) against the sum of the oracle's
    backward of the oracle's own D-SSIM gradient of its image; the two calls change no parameter."""
    R, B, _, L = mods
    from oracle import ssim as OS
    scenes, views = uneven_sh3_batch()
    bt, bufs = make_trainer(mods, scenes, views)
    p0 = [b.data.clone() for b in bufs]
    bt.render()
    lossr = R.Rasterizer()
    for k in range(len(views)):
        lossr.loss_dssim(bt.images[k], bt.targets[k], 0.2, grad=bt.dls[k])
    grads = [b.zeros_like() for b in bufs]
    bt.backward(grads)
    torch.cuda.synchronize()
    assert bt.status()[0] == 0
    for x, y in zip(p0, bufs):
        assert torch.equal(x, y.data)
    for s, sc in enumerate(scenes):
        g = sc.init
        total, keep = None, np.ones(g.n, bool)
        rast = R.Rasterizer()
        for k, (vs, cam, tgt) in enumerate(views):
            if vs != s:
                continue
            img = bt.images[k].cpu().numpy()
            assert np.array_equal(rast.render(R.GaussianBuffer.from_arrays(g), cam).cpu().numpy(), img)
            ora, forced = check_render(rast, g, cam, img)
            _, _, dl = OS.loss_and_grad(ora["image"], np.asarray(tgt, np.float64), 0.2)
            _, og = oracle.backward(g, cam, dl, forced=forced)
            total = og if total is None else {q: total[q] + og[q] for q in og}
            keep &= oracle.gaussian_flags(g, cam) == 0
        compare_grads(grads[s].numpy(), total, keep)


def test_backward_batch_needs_a_render(mods):
    R, B, _, L = mods
    scenes, views = small_batch(7)
    bt, bufs = make_trainer(mods, scenes, views)
    with pytest.raises(L.PgsError) as e:
        bt.backward([b.zeros_like() for b in bufs])
    assert e.value.code == L.PGS_ERR_NO_RENDER
    bt.render()
    bt.step()  # a step changes the parameters: the render is stale
    with pytest.raises(L.PgsError) as e:
        bt.backward([b.zeros_like() for b in bufs])
    assert e.value.code == L.PGS_ERR_NO_RENDER


def test_graph_replay_equals_eager_steps(mods):
    scenes, views = small_batch(2)
    a, pa = make_trainer(mods, scenes, views)
    b, pb = make_trainer(mods, scenes, views)
    b.capture()
    for _ in range(3):
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert a.status()[0] == 0 and b.status()[0] == 0
    assert b.launch_count() > 0
    for x, y in zip(pa, pb):
        assert rel_l2(y.data.cpu().numpy(), x.data.cpu().numpy()) < 1e-4
    for k in range(len(views)):
        assert rel_l2(b.images[k].cpu().numpy(), a.images[k].cpu().numpy()) < 1e-4


def test_all_variants_render_identically(mods):
    R, B, _, L = mods
    scenes, views = small_batch(3)
    ref = None
    for pix, depth in L.VARIANTS:
        bt, _ = make_trainer(mods, scenes, views)
        bt.set_variant(pix, depth)
        bt.step()
        torch.cuda.synchronize()
        imgs = [im.cpu().numpy() for im in bt.images]
        if ref is None:
            ref = imgs
        else:
            for a, b in zip(imgs, ref):
                assert np.array_equal(a, b), (pix, depth)


def test_autotuner_times_picks_and_caches(mods, tmp_path):
    R, B, A, L = mods
    scenes, views = small_batch(4)
    bt, _ = make_trainer(mods, scenes, views)
    cache = str(tmp_path / "tune.json")
    choice = A.tune_batch(bt, cache=cache, reps=1)
    assert choice in L.VARIANTS
    import json
    data = json.load(open(cache))
    (entry,) = data.values()
    assert (entry["pixels"], entry["depth"]) == choice and len(entry["ms"]) == 9
    bt2, _ = make_trainer(mods, scenes, views)
    assert A.tune_batch(bt2, cache=cache) == choice
    bt2.capture()
    bt2.step()
    torch.cuda.synchronize()
    assert bt2.status()[0] == 0
    # single-view tuning on one render
    rast = R.Rasterizer()
    p = R.GaussianBuffer.from_arrays(scenes[0].init)
    cam = views[0][1]
    dl = torch.from_numpy(S.random_image(1, cam.width, cam.height)).cuda()
    v = A.tune_rasterizer(rast, p, cam, dl, cache=cache, reps=1)
    assert v.fwd in L.VARIANTS and v.bwd in L.VARIANTS and v.ms > 0
    # the split timing's choice: each kernel's own fastest strip, and a render with it still matches
    tf, tb = rast.time_variants_split(dl, 1)
    assert set(tf) == set(tb) and len(tf) >= 6
    assert A.tune_rasterizer(rast, p, cam, dl, cache=cache) == v   # from the cache


def test_pair_overflow_skips_the_step_then_grows(mods):
    """A captured step whose pairs overflow the capacity leaves parameters, moments and the step
    count untouched; after the status is read and the capacity grown, the graph is captured again
    and steps proceed as in a batch planned with room from the start."""
    R, B, _, L = mods
    scenes, views = small_batch(5)
    a, pa = make_trainer(mods, scenes, views)           # measured capacity
    b, pb = make_trainer(mods, scenes, views, pair_capacity=512)
    before = [p.data.clone() for p in pb]
    b.capture()
    for _ in range(2):
        b.step()
    torch.cuda.synchronize()
    code, pairs = b.status()
    assert code == L.PGS_ERR_CAPACITY and pairs > 512
    assert b.steps() == 0
    for x, y in zip(before, pb):
        assert torch.equal(x, y.data)
    for m in b.m + b.v:
        assert not m.data.any()
    b.reserve(pairs + pairs // 4)
    for _ in range(2):
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert b.check() == 2 and a.check() == 2
    for x, y in zip(pa, pb):
        assert rel_l2(y.data.cpu().numpy(), x.data.cpu().numpy()) < 1e-4


def test_tile_edge_8_batch_matches_single_view_and_tuner_picks_an_edge(mods, tmp_path):
    """A batch planned with 8x8 tiles renders like single-view contexts with 8x8 tiles, and the
    tile autotuner returns a trainer with the edge and variant it timed fastest (and caches)."""
    R, B, A, L = mods
    scenes, views = small_batch(6)
    bt, bufs = make_trainer(mods, scenes, views, tile=8)
    bt.step()
    torch.cuda.synchronize()
    assert bt.status()[0] == 0
    rast = R.Rasterizer(tile=8)
    for k, (s, cam, _) in enumerate(views):
        img = rast.render(R.GaussianBuffer.from_arrays(scenes[s].init), cam)
        assert torch.equal(img, bt.images[k]), k
    assert bt.time_render(1) > 0
    cache = str(tmp_path / "tile.json")
    bufs2 = [R.GaussianBuffer.from_arrays(sc.init) for sc in scenes]
    tv = [(s, c, torch.from_numpy(t).cuda()) for s, c, t in views]
    tuned, tile, variant = A.tune_batch_tile(bufs2, tv, cache=cache, reps=1)
    assert tile in (8, 16, 32) and tuned.tile == tile and variant in L.VARIANTS
    import json
    entry = [v for k, v in json.load(open(cache)).items() if "-tile" in k][0]
    assert entry["tile"] == tile and set(entry["ms"]) == {"8", "16", "32"}
    tuned.capture()
    tuned.step()
    torch.cuda.synchronize()
    assert tuned.status()[0] == 0


def test_many_super_tiles_batch_renders_like_single_views(mods):
    """Four 1920x1080 renders with 8x8 tiles in one batch: 4 x 1,020 super-tiles (two grouping
    passes over 12-bit ids, ranges from the sorted keys) and 129,600 tiles (the multi-CTA tile
    order); every image equals the single-view render bit for bit."""
    R, B, _, _ = mods
    scenes, views = [], []
    for s in range(2):
        sc = S.surface_scene(40 + s, 20000, 1, 1920, 1080, 1500.0, n_cameras=4)
        scenes.append(sc)
        for v in (0, 1):
            views.append((s, sc.cameras[v], S.random_image(7 * s + v, 1920, 1080, 0.0, 1.0)))
    bt, bufs = make_trainer(mods, scenes, views, tile=8)
    bt.render()
    torch.cuda.synchronize()
    assert bt.status()[0] == 0
    rast = R.Rasterizer(tile=8)
    for k, (s, cam, _) in enumerate(views):
        img = rast.render(R.GaussianBuffer.from_arrays(scenes[s].init), cam)
        assert torch.equal(img, bt.images[k]), k
