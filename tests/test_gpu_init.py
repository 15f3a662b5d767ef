"""The initializer path on the GPU (operator I of Sec. III-B and its learned stand-in) against the
initializer oracle: exact neighbour lists, features and the paper's disc seeding, the BF16 MLP's
outputs and gradients (BF16 tolerance: rounding of activations can differ by one BF16 ulp where
the fp32 sums differ in their last bits), and the frame composition."""
import numpy as np
import pytest

import oracle
from paper_2601_17354_gb300 import synthetic as S
from tests._parity import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2601_17354_gb300 import initializer
    return initializer


def surface_points(seed, n):
    rng = np.random.default_rng(seed)
    return S.sample_surface_points(rng, S.random_surfaces(rng), n).astype(np.float32)


@pytest.mark.parametrize("k", [3, 16, 32])
def test_knn_exact(I, k):
    P = np.concatenate([surface_points(1, 3000), np.random.default_rng(2).uniform(-2, 2, (3, 1500))], 1)
    P = np.ascontiguousarray(P.astype(np.float32))
    init = I.Initializer()
    nb = init.knn(torch.from_numpy(P).cuda(), k).cpu().numpy()
    assert np.array_equal(nb, oracle.knn(P, k))


def test_features_and_paper_init(I):
    P = surface_points(3, 4000)
    init = I.Initializer()
    pi = init.paper_init(torch.from_numpy(P).cuda(), sh_degree=1)
    nb = oracle.knn(P, 32)
    assert np.array_equal(pi.nb.cpu().numpy(), nb)
    f, fq = oracle.features(P, nb)
    assert np.allclose(pi.features.cpu().numpy(), f, rtol=1e-5, atol=1e-6)
    assert np.allclose(pi.frame_q.cpu().numpy(), fq, atol=1e-6)
    assert np.array_equal(pi.features_bf16.float().cpu().numpy(),
                          pi.features.bfloat16().float().cpu().numpy())
    o = oracle.pca_init(P, nb)
    g = pi.paper.numpy()
    assert np.allclose(g["log_scales"], o["log_scales"], rtol=1e-6, atol=1e-6)
    assert np.allclose(g["quats"], o["quats"], atol=1e-6)
    assert np.allclose(g["opacity_logits"], o["opacity_logits"])
    assert np.array_equal(g["means"], P) and np.all(g["sh"] == 0)


def _mlp_with_random_weights(I, init, seed):
    mlp = I.MLP(init, seed)
    rng = np.random.default_rng(seed)
    ws = [rng.normal(0, s, shape).astype(np.float32) for s, shape in
          zip([0.3, 0.1, 0.15, 0.1, 0.15, 0.1], I.MLP.SHAPES)]
    mlp.set_weights(ws)
    return mlp, ws


def test_mlp_forward_matches_bf16_oracle(I):
    init = I.Initializer()
    mlp, ws = _mlp_with_random_weights(I, init, 1)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(5000, 16)).astype(np.float32)
    xb = torch.from_numpy(x).cuda().bfloat16()
    y = mlp.forward(xb).cpu().numpy()
    want = oracle.mlp_forward(xb.float().cpu().numpy(), ws, mode=1)
    assert rel_l2(y, want) < 5e-3
    assert rel_l2(y, oracle.mlp_forward(xb.float().cpu().numpy(), ws, mode=0)) < 2e-2


def test_mlp_gradients_match_bf16_oracle(I):
    init = I.Initializer()
    mlp, ws = _mlp_with_random_weights(I, init, 2)
    rng = np.random.default_rng(8)
    n = 3001  # not a multiple of the 64-point slice
    x = rng.normal(size=(n, 16)).astype(np.float32)
    t = np.concatenate([rng.normal(size=(n, 3)), rng.normal(size=(n, 4)), rng.normal(size=(n, 1))], 1)
    t[:, 3:7] /= np.linalg.norm(t[:, 3:7], axis=1, keepdims=True)
    t = t.astype(np.float32)
    xb = torch.from_numpy(x).cuda().bfloat16()
    mlp.loss_sum.zero_()
    mlp.grad.zero_()
    mlp.accumulate_grad(xb, torch.from_numpy(t).cuda())
    xr = xb.float().cpu().numpy()
    y = oracle.mlp_forward(xr, ws, mode=1)
    L, dy = oracle.init_loss(y, t)
    assert abs(mlp.loss_sum.item() / n - L) <= 1e-3 * L
    want = oracle.mlp_backward(xr, ws, dy, mode=1)
    got = mlp.grad.cpu().numpy()
    off = 0
    for w in want:
        k = w.size
        assert rel_l2(got[off:off + k], w.reshape(-1)) < 2e-2, off
        off += k


def test_apply_and_targets_match_oracle(I):
    P = surface_points(4, 3000)
    init = I.Initializer()
    pi = init.paper_init(torch.from_numpy(P).cuda(), sh_degree=0)
    y = np.random.default_rng(9).normal(size=(3000, 8)).astype(np.float32)
    y[5, 2] = np.nan  # falls back to the paper's initializer
    out, fallbacks = init.apply(pi, torch.from_numpy(y).cuda())
    assert fallbacks == 1
    base = pi.paper.numpy()
    o = oracle.apply_mlp(y.astype(np.float64), base)
    g = out.numpy()
    keep = np.ones(3000, bool)
    keep[5] = False
    assert np.allclose(g["quats"][:, keep], o["quats"][:, keep], atol=1e-5)
    assert np.allclose(g["log_scales"][:, keep], o["log_scales"][:, keep])
    assert np.allclose(g["quats"][:, 5], pi.paper.quats[:, 5].cpu().numpy())
    t = init.make_targets(pi, out).cpu().numpy()
    ot = oracle.make_targets(base, g)
    assert np.allclose(t, ot, atol=1e-5)


def test_training_reduces_the_loss(I):
    init = I.Initializer()
    P = surface_points(5, 20000)
    pi = init.paper_init(torch.from_numpy(P).cuda(), sh_degree=0)
    # targets: a smooth function of the point's own statistics (scale offset from density, the
    # seeded rotation itself, opacity offset from planarity)
    f = pi.features
    t = torch.zeros((f.shape[0], 8), device="cuda")
    t[:, 0:3] = 0.1 * (f[:, 15:16] - f[:, 15].mean())
    t[:, 3] = 1.0
    t[:, 7] = 2.0 * f[:, 0] - 0.5
    li = I.LearnedInit(init, seed=3)
    hist = li.fit([pi.features_bf16], [t], steps=300, batch=8192, lr=3e-3)
    assert hist[-1][1] < 0.2 * hist[0][1]
    out, fallbacks = li.infer(pi)
    assert fallbacks == 0
    assert torch.isfinite(out.data).all()
