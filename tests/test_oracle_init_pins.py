"""Pins of the initializer oracle (operator I, Sec. III-B, Eq. 5 and Eq. 6) and of the learned
stand-in's MLP: library routines (scipy cKDTree, numpy eigh, torch float64 autograd) and closed
forms on planes and spheres.  CPU only."""
import math

import numpy as np
import pytest

import oracle


def test_knn_matches_kdtree():
    cKDTree = pytest.importorskip("scipy.spatial").cKDTree
    rng = np.random.default_rng(0)
    P = rng.uniform(-1, 1, size=(3, 800)).astype(np.float32)
    nb = oracle.knn(P, 12)
    _, idx = cKDTree(P.T.astype(np.float64)).query(P.T.astype(np.float64), k=13)
    assert np.array_equal(nb, idx[:, 1:])


def test_eig3_matches_numpy():
    rng = np.random.default_rng(1)
    for _ in range(50):
        M = rng.normal(size=(3, 3))
        A = M @ M.T
        w, V = oracle.eig3(A)
        wn, Vn = np.linalg.eigh(A)
        assert np.allclose(w, wn, rtol=1e-12, atol=1e-12)
        for k in range(3):
            v = Vn[:, k] * np.sign(Vn[np.argmax(np.abs(Vn[:, k])), k])
            assert np.allclose(V[:, k], v, atol=1e-9)
            assert np.abs(V[:, k]).argmax() == np.abs(V[:, k]).argmax() and V[np.abs(V[:, k]).argmax(), k] > 0


def _rotmat(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_pca_init_on_planes_closed_form():
    """Points on a plane: the Eq. 5 normal is the plane normal, the seeded Gaussian's z axis is it
    (Sec. III-B.2), the tangential scale is the mean 3-NN distance (Eq. 6), the normal scale
    0.1 of it, and the opacity is logit(0.1)."""
    rng = np.random.default_rng(2)
    n = 500
    uv = rng.uniform(-1, 1, size=(2, n))
    for normal in [np.array([0.0, 0.0, 1.0]), np.array([0.3, -0.5, 0.81])]:
        normal = normal / np.linalg.norm(normal)
        a = np.cross(normal, [1.0, 0.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(normal, a)
        P = (np.outer(a, uv[0]) + np.outer(b, uv[1]) + 0.2).astype(np.float32)
        nb = oracle.knn(P, 32)
        init = oracle.pca_init(P, nb)
        for i in range(0, n, 37):
            R = _rotmat(init["quats"][:, i])
            assert np.allclose(np.abs(R[:, 2] @ normal), 1.0, atol=1e-4)
            d = np.linalg.norm(P[:, nb[i, :3]].astype(np.float64) - P[:, i:i + 1].astype(np.float64), axis=0)
            assert math.isclose(init["log_scales"][0, i], math.log(d.mean()), rel_tol=1e-9)
            assert math.isclose(init["log_scales"][2, i], math.log(0.1 * d.mean()), rel_tol=1e-9)
        assert np.allclose(init["opacity_logits"], math.log(0.1 / 0.9))
    # a normal along -z takes the 180-degree rotation about x
    P = np.stack([uv[0], uv[1], np.zeros(n)]).astype(np.float32)
    f, _ = oracle.features(P, oracle.knn(P, 32))
    assert np.allclose(f[:, 0], 0, atol=1e-12)


def test_features_on_a_sphere():
    """Points on a sphere: the smallest-eigenvalue eigenvector of a small neighbourhood is the
    radial direction, the eigenvalue ratios sum to 1, and the density feature tracks the mean
    neighbour distance."""
    rng = np.random.default_rng(3)
    d = rng.normal(size=(3, 4000))
    d /= np.linalg.norm(d, axis=0)
    P = (0.7 * d).astype(np.float32)
    nb = oracle.knn(P, 32)
    f, fq = oracle.features(P, nb)
    assert np.allclose(f[:, :3].sum(1), 1.0)
    assert np.all(f[:, 0] <= f[:, 1]) and np.all(f[:, 1] <= f[:, 2])
    cosang = np.abs(np.sum(f[:, 3:6] * d.T, axis=1))
    assert np.median(cosang) > 0.99
    md = np.array([np.linalg.norm(P[:, nb[i]].astype(np.float64) - P[:, i:i + 1], axis=0).mean()
                   for i in range(0, 4000, 200)])
    assert np.allclose(f[::200, 15], -3 * np.log(md), rtol=1e-9)
    for i in range(0, 4000, 500):
        R = _rotmat(fq[:, i])
        assert np.allclose(R[:, 2], f[i, 3:6], atol=1e-9)
        assert np.linalg.det(R) > 0


def _weights(seed=0):
    rng = np.random.default_rng(seed)
    return (rng.normal(0, 0.3, (64, 16)), rng.normal(0, 0.1, 64), rng.normal(0, 0.15, (64, 64)),
            rng.normal(0, 0.1, 64), rng.normal(0, 0.15, (8, 64)), rng.normal(0, 0.1, 8))


def _torch_mlp(torch, x, W):
    W1, b1, W2, b2, W3, b3 = W
    g = torch.nn.functional.gelu
    return g(g(x @ W1.T + b1) @ W2.T + b2) @ W3.T + b3


def test_mlp_forward_backward_match_torch_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = rng.normal(size=(50, 16)).astype(np.float32)
    W = [w.astype(np.float32) for w in _weights()]
    y = oracle.mlp_forward(x, W, mode=0)
    Wt = [torch.tensor(w.astype(np.float64), requires_grad=True) for w in W]
    yt = _torch_mlp(torch, torch.tensor(x.astype(np.float64)), Wt)
    assert np.allclose(y, yt.detach().numpy(), rtol=1e-12, atol=1e-12)
    t = np.concatenate([rng.normal(size=(50, 3)), rng.normal(size=(50, 4)), rng.normal(size=(50, 1))], 1)
    t[:, 3:7] /= np.linalg.norm(t[:, 3:7], axis=1, keepdims=True)
    t = t.astype(np.float32)
    L, dy = oracle.init_loss(y, t)
    tt = torch.tensor(t.astype(np.float64))
    qh = yt[:, 3:7] / yt[:, 3:7].norm(dim=1, keepdim=True)
    Lt = (((yt[:, :3] - tt[:, :3]) ** 2).sum(1) + (1 - (qh * tt[:, 3:7]).sum(1) ** 2)
          + (yt[:, 7] - tt[:, 7]) ** 2).mean()
    Lt.backward()
    assert math.isclose(L, Lt.item(), rel_tol=1e-12)
    grads = oracle.mlp_backward(x, W, dy, mode=0)
    for g, w in zip(grads, Wt):
        assert np.allclose(g, w.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_mlp_bf16_mode_is_close_to_exact():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(200, 16)).astype(np.float32)
    W = [w.astype(np.float32) for w in _weights(1)]
    a = oracle.mlp_forward(x, W, mode=1)
    b = oracle.mlp_forward(x, W, mode=0)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-2
    dy = rng.normal(size=(200, 8))
    ga = oracle.mlp_backward(x, W, dy, mode=1)
    gb = oracle.mlp_backward(x, W, dy, mode=0)
    for u, v in zip(ga, gb):
        assert np.linalg.norm(u - v) / np.linalg.norm(v) < 3e-2


def test_residual_composition_matches_scipy_and_round_trips():
    """Learned parameters = the paper's seeding corrected by the network: rotation = seeded
    rotation (x) predicted rotation (composition checked with scipy's Rotation), log-scales and
    logit offset; zero offsets with the identity rotation give the seeding back, and targets built
    from any converged Gaussians map back to them."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(6)
    n = 40
    bq = rng.normal(size=(4, n))
    bq /= np.linalg.norm(bq, axis=0)
    base = dict(log_scales=rng.normal(-4, 0.3, (3, n)), quats=bq, opacity_logits=rng.normal(-2, 0.1, n))
    y = rng.normal(size=(n, 8))
    out = oracle.apply_mlp(y, base)
    for i in range(n):
        Rb = Rot.from_quat([bq[1, i], bq[2, i], bq[3, i], bq[0, i]])
        Rl = Rot.from_quat([y[i, 4], y[i, 5], y[i, 6], y[i, 3]])
        want = (Rb * Rl).as_matrix()
        q = out["quats"][:, i]
        got = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.allclose(got, want, atol=1e-12)
    assert np.allclose(out["log_scales"], base["log_scales"] + y[:, 0:3].T)
    assert np.allclose(out["opacity_logits"], base["opacity_logits"] + y[:, 7])
    ident = np.zeros((n, 8))
    ident[:, 3] = 2.5  # any positive multiple of the identity rotation
    same = oracle.apply_mlp(ident, base)
    assert np.allclose(same["quats"], bq, atol=1e-15) and np.array_equal(same["log_scales"], base["log_scales"])
    t = oracle.make_targets(base, out)
    back = oracle.apply_mlp(t, base)
    assert np.allclose(np.abs(np.sum(back["quats"] * out["quats"], axis=0)), 1.0, atol=1e-12)
    assert np.allclose(back["log_scales"], out["log_scales"]) and np.allclose(back["opacity_logits"], out["opacity_logits"])
