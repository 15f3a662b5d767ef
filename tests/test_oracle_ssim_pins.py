"""Pins of the SSIM / D-SSIM oracle (oracle/ssim.py) against what the definition and a library
routine fix: SSIM(x, x) = 1, the closed form of constant images away from the border, the
filtered moments against scipy's Gaussian filter with the same truncation and zero padding, and
FP64 central finite differences of the loss."""
import numpy as np
import pytest

from oracle import ssim as O


def rand_img(seed, H=14, W=17):
    return np.random.default_rng(seed).uniform(0, 1, (3, H, W))


def test_identical_images_have_ssim_one():
    x = rand_img(1)
    assert np.allclose(O.ssim_map(x, x), 1.0, atol=1e-12)
    loss, ssim, g = O.loss_and_grad(x, x, 0.2)
    assert abs(ssim - 1.0) < 1e-12 and abs(loss) < 1e-12


def test_constant_images_closed_form_in_the_interior():
    a, b = 0.3, 0.7
    x = np.full((3, 15, 15), a)
    y = np.full((3, 15, 15), b)
    s = O.ssim_map(x, y)
    want = (2 * a * b + O.C1) / (a * a + b * b + O.C1)   # the variances vanish
    assert abs(s[1, 7, 7] - want) < 1e-12
    assert not np.isclose(s[1, 0, 0], want)              # the zero padding darkens the border


def test_window_taps_and_filter_match_scipy():
    ndi = pytest.importorskip("scipy.ndimage")
    w = O.window()
    assert len(w) == 11 and abs(w.sum() - 1) < 1e-15 and np.allclose(w, w[::-1])
    img = rand_img(2)[0]
    ref = ndi.gaussian_filter(img, O.SIGMA, mode="constant", cval=0.0, truncate=O.RADIUS / O.SIGMA)
    assert np.allclose(O.filt(img), ref, atol=1e-13)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_gradient_matches_central_differences(lam):
    rng = np.random.default_rng(3)
    x, y = rand_img(4, 9, 12), rand_img(5, 9, 12)
    _, _, g = O.loss_and_grad(x, y, lam)
    h = 1e-6
    for _ in range(40):
        c, i, j = rng.integers(3), rng.integers(9), rng.integers(12)
        if lam < 1 and abs(x[c, i, j] - y[c, i, j]) < 10 * h:
            continue
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (O.loss_and_grad(xp, y, lam)[0] - O.loss_and_grad(xm, y, lam)[0]) / (2 * h)
        assert abs(fd - g[c, i, j]) <= 1e-7 * max(1.0, abs(g[c, i, j]) * 1e3), (c, i, j, fd, g[c, i, j])
