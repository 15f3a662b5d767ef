"""CPU oracle of the structural-similarity loss — TEST INFRASTRUCTURE ONLY (imported by the tests
and the benchmark's CPU-baseline leg, never by the product path).

The paper reports SSIM (Sec. IV) and names no training loss; the L1 + D-SSIM loss of the 3DGS
line of work is the one written here, in FP64 numpy, straight from the definition:

  per channel, with G the 11 x 11 Gaussian window (sigma 1.5, normalised over its taps) and zero
  padding outside the image,
    mu_x = G * x,  sigma_x^2 = G * x^2 - mu_x^2,  sigma_xy = G * (x y) - mu_x mu_y   (same for y)
    SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2))
  with C1 = 0.01^2, C2 = 0.03^2;
  loss = (1 - lam) mean |x - y| + lam (1 - mean SSIM), means over all 3 H W values.

The gradient with respect to the rendered image x treats the three filtered moments of x
(m1 = G * x, m2 = G * x^2, m12 = G * (x y)) as the variables SSIM depends on: with
ds/dm1, ds/dm2, ds/dm12 per pixel, d(sum SSIM)/dx = G * ds/dm1 + 2 x (G * ds/dm2) + y (G * ds/dm12)
(the window is symmetric, so correlating with it is convolving with it).

Parity status: pinned by SSIM(x, x) = 1, the closed form of constant images, the filtered moments
against scipy.ndimage.gaussian_filter (library routine, same truncation and zero padding) and FP64
central finite differences of the loss.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
RADIUS = 5
SIGMA = 1.5


def window() -> np.ndarray:
    """The 1-D taps (2 RADIUS + 1) of the separable Gaussian window, summing to 1."""
    r = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    w = np.exp(-(r * r) / (2.0 * SIGMA * SIGMA))
    return w / w.sum()


def filt(img: np.ndarray) -> np.ndarray:
    """G * img for a [H][W] plane: a plain double loop over the 11 x 11 window, zero outside."""
    H, W = img.shape
    w = window()
    pad = np.zeros((H + 2 * RADIUS, W + 2 * RADIUS))
    pad[RADIUS:RADIUS + H, RADIUS:RADIUS + W] = img
    out = np.zeros((H, W))
    for dy in range(-RADIUS, RADIUS + 1):
        for dx in range(-RADIUS, RADIUS + 1):
            out += w[dy + RADIUS] * w[dx + RADIUS] * pad[RADIUS + dy:RADIUS + dy + H, RADIUS + dx:RADIUS + dx + W]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM per value of two [3][H][W] images."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    out = np.zeros_like(x)
    for c in range(x.shape[0]):
        mx, my = filt(x[c]), filt(y[c])
        sxx = filt(x[c] * x[c]) - mx * mx
        syy = filt(y[c] * y[c]) - my * my
        sxy = filt(x[c] * y[c]) - mx * my
        out[c] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return out


def loss_and_grad(x: np.ndarray, y: np.ndarray, lam: float = 0.2):
    """(loss, mean SSIM, dloss/dx [3][H][W]) of (1 - lam) L1 + lam (1 - SSIM)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    s_sum = 0.0
    grad = np.zeros_like(x)
    for c in range(x.shape[0]):
        xc, yc = x[c], y[c]
        mx, my = filt(xc), filt(yc)
        sxx = filt(xc * xc) - mx * mx
        syy = filt(yc * yc) - my * my
        sxy = filt(xc * yc) - mx * my
        A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
        B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
        s = A1 * A2 / (B1 * B2)
        s_sum += s.sum()
        ds_dmu = 2 * my * A2 / (B1 * B2) - s * 2 * mx / B1   # sigmas held fixed
        ds_dsxx = -s / B2
        ds_dsxy = 2 * A1 / (B1 * B2)
        dm1 = ds_dmu - 2 * mx * ds_dsxx - my * ds_dsxy      # moments m1 = G*x, m2 = G*x^2, m12 = G*xy
        dm2 = ds_dsxx
        dm12 = ds_dsxy
        grad[c] = filt(dm1) + 2 * xc * filt(dm2) + yc * filt(dm12)
    ssim = s_sum / n
    l1 = np.abs(x - y).mean()
    loss = (1 - lam) * l1 + lam * (1 - ssim)
    dl = (1 - lam) * np.sign(x - y) / n - lam * grad / n
    return loss, ssim, dl
