"""Shared comparison helpers for the GPU parity tests (CUDA path vs the CPU oracle).

Tolerances: keys, values, ranges and per-pixel last-contributor indices bit-exact; image within
1e-4 absolute on [0, 1]; gradients within 1e-3 relative L2 per parameter group.  Pixels whose
FP64 decisions (alpha vs 1/255, T vs 1e-4, the 0.99 clamp) lie within a small relative margin
of the threshold may legitimately decide differently in fp32; the oracle flags them, they are
counted, and they are excluded from the value checks (and their upstream gradient is zeroed for
the gradient checks).
"""
import numpy as np

IMAGE_TOL = 1e-4
GRAD_TOL = 1e-3


def compare_forward(img, T, last, ora, max_flagged_frac=2e-3):
    """img [3][H][W], T [H][W], last [H][W] from the GPU against oracle.render output."""
    H, W = ora["T"].shape
    flag = ora["flag"] != 0
    diff = np.abs(img.astype(np.float64) - ora["image"]).max(axis=0)
    bad = diff > IMAGE_TOL
    assert not np.any(bad & ~flag), f"{np.sum(bad & ~flag)} unflagged pixels off by up to {diff[~flag].max():.3g}"
    assert np.sum(bad & flag) <= max(2, max_flagged_frac * H * W)
    lbad = last.astype(np.int64) != ora["last"]
    assert not np.any(lbad & ~flag), f"{np.sum(lbad & ~flag)} unflagged last-index mismatches"
    tdiff = np.abs(T.astype(np.float64) - ora["T"])
    assert np.all(tdiff[~flag] <= IMAGE_TOL)
    return int(np.sum(flag)), float(diff[~flag].max() if np.any(~flag) else 0.0)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def compare_grads(gpu: dict, ora: dict, keep=None, tol=GRAD_TOL):
    """Per-group relative L2 over the Gaussians in `keep` (bool [n]); returns the errors."""
    errs = {}
    for k, want in ora.items():
        got = gpu[k]
        if keep is not None:
            got = got[..., keep]
            want = want[..., keep]
        errs[k] = rel_l2(got, want)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"gradient groups over {tol}: {bad} (all: {errs})"
    return errs
