"""Shared comparison helpers for the GPU parity tests (CUDA path vs the CPU oracle).

Tolerances: keys, values, ranges and per-pixel last-contributor indices bit-exact; image and
final transmittance within 1e-4 absolute on [0, 1]; gradients within 1e-3 relative L2 per
parameter group.

Every pixel is compared.  The compositing decisions (skip alpha < 1/255, clamp at 0.99, stop when
T (1 - alpha) < 1e-4) are integers decided in floating point; the oracle takes them in the
kernel's precision (fp32, same evaluation order) and flags a pixel when one of them lies within
the stated bound of the kernel's unreproducible steps (hardware 2^x, library exp in the opacity)
of its threshold.  For a flagged pixel the kernel's own decisions are read back through the
decision trace (pgs_trace_pixels) and the oracle composites that pixel following them; every
decision of the kernel that differs from the oracle's must be one the oracle flagged as
ambiguous.  The flagged fraction is asserted: a rate of at most 1e-4 of the pixels (1e-3 on the
dense 500k-Gaussian views), with a Poisson allowance for small images.
"""
import numpy as np

import oracle

IMAGE_TOL = 1e-4
GRAD_TOL = 1e-3
MAX_FLAGGED_FRAC = 1e-4
# Dense views (the 500k-Gaussian 1080p scene: ~80 composited entries per pixel) flag more: the
# bound of the fp32 transmittance chain grows by every composited entry's share, so more stop
# tests fall inside it (3.4e-4 of the pixels of its 256 x 256 crop); they are replayed all the same.
MAX_FLAGGED_FRAC_DENSE = 1e-3


def flag_allowance(rate, pixels):
    """Most flagged pixels accepted at a flag rate of `rate`: the expected count plus three
    Poisson standard deviations plus one (small images flag 0-2 pixels by chance)."""
    mean = rate * pixels
    return mean + 3.0 * np.sqrt(mean) + 1.0


def list_lengths(g, cam, pix, tile=16):
    """Length of the tile list of each pixel (x, y) from the oracle's own ranges."""
    _, _, r = oracle.keys(g, cam, tile)
    TX, _ = oracle.tiles(cam, tile)
    t = (pix[:, 1] // tile) * TX + pix[:, 0] // tile
    return (r[t, 1].astype(np.int64) - r[t, 0].astype(np.int64))


def kernel_decisions(rast, g, cam, pix, tile=16):
    """The kernel's decisions at pixels pix [m][2] (x, y) of the rasterizer's last render, as an
    oracle.Forced, and the raw trace."""
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    E = int(max(1, list_lengths(g, cam, pix, tile).max(initial=0)))
    tr = rast.trace_pixels(pix, E)
    cnt = tr["count"].astype(np.int64)
    assert np.all((cnt >= 0) & (cnt <= E)), "trace count outside the tile list"
    off = np.concatenate([[0], np.cumsum(cnt)])
    codes = np.concatenate([tr["code"][k, :cnt[k]] for k in range(len(pix))]) if len(pix) else np.zeros(0, np.uint8)
    return oracle.Forced(pix, off, codes), tr


def compare_forward(img, T, last, ora, ctx=None, max_flagged_frac=MAX_FLAGGED_FRAC):
    """img [3][H][W], T [H][W], last [H][W] from the GPU against oracle.render output `ora`.
    ctx = (rasterizer whose last render gave img, gaussians, camera, tile) lets flagged pixels be
    replayed with the kernel's decisions; returns (number flagged, oracle.Forced of them)."""
    H, W = ora["T"].shape
    flag = ora["flag"] != 0
    nflag = int(flag.sum())
    print(f"flagged pixels: {nflag} of {H * W} ({nflag / (H * W):.2e})")
    assert nflag <= flag_allowance(max_flagged_frac, H * W), f"{nflag} flagged pixels of {H * W}"
    diff = np.abs(img.astype(np.float64) - ora["image"]).max(axis=0)
    ok = ~flag
    assert np.all(diff[ok] <= IMAGE_TOL), f"{np.sum(diff[ok] > IMAGE_TOL)} pixels off by up to {diff[ok].max():.3g}"
    assert np.array_equal(last[ok].astype(np.int64), ora["last"][ok]), \
        f"{np.sum(last[ok].astype(np.int64) != ora['last'][ok])} last-index mismatches"
    assert np.all(np.abs(T[ok].astype(np.float64) - ora["T"][ok]) <= IMAGE_TOL)
    if nflag == 0:
        return 0, oracle.Forced.empty()
    assert ctx is not None, "flagged pixels need the kernel's decision trace"
    rast, g, cam, tile = ctx
    pix = np.argwhere(flag)[:, ::-1].astype(np.int32)  # (x, y)
    forced, tr = kernel_decisions(rast, g, cam, pix, tile)
    xs, ys = pix[:, 0], pix[:, 1]
    # the trace walks the pixels as the render did
    assert np.array_equal(tr["last"], last[ys, xs].astype(np.uint32))
    assert np.array_equal(tr["T"].view(np.uint32), T[ys, xs].astype(np.float32).view(np.uint32))
    rep = oracle.render_forced(g, cam, forced, tile)
    assert rep["illegal"].sum() == 0, f"kernel decisions outside the error bound at {np.sum(rep['illegal'] > 0)} pixels"
    got = img[:, ys, xs].T.astype(np.float64)
    assert np.all(np.abs(got - rep["rgb"]) <= IMAGE_TOL)
    assert np.all(np.abs(T[ys, xs].astype(np.float64) - rep["T"]) <= IMAGE_TOL)
    assert np.array_equal(rep["last"].astype(np.int64), last[ys, xs].astype(np.int64))
    assert np.array_equal(rep["ncomp"].astype(np.uint32), tr["ncomp"])
    return nflag, forced


def check_render(rast, g, cam, img, tile=16, ora=None, max_flagged_frac=MAX_FLAGGED_FRAC):
    """The rasterizer's last render (image img [3][H][W] as numpy) against the oracle, every pixel
    compared; returns (oracle render, oracle.Forced of the flagged pixels)."""
    from paper_2601_17354_gb300 import _lib as L
    T = rast.read_buffer(L.PGS_BUF_T_FINAL).reshape(cam.height, cam.width)
    last = rast.read_buffer(L.PGS_BUF_LAST).reshape(cam.height, cam.width)
    ora = oracle.render(g, cam, tile) if ora is None else ora
    _, forced = compare_forward(img, T, last, ora, (rast, g, cam, tile), max_flagged_frac)
    return ora, forced


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
