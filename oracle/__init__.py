"""CPU oracle for the differentiable Gaussian rasterizer — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package.  The product path (``paper_2601_17354_gb300``) never imports, links or runs it.

The arithmetic lives in ``pgs_oracle.cpp`` (plain C++17, FP64 values, fp32 decisions with a
prescribed operation order), compiled by :func:`build` with ``-ffp-contract=off`` into
``oracle/_build/liboracle.so``; its per-pixel and per-Gaussian loops run on OpenMP threads
(:func:`set_threads`), each pixel and each Gaussian computed exactly as in a serial run.  This module only marshals numpy arrays into that library.

Parity status of each function (what pins it, besides agreeing with the GPU path):
  project / render / render_pixels  closed-form single and stacked Gaussians, sum(w)+T = 1,
                                    Eq. 7 back-to-front cross-check
  render_forced / decisions         its own decisions replayed reproduce render exactly; a
                                    forced flip is legal only inside the stated error bound
  keys                              brute-force per-tile lists, hand-checked tiny case
  backward / backward_subset        FP64 central finite differences, two derivations agree
  fd_subset                         agrees with the analytic backward on small scenes (and is
                                    itself plain central differencing of the render)
  sh basis                          orthonormality by quadrature, addition theorem, zonal values
  det_expf                          FP64 exp within 2 ulp
  adam                              torch.optim.Adam (float64), closed-form first step
  l1                                closed forms
  knn                               scipy cKDTree (library routine)
  eig3                              numpy.linalg.eigh (library routine)
  pca_init / features               closed forms on planes, tilted planes and spheres
  mlp_forward / mlp_backward        torch float64 autograd of the same network (library routine)
  init_loss                         torch float64 autograd (library routine)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgs_oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "init_oracle.cpp")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++, -O2, -ffp-contract=off).  Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f)
                                              for f in _SRCS)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, *_SRCS]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OCam(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("view", C.c_float * 12),
                ("near_z", C.c_float), ("bg", C.c_float * 3)]


class OGauss(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("pad_", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logits", C.c_void_p), ("sh", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.c_void_p
            L.oracle_det_expf.restype = C.c_float
            L.oracle_decision_bound.restype = C.c_double
            L.oracle_set_threads.restype = C.c_int
            L.oracle_set_threads.argtypes = [C.c_int]
            L.oracle_decision_bound.argtypes = []
            L.oracle_det_expf.argtypes = [C.c_float]
            L.oracle_sh_basis.argtypes = [P, P, P]
            L.oracle_param_count.restype = C.c_int
            L.oracle_param_count.argtypes = [C.c_int]
            L.oracle_project.argtypes = [P, P, C.c_int] + [P] * 10
            L.oracle_keys.restype = C.c_int64
            L.oracle_keys.argtypes = [P, P, C.c_int, C.c_int64, P, P, P]
            L.oracle_render.argtypes = [P, P, C.c_int, P, P, P, P, P, P]
            L.oracle_render_pixels.argtypes = [P, P, C.c_int, C.c_int64, P, P, P, P, P]
            L.oracle_render_forced.argtypes = [P, P, C.c_int, C.c_int64, P, P, P] + [P] * 6
            L.oracle_decisions.argtypes = [P, P, C.c_int, C.c_int64, P, C.c_int64, P, P, P]
            L.oracle_backward_forced.argtypes = [P, P, C.c_int, P, C.c_int, C.c_int64, P, P, P, P, P]
            L.oracle_backward_subset_forced.argtypes = [P, P, C.c_int, P, C.c_int64, P, C.c_int64,
                                                        P, P, P, P, P]
            L.oracle_render_eq7.argtypes = [P, P, C.c_int, P]
            L.oracle_backward.argtypes = [P, P, C.c_int, P, C.c_int, P, P]
            L.oracle_backward_subset.argtypes = [P, P, C.c_int, P, C.c_int64, P, P, P]
            L.oracle_chain.argtypes = [P, P, C.c_int, P, P]
            L.oracle_fd_subset.argtypes = [P, P, C.c_int, P, C.c_int64, P, C.c_double, P]
            L.oracle_fd_subset_forced.argtypes = [P, P, C.c_int, P, C.c_int64, P, C.c_double,
                                                  C.c_int64, P, P, P, P]
            L.oracle_gaussian_flags.argtypes = [P, P, C.c_int, P]
            L.oracle_l1.argtypes = [C.c_int64, P, P, P, P, P]
            L.oracle_knn.argtypes = [C.c_int64, P, C.c_int, P]
            L.oracle_eig3.argtypes = [P, P, P]
            L.oracle_pca_init.argtypes = [C.c_int64, P, P, C.c_int, C.c_double, P, P, P]
            L.oracle_features.argtypes = [C.c_int64, P, P, C.c_int, P, P]
            L.oracle_mlp_forward.argtypes = [C.c_int64] + [P] * 7 + [C.c_int, P]
            L.oracle_init_loss.argtypes = [C.c_int64, P, P, P]
            L.oracle_init_loss.restype = C.c_double
            L.oracle_mlp_backward.argtypes = [C.c_int64] + [P] * 7 + [P, C.c_int] + [P] * 6
            L.oracle_apply_mlp.argtypes = [C.c_int64, P, P, P, P, P]
            L.oracle_make_targets.argtypes = [C.c_int64, P, P, P, P, P]
            L.oracle_adam.argtypes = [C.c_int64, P, P, P, P, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_int64]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Inputs:
    """Keeps the contiguous float32 copies alive while the C structs point at them."""

    def __init__(self, g, cam):
        self.arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in g.arrays()]
        m, ls, q, lg, sh = self.arrs
        self.g = OGauss(g.n, g.sh_degree, 0, _ptr(m).value, _ptr(ls).value, _ptr(q).value,
                        _ptr(lg).value, _ptr(sh).value)
        self.cam = OCam(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy),
                        float(cam.cx), float(cam.cy),
                        (C.c_float * 12)(*np.asarray(cam.viewmat, np.float32).reshape(-1).tolist()),
                        float(cam.near), (C.c_float * 3)(*[float(b) for b in cam.bg]))

    @property
    def gp(self):
        return C.byref(self.g)

    @property
    def cp(self):
        return C.byref(self.cam)


def tiles(cam, tile: int = 16):
    return (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile


def param_count(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


def det_expf(x) -> np.ndarray:
    L = lib()
    x = np.asarray(x, np.float32).reshape(-1)
    return np.array([L.oracle_det_expf(float(v)) for v in x], np.float32)


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (pixel rows, pixels, Gaussians); n <= 0 keeps the
    current setting.  Returns the count in effect."""
    return int(lib().oracle_set_threads(int(n)))


def decision_bound() -> float:
    """Relative bound on a compositing kernel's o G against the oracle's decision-side o 2^p
    (hardware 2^x approximation + fp32 logistic + one rounding)."""
    return float(lib().oracle_decision_bound())


def sh_basis(direction):
    """Y [16] and dY/d(x,y,z) [16][3] of the degree-3 real SH at a unit direction."""
    d = np.ascontiguousarray(direction, np.float64)
    y = np.zeros(16)
    dy = np.zeros((16, 3))
    lib().oracle_sh_basis(_ptr(d), _ptr(y), _ptr(dy))
    return y, dy


def project(g, cam, tile: int = 16) -> dict:
    inp = _Inputs(g, cam)
    n = g.n
    out = dict(visible=np.zeros(n, np.int32), radius=np.zeros((n, 2), np.int32),
               rect=np.zeros((n, 4), np.int32), depth=np.zeros(n, np.float32),
               uv=np.zeros((n, 2), np.float32), cov2d=np.zeros((n, 3), np.float32),
               mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
               rgb=np.zeros((n, 3)))
    lib().oracle_project(inp.gp, inp.cp, tile, *[_ptr(out[k]) for k in
                         ["visible", "radius", "rect", "depth", "uv", "cov2d", "mean2d", "conic",
                          "opacity", "rgb"]])
    return out


def keys(g, cam, tile: int = 16):
    """(keys uint64 [P], values uint32 [P], ranges uint32 [tiles][2])."""
    inp = _Inputs(g, cam)
    L = lib()
    P = L.oracle_keys(inp.gp, inp.cp, tile, 0, None, None, None)
    k = np.zeros(max(P, 1), np.uint64)
    v = np.zeros(max(P, 1), np.uint32)
    tx, ty = tiles(cam, tile)
    r = np.zeros((tx * ty, 2), np.uint32)
    L.oracle_keys(inp.gp, inp.cp, tile, P, _ptr(k), _ptr(v), _ptr(r))
    return k[:P], v[:P], r


def render(g, cam, tile: int = 16) -> dict:
    inp = _Inputs(g, cam)
    H, W = cam.height, cam.width
    out = dict(image=np.zeros((3, H, W)), T=np.zeros((H, W)), last=np.zeros((H, W), np.int32),
               flag=np.zeros((H, W), np.uint8), evals=np.zeros((H, W), np.int64),
               ncomp=np.zeros((H, W), np.int32))
    lib().oracle_render(inp.gp, inp.cp, tile, _ptr(out["image"]), _ptr(out["T"]),
                        _ptr(out["last"]), _ptr(out["flag"]), _ptr(out["evals"]),
                        _ptr(out["ncomp"]))
    return out


def render_pixels(g, cam, pix_xy, tile: int = 16) -> dict:
    inp = _Inputs(g, cam)
    pix = np.ascontiguousarray(pix_xy, np.int32).reshape(-1, 2)
    m = pix.shape[0]
    out = dict(rgb=np.zeros((m, 3)), T=np.zeros(m), last=np.zeros(m, np.int32),
               flag=np.zeros(m, np.uint8))
    lib().oracle_render_pixels(inp.gp, inp.cp, tile, m, _ptr(pix), _ptr(out["rgb"]),
                               _ptr(out["T"]), _ptr(out["last"]), _ptr(out["flag"]))
    return out


class Forced:
    """Decisions to follow for some pixels: pix [m][2] (x, y) int32, and per pixel the codes of its
    evaluated list entries (0 skipped, 1 composited, 2 composited clamped at 0.99, 3 stop),
    concatenated in `codes` (uint8) with pixel k's at codes[off[k]:off[k + 1]]."""

    def __init__(self, pix, off, codes):
        self.pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
        self.off = np.ascontiguousarray(off, np.int64)
        self.codes = np.ascontiguousarray(codes, np.uint8)
        assert self.off.shape == (self.pix.shape[0] + 1,) and self.off[-1] == self.codes.size

    @classmethod
    def empty(cls):
        return cls(np.zeros((0, 2), np.int32), np.zeros(1, np.int64), np.zeros(0, np.uint8))

    def __len__(self):
        return self.pix.shape[0]

    def args(self):
        b = max(1, self.codes.size)
        if self.codes.size == 0:
            self._pad = np.zeros(b, np.uint8)
            return [len(self), _ptr(self.pix), _ptr(self.off), _ptr(self._pad)]
        return [len(self), _ptr(self.pix), _ptr(self.off), _ptr(self.codes)]


def render_forced(g, cam, forced: Forced, tile: int = 16) -> dict:
    """Pixels of `forced` composited with its decisions (values FP64): rgb [m][3], T, last, ncomp,
    flips (codes differing from the oracle's own decisions) and illegal (of those, decisions the
    oracle did not find within the error bound of their threshold)."""
    inp = _Inputs(g, cam)
    m = len(forced)
    out = dict(rgb=np.zeros((m, 3)), T=np.zeros(m), last=np.zeros(m, np.int32),
               ncomp=np.zeros(m, np.int32), flips=np.zeros(m, np.int32), illegal=np.zeros(m, np.int32))
    if m:
        lib().oracle_render_forced(inp.gp, inp.cp, tile, m, _ptr(forced.pix), _ptr(forced.off),
                                   _ptr(forced.codes), *[_ptr(out[k]) for k in
                                                         ("rgb", "T", "last", "ncomp", "flips", "illegal")])
    return out


def decisions(g, cam, pix_xy, max_entries: int, tile: int = 16) -> dict:
    """The oracle's own decisions entry by entry: og [m][max_entries] (decision-side o 2^p),
    code [m][max_entries] and count [m] (evaluated entries, -1 beyond max_entries)."""
    inp = _Inputs(g, cam)
    pix = np.ascontiguousarray(pix_xy, np.int32).reshape(-1, 2)
    m = pix.shape[0]
    out = dict(og=np.zeros((m, max_entries)), code=np.full((m, max_entries), 255, np.uint8),
               count=np.zeros(m, np.int64))
    lib().oracle_decisions(inp.gp, inp.cp, tile, m, _ptr(pix), max_entries, _ptr(out["og"]),
                           _ptr(out["code"]), _ptr(out["count"]))
    return out


def render_eq7(g, cam, tile: int = 16) -> np.ndarray:
    inp = _Inputs(g, cam)
    img = np.zeros((3, cam.height, cam.width))
    lib().oracle_render_eq7(inp.gp, inp.cp, tile, _ptr(img))
    return img


def split_grads(flat: np.ndarray, n: int, sh_degree: int) -> dict:
    """Planar [P*N] parameter gradients -> named arrays."""
    K = (sh_degree + 1) ** 2
    return dict(means=flat[:3 * n].reshape(3, n), log_scales=flat[3 * n:6 * n].reshape(3, n),
                quats=flat[6 * n:10 * n].reshape(4, n), opacity_logits=flat[10 * n:11 * n],
                sh=flat[11 * n:].reshape(3, K, n))


def backward(g, cam, dL_dimage, tile: int = 16, mode: int = 0, forced: Forced | None = None):
    """(grad2d [N][9], named parameter gradients) for an upstream gradient [3][H][W]; the pixels of
    `forced` follow its decisions."""
    inp = _Inputs(g, cam)
    d = np.ascontiguousarray(dL_dimage, np.float64)
    g2 = np.zeros((g.n, 9))
    flat = np.zeros(param_count(g.sh_degree) * g.n)
    f = forced if forced is not None else Forced.empty()
    lib().oracle_backward_forced(inp.gp, inp.cp, tile, _ptr(d), mode, *f.args(), _ptr(g2), _ptr(flat))
    return g2, split_grads(flat, g.n, g.sh_degree)


def backward_subset(g, cam, dL_dimage, sel, tile: int = 16, forced: Forced | None = None):
    """(grad2d [S][9], grads [S][11 + 3K]) for the selected canonical indices; the pixels of
    `forced` follow its decisions."""
    inp = _Inputs(g, cam)
    d = np.ascontiguousarray(dL_dimage, np.float64)
    sel = np.ascontiguousarray(sel, np.int64)
    g2 = np.zeros((len(sel), 9))
    gp = np.zeros((len(sel), param_count(g.sh_degree)))
    f = forced if forced is not None else Forced.empty()
    lib().oracle_backward_subset_forced(inp.gp, inp.cp, tile, _ptr(d), len(sel), _ptr(sel), *f.args(),
                                        _ptr(g2), _ptr(gp))
    return g2, gp


def fd_subset(g, cam, dL_dimage, sel, h_rel: float = 2.0 ** -12, tile: int = 16,
              forced: Forced | None = None):
    """FP64 central differences [S][11 + 3K] of sum(dL_dimage * image) for the selected
    Gaussians; NaN where a perturbation changed a decision.  The pixels of `forced` keep its
    decisions."""
    inp = _Inputs(g, cam)
    d = np.ascontiguousarray(dL_dimage, np.float64)
    sel = np.ascontiguousarray(sel, np.int64)
    out = np.zeros((len(sel), param_count(g.sh_degree)))
    f = forced if forced is not None else Forced.empty()
    lib().oracle_fd_subset_forced(inp.gp, inp.cp, tile, _ptr(d), len(sel), _ptr(sel), h_rel, *f.args(),
                                  _ptr(out))
    return out


def chain(g, cam, grad2d, tile: int = 16) -> dict:
    inp = _Inputs(g, cam)
    g2 = np.ascontiguousarray(grad2d, np.float64)
    flat = np.zeros(param_count(g.sh_degree) * g.n)
    lib().oracle_chain(inp.gp, inp.cp, tile, _ptr(g2), _ptr(flat))
    return split_grads(flat, g.n, g.sh_degree)


def gaussian_flags(g, cam, tile: int = 16) -> np.ndarray:
    inp = _Inputs(g, cam)
    f = np.zeros(g.n, np.uint8)
    lib().oracle_gaussian_flags(inp.gp, inp.cp, tile, _ptr(f))
    return f


def l1(img, gt):
    a = np.ascontiguousarray(img, np.float64).reshape(-1)
    b = np.ascontiguousarray(gt, np.float64).reshape(-1)
    grad = np.zeros_like(a)
    loss = C.c_double()
    sse = C.c_double()
    lib().oracle_l1(a.size, _ptr(a), _ptr(b), _ptr(grad), C.byref(loss), C.byref(sse))
    return loss.value, grad.reshape(np.shape(img)), sse.value


def adam(p, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step in place on float64 arrays."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().oracle_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), lr, b1, b2, eps, t)


# ------------------------------------------------------------------------------------------------
# initializer path (operator I, Sec. III-B) and its learned stand-in
# ------------------------------------------------------------------------------------------------

def knn(points, k: int) -> np.ndarray:
    """points [3][n] float32 -> neighbour indices [n][k] (self excluded), by (fp32 d^2, index)."""
    P = np.ascontiguousarray(points, np.float32)
    n = P.shape[1]
    nb = np.zeros((n, k), np.int32)
    lib().oracle_knn(n, _ptr(P), k, _ptr(nb))
    return nb


def eig3(A):
    A = np.ascontiguousarray(A, np.float64).reshape(9)
    w = np.zeros(3)
    V = np.zeros(9)
    lib().oracle_eig3(_ptr(A), _ptr(w), _ptr(V))
    return w, V.reshape(3, 3)


def pca_init(points, nb, r_normal: float = 0.1) -> dict:
    P = np.ascontiguousarray(points, np.float32)
    nb = np.ascontiguousarray(nb, np.int32)
    n = P.shape[1]
    ls, q, lg = np.zeros((3, n)), np.zeros((4, n)), np.zeros(n)
    lib().oracle_pca_init(n, _ptr(P), _ptr(nb), nb.shape[1], r_normal, _ptr(ls), _ptr(q), _ptr(lg))
    return dict(log_scales=ls, quats=q, opacity_logits=lg)


def features(points, nb):
    """(features [n][16], eigenframe quaternions [4][n])."""
    P = np.ascontiguousarray(points, np.float32)
    nb = np.ascontiguousarray(nb, np.int32)
    n = P.shape[1]
    f = np.zeros((n, 16))
    fq = np.zeros((4, n))
    lib().oracle_features(n, _ptr(P), _ptr(nb), nb.shape[1], _ptr(f), _ptr(fq))
    return f, fq


def _w(ws):
    return [np.ascontiguousarray(w, np.float32) for w in ws]


def mlp_forward(x, weights, mode: int = 1) -> np.ndarray:
    """weights = (W1 [64][16], b1, W2 [64][64], b2, W3 [8][64], b3); x [n][16]."""
    x = np.ascontiguousarray(x, np.float32)
    W = _w(weights)
    out = np.zeros((x.shape[0], 8))
    lib().oracle_mlp_forward(x.shape[0], _ptr(x), *[_ptr(w) for w in W], mode, _ptr(out))
    return out


def init_loss(y, t):
    y = np.ascontiguousarray(y, np.float64)
    t = np.ascontiguousarray(t, np.float32)
    dy = np.zeros_like(y)
    L = lib().oracle_init_loss(y.shape[0], _ptr(y), _ptr(t), _ptr(dy))
    return L, dy


def mlp_backward(x, weights, dy, mode: int = 1):
    x = np.ascontiguousarray(x, np.float32)
    W = _w(weights)
    dy = np.ascontiguousarray(dy, np.float64)
    grads = [np.zeros(w.shape) for w in W]
    lib().oracle_mlp_backward(x.shape[0], _ptr(x), *[_ptr(w) for w in W], _ptr(dy), mode,
                              *[_ptr(g) for g in grads])
    return grads


def _base(g):
    return (np.ascontiguousarray(g["log_scales"], np.float64), np.ascontiguousarray(g["quats"], np.float64),
            np.ascontiguousarray(g["opacity_logits"], np.float64))


def apply_mlp(y, base) -> dict:
    """Learned parameters: MLP outputs y [n][8] applied as corrections of `base` (the paper's
    initializer: log_scales [3][n], quats [4][n], opacity_logits [n])."""
    y = np.ascontiguousarray(y, np.float64)
    bl, bq, bo = _base(base)
    n = y.shape[0]
    out = dict(log_scales=np.zeros((3, n)), quats=np.zeros((4, n)), opacity_logits=np.zeros(n))
    lib().oracle_apply_mlp(n, _ptr(y), _ptr(bl), _ptr(bq), _ptr(bo), _ptr(out["log_scales"]),
                           _ptr(out["quats"]), _ptr(out["opacity_logits"]))
    return out


def make_targets(base, converged) -> np.ndarray:
    """Targets [n][8] of `converged` relative to `base` (dicts as in apply_mlp)."""
    bl, bq, bo = _base(base)
    cl, cq, co = _base(converged)
    n = bq.shape[1]
    t = np.zeros((n, 8))
    lib().oracle_make_targets(n, _ptr(bl), _ptr(bq), _ptr(bo), _ptr(cl), _ptr(cq), _ptr(co), _ptr(t))
    return t
