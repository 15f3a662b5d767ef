"""Bundle adjustment of the geometry prior (Sec. III-A) on the GPU: Levenberg-Marquardt on the
robust reprojection objective of Eq. 2, each step solved through the reduced camera system of
Eq. 3 (independent 3 x 3 point inverses, dense FP64 Cholesky of the 6C x 6C camera system,
back-substitution of the points).

Cameras are world-to-camera (R [C][3][3], t [C][3]); points P [n][3]; observations (cam, pt, uv)
grouped by point (pt non-decreasing); intrinsics (fx, fy, cx, cy).  All arithmetic runs in
libpocketgs kernels; this module marshals tensors.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _p(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _f32(t: torch.Tensor, shape, name: str) -> torch.Tensor:
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor of shape {tuple(shape)}")
    return t


def _i32(t: torch.Tensor, m: int, name: str) -> torch.Tensor:
    if t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (m,):
        raise ValueError(f"{name}: expected a contiguous int32 CUDA tensor of shape ({m},)")
    return t


class BundleAdjuster:
    """Buffers for a fixed problem size (C cameras, n points, m observations) on one stream."""

    def __init__(self, n_cams: int, n_points: int, n_obs: int, stream: torch.cuda.Stream | None = None,
                 device="cuda"):
        self._lib = L.lib()
        self.C, self.n, self.m = int(n_cams), int(n_points), int(n_obs)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._b = C.c_void_p()
        L.check(self._lib.pgs_ba_create(C.byref(self._b), self.C, self.n, self.m,
                                        C.c_void_p(self.stream.cuda_stream)), "pgs_ba_create")

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._lib.pgs_ba_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _K(K):
        return (C.c_float * 4)(*[float(k) for k in K])

    def _state(self, R, t, P):
        return (_f32(R, (self.C, 3, 3), "R"), _f32(t, (self.C, 3), "t"), _f32(P, (self.n, 3), "P"))

    def project(self, R, t, P, cam, pt, K):
        """uv [k][2] and depth z [k] of the (cam, pt) pairs."""
        R, t, P = self._state(R, t, P)
        k = int(cam.shape[0])
        cam, pt = _i32(cam, k, "cam"), _i32(pt, k, "pt")
        uv = torch.empty((k, 2), dtype=torch.float32, device=self.device)
        z = torch.empty((k,), dtype=torch.float32, device=self.device)
        L.check(self._lib.pgs_ba_project(self._b, _p(R), _p(t), _p(P), _p(cam), _p(pt), k, self._K(K),
                                         _p(uv), _p(z)), "pgs_ba_project")
        return uv, z

    def _obs(self, cam, pt, uv):
        return _i32(cam, self.m, "cam"), _i32(pt, self.m, "pt"), _f32(uv, (self.m, 2), "uv")

    def step(self, R, t, P, cam, pt, uv, K, sigma: float, delta: float, lam: float):
        """One damped step at lam, not applied: (dcam [C][6] (omega, v), dP [n][3], cost)."""
        R, t, P = self._state(R, t, P)
        cam, pt, uv = self._obs(cam, pt, uv)
        dcam = torch.empty((self.C, 6), dtype=torch.float32, device=self.device)
        dP = torch.empty((self.n, 3), dtype=torch.float32, device=self.device)
        cost = C.c_double()
        L.check(self._lib.pgs_ba_step(self._b, _p(R), _p(t), _p(P), _p(cam), _p(pt), _p(uv), self._K(K),
                                      sigma, delta, lam, _p(dcam), _p(dP), C.byref(cost)), "pgs_ba_step")
        return dcam, dP, cost.value

    def solve(self, R, t, P, cam, pt, uv, K, sigma: float, delta: float, iters: int = 20, lam0: float = 1e-4):
        """Levenberg-Marquardt in place on (R, t, P); returns (costs [iters + 1], accepted)."""
        R, t, P = self._state(R, t, P)
        cam, pt, uv = self._obs(cam, pt, uv)
        costs = np.zeros(iters + 1, np.float64)
        acc = C.c_int32()
        L.check(self._lib.pgs_ba_solve(self._b, _p(R), _p(t), _p(P), _p(cam), _p(pt), _p(uv), self._K(K),
                                       sigma, delta, int(iters), lam0, costs.ctypes.data_as(C.POINTER(C.c_double)),
                                       C.byref(acc)), "pgs_ba_solve")
        return costs, int(acc.value)

    STAGES = ["linearize", "camblocks", "points", "schur", "solve", "backsub", "cost"]

    def stage_times(self, R, t, P, cam, pt, uv, K, sigma: float, delta: float, lam: float):
        """Device ms of each stage of one iteration (nothing applied), keyed by STAGES."""
        R, t, P = self._state(R, t, P)
        cam, pt, uv = self._obs(cam, pt, uv)
        ms = (C.c_float * 7)()
        L.check(self._lib.pgs_ba_stage_times(self._b, _p(R), _p(t), _p(P), _p(cam), _p(pt), _p(uv), self._K(K),
                                             sigma, delta, lam, C.cast(ms, C.c_void_p)), "pgs_ba_stage_times")
        return dict(zip(self.STAGES, list(ms)))
