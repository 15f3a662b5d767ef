"""Batched training over many views of many scenes: one planned batch per set of (scene, view,
target) renders, one training step = render + L1 + backward + Adam of every render, optionally
captured once in a CUDA graph and replayed; or its halves apart (render(), then backward() of the
caller's upstream gradients, e.g. L1 + D-SSIM).  Thin marshalling over pgs_batch_*,
pgs_render_batch and pgs_backward_batch of the C ABI."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .rasterizer import AdamConfig, GaussianBuffer, camera_struct


class BatchTrainer:
    """scenes: GaussianBuffers (one SH degree); views: (scene index, camera, target [3][H][W])
    tuples, given scene by scene."""

    def __init__(self, scenes: list, views: list, adam: AdamConfig | None = None,
                 pair_capacity: int = 0, stream: torch.cuda.Stream | None = None, tile: int = 16):
        self._lib = L.lib()
        adam = adam or AdamConfig()
        self.scenes = scenes
        self.m = [s.zeros_like() for s in scenes]
        self.v = [s.zeros_like() for s in scenes]
        order = [s for s, _, _ in views]
        if order != sorted(order):
            raise ValueError("views must be given scene by scene")
        self.views = views
        dev = scenes[0].data.device
        self.images = [torch.zeros((3, c.height, c.width), dtype=torch.float32, device=dev)
                       for _, c, _ in views]
        self.dls = [torch.zeros_like(im) for im in self.images]
        self.targets = [t.contiguous() for _, _, t in views]
        # a stream of its own: the legacy default stream cannot be captured in a graph; every
        # call is ordered after the caller's current stream and before its later work
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        S, R = len(scenes), len(views)
        P = (L.PgsGaussians * S)(*[s.struct() for s in scenes])
        M = (L.PgsGaussians * S)(*[s.struct() for s in self.m])
        V = (L.PgsGaussians * S)(*[s.struct() for s in self.v])
        D = (L.PgsRenderDesc * R)(*[
            L.PgsRenderDesc(int(s), 0, camera_struct(c), self.images[k].data_ptr(),
                            self.targets[k].data_ptr(), self.dls[k].data_ptr())
            for k, (s, c, _) in enumerate(views)])
        self.tile = int(tile)  # screen tile edge: 8, 16 or 32
        self.adam = adam
        cfg = L.PgsConfig(self.tile, 0, int(pair_capacity), adam.b1, adam.b2, adam.eps,
                          (C.c_float * 6)(*adam.lr))
        self._b = C.c_void_p()
        L.check(self._lib.pgs_batch_create(C.byref(self._b), C.byref(cfg), S, P, M, V, R, D,
                                           int(pair_capacity), C.c_void_p(self.stream.cuda_stream)),
                "pgs_batch_create")
        self.captured = False

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._lib.pgs_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _enter(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.stream.device))

    def _leave(self):
        torch.cuda.current_stream(self.stream.device).wait_stream(self.stream)

    def step(self):
        self._enter()
        L.check(self._lib.pgs_batch_step(self._b), "pgs_batch_step")
        self._leave()

    def render(self):
        """The forward of every render into self.images (no loss, no parameter change)."""
        self._enter()
        L.check(self._lib.pgs_render_batch(self._b), "pgs_render_batch")
        self._leave()

    def backward(self, grads: list):
        """The backward of the last render() for the upstream gradients in self.dls (written by the
        caller), added to grads (one GaussianBuffer per scene)."""
        if len(grads) != len(self.scenes):
            raise ValueError("one gradient buffer per scene")
        G = (L.PgsGaussians * len(grads))(*[g.struct() for g in grads])
        self._enter()
        L.check(self._lib.pgs_backward_batch(self._b, G), "pgs_backward_batch")
        self._leave()

    def capture(self):
        self._enter()
        L.check(self._lib.pgs_batch_capture(self._b), "pgs_batch_capture")
        self.captured = True

    def set_views(self, views: list):
        """New (camera, target) per render slot, same sizes; applies from the next step."""
        if len(views) != len(self.views):
            raise ValueError("one (camera, target) per render")
        cams = (L.PgsCamera * len(views))(*[camera_struct(c) for c, _ in views])
        self._keep = [t.contiguous() for _, t in views]
        ptrs = (C.c_void_p * len(views))(*[t.data_ptr() for t in self._keep])
        self._enter()
        L.check(self._lib.pgs_batch_set_views(self._b, cams, ptrs), "pgs_batch_set_views")

    def reserve(self, pair_capacity: int):
        """Grow the pair capacity (a captured graph is captured again)."""
        self._enter()
        L.check(self._lib.pgs_batch_reserve(self._b, int(pair_capacity)), "pgs_batch_reserve")

    def steps(self) -> int:
        """Completed steps (steps after a pair overflow do not count)."""
        t = C.c_int64()
        L.check(self._lib.pgs_batch_steps(self._b, C.byref(t)), "pgs_batch_steps")
        return t.value

    def check(self) -> int:
        """Read the status; after a pair overflow grow the capacity to the pairs needed + 25 %.
        Returns the completed steps."""
        code, pairs = self.status()
        if code == L.PGS_ERR_CAPACITY:
            self.reserve(pairs + pairs // 4 + 4096)
        elif code != 0:
            L.check(code, "batched step")
        return self.steps()

    def losses(self) -> np.ndarray:
        out = np.zeros((len(self.views), 2))
        L.check(self._lib.pgs_batch_losses(self._b, out.ctypes.data_as(C.c_void_p)), "pgs_batch_losses")
        return out

    def status(self):
        pairs = C.c_int64()
        code = self._lib.pgs_batch_status(self._b, C.byref(pairs))
        return code, pairs.value

    def launch_count(self) -> int:
        return int(self._lib.pgs_batch_launch_count(self._b))

    def set_variant(self, pixels_per_thread: int, depth: int):
        L.check(self._lib.pgs_batch_set_variant(self._b, int(pixels_per_thread), int(depth)),
                "pgs_batch_set_variant")
        self.captured = False

    def time_render(self, reps: int = 3) -> float:
        """ms of the render part of a step (projection .. tile order) on the current parameters."""
        self._enter()
        ms = C.c_float()
        L.check(self._lib.pgs_batch_time_render(self._b, int(reps), C.byref(ms)), "pgs_batch_time_render")
        return float(ms.value)

    def time_variants(self, reps: int = 3) -> dict:
        self._enter()
        ms = np.zeros(len(L.VARIANTS), np.float32)
        L.check(self._lib.pgs_batch_time_variants(self._b, int(reps), ms.ctypes.data_as(C.c_void_p)),
                "pgs_batch_time_variants")
        return {v: float(t) for v, t in zip(L.VARIANTS, ms) if t >= 0}  # -1: not for this tile edge
