"""Single-reference cost-volume MVS of the geometry prior (Sec. III-A) on the GPU: per target
keyframe, the depth range from the projected sparse points, the Eq. 4 reference keyframe, census
matching over a plane sweep, SGM aggregation, the 0.4 confidence filter, and fusion of the kept
depths into a dense world point cloud (the P that seeds the initializer).

All arithmetic runs in libpocketgs kernels; this module marshals tensors.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .rasterizer import camera_struct


def _p(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class MultiViewStereo:
    """Buffers for one target at a time at a fixed resolution and plane count."""

    def __init__(self, width: int, height: int, planes: int = 64, stream: torch.cuda.Stream | None = None,
                 device="cuda"):
        self._lib = L.lib()
        self.W, self.H, self.D = int(width), int(height), int(planes)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._m = C.c_void_p()
        L.check(self._lib.pgs_mvs_create(C.byref(self._m), self.W, self.H, self.D,
                                         C.c_void_p(self.stream.cuda_stream)), "pgs_mvs_create")

    def close(self):
        if getattr(self, "_m", None) is not None and self._m.value:
            self._lib.pgs_mvs_destroy(self._m)
            self._m = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _image(self, img: torch.Tensor, name: str) -> torch.Tensor:
        if img.dtype != torch.float32 or not img.is_cuda or not img.is_contiguous() or tuple(img.shape) != (3, self.H, self.W):
            raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor of shape (3, {self.H}, {self.W})")
        return img

    def depth_range(self, cam, points: torch.Tensor):
        """(d_min, d_max, median) of a target from sparse points [n][3] (float32 CUDA)."""
        if (points.dtype != torch.float32 or not points.is_cuda or not points.is_contiguous() or points.dim() != 2
                or points.shape[1] != 3):
            raise ValueError("points: expected a contiguous float32 CUDA tensor of shape (n, 3)")
        out = (C.c_double * 3)()
        cs = camera_struct(cam)
        L.check(self._lib.pgs_mvs_depth_range(self._m, C.byref(cs), _p(points), int(points.shape[0]), out),
                "pgs_mvs_depth_range")
        return out[0], out[1], out[2]

    def select_reference(self, cams, target: int, median_depth: float):
        """(reference index, scores [len(cams)]) by Eq. 4."""
        arr = (L.PgsCamera * len(cams))(*[camera_struct(c) for c in cams])
        scores = np.zeros(len(cams), np.float64)
        ref = C.c_int32()
        L.check(self._lib.pgs_mvs_select_reference(self._m, arr, len(cams), int(target), float(median_depth),
                                                   scores.ctypes.data_as(C.POINTER(C.c_double)), C.byref(ref)),
                "pgs_mvs_select_reference")
        return int(ref.value), scores

    def depth(self, cam_t, cam_r, image_t: torch.Tensor, image_r: torch.Tensor, d_min: float, d_max: float,
              out: torch.Tensor | None = None, count: bool = True):
        """Depth map [H][W] (NaN where not kept) and the kept count (None with count=False)."""
        image_t, image_r = self._image(image_t, "image_t"), self._image(image_r, "image_r")
        if out is None:
            out = torch.empty((self.H, self.W), dtype=torch.float32, device=self.device)
        ct, cr = camera_struct(cam_t), camera_struct(cam_r)
        kept = C.c_int64()
        L.check(self._lib.pgs_mvs_depth(self._m, C.byref(ct), C.byref(cr), _p(image_t), _p(image_r), float(d_min),
                                        float(d_max), _p(out), C.byref(kept) if count else None), "pgs_mvs_depth")
        return out, (int(kept.value) if count else None)

    STAGES = ["census", "cost", "sgm", "select"]

    def stage_times(self, cam_t, cam_r, image_t: torch.Tensor, image_r: torch.Tensor, d_min: float, d_max: float):
        """Device ms of each stage of depth(), keyed by STAGES."""
        image_t, image_r = self._image(image_t, "image_t"), self._image(image_r, "image_r")
        out = torch.empty((self.H, self.W), dtype=torch.float32, device=self.device)
        ct, cr = camera_struct(cam_t), camera_struct(cam_r)
        ms = (C.c_float * 4)()
        L.check(self._lib.pgs_mvs_stage_times(self._m, C.byref(ct), C.byref(cr), _p(image_t), _p(image_r),
                                              float(d_min), float(d_max), _p(out), C.cast(ms, C.c_void_p)),
                "pgs_mvs_stage_times")
        return dict(zip(self.STAGES, list(ms)))

    def read(self, what: int) -> torch.Tensor:
        shapes = {L.PGS_MVS_CENSUS_TARGET: ((self.H, self.W), torch.int64),
                  L.PGS_MVS_CENSUS_REFERENCE: ((self.H, self.W), torch.int64),
                  L.PGS_MVS_COST: ((self.H, self.W, self.D), torch.uint8),
                  L.PGS_MVS_AGGREGATED: ((self.H, self.W, self.D), torch.int16),
                  L.PGS_MVS_PLANE_MAPS: ((self.D, 9), torch.float32)}
        shape, dt = shapes[what]
        t = torch.empty(shape, dtype=dt, device=self.device)
        L.check(self._lib.pgs_mvs_read(self._m, int(what), _p(t), t.numel() * t.element_size()), "pgs_mvs_read")
        return t

    def fuse(self, cam, depth: torch.Tensor, capacity: int | None = None):
        """World points [n][3] and pixel indices [n] of the kept depths, in pixel order."""
        cap = self.W * self.H if capacity is None else int(capacity)
        pts = torch.empty((max(cap, 1), 3), dtype=torch.float32, device=self.device)
        pix = torch.empty((max(cap, 1),), dtype=torch.int32, device=self.device)
        n = C.c_int64()
        cs = camera_struct(cam)
        L.check(self._lib.pgs_mvs_fuse(self._m, C.byref(cs), _p(depth), _p(pts), _p(pix), cap, C.byref(n)),
                "pgs_mvs_fuse")
        return pts[:n.value], pix[:n.value]

    def reconstruct(self, cams, images, target: int, points: torch.Tensor):
        """The whole single-reference MVS of one target keyframe: (reference, (d_min, d_max),
        depth map, world points, pixel indices).  images: a sequence indexed like cams holding at
        least the target's and the chosen reference's [3][H][W] CUDA images."""
        d_min, d_max, med = self.depth_range(cams[target], points)
        ref, _ = self.select_reference(cams, target, med)
        depth, _ = self.depth(cams[target], cams[ref], images[target], images[ref], d_min, d_max, count=False)
        pts, pix = self.fuse(cams[target], depth)
        return ref, (d_min, d_max), depth, pts, pix
