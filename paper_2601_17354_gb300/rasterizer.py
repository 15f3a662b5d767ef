"""Python face of the rasterizer: parameter buffers, a context, and the render / loss /
backward / step calls of one training iteration (operator T of Sec. III,
T : (Theta_0, {I_t, T_t}) -> Theta*).

PyTorch supplies device memory and the CUDA stream; every computation runs in libpocketgs.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")

# Learning rates of the parameter groups (the paper states none): means 1.6e-4 x scene extent 2,
# log-scales 5e-3, rotations 1e-3, opacity logits 2.5e-2, SH DC 2.5e-3, higher SH 1.25e-4.
DEFAULT_LR = (3.2e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4)


def rows_of(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


class GaussianBuffer:
    """One contiguous fp32 device buffer [11 + 3K][n] holding the planar groups
    means [3][n], log_scales [3][n], quats [4][n], opacity_logits [n], sh [3][K][n]."""

    def __init__(self, n: int, sh_degree: int, device="cuda", data: torch.Tensor | None = None):
        self.n = int(n)
        self.sh_degree = int(sh_degree)
        K = (sh_degree + 1) ** 2
        rows = rows_of(sh_degree)
        if data is None:
            data = torch.zeros((rows, self.n), dtype=torch.float32, device=device)
        assert data.shape == (rows, self.n) and data.dtype == torch.float32 and data.is_contiguous()
        self.data = data
        self.means = data[0:3]
        self.log_scales = data[3:6]
        self.quats = data[6:10]
        self.opacity_logits = data[10]
        self.sh = data[11:].view(3, K, self.n)
        self._struct = None

    @classmethod
    def from_arrays(cls, g, device="cuda") -> "GaussianBuffer":
        """From any object with numpy/torch attributes means, log_scales, quats, opacity_logits,
        sh and sh_degree (e.g. synthetic.Gaussians)."""
        n = int(np.asarray(g.means).shape[1]) if not torch.is_tensor(g.means) else g.means.shape[1]
        buf = cls(n, g.sh_degree, device)
        for name in GROUPS:
            src = getattr(g, name)
            t = src if torch.is_tensor(src) else torch.from_numpy(np.ascontiguousarray(src, np.float32))
            getattr(buf, name).copy_(t.to(device).view_as(getattr(buf, name)))
        return buf

    def zeros_like(self) -> "GaussianBuffer":
        return GaussianBuffer(self.n, self.sh_degree, self.data.device)

    def clone(self) -> "GaussianBuffer":
        return GaussianBuffer(self.n, self.sh_degree, self.data.device, self.data.clone())

    def struct(self) -> L.PgsGaussians:
        if self._struct is None:
            self._struct = L.PgsGaussians(self.n, self.sh_degree, 0, *[
                getattr(self, k).data_ptr() for k in GROUPS])
        return self._struct

    def numpy(self) -> dict:
        return {k: getattr(self, k).detach().cpu().numpy() for k in GROUPS}


def tensors_struct(n, sh_degree, means, log_scales, quats, opacity_logits, sh) -> L.PgsGaussians:
    """Struct over separate contiguous fp32 CUDA tensors (autograd path)."""
    ts = (means, log_scales, quats, opacity_logits, sh)
    for t in ts:
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("parameters must be contiguous float32 CUDA tensors")
    return L.PgsGaussians(n, sh_degree, 0, *[t.data_ptr() for t in ts])


def camera_struct(cam) -> L.PgsCamera:
    vm = np.asarray(cam.viewmat, np.float32).reshape(-1)
    bg = getattr(cam, "bg", (0.0, 0.0, 0.0))
    return L.PgsCamera(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy),
                       float(cam.cx), float(cam.cy), (C.c_float * 12)(*vm.tolist()),
                       float(getattr(cam, "near", 0.2)), (C.c_float * 3)(*[float(b) for b in bg]))


@dataclass
class AdamConfig:
    lr: tuple = DEFAULT_LR
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-15


class Rasterizer:
    """A libpocketgs context bound to one CUDA stream (default: the current torch stream)."""

    def __init__(self, pair_capacity: int = 0, adam: AdamConfig | None = None,
                 stream: torch.cuda.Stream | None = None, device="cuda", tile: int = 16):
        self._lib = L.lib()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.tile = int(tile)  # screen tile edge: 8, 16 or 32
        adam = adam or AdamConfig()
        cfg = L.PgsConfig(self.tile, 0, int(pair_capacity), adam.b1, adam.b2, adam.eps,
                          (C.c_float * 6)(*adam.lr))
        self._ctx = C.c_void_p()
        L.check(self._lib.pgs_create(C.byref(self._ctx), C.byref(cfg),
                                     C.c_void_p(self.stream.cuda_stream)), "pgs_create")
        self.render_id = 0
        self._last_shape = None

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.pgs_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------------------------- calls
    def reserve(self, n: int, width: int, height: int, pair_capacity: int):
        L.check(self._lib.pgs_reserve(self._ctx, int(n), int(width), int(height),
                                      int(pair_capacity)), "pgs_reserve")

    def render_struct(self, g: L.PgsGaussians, cam, out: torch.Tensor | None = None) -> torch.Tensor:
        cs = cam if isinstance(cam, L.PgsCamera) else camera_struct(cam)
        if out is None:
            out = torch.empty((3, cs.height, cs.width), dtype=torch.float32, device=self.device)
        L.check(self._lib.pgs_render(self._ctx, C.byref(g), C.byref(cs), C.c_void_p(out.data_ptr())),
                "pgs_render")
        self.render_id += 1
        self._last_shape = (cs.height, cs.width)
        return out

    def render(self, params: GaussianBuffer, cam, out: torch.Tensor | None = None) -> torch.Tensor:
        return self.render_struct(params.struct(), cam, out)

    def render_l1(self, params: GaussianBuffer, cam, target: torch.Tensor, out: torch.Tensor | None = None,
                  grad: torch.Tensor | None = None, loss: torch.Tensor | None = None):
        """render + loss_l1 in one pass (pgs_render_l1): (image, dL/dimage, device tensor [l1, sse])."""
        cs = cam if isinstance(cam, L.PgsCamera) else camera_struct(cam)
        shape = (3, cs.height, cs.width)
        assert target.is_contiguous() and tuple(target.shape) == shape and target.dtype == torch.float32
        out = torch.empty(shape, dtype=torch.float32, device=self.device) if out is None else out
        grad = torch.empty(shape, dtype=torch.float32, device=self.device) if grad is None else grad
        loss = torch.empty(2, dtype=torch.float32, device=self.device) if loss is None else loss
        g = params.struct()
        L.check(self._lib.pgs_render_l1(self._ctx, C.byref(g), C.byref(cs), C.c_void_p(target.data_ptr()),
                                        C.c_void_p(out.data_ptr()), C.c_void_p(grad.data_ptr()),
                                        C.c_void_p(loss.data_ptr())), "pgs_render_l1")
        self.render_id += 1
        self._last_shape = (cs.height, cs.width)
        return out, grad, loss

    def loss_l1(self, image: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None,
                out: torch.Tensor | None = None):
        """(dL/dimage, device tensor [l1, sse])."""
        assert image.is_contiguous() and target.is_contiguous() and image.numel() == target.numel()
        grad = torch.empty_like(image) if grad is None else grad
        out = torch.empty(2, dtype=torch.float32, device=self.device) if out is None else out
        L.check(self._lib.pgs_loss_l1(self._ctx, C.c_void_p(image.data_ptr()),
                                      C.c_void_p(target.data_ptr()), image.numel(),
                                      C.c_void_p(grad.data_ptr()), C.c_void_p(out.data_ptr())),
                "pgs_loss_l1")
        return grad, out

    def loss_dssim(self, image: torch.Tensor, target: torch.Tensor, lam: float = 0.2,
                   grad: torch.Tensor | None = None, out: torch.Tensor | None = None):
        """(1 - lam) L1 + lam (1 - SSIM) of [3][H][W] images: (dL/dimage, device tensor
        [loss, mean SSIM])."""
        assert image.is_contiguous() and target.is_contiguous() and image.shape == target.shape
        _, H, W = image.shape
        grad = torch.empty_like(image) if grad is None else grad
        out = torch.empty(2, dtype=torch.float32, device=self.device) if out is None else out
        L.check(self._lib.pgs_loss_dssim(self._ctx, C.c_void_p(image.data_ptr()), C.c_void_p(target.data_ptr()),
                                         int(W), int(H), float(lam), C.c_void_p(grad.data_ptr()),
                                         C.c_void_p(out.data_ptr())), "pgs_loss_dssim")
        return grad, out

    def backward_struct(self, dL_dimage: torch.Tensor, grads: L.PgsGaussians):
        assert dL_dimage.is_contiguous() and dL_dimage.dtype == torch.float32
        L.check(self._lib.pgs_backward(self._ctx, C.c_void_p(dL_dimage.data_ptr()), C.byref(grads)),
                "pgs_backward")

    def backward(self, dL_dimage: torch.Tensor, grads: GaussianBuffer):
        self.backward_struct(dL_dimage, grads.struct())

    def step(self, params: GaussianBuffer, grads: GaussianBuffer, m: GaussianBuffer,
             v: GaussianBuffer, t: int):
        L.check(self._lib.pgs_step(self._ctx, C.byref(params.struct()), C.byref(grads.struct()),
                                   C.byref(m.struct()), C.byref(v.struct()), int(t)), "pgs_step")

    def backward_step(self, dL_dimage: torch.Tensor, params: GaussianBuffer, m: GaussianBuffer,
                      v: GaussianBuffer, t: int):
        """Backward of the last render fused with one Adam step (no gradient buffer)."""
        assert dL_dimage.is_contiguous() and dL_dimage.dtype == torch.float32
        L.check(self._lib.pgs_backward_step(self._ctx, C.c_void_p(dL_dimage.data_ptr()),
                                            C.byref(params.struct()), C.byref(m.struct()),
                                            C.byref(v.struct()), int(t)), "pgs_backward_step")

    def status(self):
        """(code, pairs of the last render); synchronises."""
        pairs = C.c_int64()
        code = self._lib.pgs_status(self._ctx, C.byref(pairs))
        return code, pairs.value

    def check_status(self):
        code, pairs = self.status()
        L.check(code, "device status")
        return pairs

    def profile(self, enable: bool = True):
        L.check(self._lib.pgs_profile(self._ctx, int(bool(enable))), "pgs_profile")

    def stage_times(self) -> dict:
        """{stage: (total ms, count)} since the last read; synchronises."""
        ms = np.zeros(len(L.PGS_STAGES), np.float64)
        cnt = np.zeros(len(L.PGS_STAGES), np.int64)
        L.check(self._lib.pgs_stage_times(self._ctx, ms.ctypes.data_as(C.c_void_p),
                                          cnt.ctypes.data_as(C.c_void_p)), "pgs_stage_times")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(L.PGS_STAGES)}

    def set_replay_cache(self, k_max: int):
        """The paper's per-pixel replay cache (k_max entries per pixel) instead of the recompute
        backward from the next render on; 0 turns it off."""
        L.check(self._lib.pgs_set_replay_cache(self._ctx, int(k_max)), "pgs_set_replay_cache")

    def set_variant(self, pixels_per_thread: int, depth: int):
        L.check(self._lib.pgs_set_variant(self._ctx, int(pixels_per_thread), int(depth)), "pgs_set_variant")

    def time_variants(self, dL_dimage: torch.Tensor, reps: int = 3) -> dict:
        """{(pixels per thread, depth): ms} of forward + backward compositing on the last render."""
        ms = np.zeros(len(L.VARIANTS), np.float32)
        scratch = torch.empty_like(dL_dimage)
        L.check(self._lib.pgs_time_variants(self._ctx, C.c_void_p(scratch.data_ptr()),
                                            C.c_void_p(dL_dimage.data_ptr()), int(reps),
                                            ms.ctypes.data_as(C.c_void_p)), "pgs_time_variants")
        return {v: float(t) for v, t in zip(L.VARIANTS, ms) if t >= 0}  # -1: not for this tile edge

    def set_variants(self, fwd: tuple, bwd: tuple):
        """Compositing variants (pixels per thread, depth) of the forward and of the backward."""
        L.check(self._lib.pgs_set_variants(self._ctx, int(fwd[0]), int(fwd[1]), int(bwd[0]), int(bwd[1])),
                "pgs_set_variants")

    def time_variants_split(self, dL_dimage: torch.Tensor, reps: int = 3) -> tuple:
        """({variant: forward ms}, {variant: backward ms}) of compositing on the last render."""
        mf = np.zeros(len(L.VARIANTS), np.float32)
        mb = np.zeros(len(L.VARIANTS), np.float32)
        scratch = torch.empty_like(dL_dimage)
        L.check(self._lib.pgs_time_variants_split(self._ctx, C.c_void_p(scratch.data_ptr()),
                                                  C.c_void_p(dL_dimage.data_ptr()), int(reps),
                                                  mf.ctypes.data_as(C.c_void_p), mb.ctypes.data_as(C.c_void_p)),
                "pgs_time_variants_split")
        keep = [i for i, t in enumerate(mf) if t >= 0]
        return ({L.VARIANTS[i]: float(mf[i]) for i in keep}, {L.VARIANTS[i]: float(mb[i]) for i in keep})

    def trace_pixels(self, pixels, max_entries: int) -> dict:
        """Decision trace of the last render at pixels [m][2] (x, y): per evaluated entry o G
        (og [m][max_entries]) and the decision code (code [m][max_entries]: 0 skipped, 1
        composited, 2 composited clamped, 3 stop), per pixel count, T_final, last, ncomp
        (numpy arrays; synchronises)."""
        host = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
        m, E = host.shape[0], int(max_entries)
        dev = self.device
        ptr = lambda t: C.c_void_p(t.data_ptr())
        with torch.cuda.stream(self.stream):
            pix = torch.as_tensor(host, device=dev)
            og = torch.zeros((m, max(E, 1)), dtype=torch.float32, device=dev)
            code = torch.full((m, max(E, 1)), 255, dtype=torch.uint8, device=dev)
            count = torch.zeros(m, dtype=torch.int32, device=dev)
            T = torch.zeros(m, dtype=torch.float32, device=dev)
            last = torch.zeros(m, dtype=torch.int32, device=dev)
            ncomp = torch.zeros(m, dtype=torch.int32, device=dev)
            L.check(self._lib.pgs_trace_pixels(self._ctx, ptr(pix), m, E, ptr(og), ptr(code), ptr(count), ptr(T),
                                               ptr(last), ptr(ncomp)), "pgs_trace_pixels")
        self.stream.synchronize()
        return dict(og=og[:, :E].cpu().numpy(), code=code[:, :E].cpu().numpy(), count=count.cpu().numpy(),
                    T=T.cpu().numpy(), last=last.cpu().numpy().astype(np.uint32),
                    ncomp=ncomp.cpu().numpy().astype(np.uint32))

    def selftest_timeout(self) -> int:
        """Failure-detection self-test of the sort's bounded waits (about a second); returns the
        status code it reads (PGS_ERR_TIMEOUT when the detection works)."""
        return int(self._lib.pgs_selftest_timeout(self._ctx))

    def launch_count(self) -> int:
        return int(self._lib.pgs_launch_count(self._ctx))

    def read_buffer(self, which: int) -> np.ndarray:
        size = C.c_int64()
        L.check(self._lib.pgs_read_buffer(self._ctx, which, None, 0, C.byref(size)), "pgs_read_buffer")
        dtype = {L.PGS_BUF_KEYS: np.uint64, L.PGS_BUF_T_FINAL: np.float32,
                 L.PGS_BUF_GRAD2D: np.float32}.get(which, np.uint32)
        out = np.zeros(size.value // np.dtype(dtype).itemsize, dtype)
        L.check(self._lib.pgs_read_buffer(self._ctx, which, out.ctypes.data_as(C.c_void_p),
                                          size.value, C.byref(size)), "pgs_read_buffer")
        return out


class Trainer:
    """Plain training iteration on one view: render -> L1 -> backward -> Adam (Sec. IV, 500
    iterations, one view per iteration)."""

    def __init__(self, params: GaussianBuffer, rasterizer: Rasterizer | None = None,
                 adam: AdamConfig | None = None, fused: bool = True, dssim: float = 0.0):
        """dssim: weight lambda of the D-SSIM term ((1 - lambda) L1 + lambda D-SSIM); 0 = L1."""
        self.params = params
        self.dssim = float(dssim)
        self.r = rasterizer or Rasterizer(adam=adam)
        self.fused = fused
        self.grads = None if fused else params.zeros_like()
        self.m = params.zeros_like()
        self.v = params.zeros_like()
        self.t = 0
        self.image = None
        self.dl = None
        self.loss = torch.zeros(2, dtype=torch.float32, device=params.data.device)

    def step(self, cam, target: torch.Tensor) -> torch.Tensor:
        shape = (3, cam.height, cam.width)
        if self.image is None or tuple(self.image.shape) != shape:
            self.image = torch.empty(shape, dtype=torch.float32, device=self.params.data.device)
            self.dl = torch.empty_like(self.image)
        if self.dssim > 0.0:
            self.r.render(self.params, cam, self.image)
            self.r.loss_dssim(self.image, target, self.dssim, self.dl, self.loss)
        else:  # the L1 loss and its gradient come out of the compositing forward
            self.r.render_l1(self.params, cam, target, self.image, self.dl, self.loss)
        self.t += 1
        if self.fused:
            self.r.backward_step(self.dl, self.params, self.m, self.v, self.t)
        else:
            self.r.backward(self.dl, self.grads)
            self.r.step(self.params, self.grads, self.m, self.v, self.t)
        return self.loss


class ImageFeed:
    """Host images (pinned) fed to training steps through `depth` device buffers that a copy
    stream of their own fills ahead of use, so the host-to-device copy of the next view overlaps
    the current step on the copy engine.  put(k, host) queues image k into slot k % depth (after
    the step that last used the slot); take(k, stream) orders `stream` after that copy and returns
    the device image; release(k, stream) marks the slot free once `stream`'s queued work is done."""

    def __init__(self, shape, device="cuda", depth: int = 2):
        self.bufs = [torch.empty(shape, dtype=torch.float32, device=device) for _ in range(depth)]
        self.copy_stream = torch.cuda.Stream(torch.device(device))
        self.ready = [torch.cuda.Event() for _ in range(depth)]
        self.free = [torch.cuda.Event() for _ in range(depth)]

    def put(self, k: int, host: torch.Tensor):
        s = k % len(self.bufs)
        self.copy_stream.wait_event(self.free[s])
        with torch.cuda.stream(self.copy_stream):
            self.bufs[s].copy_(host, non_blocking=True)
        self.ready[s].record(self.copy_stream)

    def take(self, k: int, stream: torch.cuda.Stream) -> torch.Tensor:
        s = k % len(self.bufs)
        stream.wait_event(self.ready[s])
        return self.bufs[s]

    def release(self, k: int, stream: torch.cuda.Stream):
        self.free[k % len(self.bufs)].record(stream)
