"""Initialization (operator I of Sec. III-B) and its learned stand-in, on the GPU.

Initializer.paper_init: kNN -> Eq. 5 normal (16 neighbours) and Eq. 6 tangential scale
(3 neighbours) -> thin disc Gaussians (the paper's initializer, also the learned path's fallback).
LearnedInit: a 16-64-64-8 GELU MLP (BF16 weights and activations, FP32 accumulation, FP32 master
weights with Adam) mapping 32-neighbour features to log-scales, rotation and opacity logit, each
expressed as a correction of the paper's initializer of the same point (log-scale and logit
offsets, rotation composed after the seeded one), so the network learns what training changes in
the seeding; trained on converged Gaussians produced by the plain method.
All arithmetic runs in libpocketgs kernels; this module marshals tensors.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .rasterizer import GaussianBuffer

R_NORMAL = 0.1  # normal-to-tangential scale ratio of the disc seeding (the paper leaves it open)


def _p(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


@dataclass
class PointInit:
    paper: GaussianBuffer         # the paper's initializer (Eq. 5 / Eq. 6)
    features: torch.Tensor        # [n][16] fp32
    features_bf16: torch.Tensor   # [n][16] bf16
    frame_q: torch.Tensor         # [4][n] eigenframe quaternions
    nb: torch.Tensor              # [n][32] neighbour indices


class Initializer:
    def __init__(self, stream: torch.cuda.Stream | None = None, device="cuda"):
        self._lib = L.lib()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._c = C.c_void_p()
        L.check(self._lib.pgs_init_create(C.byref(self._c), C.c_void_p(self.stream.cuda_stream)),
                "pgs_init_create")

    def close(self):
        if getattr(self, "_c", None) is not None and self._c.value:
            self._lib.pgs_init_destroy(self._c)
            self._c = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def knn(self, points: torch.Tensor, k: int) -> torch.Tensor:
        points = points.contiguous().float()
        n = points.shape[1]
        nb = torch.empty((n, k), dtype=torch.int32, device=self.device)
        L.check(self._lib.pgs_knn(self._c, _p(points), n, int(k), _p(nb)), "pgs_knn")
        return nb

    def paper_init(self, points: torch.Tensor, sh_degree: int = 3, r_normal: float = R_NORMAL) -> PointInit:
        points = points.contiguous().float()
        n = points.shape[1]
        nb = self.knn(points, 32)
        init = GaussianBuffer(n, sh_degree, self.device)
        feats = torch.empty((n, 16), dtype=torch.float32, device=self.device)
        fb = torch.empty((n, 16), dtype=torch.bfloat16, device=self.device)
        fq = torch.empty((4, n), dtype=torch.float32, device=self.device)
        L.check(self._lib.pgs_features_init(self._c, _p(points), n, _p(nb), float(r_normal), _p(feats),
                                            _p(fb), _p(fq), C.byref(init.struct())), "pgs_features_init")
        return PointInit(init, feats, fb, fq, nb)

    def make_targets(self, pi: PointInit, converged: GaussianBuffer) -> torch.Tensor:
        t = torch.empty((converged.n, 8), dtype=torch.float32, device=self.device)
        L.check(self._lib.pgs_make_targets(self._c, C.byref(pi.paper.struct()), C.byref(converged.struct()),
                                           _p(t)), "pgs_make_targets")
        return t

    def apply(self, pi: PointInit, y: torch.Tensor) -> tuple:
        """Learned initial parameters from MLP outputs y [n][8]; (GaussianBuffer, fallbacks)."""
        out = pi.paper.clone()
        fb = torch.zeros(1, dtype=torch.int32, device=self.device)
        L.check(self._lib.pgs_apply_mlp(self._c, _p(y.contiguous()), C.byref(pi.paper.struct()),
                                        C.byref(out.struct()), _p(fb)), "pgs_apply_mlp")
        return out, int(fb.item())


class MLP:
    """16-64-64-8 GELU MLP: FP32 master parameters [W1|b1|W2|b2|W3|b3] with Adam moments and BF16
    copies of the weight matrices used by the kernels."""

    SHAPES = [(64, 16), (64,), (64, 64), (64,), (8, 64), (8,)]

    def __init__(self, init: Initializer, seed: int = 0):
        self.init = init
        lib = init._lib
        self.count = int(lib.pgs_mlp_param_count())
        dev = init.device
        g = torch.Generator(device="cpu").manual_seed(seed)
        parts = []
        for shape in self.SHAPES:
            if len(shape) == 2:  # uniform +-sqrt(6 / (fan_in + fan_out)) (Glorot)
                lim = math.sqrt(6.0 / (shape[0] + shape[1]))
                parts.append((torch.rand(shape, generator=g) * 2 - 1) * lim)
            else:
                parts.append(torch.zeros(shape))
        self.master = torch.cat([p.reshape(-1) for p in parts]).float().to(dev).contiguous()
        assert self.master.numel() == self.count
        self.grad = torch.zeros_like(self.master)
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.W1 = torch.empty((64, 16), dtype=torch.bfloat16, device=dev)
        self.W2 = torch.empty((64, 64), dtype=torch.bfloat16, device=dev)
        self.W3 = torch.empty((8, 64), dtype=torch.bfloat16, device=dev)
        self.t = 0
        self.loss_sum = torch.zeros(1, dtype=torch.float64, device=dev)
        self._s = L.PgsMlp(self.master.data_ptr(), self.W1.data_ptr(), self.W2.data_ptr(), self.W3.data_ptr())
        L.check(lib.pgs_mlp_pack(init._c, C.byref(self._s)), "pgs_mlp_pack")

    def weights(self):
        """Master parameters as (W1, b1, W2, b2, W3, b3) numpy arrays."""
        out, off = [], 0
        flat = self.master.detach().cpu().numpy()
        for shape in self.SHAPES:
            k = int(np.prod(shape))
            out.append(flat[off:off + k].reshape(shape))
            off += k
        return out

    def set_weights(self, ws):
        flat = np.concatenate([np.asarray(w, np.float32).reshape(-1) for w in ws])
        self.master.copy_(torch.from_numpy(flat))
        L.check(self.init._lib.pgs_mlp_pack(self.init._c, C.byref(self._s)), "pgs_mlp_pack")

    def forward(self, x_bf16: torch.Tensor) -> torch.Tensor:
        n = x_bf16.shape[0]
        out = torch.empty((n, 8), dtype=torch.float32, device=x_bf16.device)
        L.check(self.init._lib.pgs_mlp_forward(self.init._c, C.byref(self._s), _p(x_bf16.contiguous()), n,
                                               _p(out)), "pgs_mlp_forward")
        return out

    def accumulate_grad(self, x_bf16: torch.Tensor, targets: torch.Tensor):
        L.check(self.init._lib.pgs_mlp_grad(self.init._c, C.byref(self._s), _p(x_bf16.contiguous()),
                                            _p(targets.contiguous()), x_bf16.shape[0], _p(self.grad),
                                            _p(self.loss_sum)), "pgs_mlp_grad")

    def adam(self, lr: float):
        self.t += 1
        L.check(self.init._lib.pgs_mlp_adam(self.init._c, C.byref(self._s), _p(self.grad), _p(self.m),
                                            _p(self.v), float(lr), self.t), "pgs_mlp_adam")


class LearnedInit:
    """fit(): MLP regression from features to converged parameters; infer(): initial Gaussians."""

    def __init__(self, initializer: Initializer | None = None, seed: int = 0):
        self.init = initializer or Initializer()
        self.mlp = MLP(self.init, seed)
        self.history = []

    def fit(self, features: list, targets: list, steps: int = 400, batch: int = 65536,
            lr: float = 3e-3, seed: int = 0) -> list:
        """features: list of [n_i][16] bf16; targets: list of [n_i][8]; minibatch Adam steps."""
        X = torch.cat(features).contiguous()
        T = torch.cat(targets).contiguous()
        n = X.shape[0]
        g = torch.Generator(device=X.device).manual_seed(seed)
        for s in range(steps):
            idx = torch.randint(0, n, (min(batch, n),), device=X.device, generator=g)
            self.mlp.loss_sum.zero_()
            self.mlp.accumulate_grad(X[idx], T[idx])
            # cosine learning-rate decay
            self.mlp.adam(lr * 0.5 * (1 + math.cos(math.pi * s / steps)))
            if s % 50 == 0 or s == steps - 1:
                self.history.append((s, float(self.mlp.loss_sum.item()) / min(batch, n)))
        return self.history

    def infer(self, pi: PointInit) -> tuple:
        y = self.mlp.forward(pi.features_bf16)
        return self.init.apply(pi, y)
