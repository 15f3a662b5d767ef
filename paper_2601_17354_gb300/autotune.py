"""Autotuner of the rasterizer: picks the screen tile edge (8, 16, 32 pixels), the pixels-per-thread
strip (1, 2, 4) and the number of list entries staged in shared memory per batch (64, 128, 256) by
timing them on the caller's own workload (every variant's forward + backward compositing, and per
tile edge the render part of the step), and caches the choices in a JSON file keyed by GPU and
workload class (batch shape, resolution class, Gaussian count), so later runs skip the timing."""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import torch

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pocketgs_gb300", "autotune.json")


def _cache_path(path: str | None) -> str:
    return path or os.environ.get("PGS_AUTOTUNE_CACHE", DEFAULT_CACHE)


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, key: str, entry: dict) -> None:
    data = _load(path)
    data[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def resolution_class(width: int, height: int) -> str:
    return f"{width}x{height}"


def workload_key(kind: str, resolutions, n_gaussians: int, sh_degree: int) -> str:
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    res = "+".join(sorted(set(resolutions)))
    return f"{gpu}|{kind}|{res}|N~2^{round(math.log2(max(n_gaussians, 1)))}|sh{sh_degree}"


def pick(timings: dict) -> tuple:
    return min(timings, key=lambda v: timings[v])


@dataclass(frozen=True)
class Variants:
    """The compositing variants (pixels per thread, staging depth) of the forward and the backward
    of single-view training, each the fastest for its own kernel."""
    fwd: tuple
    bwd: tuple
    ms: float = 0.0  # forward + backward compositing time at this choice

    def apply(self, rast):
        rast.set_variants(self.fwd, self.bwd)


def tune_rasterizer(rast, params, cam, dL_dimage: torch.Tensor, cache: str | None = None,
                    reps: int = 3, force: bool = False) -> Variants:
    """Choose and set the forward and backward variants for single-view training of `params`
    through `cam` (each kernel timed on its own)."""
    path = _cache_path(cache)
    key = workload_key(f"single-T{rast.tile}", [resolution_class(cam.width, cam.height)], params.n,
                       params.sh_degree)
    entry = None if force else _load(path).get(key)
    if entry is None or "fwd" not in entry:
        rast.render(params, cam)
        tf, tb = rast.time_variants_split(dL_dimage, reps)
        f, b = pick(tf), pick(tb)
        entry = {"fwd": list(f), "bwd": list(b), "ms": tf[f] + tb[b],
                 "ms_fwd": {f"{p}x{d}": ms for (p, d), ms in tf.items()},
                 "ms_bwd": {f"{p}x{d}": ms for (p, d), ms in tb.items()}}
        _store(path, key, entry)
    v = Variants(tuple(entry["fwd"]), tuple(entry["bwd"]), float(entry["ms"]))
    v.apply(rast)
    return v


def tune_rasterizer_tile(params, cam, dL_dimage: torch.Tensor, adam=None, tiles=(8, 16, 32),
                         cache: str | None = None, reps: int = 3, force: bool = False):
    """The tile edge and compositing variants that minimise render + forward and backward
    compositing time for single-view training of `params` through `cam`, each timed on this
    workload (the candidates grow their pair buffers on demand).  Returns (rasterizer with that
    edge and those variants, tile, Variants)."""
    from .rasterizer import Rasterizer
    path = _cache_path(cache)
    key = workload_key("single-tile", [resolution_class(cam.width, cam.height)], params.n, params.sh_degree)
    entry = None if force else _load(path).get(key)

    def build(T):
        return Rasterizer(adam=adam, tile=T)

    if entry is not None and int(entry["tile"]) in tiles:
        rast = build(int(entry["tile"]))
        return rast, rast.tile, tune_rasterizer(rast, params, cam, dL_dimage, cache=cache, reps=reps)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, costs = None, {}
    for T in tiles:
        rast = build(T)
        variant = tune_rasterizer(rast, params, cam, dL_dimage, cache=cache, reps=reps, force=force)
        comp = variant.ms
        render = []
        for _ in range(reps + 1):
            ev0.record(rast.stream)
            rast.render(params, cam)
            ev1.record(rast.stream)
            ev1.synchronize()
            render.append(ev0.elapsed_time(ev1))
        costs[T] = min(render[1:]) + comp  # the render includes one forward composite
        if best is None or costs[T] < costs[best[0]]:
            if best is not None:
                best[1].close()
            best = (T, rast, variant)
        else:
            rast.close()
    _store(path, key, {"tile": best[0], "ms": {str(t): c for t, c in costs.items()}})
    return best[1], best[0], best[2]


def tune_batch(bt, cache: str | None = None, reps: int = 3, force: bool = False) -> tuple:
    """Choose and set the variant of a BatchTrainer's persistent compositing launches."""
    path = _cache_path(cache)
    res = [resolution_class(c.width, c.height) for _, c, _ in bt.views]
    n = sum(s.n for s in bt.scenes)
    key = workload_key(f"batch{len(bt.views)}-T{bt.tile}", res, n, bt.scenes[0].sh_degree)
    entry = None if force else _load(path).get(key)
    if entry is None:
        t = bt.time_variants(reps)
        best = pick(t)
        entry = {"pixels": best[0], "depth": best[1],
                 "ms": {f"{p}x{d}": ms for (p, d), ms in t.items()}}
        _store(path, key, entry)
    bt.set_variant(entry["pixels"], entry["depth"])
    return entry["pixels"], entry["depth"]


def tune_batch_tile(scenes: list, views: list, adam=None, tiles=(8, 16, 32), cache: str | None = None,
                    reps: int = 3, force: bool = False, pair_headroom: float = 1.0):
    """A BatchTrainer for (scenes, views) with the tile edge and compositing variant that minimise
    the render part of a step plus the forward + backward compositing, each timed on this workload
    (parameters are not changed).  pair_headroom > 1 grows the pair capacity over the measured
    count.  Returns (trainer, tile, (pixels_per_thread, depth))."""
    from .batch import BatchTrainer
    path = _cache_path(cache)
    res = [resolution_class(c.width, c.height) for _, c, _ in views]
    n = sum(s.n for s in scenes)
    key = workload_key(f"batch{len(views)}-tile", res, n, scenes[0].sh_degree)
    entry = None if force else _load(path).get(key)

    def build(T):
        bt = BatchTrainer(scenes, views, adam=adam, tile=T)
        if pair_headroom > 1.0:
            bt.reserve(int(pair_headroom * bt.status()[1]) + 4096)
        return bt

    if entry is not None and int(entry["tile"]) in tiles:
        bt = build(int(entry["tile"]))
        return bt, bt.tile, tune_batch(bt, cache=cache, reps=reps)
    best, costs = None, {}
    for T in tiles:
        bt = build(T)
        variant = tune_batch(bt, cache=cache, reps=reps, force=force)
        timed = _load(path).get(workload_key(f"batch{len(views)}-T{T}", res, n, scenes[0].sh_degree), {})
        comp = timed.get("ms", {}).get(f"{variant[0]}x{variant[1]}")
        if comp is None:
            comp = bt.time_variants(reps)[variant]
        costs[T] = bt.time_render(reps) + comp
        if best is None or costs[T] < costs[best[0]]:
            if best is not None:
                best[1].close()
            best = (T, bt, variant)
        else:
            bt.close()
    _store(path, key, {"tile": best[0], "ms": {str(t): c for t, c in costs.items()}})
    return best[1], best[0], best[2]
