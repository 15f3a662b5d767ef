"""Training and evaluation drivers on synthetic surface scenes: the plain method (paper
initializer + one view per iteration), the learned initializer fitted on converged Gaussians of
plain runs, and held-out-view PSNR at fixed iteration budgets."""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import synthetic as S
from .autotune import tune_batch_tile, tune_rasterizer_tile
from .initializer import Initializer, LearnedInit, PointInit
from .rasterizer import DEFAULT_LR, AdamConfig, GaussianBuffer, Rasterizer, Trainer


@dataclass
class SceneData:
    scene: S.SurfaceScene
    points: torch.Tensor              # [3][n] trainable start positions
    targets: dict                     # view index -> [3][H][W] ground-truth render
    pi: PointInit | None = None


def make_scene(seed: int, n: int, width: int, height: int, focal: float, n_cameras: int = 64,
               sh_degree: int = 3) -> SceneData:
    sc = S.surface_scene(seed, n, sh_degree, width, height, focal, n_cameras=n_cameras)
    rast = Rasterizer()
    gt = GaussianBuffer.from_arrays(sc.gt)
    targets = {v: rast.render(gt, sc.cameras[v]).clone() for v in range(len(sc.cameras))}
    torch.cuda.synchronize()
    return SceneData(sc, torch.from_numpy(np.ascontiguousarray(sc.init.means)).cuda(), targets)


def with_colour(params: GaussianBuffer) -> GaussianBuffer:
    """Initial colour: grey (all SH coefficients 0)."""
    params.sh.zero_()
    return params


def psnr(img: torch.Tensor, ref: torch.Tensor) -> float:
    mse = torch.mean((img.clamp(0, 1) - ref.clamp(0, 1)) ** 2).item()
    return float("inf") if mse == 0 else -10.0 * math.log10(mse)


def eval_psnr(rast: Rasterizer, params: GaussianBuffer, sd: SceneData) -> float:
    vals = [psnr(rast.render(params, sd.scene.cameras[v]), sd.targets[v]) for v in sd.scene.test_views()]
    return float(np.mean(vals))


def pair_capacity(params: GaussianBuffer, sd: SceneData, views: int = 8, headroom: float = 2.0,
                  tile: int = 16) -> int:
    """A fixed pair capacity for training: the most pairs over the first training views of the
    starting parameters, times the headroom (the pairs grow as the Gaussians train)."""
    probe = Rasterizer(tile=tile)
    most = 0
    for v in sd.scene.train_views()[:views]:
        probe.render(params, sd.scene.cameras[v])
        most = max(most, probe.status()[1])
    probe.close()
    return int(most * headroom) + 4096


def tuned_rasterizer(params: GaussianBuffer, sd: SceneData) -> Rasterizer:
    """A rasterizer for training `params` on `sd`: tile edge and compositing variant chosen by the
    autotuner on the first training view, fixed pair capacity for that edge."""
    v = sd.scene.train_views()[0]
    probe = Rasterizer()
    img = probe.render(params, sd.scene.cameras[v])
    dl, _ = probe.loss_l1(img, sd.targets[v])
    tuned, tile, variant = tune_rasterizer_tile(params, sd.scene.cameras[v], dl.clone())
    tuned.close()
    probe.close()
    rast = Rasterizer(pair_capacity=pair_capacity(params, sd, tile=tile), tile=tile)
    variant.apply(rast)
    return rast


def train_plain(params: GaussianBuffer, sd: SceneData, iters: int, checkpoints=(), seed: int = 0,
                rast: Rasterizer | None = None):
    """Plain training: Adam, L1, one view per iteration from a seeded permutation of the training
    views, reshuffled every epoch.  Returns ({iteration: held-out PSNR}, GPU seconds of training).
    The rasterizer has a fixed pair capacity, so no iteration waits on the host (an overflow is
    reported at the end), and the autotuner's compositing variant."""
    rast = rast or tuned_rasterizer(params, sd)
    tr = Trainer(params, rast)
    views = sd.scene.train_views()
    rng = np.random.default_rng(seed)
    order = []
    out = {}
    gpu_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eval_rast = Rasterizer()
    e0.record()
    for it in range(1, iters + 1):
        if not order:
            order = list(rng.permutation(views))
        v = order.pop()
        tr.step(sd.scene.cameras[v], sd.targets[v])
        if it in checkpoints:
            e1.record()
            torch.cuda.synchronize()
            gpu_ms += e0.elapsed_time(e1)
            out[it] = eval_psnr(eval_rast, params, sd)
            e0.record()
    e1.record()
    torch.cuda.synchronize()
    gpu_ms += e0.elapsed_time(e1)
    code, _ = rast.status()
    if code != 0:
        raise RuntimeError(f"training status {code}")
    return out, gpu_ms / 1000.0


@dataclass
class InitComparison:
    budgets: tuple
    paper: list = field(default_factory=list)    # per eval scene {budget: PSNR}
    learned: list = field(default_factory=list)
    fit_history: list = field(default_factory=list)
    fallbacks: int = 0
    seconds: dict = field(default_factory=dict)
    learned_init: LearnedInit | None = None

    def mean(self, which: str) -> dict:
        rows = getattr(self, which)
        return {b: float(np.mean([r[b] for r in rows])) for b in self.budgets}


def compare_initializers(train_seeds, eval_seeds, n: int, width: int, height: int, focal: float,
                         budgets=(100, 250, 500), converge_iters: int = 500, fit_steps: int = 600,
                         n_cameras: int = 64, sh_degree: int = 3, keep_learned: bool = False) -> InitComparison:
    """Fit the learned initializer on converged Gaussians of plain runs on the training scenes,
    then compare it with the paper's initializer on the held-out views of the evaluation scenes."""
    t0 = time.time()
    init = Initializer()
    feats, targs = [], []
    for seed in train_seeds:
        sd = make_scene(seed, n, width, height, focal, n_cameras, sh_degree)
        pi = init.paper_init(sd.points, sh_degree)
        params = with_colour(pi.paper.clone())
        train_plain(params, sd, converge_iters, seed=seed)
        feats.append(pi.features_bf16)
        targs.append(init.make_targets(pi, params))
    t1 = time.time()
    li = LearnedInit(init, seed=1)
    li.fit(feats, targs, steps=fit_steps)
    res = InitComparison(tuple(budgets), fit_history=list(li.history))
    t2 = time.time()
    for seed in eval_seeds:
        sd = make_scene(seed, n, width, height, focal, n_cameras, sh_degree)
        pi = init.paper_init(sd.points, sh_degree)
        paper = with_colour(pi.paper.clone())
        p, _ = train_plain(paper, sd, max(budgets), checkpoints=budgets, seed=seed)
        learned, fb = li.infer(pi)
        learned = with_colour(learned)
        q, _ = train_plain(learned, sd, max(budgets), checkpoints=budgets, seed=seed)
        res.paper.append(p)
        res.learned.append(q)
        res.fallbacks += fb
    res.seconds = {"converge_runs": t1 - t0, "fit": t2 - t1, "eval": time.time() - t2}
    if keep_learned:
        res.learned_init = li
    return res


def batched_adam(views_per_step: int) -> AdamConfig:
    """Adam settings for a step that averages the gradients of `views_per_step` views of a scene:
    the square-root learning-rate rule and momentum decay per view (beta ** views_per_step) of
    the batch-size scaling study for Gaussian splatting by Zhao et al. (2024), so that one step
    stands in for that many single-view iterations."""
    return AdamConfig(lr=tuple(l * math.sqrt(views_per_step) for l in DEFAULT_LR),
                      b1=0.9 ** views_per_step, b2=0.999 ** views_per_step)


def time_to_target(seeds, n: int, width: int, height: int, focal: float, plain_iters: int = 500,
                   views_per_step: int = 4, learned: LearnedInit | None = None, check_every: int = 10,
                   max_steps: int = 500, n_cameras: int = 64, sh_degree: int = 3,
                   adam=None) -> dict:
    """GPU seconds for the plain form (paper initializer, one view per iteration, each scene on its
    own for plain_iters iterations) against the batched form (every scene in one captured batch,
    views_per_step views of each scene per step, learned initializer when given) to reach, for
    every scene, the plain form's held-out PSNR.  adam: the batched form's Adam settings (default:
    the plain form's).  Evaluation renders are not counted."""
    init = learned.init if learned is not None else Initializer()
    scenes = [make_scene(s, n, width, height, focal, n_cameras, sh_degree) for s in seeds]
    plain_psnr, plain_s = [], 0.0
    for k, sd in enumerate(scenes):
        sd.pi = init.paper_init(sd.points, sh_degree)
        params = with_colour(sd.pi.paper.clone())
        out, secs = train_plain(params, sd, plain_iters, checkpoints=(plain_iters,), seed=seeds[k])
        plain_psnr.append(out[plain_iters])
        plain_s += secs
    starts = []
    fallbacks = 0
    for sd in scenes:
        if learned is not None:
            p, fb = learned.infer(sd.pi)
            fallbacks += fb
        else:
            p = sd.pi.paper.clone()
        starts.append(with_colour(p))
    rng = np.random.default_rng(0)
    orders = [[] for _ in scenes]

    def next_views():
        out = []
        for k, sd in enumerate(scenes):
            for _ in range(views_per_step):
                if not orders[k]:
                    orders[k] = list(rng.permutation(sd.scene.train_views()))
                v = orders[k].pop()
                out.append((k, sd.scene.cameras[v], sd.targets[v]))
        return out

    first = next_views()
    bt, _, _ = tune_batch_tile(starts, first, adam=adam, pair_headroom=2.0)
    bt.capture()
    eval_rast = Rasterizer()
    reached = [None] * len(scenes)
    batched_s = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step, issued = 0, 0
    while step < max_steps and any(r is None for r in reached):
        e0.record(bt.stream)
        for _ in range(check_every):
            if issued > 0:
                bt.set_views([(c, t) for _, c, t in next_views()])
            bt.step()
            issued += 1
        e1.record(bt.stream)
        torch.cuda.synchronize()
        batched_s += e0.elapsed_time(e1) / 1000.0
        step = bt.check()  # completed steps; a pair overflow grows the capacity
        for k, sd in enumerate(scenes):
            if reached[k] is None and eval_psnr(eval_rast, starts[k], sd) >= plain_psnr[k]:
                reached[k] = (step, batched_s)
    done = all(r is not None for r in reached)
    return {"plain_psnr": plain_psnr, "plain_gpu_s": plain_s, "batched_gpu_s": batched_s,
            "steps": step, "issued": issued, "reached": reached, "all_reached": done, "fallbacks": fallbacks,
            "ratio": batched_s / plain_s if done else None}


def geometry_prior(sc: S.MVSScene, images: list, every: int = 4, planes: int = 64):
    """The geometry prior of Sec. III-A on a synthetic keyframe ring: single-reference MVS on every
    `every`-th keyframe (depth range from the sparse points, Eq. 4 reference), fused into one
    dense cloud [n][3].  images: CUDA [3][H][W] per keyframe."""
    from .mvs import MultiViewStereo
    cams = sc.cameras
    mv = MultiViewStereo(cams[0].width, cams[0].height, planes)
    sparse = torch.from_numpy(sc.sparse.astype(np.float32)).cuda()
    clouds = [mv.reconstruct(cams, images, t, sparse)[3] for t in range(0, len(cams), every)]
    mv.close()
    return torch.cat(clouds, 0)


def train_views_psnr(params: GaussianBuffer, cams: list, images: list, iters: int, seed: int = 0) -> float:
    """Plain training (Adam, L1, one view per iteration from a seeded permutation of the views
    i % 8 != 0), then the mean PSNR over the held-out views i % 8 == 0."""
    rast = Rasterizer()
    tr = Trainer(params, rast)
    views = [i for i in range(len(cams)) if i % 8 != 0]
    rng = np.random.default_rng(seed)
    order = []
    for _ in range(iters):
        if not order:
            order = list(rng.permutation(views))
        v = order.pop()
        tr.step(cams[v], images[v])
    code, _ = rast.status()
    if code != 0:
        raise RuntimeError(f"training status {code}")
    return float(np.mean([psnr(rast.render(params, cams[v]), images[v]) for v in range(0, len(cams), 8)]))


def prior_experiment(seed: int = 3, width: int = 320, height: int = 180, focal: float = 250.0, n_points: int = 60000,
                     iters: int = 300, sh_degree: int = 0) -> dict:
    """The G -> I -> T loop on a synthetic keyframe ring: the MVS cloud (subsampled to n_points)
    seeds the paper's initializer (Eq. 5-6) and trains for `iters` iterations; the same budget
    from as many points drawn uniformly in the cloud's bounding box is the comparison.  Returns
    the held-out PSNRs and the cloud size."""
    sc = S.mvs_scene(seed, width=width, height=height, focal=focal)
    images = [torch.from_numpy(im).cuda() for im in sc.images]
    cloud = geometry_prior(sc, images)
    rng = np.random.default_rng(seed)
    pick = torch.from_numpy(rng.choice(cloud.shape[0], size=min(n_points, cloud.shape[0]), replace=False)).cuda()
    pts = cloud[pick].t().contiguous()
    init = Initializer()
    out = {"cloud_points": int(cloud.shape[0])}
    lo, hi = pts.min(dim=1).values.cpu().numpy(), pts.max(dim=1).values.cpu().numpy()
    box = torch.from_numpy(rng.uniform(lo[:, None], hi[:, None], size=(3, pts.shape[1])).astype(np.float32)).cuda()
    for name, p in (("mvs_prior", pts), ("bounding_box", box)):
        params = with_colour(init.paper_init(p, sh_degree).paper)
        out[name] = train_views_psnr(params, sc.cameras, images, iters)
    init.close()
    return out


def learned_init_experiment(scenes: int = 32, held_out: int = 8, points: int = 200_000, width: int = 1280,
                            height: int = 720, focal: float = 1000.0, fit_steps: int = 1000,
                            views_per_step=(1, 2), check_every: int = 5, with_paper_batched: bool = True) -> dict:
    """Learned-initializer experiment on surface scenes of `points` points: the network is fitted on
    the converged Gaussians of plain 500-iteration runs of the training scenes (seeds 1000..) and
    compared with the paper's initializer on the held-out views of the held-out scenes (seeds 2000..)
    at 100/250/500 iterations; then the batched form is timed to the plain form's 500-iteration
    PSNR on the held-out scenes, with the learned initializer (and, for reference, the paper's)."""
    t0 = time.time()
    train = list(range(1000, 1000 + scenes - held_out))
    held = list(range(2000, 2000 + held_out))
    res = compare_initializers(train, held, points, width, height, focal, fit_steps=fit_steps, keep_learned=True)
    out = {"experiment": "learned initializer", "train_seeds": [train[0], train[-1]],
           "held_out_seeds": [held[0], held[-1]], "points": points, "resolution": f"{width}x{height}",
           "focal": focal, "psnr_paper_init": res.mean("paper"), "psnr_learned_init": res.mean("learned"),
           "fit_steps": fit_steps, "fit_loss": res.fit_history[-1][1], "fallbacks": res.fallbacks,
           "time_to_plain_psnr": []}
    for vps in views_per_step:
        for learned in ((res.learned_init, None) if with_paper_batched else (res.learned_init,)):
            tt = time_to_target(held, points, width, height, focal, views_per_step=vps, learned=learned,
                                adam=batched_adam(vps) if vps > 1 else None, check_every=check_every)
            out["time_to_plain_psnr"].append(
                {"views_per_step": vps, "learned": learned is not None,
                 **{k: tt[k] for k in ("plain_gpu_s", "batched_gpu_s", "steps", "all_reached", "ratio")}})
    out["wall_s"] = time.time() - t0
    return out


def main(argv=None):
    """Runs learned_init_experiment (default: 32 surface scenes of 200k points, 1280x720, fx = 1000,
    8 held out) and prints one JSON line."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=32)
    ap.add_argument("--held-out", type=int, default=8)
    ap.add_argument("--points", type=int, default=200_000)
    ap.add_argument("--width", type=int, default=1280)
    ap.add_argument("--height", type=int, default=720)
    ap.add_argument("--focal", type=float, default=1000.0)
    ap.add_argument("--fit-steps", type=int, default=1000)
    ap.add_argument("--views-per-step", type=int, nargs="+", default=[1, 2])
    ap.add_argument("--check-every", type=int, default=5, help="batched steps between PSNR checks")
    args = ap.parse_args(argv)
    print(json.dumps(learned_init_experiment(args.scenes, args.held_out, args.points, args.width, args.height,
                                             args.focal, args.fit_steps, tuple(args.views_per_step),
                                             args.check_every)))


if __name__ == "__main__":
    main()
