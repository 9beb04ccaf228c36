"""Optimiser ablations as convergence curves (Sec. 5, optimiser ablation, and
App. A): paths per pixel for the colour estimate, the split of a fixed path
budget between colour and derivative samples, the pixel-batch size at equal
time, multiple importance sampling, and the number of bounces fitted to a
10-bounce target.

Each setting optimises the same scene from the same start for the same
GPU time budget on the batch-graph step (one scene, stochastic pixel
batches, the L1 loss of Sec. 3.2).  At checkpoints it records the iteration,
the elapsed optimisation time (CUDA-synchronised, reads excluded), the
parameter error (relative L2 over the scored parameters) and the full-image
L1 loss of the current parameters against the target, estimated with a fixed
sample set so that every setting is scored on the same random numbers.
"""
from __future__ import annotations

import time
from dataclasses import replace

import torch

from . import convergence, metrics
from .tracer import AdamOptions, TraceOptions, Tracer

# depth = vertices with light gathering: 1 = direct light only, 2 = one
# indirect bounce (the paper's "bounces")
BASE = TraceOptions(spp_r=128, spp_d=1, max_depth=2, loss="l1", pixel_batch=256)

SWEEPS = {
    # Fig. plot_srays: colour paths per pixel (1 fails)
    "paths": [("spp_r=%d" % s, replace(BASE, spp_r=s)) for s in (1, 8, 128, 1024)],
    # Fig. plot_samples: 128 paths split between colour and derivatives
    "split": [("spp_r=%d,spp_d=%d" % (r, d), replace(BASE, spp_r=r, spp_d=d))
              for r, d in ((127, 1), (112, 16), (64, 64), (16, 112))],
    # Fig. plot_batch: pixels per step at equal time
    "batch": [("B=%d" % b, replace(BASE, pixel_batch=b)) for b in (8, 64, 512, 4096)],
    # Fig. plot_mis: light sampling with and without MIS, and BSDF sampling only
    "mis": [("nee+mis", BASE), ("nee,no mis", replace(BASE, mis=False)),
            ("bsdf only", replace(BASE, nee=False))],
    # Fig. plot_bounces: 1, 2, 3 bounces against a 10-bounce target
    "bounces": [("depth=%d" % d, replace(BASE, max_depth=d)) for d in (1, 2, 3)],
}
TARGET_DEPTH = {"bounces": 10}


def _eval_loss(ev: Tracer, target, params, opts: TraceOptions, iteration: int) -> float:
    """Image L1 loss (1/N) sum |I - I_C| over all pixel-channels, I rendered
    with residual sample set 0 at a fixed iteration."""
    ev.set_params(params)
    img = ev.render(opts, view=-1, set_id=0, spp=opts.spp_r, iteration=iteration)
    return float(torch.mean(torch.abs(img - target)))


def curve(scene, opts: TraceOptions, adam: AdamOptions, seconds: float, target_depth: int, points: int = 24,
          eval_spp: int = 64, target_spp: int = 1024, seed: int = 7, max_iters: int = 200_000):
    """Optimises `scene` from zero diffuse albedo and emission with `opts`
    for `seconds` of GPU time; returns [(iteration, seconds, parameter error,
    image L1 loss)] at about `points` checkpoints, the first at iteration 0."""
    tgt = TraceOptions(max_depth=target_depth)
    ss, masks = convergence.prepare([scene], tgt, target_spp=target_spp, init=0.0, seed=seed)
    ss.configure(integrator="wavefront")
    ev = Tracer(scene, seed=seed + 1)
    ev.set_params(scene.gt_params)
    target = ev.render(tgt, view=-1, set_id=2, spp=target_spp)
    eval_opts = TraceOptions(spp_r=eval_spp, spp_d=1, max_depth=target_depth, loss="l1")
    eval_it = 1 << 24  # the same sample set for every setting and checkpoint
    ss.make_batch()
    p = ss.batch_params(0)
    out = [(0, 0.0, metrics.param_error(p, scene.gt_params, masks[0]),
            _eval_loss(ev, target, p, eval_opts, eval_it))]
    # step cost from a short run (not part of the curve), then a fresh batch
    # from the same start (the scene's own parameters are still the start)
    probe = 20
    torch.cuda.synchronize(ss.device)
    t0 = time.perf_counter()
    for k in range(probe):
        ss.batch_step(opts, adam, want_losses=False)
    torch.cuda.synchronize(ss.device)
    per_step = (time.perf_counter() - t0) / probe
    ss.make_batch()
    chunk = max(1, int(seconds / points / max(per_step, 1e-6)))
    it, elapsed = 0, 0.0
    while elapsed < seconds and it < max_iters:
        torch.cuda.synchronize(ss.device)
        t0 = time.perf_counter()
        for _ in range(chunk):
            ss.batch_step(opts, adam, want_losses=False)
        torch.cuda.synchronize(ss.device)
        elapsed += time.perf_counter() - t0
        it += chunk
        p = ss.batch_params(0)
        out.append((it, elapsed, metrics.param_error(p, scene.gt_params, masks[0]),
                    _eval_loss(ev, target, p, eval_opts, eval_it)))
    ev.close()
    ss.close()
    return out


def sweep(kind: str, scene, adam: AdamOptions, seconds: float, points: int = 24, seed: int = 7):
    """Curves of every setting of one ablation on the same scene and budget."""
    depth = TARGET_DEPTH.get(kind)
    res = {}
    for name, opts in SWEEPS[kind]:
        res[name] = curve(scene, opts, adam, seconds, depth or opts.max_depth, points=points, seed=seed)
    return res
