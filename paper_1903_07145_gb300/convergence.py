"""Time to a parameter-error threshold for one scene or a batch.

The measured quantity is the wall time (and the number of iterations) until
a member's parameter error first falls to the threshold.  The unknowns are
the diffuse albedo and emission of every segment (the quantities the paper
evaluates, Table 1); specular albedo and roughness are held at their true
values through the free mask, because without a Fresnel term a rough GGX
lobe can stand in for a Lambertian one and a few views cannot tell them
apart.  Iterations run as batch-graph replays; the error is read every
`check_every` iterations (the reads are outside the timed iterations).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import metrics
from .batch import SceneSet
from .tracer import AdamOptions, TraceOptions, Tracer


def diffuse_and_emission_mask(scene) -> np.ndarray:
    m = np.zeros((scene.n_segments, 10), bool)
    m[:, 0:3] = True
    m[:, 7:10] = True
    return m


def prepare(scenes, opts: TraceOptions, target_spp: int = 1024, init: float = 0.0, seed: int = 0,
            configure=None):
    """Context with every scene uploaded, targets rendered from the ground
    truth (sample set 2), and the unknowns reset to `init`."""
    ss = SceneSet(scenes, seed=seed)
    if configure:
        configure(ss)
    masks = []
    for i, sc in enumerate(scenes):
        ss.set_params(i, sc.gt_params)
        ss.set_targets(i, ss.render(i, opts, spp=target_spp))
        free = diffuse_and_emission_mask(sc)
        p0 = sc.gt_params.copy()
        p0[free] = init
        ss.set_params(i, p0, free_mask=free.astype(np.uint8))
        tr = Tracer(sc)
        vis = metrics.visible_segments(tr, sc)
        tr.close()
        m = free.copy()
        m[~vis] = False
        masks.append(m)
    return ss, masks


def time_to_error(ss: SceneSet, masks, opts: TraceOptions, adam: AdamOptions, threshold: float = 0.01,
                  max_iters: int = 20000, check_every: int = 50):
    """Runs the batch until every member reaches the threshold (or
    max_iters).  Returns per-member (iterations, seconds) of the first
    crossing (None if never) and the error history."""
    n = len(ss.scenes)
    ss.make_batch()
    first = [None] * n
    history = []
    elapsed = 0.0
    it = 0
    while it < max_iters and any(f is None for f in first):
        torch.cuda.synchronize(ss.device)
        t0 = time.perf_counter()
        for _ in range(check_every):
            ss.batch_step(opts, adam, want_losses=False)
        torch.cuda.synchronize(ss.device)
        elapsed += time.perf_counter() - t0
        it += check_every
        errs = [metrics.param_error(ss.batch_params(i), ss.scenes[i].gt_params, masks[i]) for i in range(n)]
        history.append((it, elapsed, errs))
        for i, e in enumerate(errs):
            if first[i] is None and e <= threshold:
                first[i] = (it, elapsed)
    return first, history
