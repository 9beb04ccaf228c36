"""Time to a parameter-error threshold for one scene or a batch.

The measured quantity is the wall time (and the number of iterations) until
a member's parameter error first falls to the threshold.  By default the
unknowns are the diffuse albedo and emission of every segment (the
quantities the paper evaluates, Table 1); specular albedo and roughness are
held at their true values through the free mask, because without a Fresnel
term a rough GGX lobe can stand in for a Lambertian one and a few views
cannot tell them apart (unknowns_mask and scored_mask select other sets).  The error covers segments that a pixel centre sees, except the
diffuse albedo of emitting segments: an emitter's appearance is almost all
emission (Sec. 4 notes the same emission/albedo trade-off for objects in
few pixels), so its albedo is left free but not scored.  Iterations run as batch-graph replays; the error is read every
`check_every` iterations (the reads are outside the timed iterations).
"""
from __future__ import annotations

import time
from dataclasses import replace

import numpy as np
import torch

from . import metrics
from .batch import SceneSet
from .tracer import AdamOptions, TraceOptions, Tracer


def diffuse_and_emission_mask(scene) -> np.ndarray:
    return unknowns_mask(scene, "kd_e")


def unknowns_mask(scene, kind: str = "kd_e") -> np.ndarray:
    """The free parameters of an optimisation: "kd_e" diffuse albedo and
    emission (the rest at the truth), "kd" diffuse albedo only, "material"
    diffuse and specular albedo and roughness (emission at the truth)."""
    m = np.zeros((scene.n_segments, 10), bool)
    m[:, 0:3] = True
    if kind == "kd_e":
        m[:, 7:10] = True
    elif kind == "material":
        m[:, 3:7] = True
    elif kind != "kd":
        raise ValueError(kind)
    return m


def scored_mask(scene, free, visible, score: str = "legacy") -> np.ndarray:
    """Parameters the error scores.  "legacy": free ones of visible segments,
    without the diffuse albedo of emitting segments.  "survey": the
    identifiable set of metrics.identifiable_mask (diffuse and specular
    albedo and emission of visible segments, roughness where the true
    specular albedo has luminance >= 0.05) among the free parameters."""
    if score == "survey":
        return metrics.identifiable_mask(scene.gt_params, visible) & free
    m = free.copy()
    m[~visible] = False
    m[np.asarray(scene.light_segments, int), 0:3] = False
    return m


def prepare(scenes, opts: TraceOptions, target_spp: int = 1024, init: float = 0.0, seed: int = 0,
            configure=None, unknowns: str = "kd_e", score: str = "legacy"):
    """Context with every scene uploaded, targets rendered from the ground
    truth (sample set 2), and the unknowns reset to `init`."""
    ss = SceneSet(scenes, seed=seed)
    if configure:
        configure(ss)
    masks = []
    for i, sc in enumerate(scenes):
        ss.set_params(i, sc.gt_params)
        ss.set_targets(i, ss.render(i, opts, spp=target_spp))
        free = unknowns_mask(sc, unknowns)
        p0 = sc.gt_params.copy()
        p0[free] = init
        ss.set_params(i, p0, free_mask=free.astype(np.uint8))
        tr = Tracer(sc)
        vis = metrics.visible_segments(tr, sc)
        tr.close()
        masks.append(scored_mask(sc, free, vis, score))
    return ss, masks


def adam_at(adam: AdamOptions, it: int, halve_every: int) -> AdamOptions:
    """The learning rate halved every `halve_every` iterations (0: constant)."""
    if not halve_every:
        return adam
    return replace(adam, lr=adam.lr * 0.5 ** (it // halve_every))


def time_to_error(ss: SceneSet, masks, opts: TraceOptions, adam: AdamOptions, threshold: float = 0.01,
                  max_iters: int = 20000, check_every: int = 50, halve_every: int = 0, retire: bool = False):
    """Runs the batch until every member reaches the threshold (or
    max_iters).  With retire, a member that has crossed stops taking part
    (ipt_batch_set_active), as a scene optimised alone stops at its own
    crossing.  Returns per-member (iterations, seconds) of the first
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
        for k in range(check_every):
            ss.batch_step(opts, adam_at(adam, it + k, halve_every), want_losses=False)
        torch.cuda.synchronize(ss.device)
        elapsed += time.perf_counter() - t0
        it += check_every
        errs = [metrics.param_error(ss.batch_params(i), ss.scenes[i].gt_params, masks[i]) for i in range(n)]
        history.append((it, elapsed, errs))
        for i, e in enumerate(errs):
            if first[i] is None and e <= threshold:
                first[i] = (it, elapsed)
        if retire:
            ss.set_active([f is None for f in first])
    return first, history


def prepare_single(scene, opts: TraceOptions, target_spp: int = 1024, init: float = 0.0, seed: int = 0,
                   device: int = 0, unknowns: str = "kd_e", score: str = "legacy"):
    """One-scene counterpart of prepare(): a Tracer with targets rendered from
    the ground truth (sample set 2) and the unknowns reset to `init`."""
    tr = Tracer(scene, device=device, seed=seed)
    tr.set_params(scene.gt_params)
    tr.set_targets(tr.render(opts, view=-1, set_id=2, spp=target_spp))
    free = unknowns_mask(scene, unknowns)
    p0 = scene.gt_params.copy()
    p0[free] = init
    tr.set_params(p0, free_mask=free.astype(np.uint8))
    return tr, scored_mask(scene, free, metrics.visible_segments(tr, scene), score)


def time_to_error_single(tr: Tracer, mask, opts: TraceOptions, adam: AdamOptions, threshold: float = 0.01,
                         max_iters: int = 20000, check_every: int = 50, monitor_every: int = 0,
                         monitor_spp: int = 64, halve_every: int = 0):
    """ipt_step on one scene until its parameter error falls to the
    threshold.  With the radiance cache active, every `monitor_every`
    iterations ipt_cache_bias compares the cached and plain estimators (set 0
    at monitor_spp, the step's spp_d) and turns the cache off once the bias
    exceeds the cache's threshold; the monitor's time counts.  Returns
    ((iterations, seconds) or None, history of (iteration, seconds, error,
    cache active))."""
    history = []
    elapsed = 0.0
    it = 0
    first = None
    cached = monitor_every > 0
    while it < max_iters and first is None:
        torch.cuda.synchronize(tr.device)
        t0 = time.perf_counter()
        for _ in range(check_every):
            tr.step(opts, adam_at(adam, it, halve_every), want_loss=False)
            it += 1
            if cached and it % monitor_every == 0:
                tr.cache_bias(opts, monitor_spp, iteration=1_000_000 + it)
                cached = tr.cache_status()["active"]
        torch.cuda.synchronize(tr.device)
        elapsed += time.perf_counter() - t0
        err = metrics.param_error(tr.get_params(), tr.scene.gt_params, mask)
        history.append((it, elapsed, err, cached))
        if err <= threshold:
            first = (it, elapsed)
    return first, history



def _fine_free_mask(sc) -> np.ndarray:
    """Per-triangle phases: the diffuse albedo of every non-light triangle and
    the emission of the light triangles are free (App. E keeps the lights
    fixed but lets their emission change)."""
    lights = np.zeros(sc.n_segments, bool)
    lights[np.asarray(sc.light_segments, int)] = True
    free = np.zeros((sc.n_segments, 10), bool)
    free[~lights, 0:3] = True
    free[lights, 7:10] = True
    return free


def coarse_to_fine(scene, opts: TraceOptions, adam: AdamOptions, iters=(300, 300, 300), split_fraction=0.25,
                   target_spp: int = 256, seed: int = 0, device: int = 0):
    """The paper's coarse-to-fine schedule (App. E, App. B) on one scene:
    (1) one albedo and one emission per object, from zero; (2) every
    triangle its own segment, started from (1), lights fixed except their
    emission; (3) the triangles whose covered pixels have the highest mean
    squared error (the top `split_fraction` of those seen) split in four,
    children started from their parent.  The captured images are rendered
    from the per-triangle truth (the scene's texture when it has one).
    Returns per phase (scene, recovered parameters, image relative L2 error
    against the captured images)."""
    from .scenes import per_triangle, subdivide
    truth = per_triangle(scene)
    tr = Tracer(truth, device=device, seed=seed)
    tr.set_params(truth.gt_params)
    tgt = tr.render(opts, view=-1, set_id=2, spp=target_spp)
    tr.close()

    def optimise(sc, p0, free, n):
        t = Tracer(sc, device=device, seed=seed)
        t.set_targets(tgt)
        t.set_params(p0, free_mask=free.astype(np.uint8))
        for _ in range(n):
            t.step(opts, adam, want_loss=False)
        img = t.render(opts, view=-1, set_id=0, spp=target_spp)
        return t, img, float(torch.linalg.norm(img - tgt) / torch.linalg.norm(tgt))

    phases = []
    free = diffuse_and_emission_mask(scene)
    p0 = scene.gt_params.copy()
    p0[free] = 0.0
    t, _, err = optimise(scene, p0, free, iters[0])
    p1 = t.get_params()
    t.close()
    phases.append((scene, p1, err))
    fine = per_triangle(scene, p1)
    t, img, err = optimise(fine, fine.start_params, _fine_free_mask(fine), iters[1])
    p2 = t.get_params()
    e = metrics.triangle_pixel_errors(t, fine, img, tgt)
    t.close()
    phases.append((fine, p2, err))
    lights = np.zeros(fine.n_segments, bool)
    lights[np.asarray(fine.light_segments, int)] = True
    seen = np.isfinite(e) & ~lights
    k = max(1, int(split_fraction * seen.sum()))
    thr = np.sort(e[seen])[::-1][k - 1]
    fine3 = subdivide(fine, seen & (e >= thr), p2)
    t, _, err = optimise(fine3, fine3.start_params, _fine_free_mask(fine3), iters[2])
    phases.append((fine3, t.get_params(), err))
    t.close()
    return phases
