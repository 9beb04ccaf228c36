"""Picks the integrator configuration of a context by measurement.

Candidates: the megakernel, and the wavefront integrator with the three BVH
widths (binary, 4-wide sorted by distance, 8-wide in octant order), two chunk
sizes (2M path slots, and 32M, which holds a whole pass of most workloads in
one chunk: no drain tail between chunks, fewer launches) and two traversal
refill granularities; with 32M slots and the wide BVHs also the reordering
of secondary rays by origin and direction cell (6^3 cells x 24 directions).  Each candidate runs one
loss-and-gradient evaluation of the caller's workload (after one untimed
run that allocates its buffers); the fastest by CUDA-event time wins and is
left configured.  Every candidate traces the same paths, so the choice
changes speed only.
"""
from __future__ import annotations

import itertools

import torch

DEFAULT_CANDIDATES = (
    [dict(integrator="megakernel")]
    + [dict(integrator="wavefront", wavefront_slots=s, trace_steps=k, bvh_width=b)
       for b, s, k in itertools.product([2, 4, 8], [1 << 21, 1 << 25], [16, 24])]
    + [dict(integrator="wavefront", wavefront_slots=1 << 25, trace_steps=k, bvh_width=b, sort_cells=6, sort_dirs=2)
       for b, k in itertools.product([4, 8], [16, 24])]
)


def _time_once(tracer, run):
    stream = torch.cuda.current_stream(tracer.device)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    run()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def tune(tracer, run, candidates=DEFAULT_CANDIDATES, repeats=1, wavefront_only=False):
    """run(): one evaluation of the workload on `tracer` (no host sync
    needed).  Returns (best config dict, {repr(config): ms}).  wavefront_only
    skips megakernel candidates (the cached passes always run wavefront)."""
    if wavefront_only:
        candidates = [c for c in candidates if c.get("integrator", "wavefront") != "megakernel"]
    results = {}
    best, best_ms = None, float("inf")
    for cfg in candidates:
        tracer.configure(**cfg)
        run()  # first use allocates the candidate's buffers
        torch.cuda.synchronize(tracer.device)
        ms = min(_time_once(tracer, run) for _ in range(repeats))
        results[repr(cfg)] = ms
        if ms < best_ms:
            best, best_ms = cfg, ms
    tracer.configure(**best)
    return best, results
