"""Benchmark: forward + adjoint Mpaths/s of one nested-SGD iteration of
inverse path tracing on the 61k-triangle procedural room (8 views of
320x240, 32 residual + 32 derivative samples per pixel, depth 5, NEE + MIS,
L2 loss, Adam).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = light tables + forward (residual set) + fused residual + adjoint
(derivative set) + loss/gradient reduction + Adam, with every input resident
in device memory.  L2 is flushed (a 256 MiB write) between timed steps and
the flush is outside each step's CUDA-event bracket.  Rank 0 prints one JSON
line.  Under torchrun each rank optimises its own independent room (weak
scaling, no collective in the data path).

``--cache B`` runs the same step with the learned radiance cache: paths end
at vertex B (1 or 2) in the cache, which is trained online on 1 in 16
full-length paths (a training pass per step, counted in the step's time;
the metric still counts residual plus derivative paths).

``--shard`` instead shards one room by pixels over the ranks: each rank
traces both sample sets of a contiguous range of the views' pixels with the
room's Philox key, one all-reduce of the S x 10 gradient and the loss joins
them, and every rank takes the same Adam step (strong scaling).

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the benchmark line: the 61k-triangle room with 8 views
    "room61k": dict(workload="room_61k_tri", triangles=61160, segments=48, views=8, width=320,
                    height=240, spp_r=32, spp_d=32, max_depth=5, nee=True, mis=True, loss="l2",
                    init=0.5, target_spp=1024),
    # differentiation at scale: the 516k-triangle room with 16 views (targets at 256 spp to keep
    # the run within minutes)
    "room516k": dict(workload="room_516k_tri", triangles=515728, segments=150, views=16, width=640,
                     height=480, spp_r=16, spp_d=16, max_depth=6, nee=True, mis=True, loss="l2",
                     init=0.5, target_spp=256),
}
WORKLOAD = dict(WORKLOADS["room61k"])
METRIC = "fwd+adjoint Mpaths/s"
NODE_BYTES, TRI_BYTES = 64, 48


def make_scene(seed_offset=0):
    """The workload's scene (seed of the generator + seed_offset)."""
    from paper_1903_07145_gb300 import scenes
    if WORKLOAD["workload"].startswith("room_516k"):
        return scenes.room_500k(1002 + seed_offset)
    return scenes.room_60k(1001 + seed_offset)


def paths_per_step():
    w = WORKLOAD
    return (w["spp_r"] + w["spp_d"]) * w["views"] * w["width"] * w["height"]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for s in self.samples for n, v in zip(names, s[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# DRAM traffic of the dominant kernel comes from a committed ncu capture (the
# benchmark cannot read hardware counters itself).  It is reported only while
# the capture matches: same kernel, workload and wavefront configuration, and
# the traversal kernel's sources unchanged since (their SHA-256 is recorded
# with it): the device header, the wavefront header, and the traversal
# section of the wavefront source.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "wf_closest_room61k_traffic.txt")
CSRC = os.path.join(ROOT, "paper_1903_07145_gb300", "csrc")
TRAVERSAL_SECTION = ("// Persistent traversal with warp refills", "// Forward shading of queue")


def kernel_sources_sha256():
    h = hashlib.sha256()
    for f in ("ipt_device.cuh", "ipt_wavefront.h"):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(CSRC, "ipt_wavefront.cu")) as fh:
        text = fh.read()
    a, b = text.find(TRAVERSAL_SECTION[0]), text.find(TRAVERSAL_SECTION[1])
    if a < 0 or b < a:
        return None  # section markers moved: no record can match
    h.update(text[a:b].encode())
    return h.hexdigest()


def recorded_traffic(kernel, cfg, slots_per_launch):
    """DRAM bytes (read + write) per launch, or None: the committed record's
    bytes per path slot, from an ncu capture of the same kernel on a small
    case of the workload, times the slots of this run's chunks.  The traffic
    is the per-slot ray state read in 32-byte sectors across a chunk's slot
    range (the nodes and triangles stay in L2), so it scales with the chunk,
    not with the rays still alive in it."""
    try:
        with open(TRAFFIC_FILE) as fh:
            lines = fh.read().splitlines()
    except OSError:
        return None
    kv = {}
    for line in lines:
        if ":" in line and not line.lstrip().startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    want = {"kernel": kernel, "workload": WORKLOAD["workload"], "bvh_width": str(cfg.get("bvh_width")),
            "sort_cells": str(cfg.get("sort_cells", 0)), "sort_dirs": str(cfg.get("sort_dirs", 0)),
            "kernel_sources_sha256": kernel_sources_sha256()}
    if want["kernel_sources_sha256"] is None or any(kv.get(k) != v for k, v in want.items()):
        return None
    try:
        return float(kv["dram_bytes_per_slot"]) * slots_per_launch
    except (KeyError, ValueError):
        return None


def cpu_baseline(target_seconds=15.0):
    """The FP64 oracle (as it stands) on a bounded pixel sample of the same
    workload: loss + gradient on the sampled pixels of all views."""
    from oracle import oracle as O
    from paper_1903_07145_gb300 import scenes
    w = WORKLOAD
    sc = make_scene()
    osc = O.OracleScene(sc)
    p = scenes.initial_params(sc, w["init"])
    rng = np.random.default_rng(0)
    threads = O.default_threads()

    def run(per_view):
        pix = [rng.choice(w["width"] * w["height"], per_view, replace=False).astype(np.uint32)
               for _ in sc.cameras]
        targets = [np.full((w["width"] * w["height"], 3), 0.5) for _ in sc.cameras]
        t0 = time.perf_counter()
        O.loss_grad(osc, p, targets, w["spp_r"], w["spp_d"], w["max_depth"], seed=7, pixels=pix,
                    threads=threads)
        return time.perf_counter() - t0
    per_view = 32
    dt = run(per_view)
    per_view = int(min(w["width"] * w["height"], max(32, per_view * target_seconds / max(dt, 1e-3))))
    dt = run(per_view)
    n_paths = per_view * len(sc.cameras) * (w["spp_r"] + w["spp_d"])
    return {"value": n_paths / dt / 1e6, "unit": "Mpaths/s", "cores": threads, "kind": "oracle",
            "sample": f"{per_view} random pixels per view x {len(sc.cameras)} views, "
                      f"{w['spp_r']}+{w['spp_d']} paths each ({n_paths} paths, {dt:.1f} s)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    base = None
    times = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(target_seconds=max(2.0, 60.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            times.append(r["value"])
        base = r
    value = float(np.mean(times))
    w = WORKLOAD
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpaths/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": paths_per_step() / (value * 1e6) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": w["workload"], **{k: v for k, v in w.items() if k != "workload"},
                                           "sample": base["sample"]},
           "cpu_baseline": {**base, "value": value},
           "e2e": {"value": value, "unit": "Mpaths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world, local):
    import torch
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        __graft_entry__.build()
    from paper_1903_07145_gb300 import scenes
    from paper_1903_07145_gb300 import _lib as L
    from paper_1903_07145_gb300.tracer import AdamOptions, CacheOptions, TraceOptions, Tracer

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOAD
    # --shard: every rank holds the same room and traces a contiguous range
    # of its pixels with the same Philox key; otherwise each rank its own room
    sc = make_scene(0 if args.shard else rank)
    if args.per_triangle:
        sc = scenes.per_triangle(sc)
    sc.cameras = sc.cameras[:w["views"]]
    opts = TraceOptions(spp_r=w["spp_r"], spp_d=w["spp_d"], max_depth=w["max_depth"], nee=True, mis=True)
    adam = AdamOptions()
    seed = 1903 if args.shard else 1903 + rank
    tr = Tracer(sc, device=local, seed=seed, flags=L.IPT_FLAG_KERNEL_TIMING)
    # targets: the ground truth rendered with an independent sample set
    tr.set_params(sc.gt_params)
    target = tr.render(opts, view=-1, set_id=L.IPT_SET_TARGET, spp=w["target_spp"])
    tr.set_targets(target)
    tr.set_params(scenes.initial_params(sc, w["init"]))
    if args.cache:
        tr.configure_cache(CacheOptions(enabled=True, b_term=args.cache, train_spp=max(1, w["spp_r"] // 16),
                                        train_steps=4))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = {}
    if args.integrator == "auto":
        from paper_1903_07145_gb300 import autotune
        best, tuned = autotune.tune(tr, lambda: tr.loss_grad(opts, iteration=0),
                                    wavefront_only=bool(args.cache))
        tr.set_params(scenes.initial_params(sc, w["init"]))
    else:
        tr.configure(args.integrator, wavefront_slots=args.slots, trace_steps=args.trace_steps,
                     bvh_width=args.bvh_width, sort_cells=args.sort_cells, sort_dirs=args.sort_dirs)
    chosen = tr.config()
    shard_iter = [0]

    def step(want_loss=False):
        """One nested-SGD iteration: the whole room on this GPU, or (--shard)
        this rank's pixel shard, one all-reduce of the S x 10 gradient and the
        loss over the ranks, and the same Adam step on every rank."""
        if args.shard:
            from paper_1903_07145_gb300 import parallel
            loss = parallel.sharded_step(tr, opts, adam, shard_iter[0])
            shard_iter[0] += 1
            return loss
        return tr.step(opts, adam, want_loss=want_loss)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    tr.kernel_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        # an NVTX range around the timed steps lets a profiler select them
        # (ncu --nvtx --nvtx-include "timed_steps/")
        torch.cuda.nvtx.range_push("timed_steps")
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ktimes = tr.kernel_times(reset=True)
    loss_end = tr.loss_grad(opts, iteration=10_000)[0]
    # achievable gather bandwidth over a buffer the size of the scene's nodes
    # and triangles (the traversal kernels' L2-resident working set)
    info = tr.info()
    footprint = max(1 << 16, info["n_nodes"] * NODE_BYTES + info["n_tri"] * TRI_BYTES)
    l2_gather_gbs = L.ipt_probe_gather(local, footprint)

    # algorithmic traffic of the dominant kernel: node and triangle fetches per
    # launch, counted by a separate context with counters (same seeds, same paths)
    ct = Tracer(sc, device=local, seed=seed, flags=L.IPT_FLAG_COUNTERS)
    ct.configure(**chosen)
    ct.set_targets(target)
    ct.set_params(scenes.initial_params(sc, w["init"]))
    if args.cache:  # the same cut paths as the timed context
        ct.configure_cache(CacheOptions(enabled=True, b_term=args.cache, train_spp=max(1, w["spp_r"] // 16),
                                        train_steps=4))
    ct.counters(reset=True)
    ct.render(opts, view=-1, set_id=L.IPT_SET_RESIDUAL, spp=w["spp_r"])
    fwd_cnt = ct.counters(reset=True)
    g = torch.full((tr.n_pix, 3), 1.0, device=dev)
    ct.backward(g, opts, set_id=L.IPT_SET_DERIVATIVE)
    if args.cache:  # the step's training pass traces too
        ct.cache_train(opts, iteration=0)
    adj_cnt = ct.counters(reset=True)
    ct.close()

    # end to end through the C ABI with host buffers: targets uploaded from
    # pinned memory, loss and parameters read back, every step
    host_target = target.cpu().pin_memory()
    host_params = np.zeros((sc.n_segments, 10), np.float32)
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        L.ipt_targets_set(tr.ctx, tr.sid, host_target.data_ptr(), 0)
        step(want_loss=True)
        L.ipt_params_get(tr.ctx, tr.sid, host_params.ctypes.data)
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    cache_bias = None
    if args.cache:
        # bias of the cached estimator against the plain one (image and loss
        # gradient, both at 4096 spp), after further training outside the
        # timed region
        extra = 300
        for it in range(extra):
            tr.cache_train(opts, iteration=100_000 + it)
        ib, gb = tr.cache_bias(opts, 4096, iteration=200_000)
        cache_bias = {"training_passes": args.warmup + args.steps + e2e_steps + extra, "spp": 4096,
                      "image_rel": ib, "grad_rel": gb}
    tr.close()

    if rank != 0:
        return
    # --shard: the ranks share one room's paths (strong scaling); otherwise
    # each rank steps its own room (weak scaling)
    n_paths = paths_per_step() * (1 if args.shard else world)
    value = n_paths / (ms * 1e-3) / 1e6
    # dominant kernel by total device time in the timed region
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    dom_total_ms, dom_launches = ktimes[dom]
    # counters cover the whole room; a shard traces its share of the rays
    share = world if args.shard else 1
    both = {k: (fwd_cnt[k] + adj_cnt[k]) / share for k in fwd_cnt}
    if dom in ("wf_closest", "wf_shadow"):
        kind = "closest" if dom == "wf_closest" else "shadow"
        nodes, tris = both[f"{kind}_node_visits"], both[f"{kind}_tri_tests"]
        rays = both[f"{kind}_rays"]
    elif dom in ("forward", "adjoint"):
        c = fwd_cnt if dom == "forward" else adj_cnt
        nodes = c["closest_node_visits"] + c["shadow_node_visits"]
        tris = c["closest_tri_tests"] + c["shadow_tri_tests"]
        rays = c["closest_rays"] + c["shadow_rays"]
    else:
        nodes = tris = rays = 0
    # counters cover one step's passes; the timed region ran args.steps steps
    launches_per_step = dom_launches / args.steps
    # slots of one wavefront chunk: a pass of P paths in ceil(P / cap) chunks
    pass_paths = w["spp_r"] * w["views"] * w["width"] * w["height"] / share
    cap = chosen.get("wavefront_slots") or (1 << 20)
    chunk_slots = pass_paths / math.ceil(pass_paths / cap)
    alg_bytes_step = nodes * NODE_BYTES + tris * TRI_BYTES
    alg_bytes_launch = alg_bytes_step / max(launches_per_step, 1)
    dom_ms = dom_total_ms / max(1, dom_launches)
    peak, src = measured_peaks()
    achieved = alg_bytes_launch / (dom_ms * 1e-3) / 1e9 if alg_bytes_launch else 0.0
    launches = sum(n for _, n in ktimes.values())
    rays_step = both["closest_rays"] + both["shadow_rays"]
    out = {
        "metric": METRIC, "value": value, "unit": "Mpaths/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], **{k: v for k, v in WORKLOAD.items() if k != "workload"},
                   "l2": "256 MiB flush between timed steps (outside the step events)",
                   "parallelism": (f"one room in {world} pixel shards, one NCCL all-reduce of the S x 10 "
                                   f"gradient and the loss per step" if args.shard
                                   else f"{world} independent rooms, one per GPU"),
                   "integrator": {**chosen, "integrator": ["megakernel", "wavefront"][chosen["integrator"]]},
                   "autotune_ms": tuned},
        "mrays_per_s": rays_step / (ms * 1e-3) / 1e6,
        "kernel_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in ktimes.items() if v[1]},
        "kernel_launches_per_step": {k: v[1] / args.steps for k, v in ktimes.items() if v[1]},
        # the node and triangle bytes are served by L2 and L1 (the scene's few
        # MB stay resident): the bound is the L2 gather rate.  `peak` and
        # `frac` are against the measured HBM copy bandwidth; `l2_frac`
        # against the gather probe measured in this run with the traversal's
        # own 256-bit node loads
        "roofline": {"bound": "l2", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": recorded_traffic(dom, chosen, chunk_slots),
                     "peak_source": f"{src} (HBM copy)",
                     "l2_gather_peak": l2_gather_gbs,
                     "l2_frac": achieved / l2_gather_gbs if l2_gather_gbs else None,
                     "algorithmic_bytes_per_launch": alg_bytes_launch,
                     "avg_launch_ms": dom_ms,
                     "units_per_step": {"node_visits": nodes, "tri_tests": tris, "rays": rays}},
        "roofline_l2": {"bound": "l2_gather", "kernel": dom, "achieved": achieved, "peak": l2_gather_gbs,
                        "unit": "GB/s", "frac": achieved / l2_gather_gbs if l2_gather_gbs else None,
                        "probe_bytes": footprint,
                        "peak_source": "ipt_probe_gather: random 64-byte lines over a buffer of the scene's "
                                       "node + triangle bytes, each read with two 256-bit loads as the "
                                       "traversal reads a node, measured in this run"},
        "e2e": {"value": paths_per_step() / e2e_s / 1e6, "unit": "Mpaths/s",
                "h2d_bytes_per_step": int(host_target.numel() * 4),
                "d2h_bytes_per_step": int(8 + host_params.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "loss_after": loss_end,
        "wall_s_timed_region": t_wall,
    }
    if cache_bias is not None:
        out["cache_bias"] = cache_bias
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)


def run_batch64(args):
    """Aggregate fwd+adjoint Mpaths/s of one batch iteration over the 64
    uneven rooms (one launch per stage over all rooms, replayed as a CUDA
    graph), or, with --workload cornell64, over the 64 Cornell variants in
    the paper's pixel-batch regime (--pixel-batch, --batch-spp, --spp-d) on
    --batch-integrator."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_07145_gb300 import scenes
    from paper_1903_07145_gb300.batch import SceneSet
    from paper_1903_07145_gb300.tracer import AdamOptions, TraceOptions
    t0 = time.perf_counter()
    cornell = args.workload == "cornell64"
    rooms = ([scenes.cornell_variant(k) for k in range(64)] if cornell
             else [scenes.batch_room(k, args.res_div) for k in range(64)])
    gen_s = time.perf_counter() - t0
    spp_d = args.spp_d or args.batch_spp
    opts = TraceOptions(spp_r=args.batch_spp, spp_d=spp_d, max_depth=args.batch_depth,
                        pixel_batch=args.pixel_batch)
    ss = SceneSet(rooms, seed=1903)
    integ = "wavefront" if args.batch_integrator == "auto" else args.batch_integrator
    ss.configure(integrator=integ, wavefront_slots=1 << 25, bvh_width=4, sort_cells=args.sort_cells,
                 sort_dirs=args.sort_dirs)
    for i, sc in enumerate(rooms):
        ss.set_params(i, sc.gt_params)
        ss.set_targets(i, ss.render(i, TraceOptions(max_depth=args.batch_depth), spp=16))
        ss.set_params(i, scenes.initial_params(sc, 0.5))
    ss.make_batch()
    adam = AdamOptions()
    dev = ss.device
    for _ in range(args.warmup):
        ss.batch_step(opts, adam, want_losses=False)
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            ss.batch_step(opts, adam, want_losses=False)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    pix = sum(c.width * c.height for sc in rooms for c in sc.cameras)
    entries = 64 * args.pixel_batch if args.pixel_batch else pix
    paths = (args.batch_spp + spp_d) * entries
    name = (f"cornell64_variants_pixbatch{args.pixel_batch}" if cornell else f"batch64_rooms_div{args.res_div}")
    out = {"metric": METRIC, "value": paths / (ms * 1e-3) / 1e6, "unit": "Mpaths/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": name, "rooms": 64, "integrator": integ,
                      "triangles": int(sum(sc.indices.shape[0] for sc in rooms)),
                      "segments": int(sum(sc.n_segments for sc in rooms)), "pixels": int(pix),
                      "pixel_batch": args.pixel_batch, "entries_per_step": int(entries),
                      "spp_r": args.batch_spp, "spp_d": spp_d, "max_depth": args.batch_depth,
                      "l2": "256 MiB flush between timed steps (outside the step events)",
                      "generation_s": gen_s},
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_time_to_error(args):
    """Wall time to 1% parameter error.  Without --cache: the 64 rooms
    (resolution / res_div) optimised together in the batch graph, against
    the same rooms optimised one after another by the plain single-scene
    step.  With --cache B: the 61k-triangle room (resolution / res_div) with
    the cache and its bias monitor (fallback to the plain tracer above 2%),
    against the plain tracer."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_07145_gb300 import convergence, scenes
    from paper_1903_07145_gb300.tracer import AdamOptions, CacheOptions, TraceOptions
    adam = AdamOptions(lr=args.lr)
    res = {}
    if args.cache:
        sc = scenes.room_60k(1001)
        for c in sc.cameras:
            c.width //= args.res_div
            c.height //= args.res_div
        opts = TraceOptions(spp_r=args.batch_spp, spp_d=args.batch_spp, max_depth=5)
        for arm in ["plain", "cached"]:
            tr, mask = convergence.prepare_single(sc, opts, target_spp=1024, seed=7)
            tr.configure("wavefront")
            if arm == "cached":
                tr.configure_cache(CacheOptions(enabled=True, b_term=args.cache,
                                                train_spp=max(1, args.batch_spp // 16), train_steps=4,
                                                bias_threshold=0.02))
            first, hist = convergence.time_to_error_single(
                tr, mask, opts, adam, threshold=0.01, max_iters=args.max_iters, check_every=50,
                monitor_every=args.monitor_every if arm == "cached" else 0, monitor_spp=args.monitor_spp)
            res[arm] = {"first": first, "history": [(h[0], round(h[1], 3), round(h[2], 5), h[3]) for h in hist]}
            tr.close()
        workload = f"room_61k_tri_div{args.res_div}_cache_b{args.cache}"
    else:
        if args.workload == "cornell64":
            rooms = [scenes.cornell_variant(k) for k in range(64)]
            target_spp = 1024
        else:
            rooms = [scenes.batch_room(k, args.res_div) for k in range(args.rooms)]
            target_spp = 256
        opts = TraceOptions(spp_r=args.batch_spp, spp_d=args.spp_d or args.batch_spp,
                            max_depth=args.batch_depth, pixel_batch=args.pixel_batch)
        tgt = TraceOptions(max_depth=args.batch_depth)
        ss, masks = convergence.prepare(rooms, tgt, target_spp=target_spp, init=args.init, seed=7,
                                        unknowns=args.unknowns, score=args.score)
        # the batch's integrator: as given, or the faster of the two on 20
        # batch steps from the start (outside the timing; make_batch restarts
        # from the scenes' own parameters, which the steps do not touch)
        batch_ms = {}
        for integ in (["wavefront", "megakernel"] if args.batch_integrator == "auto" else [args.batch_integrator]):
            ss.configure(integrator=integ, wavefront_slots=1 << 21, bvh_width=4)
            ss.make_batch()
            ss.batch_step(opts, adam, want_losses=False)
            torch.cuda.synchronize(ss.device)
            t0 = time.perf_counter()
            for _ in range(20):
                ss.batch_step(opts, adam, want_losses=False)
            torch.cuda.synchronize(ss.device)
            batch_ms[integ] = (time.perf_counter() - t0) / 20 * 1e3
        batch_integ = min(batch_ms, key=batch_ms.get)
        ss.configure(integrator=batch_integ, wavefront_slots=1 << 21, bvh_width=4)
        # a scene leaves the batch when it reaches the threshold, as one optimised
        # alone stops at its own crossing
        first, hist = convergence.time_to_error(ss, masks, opts, adam, threshold=args.threshold,
                                                max_iters=args.max_iters, check_every=args.check_every,
                                                halve_every=args.halve_every, retire=not args.no_retire)
        res["batched"] = {"first": first, "history_last": hist[-1][:2], "integrator": batch_integ,
                          "ms_per_step_probe": batch_ms}
        ss.close()
        # the plain arm: each scene alone with its fastest integrator
        # configuration (autotuned on its own workload, outside the timing)
        from paper_1903_07145_gb300 import autotune
        seq, seq_cfg, seq_hist = [], [], []
        for i, sc in enumerate(rooms[:args.seq_rooms]):
            tr, m = convergence.prepare_single(sc, tgt, target_spp=target_spp, seed=7, init=args.init,
                                               unknowns=args.unknowns, score=args.score)
            p0 = tr.get_params()
            best, _ = autotune.tune(tr, lambda: tr.loss_grad(opts, iteration=0), repeats=3)
            tr.set_params(p0, free_mask=convergence.unknowns_mask(sc, args.unknowns).astype(np.uint8))
            seq_cfg.append(best.get("integrator"))
            f, h = convergence.time_to_error_single(tr, m, opts, adam, threshold=args.threshold,
                                                    max_iters=args.max_iters,
                                                    check_every=args.check_every, halve_every=args.halve_every)
            seq.append(f)
            seq_hist.append(h)
            tr.close()
        res["sequential_plain"] = {"first": seq, "integrators": seq_cfg,
                                   "final_error": [h[-1][2] for h in seq_hist]}
        res["batched"]["final_error"] = hist[-1][2]

        # first crossings of looser thresholds, from the error histories (the
        # runs stop at --threshold or --max-iters)
        def crossings(thr):
            b = [next(((it, t) for it, t, errs in hist if errs[i] <= thr), None) for i in range(len(rooms))]
            q = [next(((h_[0], h_[1]) for h_ in hh if h_[2] <= thr), None) for hh in seq_hist]
            return b, q

        def summary(fs):
            t = np.array([f[1] for f in fs if f is not None])
            return {"reached": int(t.size), "of": len(fs),
                    "p50_s": float(np.percentile(t, 50)) if t.size else None,
                    "p99_s": float(np.percentile(t, 99)) if t.size else None}
        k = len(seq)
        # measured: the scenes among the first k that reached the threshold in
        # both arms; the batch's wall time until the last of them crossed (the
        # batch kept all 64 scenes running) against the sum of their
        # one-after-another times
        common = [i for i in range(k) if first[i] is not None and seq[i] is not None]
        b_wall = max((first[i][1] for i in common), default=None)
        s_sum = sum(seq[i][1] for i in common) if common else None
        # per-iteration cost of one scene alone and of the 64-scene batch
        it_alone = (float(np.mean([f[1] / f[0] for f in seq if f is not None]))
                    if any(f is not None for f in seq) else None)
        it_batch = hist[-1][1] / hist[-1][0]
        reached = [f for f in first if f is not None]
        res["summary"] = {
            "batched": summary(first), "sequential_plain": summary(seq),
            "scenes_compared": len(common),
            "batched_wall_s_compared": b_wall, "sequential_sum_s_compared": s_sum,
            "speedup_compared": (s_sum / b_wall) if common else None,
            "ms_per_iteration_one_scene_alone": None if it_alone is None else it_alone * 1e3,
            "ms_per_iteration_batch_of_64": it_batch * 1e3,
            # whole job, estimated: every scene that reached the threshold in
            # the batch, at its crossing iteration and the one-scene-alone
            # cost per iteration, against the batch's wall time to its last
            # crossing
            "whole_job_estimate": None if (it_alone is None or not reached) else {
                "scenes": len(reached), "batched_wall_s": max(f[1] for f in reached),
                "sequential_s_estimate": sum(f[0] for f in reached) * it_alone,
                "speedup": sum(f[0] for f in reached) * it_alone / max(f[1] for f in reached)}}
        res["thresholds"] = {}
        for thr in sorted({args.threshold, 0.02, 0.05, 0.1}):
            b, q = crossings(thr)
            both = [i for i in range(len(q)) if b[i] is not None and q[i] is not None]
            res["thresholds"][f"{thr:g}"] = {
                "batched": summary(b), "sequential_plain": summary(q), "scenes_compared": len(both),
                "batched_wall_s_compared": max((b[i][1] for i in both), default=None),
                "sequential_sum_s_compared": sum(q[i][1] for i in both) if both else None}
        workload = ("cornell64_variants" if args.workload == "cornell64" else f"batch64_rooms_div{args.res_div}")
        workload += f"_pixbatch{args.pixel_batch}" if args.pixel_batch else ""
    print(json.dumps({"metric": f"time to {100 * args.threshold:g}% parameter error", "unit": "s",
                      "workload": workload, "unknowns": args.unknowns, "score": args.score, "init": args.init,
                      "lr": args.lr, "halve_every": args.halve_every, "retire": not args.no_retire,
                      "spp": args.batch_spp,
                      "spp_d": args.spp_d or args.batch_spp, "pixel_batch": args.pixel_batch,
                      "results": res}), flush=True)


def run_disney(args):
    """fwd+adjoint Mpaths/s of the Disney material model (Sec. 4.1; wavefront,
    or the megakernel with --integrator megakernel) on the benchmark room with
    random Disney materials: one step = loss,
    gradient and Adam over all views; per-kernel device times from the
    library's own events (a second, identical timing pass)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_07145_gb300 import _lib as L
    from paper_1903_07145_gb300 import scenes
    from paper_1903_07145_gb300.tracer import AdamOptions, TraceOptions, Tracer
    w = WORKLOAD
    sc = make_scene()
    sc.cameras = sc.cameras[: w["views"]]
    truth = scenes.disney_materials(sc, 77)
    opts = TraceOptions(spp_r=w["spp_r"], spp_d=w["spp_d"], max_depth=w["max_depth"])
    adam = AdamOptions()
    res = {}
    integ = "megakernel" if args.integrator == "megakernel" else "wavefront"
    for timing in (False, True):
        tr = Tracer(sc, seed=1903, flags=L.IPT_FLAG_KERNEL_TIMING if timing else 0)
        if integ == "wavefront":  # the configuration the autotuner picks for this room
            tr.configure("wavefront", wavefront_slots=1 << 25, trace_steps=24, bvh_width=4, sort_cells=6,
                         sort_dirs=2)
        else:
            tr.configure("megakernel")
        tr.disney_set_params(truth)
        tr.set_targets(tr.disney_render(TraceOptions(max_depth=w["max_depth"]), set_id=L.IPT_SET_TARGET, spp=16))
        p0 = truth.copy()
        p0[:, 0:13] = 0.5
        tr.disney_set_params(p0)
        for _ in range(args.warmup):
            tr.disney_step(opts, adam, want_loss=False)
        dev = tr.device
        torch.cuda.synchronize(dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        stream = torch.cuda.current_stream(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if timing:
            tr.kernel_times(reset=True)
        with ClockSampler(0) as clk:
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                tr.disney_step(opts, adam, want_loss=False)
                ev[i][1].record(stream)
            torch.cuda.synchronize(dev)
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        if timing:
            kt = tr.kernel_times()
            res["kernel_ms_per_step"] = {k: round(v[0] / args.steps, 3) for k, v in kt.items() if v[1]}
        else:
            res["ms"], res["clocks"] = ms, clk.summary()
        tr.close()
    paths = paths_per_step()
    out = {"metric": METRIC + " (Disney material model)", "value": paths / (res["ms"] * 1e-3) / 1e6,
           "unit": "Mpaths/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w["workload"] + "_disney", "views": w["views"], "width": w["width"],
                      "height": w["height"], "spp_r": w["spp_r"], "spp_d": w["spp_d"],
                      "max_depth": w["max_depth"], "integrator": integ,
                      "l2": "256 MiB flush between timed steps (outside the step events)"},
           "kernel_ms_per_step": res["kernel_ms_per_step"], "clocks": res["clocks"]}
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """Convergence curves of the optimiser ablations on a 64 x 64 Cornell box:
    per setting (iteration, seconds, parameter error, image L1 loss) at equal
    optimisation time, and the final errors."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_07145_gb300 import ablation, scenes
    from paper_1903_07145_gb300.tracer import AdamOptions
    kinds = list(ablation.SWEEPS) if args.sweep == "all" else [args.sweep]
    for kind in kinds:
        sc = scenes.cornell_box(1000, 64, 64)
        curves = ablation.sweep(kind, sc, AdamOptions(lr=args.lr), args.sweep_seconds)
        def first_below(v, thr):
            return next((round(c[1], 3) for c in v if c[2] <= thr), None)

        def tail(v, i):  # mean over the last quarter of the checkpoints
            t = v[-max(1, len(v) // 4):]
            return float(np.mean([c[i] for c in t]))
        final = {k: {"iterations": v[-1][0], "seconds": round(v[-1][1], 3),
                     "param_error_last_quarter_mean": round(tail(v, 2), 5),
                     "image_l1_last_quarter_mean": round(tail(v, 3), 5),
                     "best_param_error": round(min(c[2] for c in v), 5),
                     "seconds_to_5pct": first_below(v, 0.05), "seconds_to_2pct": first_below(v, 0.02)}
                 for k, v in curves.items()}
        print(json.dumps({"metric": "convergence at equal time", "sweep": kind,
                          "workload": "cornell_64x64_pixel_batches_l1", "seconds_per_setting": args.sweep_seconds,
                          "lr": args.lr, "final": final,
                          "curves": {k: [(c[0], round(c[1], 4), round(c[2], 5), c[3]) for c in v]
                                     for k, v in curves.items()}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--integrator", default="auto", choices=["auto", "megakernel", "wavefront"])
    ap.add_argument("--cache", type=int, default=0, choices=[0, 1, 2],
                    help="end paths at this vertex in the learned radiance cache (0: plain tracer)")
    ap.add_argument("--workload", default="room61k", choices=["room61k", "room516k", "batch64", "cornell64"],
                    help="batch64: aggregate throughput of the 64 uneven rooms (a separate line)")
    ap.add_argument("--time-to-error", action="store_true",
                    help="wall time to 1%% parameter error (batched vs sequential, or cached vs plain)")
    ap.add_argument("--res-div", type=int, default=1, help="resolution divisor of the extra workloads")
    ap.add_argument("--batch-spp", type=int, default=8)
    ap.add_argument("--batch-depth", type=int, default=3)
    ap.add_argument("--lr", type=float, default=5e-3)
    ap.add_argument("--pixel-batch", type=int, default=0,
                    help="time-to-error: B pixels drawn per iteration (Sec. 4.5; 0 = whole images)")
    ap.add_argument("--spp-d", type=int, default=0, help="time-to-error: derivative samples (0 = --batch-spp)")
    ap.add_argument("--seq-rooms", type=int, default=64,
                    help="time-to-error: rooms optimised one after another for the plain arm")
    ap.add_argument("--check-every", type=int, default=50, help="time-to-error: iterations between error reads")
    ap.add_argument("--batch-integrator", default="auto", choices=["auto", "wavefront", "megakernel"],
                    help="time-to-error: the batch graph's integrator (auto: the faster on 20 steps)")
    ap.add_argument("--no-retire", action="store_true",
                    help="time-to-error: keep stepping batch members that reached the threshold")
    ap.add_argument("--halve-every", type=int, default=0,
                    help="time-to-error: halve the learning rate every N iterations (0 = constant)")
    ap.add_argument("--max-iters", type=int, default=6000)
    ap.add_argument("--threshold", type=float, default=0.01, help="time-to-error: relative parameter error")
    ap.add_argument("--unknowns", default="kd_e", choices=["kd_e", "kd", "material"],
                    help="time-to-error: free parameters (kd_e: diffuse albedo + emission; kd: diffuse albedo; "
                         "material: diffuse, specular albedo, roughness); the rest held at the truth")
    ap.add_argument("--score", default="legacy", choices=["legacy", "survey"],
                    help="time-to-error: legacy (free parameters of seen segments, not the lights' albedo) or "
                         "survey (albedos, emission of seen segments, roughness where lum(ks) >= 0.05)")
    ap.add_argument("--init", type=float, default=0.0, help="time-to-error: start value of the unknowns")
    ap.add_argument("--rooms", type=int, default=64, help="time-to-error: the first N of the 64 procedural rooms")
    ap.add_argument("--sweep", default=None, choices=["paths", "split", "batch", "mis", "bounces", "all"],
                    help="optimiser ablation curves (paths per pixel, sample split, batch size, MIS, bounces)")
    ap.add_argument("--sweep-seconds", type=float, default=8.0, help="optimisation time per sweep setting")
    ap.add_argument("--per-triangle", action="store_true",
                    help="every triangle its own segment (App. E refinement): gradient scatter over T segments")
    ap.add_argument("--material", default="lambert_ggx", choices=["lambert_ggx", "disney"],
                    help="disney: time the Disney material model's step (megakernel) on the workload")
    ap.add_argument("--monitor-every", type=int, default=250)
    ap.add_argument("--monitor-spp", type=int, default=1024)
    ap.add_argument("--views", type=int, default=None,
                    help="profiling only: use the first V views (not a benchmark line)")
    ap.add_argument("--spp", type=int, default=None,
                    help="profiling only: spp_r = spp_d = S (not a benchmark line)")
    ap.add_argument("--shard", action="store_true",
                    help="one room sharded by pixels over the GPUs (strong scaling), NCCL all-reduce per step")
    ap.add_argument("--bvh-width", type=int, default=0, choices=[0, 2, 4, 8],
                    help="profiling only: BVH width with --integrator wavefront or megakernel")
    ap.add_argument("--slots", type=int, default=0,
                    help="profiling only: wavefront path slots per chunk with --integrator wavefront")
    ap.add_argument("--trace-steps", type=int, default=0,
                    help="profiling only: traversal refill point with --integrator wavefront")
    ap.add_argument("--sort-cells", type=int, default=0,
                    help="with --integrator wavefront: reorder secondary closest-hit rays by origin cell "
                         "(cells per axis; 0: queue order)")
    ap.add_argument("--sort-dirs", type=int, default=0,
                    help="direction cells per cube-map face side of the reordering (0: origin cells only)")
    args = ap.parse_args()
    if args.workload in WORKLOADS:
        WORKLOAD.clear()
        WORKLOAD.update(WORKLOADS[args.workload])
    if args.views:
        WORKLOAD["views"] = args.views
        WORKLOAD["workload"] += f"_first{args.views}views"
    if args.spp:
        WORKLOAD["spp_r"] = WORKLOAD["spp_d"] = args.spp
        WORKLOAD["workload"] += f"_spp{args.spp}"
        WORKLOAD["target_spp"] = min(WORKLOAD["target_spp"], 64)
    if args.per_triangle:
        WORKLOAD["workload"] += "_per_triangle"
        WORKLOAD["segments"] = WORKLOAD["triangles"]
    if args.cache:
        WORKLOAD["workload"] += f"_cache_b{args.cache}"
        WORKLOAD["cache"] = dict(b_term=args.cache, train_spp=max(1, WORKLOAD["spp_r"] // 16), train_steps=4,
                                 lr=1e-2)
    rank, world, local = dist_env()
    if args.impl == "ours" and args.workload == "cornell64" and not args.time_to_error:
        run_batch64(args)
        return
    if args.impl == "ours" and args.time_to_error:
        run_time_to_error(args)
        return
    if args.impl == "ours" and args.sweep:
        run_sweep(args)
        return
    if args.impl == "ours" and args.material == "disney":
        run_disney(args)
        return
    if args.impl == "ours" and args.workload == "batch64":
        run_batch64(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.shard and args.cache:
        raise SystemExit("--shard runs the plain estimator (no --cache)")
    dist_on = world > 1 or args.shard
    if dist_on:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        if world > 1:
            dist.init_process_group("nccl")
        else:  # one shard: a single-rank group, so the step runs the same all-reduce
            import socket
            with socket.socket() as so:
                so.bind(("127.0.0.1", 0))
                port = so.getsockname()[1]
            dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        run_ours(args, rank, world, local)
    finally:
        if dist_on:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
