"""Sharding logic on two gloo ranks (CPU): the sharded loss and gradient,
summed over ranks, equal the unsharded ones up to summation order.  The
per-shard compute is the oracle, so the test exercises the sharding,
normalisation and all-reduce of paper_1903_07145_gb300.parallel."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1903_07145_gb300.parallel import shard_range, sharded_loss_grad


def test_shard_range_covers_pixels_once():
    for n in [0, 1, 7, 64, 1001]:
        for w in [1, 2, 3, 8]:
            seen = np.zeros(n, int)
            for r in range(w):
                b, c = shard_range(n, w, r)
                seen[b:b + c] += 1
            assert np.all(seen == 1)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _scene():
    from paper_1903_07145_gb300 import scenes
    sc = scenes.indoor_room(5, n_cuboids=4, cuboid_sub=2, room_sub=2, n_lights=2, n_views=3,
                            width=9, height=7)
    return sc


def _oracle_shard(osc, params, targets, begin, count, n_total, it):
    """Oracle loss/gradient over global pixel range [begin, begin+count)."""
    from oracle import oracle as O
    offs = osc.offsets
    loss = 0.0
    grad = np.zeros((osc.n_seg, 10))
    for v in range(len(osc.cams)):
        lo, hi = max(begin, offs[v]), min(begin + count, offs[v + 1])
        if lo >= hi:
            continue
        px = np.arange(lo - offs[v], hi - offs[v], dtype=np.uint32)
        img, _ = osc.render(params, view=v, pixels=px, spp=4, max_depth=3, set_id=0, iteration=it,
                            seed=3, threads=1)
        g, l_v = O.residual(img, targets[v][px], 3 * n_total)
        loss += l_v
        grad += osc.gradient(params, g, view=v, pixels=px, spp=4, max_depth=3, set_id=1,
                             iteration=it, seed=3, threads=1)
    return loss, grad


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        sc = _scene()
        osc = O.OracleScene(sc)
        p = sc.gt_params.astype(np.float64) * 0.9
        rng = np.random.default_rng(0)
        targets = [rng.uniform(0, 1, (c.width * c.height, 3)) for c in sc.cameras]
        n_pix = int(osc.offsets[-1])
        loss, grad = sharded_loss_grad(
            lambda b, c, n: _oracle_shard(osc, p, targets, b, c, n, 2), n_pix, sc.n_segments)
        if rank == 0:
            q.put((loss, grad.numpy()))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world", [2])
def test_sharded_equals_unsharded(world):
    from oracle import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    loss, grad = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    sc = _scene()
    osc = O.OracleScene(sc)
    p = sc.gt_params.astype(np.float64) * 0.9
    rng = np.random.default_rng(0)
    targets = [rng.uniform(0, 1, (c.width * c.height, 3)) for c in sc.cameras]
    n = int(osc.offsets[-1])
    ref_loss, ref_grad = _oracle_shard(osc, p, targets, 0, n, n, 2)
    l2, g2 = O.loss_grad(osc, p, targets, 4, 4, 3, iteration=2, seed=3, threads=1)
    assert abs(ref_loss - l2) <= 1e-12 * abs(l2) and np.allclose(ref_grad, g2, rtol=1e-12, atol=1e-14)
    assert abs(loss - ref_loss) <= 1e-12 * abs(ref_loss)
    assert np.allclose(grad, ref_grad, rtol=1e-10, atol=1e-12)


class _OracleTracer:
    """The attributes and calls parallel.sharded_step uses (device, n_pix,
    n_seg, loss_grad_shard, adam_step), computed by the oracle on the CPU:
    a GPU rank's Tracer stands in for it on a GPU machine."""

    def __init__(self, osc, params, targets):
        self.osc, self.targets = osc, targets
        self.device = torch.device("cpu")
        self.n_pix = int(osc.offsets[-1])
        self.n_seg = osc.n_seg
        self.params = np.array(params, np.float64)
        self.m = np.zeros_like(self.params)
        self.v = np.zeros_like(self.params)
        self.t = 0

    def loss_grad_shard(self, opts, iteration, begin, count, n_total):
        return _oracle_shard(self.osc, self.params, self.targets, begin, count, n_total, iteration)

    def adam_step(self, adam, grad):
        from oracle import oracle as O
        self.t += 1
        self.params, self.m, self.v = O.adam_update(self.params, grad.numpy().astype(np.float64), self.m, self.v,
                                                    self.t, lr=adam["lr"])


def _step_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_1903_07145_gb300.parallel import sharded_step
        sc = _scene()
        osc = O.OracleScene(sc)
        rng = np.random.default_rng(0)
        targets = [rng.uniform(0, 1, (c.width * c.height, 3)) for c in sc.cameras]
        tr = _OracleTracer(osc, sc.gt_params.astype(np.float64) * 0.9, targets)
        losses = [sharded_step(tr, None, {"lr": 1e-2}, it) for it in range(3)]
        q.put((rank, losses, tr.params))
    finally:
        dist.destroy_process_group()


def test_sharded_step_equals_unsharded_optimisation():
    """Three iterations of parallel.sharded_step on two gloo ranks: every rank
    ends with the same parameters, and they equal three unsharded oracle
    iterations (loss, gradient cast to FP32 as a GPU rank hands it to Adam,
    Adam)."""
    from oracle import oracle as O
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_step_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict((r, (l, p)) for r, l, p in (q.get(timeout=300) for _ in range(world)))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert np.array_equal(got[0][1], got[1][1])
    sc = _scene()
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(0)
    targets = [rng.uniform(0, 1, (c.width * c.height, 3)) for c in sc.cameras]
    p = sc.gt_params.astype(np.float64) * 0.9
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    n = int(osc.offsets[-1])
    for it in range(3):
        loss, grad = _oracle_shard(osc, p, targets, 0, n, n, it)
        assert abs(got[0][0][it] - loss) <= 1e-12 * abs(loss)
        p, m, v = O.adam_update(p, grad.astype(np.float32).astype(np.float64), m, v, it + 1, lr=1e-2)
    assert np.allclose(got[0][1], p, rtol=0, atol=1e-7), np.abs(got[0][1] - p).max()
