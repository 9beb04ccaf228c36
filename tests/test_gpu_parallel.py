"""parallel.sharded_step on the CUDA path over NCCL, with one rank (a shard
holding every pixel): the same paths, gradient, loss and Adam step as the
unsharded ipt_step, up to the rounding of the gradient's float sums.  Several ranks are covered on the CPU with gloo
(tests/test_parallel_cpu.py); on one GPU no rank waits for another."""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import torch.distributed as dist  # noqa: E402

from paper_1903_07145_gb300 import scenes  # noqa: E402
from paper_1903_07145_gb300.parallel import sharded_step  # noqa: E402
from paper_1903_07145_gb300.tracer import AdamOptions, TraceOptions, Tracer  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


def test_one_rank_sharded_step_equals_step(built):
    if not dist.is_nccl_available():
        pytest.skip("torch without NCCL")
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        sc = scenes.cornell_box(1000, 32, 32)
        opts = TraceOptions(spp_r=8, spp_d=8, max_depth=3)
        adam = AdamOptions(lr=1e-2)
        out = []
        for sharded in (False, True):
            tr = Tracer(sc, seed=5)
            tr.set_params(sc.gt_params)
            tr.set_targets(tr.render(opts, set_id=2, spp=64))
            tr.set_params(scenes.initial_params(sc, 0.5))
            losses = []
            for it in range(3):
                if sharded:
                    losses.append(sharded_step(tr, opts, adam, it))
                else:
                    # ipt_step draws iteration `it` from its own counter, as the shard call is given it
                    losses.append(tr.step(opts, adam))
            out.append((losses, tr.get_params()))
            tr.close()
        (l0, p0), (l1, p1) = out
        # the first loss comes from identical paths and parameters; later ones
        # from parameters that differ only where the float sums of the
        # gradient (accumulated in a scheduling-dependent order) round
        # differently and Adam normalised a gradient at that noise level
        assert abs(l0[0] - l1[0]) <= 1e-9 * abs(l0[0]), (l0, l1)
        assert np.allclose(l0, l1, rtol=1e-4, atol=0), (l0, l1)
        d = np.abs(p0 - p1)
        assert np.mean(d < 1e-5) >= 0.95 and d.max() <= 6 * adam.lr, d.max()
    finally:
        dist.destroy_process_group()
