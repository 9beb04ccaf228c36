"""Stochastic pixel batches (Sec. 4.5) on the CUDA path, through the C ABI:
the draw is bit-identical to the oracle's, the batch loss and gradient match
the FP64 oracle on the same sample counters (including batches that draw a
pixel several times), a batch of scenes gives every member what it gets
alone, and optimisation on pixel batches lowers the loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_1903_07145_gb300 import _lib as L  # noqa: E402
from paper_1903_07145_gb300 import scenes  # noqa: E402
from paper_1903_07145_gb300.batch import SceneSet  # noqa: E402
from paper_1903_07145_gb300.tracer import AdamOptions, CacheOptions, TraceOptions, Tracer  # noqa: E402

pytestmark = pytest.mark.gpu
SEED = 0x1903_0714


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


def two_view_cornell(w, h):
    sc = scenes.cornell_box(1000, w, h)
    cam = sc.cameras[0]
    cam2 = scenes.Camera(np.array(cam.cam_to_world, np.float64).copy(), 50.0, w, h)
    sc.cameras = [cam, cam2]
    return sc


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_pick_matches_oracle(built):
    sc = two_view_cornell(24, 20)
    tr = Tracer(sc, seed=SEED)
    n = 2 * 24 * 20
    for it in (0, 1, 77, 1 << 23):
        got = tr.pick_pixels(1000, it).cpu().numpy().astype(np.uint32)
        assert np.array_equal(got, O.pick_pixels(n, 1000, it, seed=SEED, scene_id=0)), it
    tr.close()


@pytest.mark.parametrize("integrator", ["wavefront", "megakernel"])
@pytest.mark.parametrize("loss,same_set,batch", [("l2", False, 600), ("l1", False, 600), ("l2", True, 600),
                                                 ("l2", False, 300)])
def test_batch_loss_and_gradient_match_oracle(built, loss, same_set, batch, integrator):
    """batch 300 over 2 x 12 x 10 = 240 pixels draws most pixels more than once:
    each entry keeps its own samples and upstream gradient."""
    w, h = (12, 10) if batch == 300 else (32, 24)
    sc = two_view_cornell(w, h)
    rng = np.random.default_rng(4)
    targets = [rng.uniform(0.0, 0.8, (w * h, 3)) for _ in range(2)]
    p = sc.gt_params.astype(np.float64).copy()
    p[:, 0:3] = rng.uniform(0.2, 0.8, (sc.n_segments, 3))
    spp_r, spp_d, D = 16, 4, 3
    it = 9
    osc = O.OracleScene(sc)
    lo, go, ids = O.loss_grad_batch(osc, p, targets, batch, spp_r, spp_d, D, iteration=it, seed=SEED, loss=loss,
                                    same_set=same_set)
    if batch == 300:
        assert len(np.unique(ids)) < batch
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator)
    tr.set_params(p.astype(np.float32))
    tr.set_targets(torch.from_numpy(np.concatenate(targets).astype(np.float32)).cuda())
    opts = TraceOptions(spp_r=spp_r, spp_d=spp_d, max_depth=D, loss=loss, gradcheck_same_set=same_set,
                        pixel_batch=batch)
    lg, gg = tr.loss_grad(opts, iteration=it)
    gg = gg.cpu().numpy().astype(np.float64)
    assert abs(lg - lo) <= 1e-3 * abs(lo), (lg, lo)
    cos = float((gg * go).sum() / (np.linalg.norm(gg) * np.linalg.norm(go)))
    assert cos >= 0.999 and rel(gg, go) <= 1e-2, (cos, rel(gg, go))
    tr.close()


def test_batch_of_scenes_equals_members_alone(built):
    scs = [scenes.cornell_box(1000, 24, 20),
           scenes.indoor_room(21, n_cuboids=5, cuboid_sub=2, room_sub=3, n_lights=2, n_views=2, width=30, height=22)]
    ss = SceneSet(scs, seed=5)
    ss.configure("wavefront")
    for i, sc in enumerate(scs):
        ss.set_params(i, sc.gt_params)
        ss.set_targets(i, ss.render(i, TraceOptions(max_depth=3), spp=32))
        ss.set_params(i, scenes.initial_params(sc, 0.5))
    opts = TraceOptions(spp_r=32, spp_d=2, max_depth=3, pixel_batch=64)
    adam = AdamOptions()
    init = [ss.params(i) for i in range(2)]
    ref = [[ss.step(i, opts, adam) for _ in range(3)] for i in range(2)]
    ref_params = [ss.params(i) for i in range(2)]
    for i in range(2):
        ss.set_params(i, init[i])
    ss.make_batch()
    losses = [ss.batch_step(opts, adam) for _ in range(3)]
    for i in range(2):
        assert abs(losses[0][i] - ref[i][0]) <= 1e-6 * abs(ref[i][0]), i
        d = np.abs(ss.batch_params(i) - ref_params[i])
        assert np.mean(d < 1e-5) >= 0.95 and d.max() <= 6 * adam.lr, (i, d.max())
    ss.close()


def test_pixel_batch_optimisation_lowers_the_loss(built):
    sc = scenes.cornell_box(1000, 32, 32)
    tr = Tracer(sc, seed=SEED)
    tr.set_params(sc.gt_params)
    tr.set_targets(tr.render(TraceOptions(max_depth=3), set_id=L.IPT_SET_TARGET, spp=256))
    tr.set_params(scenes.initial_params(sc, 0.5))
    opts = TraceOptions(spp_r=64, spp_d=1, max_depth=3, pixel_batch=128)
    full = TraceOptions(spp_r=16, spp_d=1, max_depth=3)
    before = tr.loss_grad(full, iteration=10_000)[0]
    for _ in range(300):
        tr.step(opts, AdamOptions(lr=2e-2), want_loss=False)
    after = tr.loss_grad(full, iteration=10_001)[0]
    assert after < 0.5 * before, (before, after)
    tr.close()


def test_pixel_batch_argument_checks(built):
    sc = scenes.cornell_box(1000, 8, 8)
    tr = Tracer(sc, seed=1)
    tr.set_params(sc.gt_params)
    tr.set_targets(torch.zeros((64, 3), device="cuda"))
    with pytest.raises(L.IptError):
        tr.render(TraceOptions(pixel_batch=4), set_id=0, spp=4)
    with pytest.raises(L.IptError):
        tr.loss_grad(TraceOptions(spp_r=1 << 20, spp_d=1, pixel_batch=1 << 12))
    tr.configure_cache(CacheOptions(enabled=True, b_term=1))
    with pytest.raises(L.IptError):
        tr.loss_grad(TraceOptions(spp_r=4, spp_d=4, pixel_batch=8))
    tr.close()
