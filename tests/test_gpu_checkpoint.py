"""Checkpoints: an optimisation saved after some steps and loaded into a
fresh context continues as the original does (same losses and parameters up
to the float-summation noise the batch tests also allow), with and without
the radiance cache; malformed or mismatched checkpoints are rejected before
any state changes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_07145_gb300 import _lib as L  # noqa: E402
from paper_1903_07145_gb300 import scenes  # noqa: E402
from paper_1903_07145_gb300.tracer import AdamOptions, CacheOptions, TraceOptions, Tracer  # noqa: E402

pytestmark = pytest.mark.gpu
OPTS = TraceOptions(spp_r=8, spp_d=8, max_depth=3)
ADAM = AdamOptions(lr=1e-2)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


def fresh(sc, target, cache):
    tr = Tracer(sc, seed=11)
    tr.configure("wavefront")
    tr.set_targets(target)
    if cache:
        tr.configure_cache(CacheOptions(enabled=True, b_term=1, train_spp=2, train_steps=2))
    return tr


@pytest.mark.parametrize("cache", [False, True])
def test_resume_continues_the_run(built, cache):
    sc = scenes.cornell_box(1000, 32, 32)
    t0 = Tracer(sc, seed=11)
    t0.set_params(sc.gt_params)
    target = t0.render(OPTS, set_id=L.IPT_SET_TARGET, spp=256)
    t0.close()
    a = fresh(sc, target, cache)
    a.set_params(scenes.initial_params(sc, 0.5))
    for _ in range(6):
        a.step(OPTS, ADAM)
    ck = a.checkpoint()
    b = fresh(sc, target, cache)
    b.restore(ck)
    # the state round-trips exactly
    assert np.array_equal(b.get_params(), a.get_params())
    assert b.checkpoint() == ck
    if cache:
        (wa, ta), (wb, tb) = a.cache_weights(table=True), b.cache_weights(table=True)
        assert np.array_equal(wa, wb) and np.array_equal(ta, tb)
    ref_loss = [a.step(OPTS, ADAM) for _ in range(4)]
    ref_params = a.get_params()
    loss = [b.step(OPTS, ADAM) for _ in range(4)]
    # the first resumed step sees identical parameters, tables and sample sets
    assert abs(loss[0] - ref_loss[0]) <= 1e-6 * abs(ref_loss[0]), (loss[0], ref_loss[0])
    # later steps differ by the order of float atomics; with the cache, Adam's
    # normalisation turns that noise on near-zero hash-table gradients into
    # full-size steps of either sign, so the cached estimate drifts further
    tol = 1e-2 if cache else 1e-3
    for i in range(1, 4):
        assert abs(loss[i] - ref_loss[i]) <= tol * abs(ref_loss[i]), (i, loss[i], ref_loss[i])
    d = np.abs(b.get_params() - ref_params)
    assert np.mean(d < 1e-5) >= 0.95 and d.max() <= 6 * ADAM.lr
    if cache:
        assert b.cache_status()["train_steps"] == a.cache_status()["train_steps"]
        dw = np.abs(a.cache_weights() - b.cache_weights())
        assert np.mean(dw < 1e-3) >= 0.95 and dw.max() <= 0.1  # training noise of float atomics
    a.close()
    b.close()


def test_bad_checkpoints_are_rejected(built):
    sc = scenes.cornell_box(1000, 16, 16)
    a = Tracer(sc, seed=1)
    a.set_params(sc.gt_params)
    ck = a.checkpoint()
    p = a.get_params()
    with pytest.raises(L.IptError):
        a.restore(ck[:-1])                      # wrong size
    with pytest.raises(L.IptError):
        a.restore(b"NOTACKPT" + ck[8:])          # wrong magic
    other = scenes.furnace_box()
    b = Tracer(other, seed=1)
    with pytest.raises(L.IptError):
        b.restore(ck)                           # segment count differs
    c = Tracer(sc, seed=1)
    c.configure_cache(CacheOptions(enabled=True, b_term=1))
    ck_cache = c.checkpoint()
    with pytest.raises(L.IptError):
        a.restore(ck_cache)                     # carries a cache the target lacks
    assert np.array_equal(a.get_params(), p)    # nothing changed
    for t in (a, b, c):
        t.close()


def test_disney_state_round_trips(built):
    """A checkpoint carries the Disney parameters and optimiser state: a fresh
    context restored from it steps exactly as the original."""
    sc = scenes.cornell_box(1000, 24, 24)
    truth = scenes.disney_materials(sc, 2)
    a = Tracer(sc, seed=3)
    a.disney_set_params(truth)
    target = a.disney_render(TraceOptions(max_depth=3), set_id=L.IPT_SET_TARGET, spp=64)
    a.set_targets(target)
    p0 = truth.copy()
    p0[:, 0:3] = 0.5
    a.disney_set_params(p0)
    opts = TraceOptions(spp_r=8, spp_d=4, max_depth=3)
    for _ in range(5):
        a.disney_step(opts, ADAM)
    ck = a.checkpoint()
    b = Tracer(sc, seed=3)
    b.set_targets(target)
    b.restore(ck)
    assert np.array_equal(b.disney_params(), a.disney_params())
    assert b.checkpoint() == ck
    la, lb = a.disney_step(opts, ADAM), b.disney_step(opts, ADAM)
    assert abs(la - lb) <= 1e-6 * abs(la), (la, lb)
    a.close()
    b.close()
