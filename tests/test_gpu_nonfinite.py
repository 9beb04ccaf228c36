"""Non-finite guard of the Adam step: a NaN or infinite loss or gradient
(here from a NaN pixel planted in the captured image on the host, or a NaN
planted in a gradient handed to ipt_adam_step) makes the step a no-op on the
device -- parameters, Adam moments and step count stay those of the last good
step -- and the next synchronising call returns IPT_ERR_NONFINITE.  Nothing
faults: the check is arithmetic in the Adam kernels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1903_07145_gb300 import _lib as L  # noqa: E402
from paper_1903_07145_gb300 import scenes  # noqa: E402
from paper_1903_07145_gb300.batch import SceneSet  # noqa: E402
from paper_1903_07145_gb300.tracer import AdamOptions, TraceOptions, Tracer  # noqa: E402

pytestmark = pytest.mark.gpu
NONFINITE = 5
HEADER = 64  # checkpoint header (counters); the arrays follow it


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


def _target(tr, sc):
    tr.set_params(sc.gt_params)
    t = tr.render(TraceOptions(max_depth=3), set_id=L.IPT_SET_TARGET, spp=64)
    tr.set_params(scenes.initial_params(sc, 0.5))
    return t


@pytest.mark.parametrize("integrator", ["megakernel", "wavefront"])
def test_nan_target_pixel_skips_the_step(built, integrator):
    sc = scenes.cornell_box(1000, 16, 16)
    tr = Tracer(sc, seed=3)
    tr.configure(integrator)
    good = _target(tr, sc)
    tr.set_targets(good)
    opts, adam = TraceOptions(spp_r=8, spp_d=8, max_depth=3), AdamOptions(lr=1e-2)
    tr.step(opts, adam)                       # non-zero Adam moments
    before_p, before_ck = tr.get_params(), tr.checkpoint()
    bad = good.clone()
    bad[37, 1] = float("nan")
    tr.set_targets(bad)
    with pytest.raises(L.IptError) as e:
        tr.step(opts, adam)
    assert e.value.status == NONFINITE
    assert np.array_equal(tr.get_params(), before_p)
    # parameters, free mask and both Adam moments unchanged; the header's
    # step count too (only the sample iteration counter advanced)
    after_ck = tr.checkpoint()
    assert after_ck[HEADER:] == before_ck[HEADER:]
    # the error is reported once; a finite target steps again
    tr.set_targets(good)
    tr.step(opts, adam)
    assert not np.array_equal(tr.get_params(), before_p)
    tr.close()


def test_nan_gradient_to_adam_step_is_rejected(built):
    sc = scenes.cornell_box(1000, 16, 16)
    tr = Tracer(sc, seed=3)
    tr.set_params(scenes.initial_params(sc, 0.5))
    g = torch.full((sc.n_segments, 10), 0.1, device="cuda")
    tr.adam_step(AdamOptions(), g)
    tr.synchronize()
    before = tr.checkpoint()
    g[2, 4] = float("inf")
    tr.adam_step(AdamOptions(), g)
    with pytest.raises(L.IptError) as e:
        tr.synchronize()
    assert e.value.status == NONFINITE
    assert tr.checkpoint() == before          # header (step count) included
    g[2, 4] = 0.1
    tr.adam_step(AdamOptions(), g)
    tr.synchronize()
    assert tr.checkpoint() != before
    tr.close()


def test_nan_gradient_wide_scene(built):
    """Above 4096 segments Adam runs over a grid behind a separate check."""
    sc = scenes.per_triangle(scenes.indoor_room(3, n_cuboids=8, cuboid_sub=4, room_sub=16, n_lights=1,
                                                n_views=1, width=8, height=8))
    assert sc.n_segments > 4096
    tr = Tracer(sc, seed=1)
    tr.set_params(sc.start_params)
    g = torch.full((sc.n_segments, 10), 0.05, device="cuda")
    tr.adam_step(AdamOptions(), g)
    tr.synchronize()
    before = tr.checkpoint()
    g[sc.n_segments - 1, 9] = float("nan")
    tr.adam_step(AdamOptions(), g)
    with pytest.raises(L.IptError) as e:
        tr.synchronize()
    assert e.value.status == NONFINITE
    assert tr.checkpoint() == before
    tr.close()


def test_batch_member_with_nan_target_is_held(built):
    scs = [scenes.cornell_box(1000, 16, 16), scenes.cornell_variant(1), scenes.cornell_variant(2)]
    opts, adam = TraceOptions(spp_r=4, spp_d=4, max_depth=3), AdamOptions(lr=1e-2)

    def prepared(plant):
        ss = SceneSet(scs, seed=9)
        ss.configure("wavefront")
        for i, sc in enumerate(scs):
            ss.set_params(i, sc.gt_params)
            t = ss.render(i, TraceOptions(max_depth=3), spp=16)
            if plant and i == 1:
                t[5, 0] = float("nan")
            ss.set_targets(i, t)
            ss.set_params(i, scenes.initial_params(sc, 0.5))
        ss.make_batch()
        return ss

    ref = prepared(False)
    ref.batch_step(opts, adam)
    ss = prepared(True)
    with pytest.raises(L.IptError) as e:
        ss.batch_step(opts, adam)
    assert e.value.status == NONFINITE
    # the member with the NaN keeps its start; the others step as in a clean batch
    assert np.array_equal(ss.batch_params(1), scenes.initial_params(scs[1], 0.5).astype(np.float32))
    for i in (0, 2):
        assert np.array_equal(ss.batch_params(i), ref.batch_params(i))


def test_disney_nan_target_skips_the_step(built):
    sc = scenes.cornell_box(1000, 16, 16)
    tr = Tracer(sc, seed=3)
    p = scenes.disney_materials(sc, 2)
    tr.disney_set_params(p)
    t = tr.disney_render(TraceOptions(max_depth=2), set_id=L.IPT_SET_TARGET, spp=16)
    t[3, 2] = float("inf")
    tr.set_targets(t)
    q = p.copy()
    q[:, 0:3] = 0.5
    tr.disney_set_params(q)
    with pytest.raises(L.IptError) as e:
        tr.disney_step(TraceOptions(spp_r=4, spp_d=4, max_depth=2), AdamOptions())
    assert e.value.status == NONFINITE
    assert np.array_equal(tr.disney_params(), q.astype(np.float32))
    tr.close()
