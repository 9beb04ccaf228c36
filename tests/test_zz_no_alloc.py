"""ipt_backward_noalloc: the vector-Jacobian product for callers that may not
allocate device memory when they call it (under stream capture, in real-time
loops, or inside an embedder that owns the memory budget).  Its scratch is a
fixed file-scope device array, so the test checks that it gives the same
gradient as ipt_backward on two calls in a row (the second call must not see
the first call's sums) and that scenes beyond its segment limit are rejected.
This file is collected last so a failure here leaves every other test run."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_backward_noalloc_matches_backward_twice():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_07145_gb300 import _lib as L
    from paper_1903_07145_gb300 import scenes
    from paper_1903_07145_gb300.tracer import TraceOptions, Tracer

    sc = scenes.cornell_box(1000, 32, 32)
    tr = Tracer(sc, seed=11)
    # the reference runs on the integrator the no-allocation call always uses
    tr.configure("megakernel")
    p = sc.gt_params.copy()
    p[:, 7:10] += 0.1
    tr.set_params(p)
    opts = TraceOptions(spp_r=8, spp_d=8, max_depth=3)
    w = torch.randn(tr.n_pix, 3, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    ref = tr.backward(w, opts, set_id=L.IPT_SET_DERIVATIVE)
    torch.cuda.synchronize()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        L.ipt_backward_noalloc(tr.ctx, tr.sid, opts.c(), L.IPT_SET_DERIVATIVE, 0, None, None,
                               C.c_void_p(w.data_ptr()), C.c_void_p(out.data_ptr()))
        tr.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= 1e-5, _rel(out, ref)
    tr.close()


def test_backward_noalloc_rejects_too_many_segments():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1903_07145_gb300 import _lib as L
    from paper_1903_07145_gb300 import scenes
    from paper_1903_07145_gb300.tracer import TraceOptions, Tracer

    # one segment per triangle: 1200 segments, above the 1024 limit
    sc = scenes.indoor_room(3, n_cuboids=1, cuboid_sub=1, room_sub=10, n_lights=1, n_views=1,
                            width=8, height=8)
    sc.tri_segment = np.arange(sc.n_tri, dtype=np.uint32)
    sc.n_segments = sc.n_tri
    sc.gt_params = np.full((sc.n_tri, 10), 0.3, np.float32)
    assert sc.n_segments > 1024
    tr = Tracer(sc, seed=1)
    tr.set_params(sc.gt_params)
    w = torch.ones(tr.n_pix, 3, device="cuda")
    out = torch.empty((sc.n_segments, 10), device="cuda")
    with pytest.raises(L.IptError) as e:
        L.ipt_backward_noalloc(tr.ctx, tr.sid, TraceOptions(spp_d=1).c(), 1, 0, None, None,
                               C.c_void_p(w.data_ptr()), C.c_void_p(out.data_ptr()))
    assert e.value.status == 1
    tr.close()
