"""The paper's optimiser ablation on the CUDA path (Sec. 5, Fig. plot_srays
and plot_mis): at equal optimisation time, a single colour path per pixel
does not converge under the L1 loss while 128 do, and light sampling without
MIS converges far worse than with it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from dataclasses import replace  # noqa: E402

from paper_1903_07145_gb300 import ablation, scenes  # noqa: E402
from paper_1903_07145_gb300.tracer import AdamOptions  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


def tail_error(curve):
    t = curve[-max(1, len(curve) // 4):]
    return float(np.mean([c[2] for c in t]))


def test_single_path_and_no_mis_fail(built):
    sc = scenes.cornell_box(1000, 64, 64)
    adam = AdamOptions(lr=1e-2)
    run = {name: ablation.curve(sc, o, adam, 2.0, o.max_depth, points=12)
           for name, o in [("one path", replace(ablation.BASE, spp_r=1)), ("128 paths", ablation.BASE),
                           ("no mis", replace(ablation.BASE, mis=False))]}
    for name, c in run.items():
        assert c[0][0] == 0 and c[-1][1] >= 2.0 and all(b[1] >= a[1] for a, b in zip(c, c[1:])), name
    e = {k: tail_error(v) for k, v in run.items()}
    assert e["128 paths"] < 0.05, e
    assert e["one path"] > 3 * e["128 paths"], e
    assert e["no mis"] > 3 * e["128 paths"], e
