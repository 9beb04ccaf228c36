"""The optimiser-ablation settings (Sec. 5 and App. A) are the experiments
they name: the paths sweep varies only the colour paths, the split keeps the
128-path budget, the batch sweep varies only the batch size, the MIS sweep
switches light sampling and MIS, and the bounces sweep fits depths 1-3 to a
10-bounce target; every setting optimises the L1 loss."""
from dataclasses import asdict

from paper_1903_07145_gb300 import ablation


def differing(a, b):
    da, db = asdict(a), asdict(b)
    return {k for k in da if da[k] != db[k]}


def test_sweeps_vary_one_thing():
    base = ablation.BASE
    assert base.loss == "l1" and base.spp_d == 1 and base.pixel_batch > 0
    for kind, allowed in (("paths", {"spp_r"}), ("batch", {"pixel_batch"}), ("bounces", {"max_depth"}),
                          ("mis", {"nee", "mis"}), ("split", {"spp_r", "spp_d"})):
        for _, o in ablation.SWEEPS[kind]:
            assert differing(base, o) <= allowed, (kind, o)
    assert [o.spp_r for _, o in ablation.SWEEPS["paths"]][0] == 1
    assert all(o.spp_r + o.spp_d == 128 for _, o in ablation.SWEEPS["split"])
    assert [o.max_depth for _, o in ablation.SWEEPS["bounces"]] == [1, 2, 3]
    assert ablation.TARGET_DEPTH["bounces"] == 10
    names = [n for s in ablation.SWEEPS.values() for n, _ in s]
    assert len(names) == len(set(names))
