"""Seeded input generators: sizes and structure of the workloads' scenes."""
import numpy as np

from paper_1903_07145_gb300 import scenes


def test_cornell_variants_are_uneven_cornell_boxes():
    res = set()
    for k in range(64):
        sc = scenes.cornell_variant(k)
        assert sc.indices.shape[0] == 34 and sc.n_segments == 7 and sc.light_segments == [1]
        assert len(sc.cameras) == 1 and sc.cameras[0].width == sc.cameras[0].height
        res.add(sc.cameras[0].width)
        p = sc.gt_params
        assert np.all((p[:, 0:3] >= 0.1) & (p[:, 0:3] <= 0.9))
        assert np.all(p[np.arange(7) != 1, 7:10] == 0) and np.all(p[1, 7:10] > 0)
        # every vertex stays inside the unit box
        assert sc.positions.min() >= -1e-6 and sc.positions.max() <= 1 + 1e-6
    assert res == {32, 48, 64, 96, 128}
    a, b = scenes.cornell_variant(3), scenes.cornell_variant(3)
    assert np.array_equal(a.positions, b.positions) and np.array_equal(a.gt_params, b.gt_params)
    assert not np.array_equal(a.positions, scenes.cornell_variant(4).positions)
