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


def tri_areas(sc):
    p = np.asarray(sc.positions, np.float64)[np.asarray(sc.indices, np.int64)]
    return 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)


def test_per_triangle_and_subdivision_structure():
    sc = scenes.cornell_textured(1000, 4, 16, 16)
    assert sc.n_tri == 5 * 2 * 16 + 24 and sc.n_segments == 7
    # the checker's mean is the per-object albedo of floor and back wall
    for s in (0, 2):
        assert np.allclose(sc.gt_params[s, 0:3], sc.tri_albedo[sc.tri_segment == s].mean(0), atol=1e-6)
    pt = scenes.per_triangle(sc, params=np.full((7, 10), 0.25, np.float32))
    assert pt.n_segments == sc.n_tri and np.array_equal(pt.tri_segment, np.arange(sc.n_tri))
    assert np.array_equal(pt.gt_params[:, 0:3], sc.tri_albedo)
    assert np.all(pt.start_params == 0.25)
    assert sorted(pt.light_segments) == list(np.nonzero(sc.tri_segment == 1)[0])
    split = np.zeros(pt.n_tri, bool)
    split[[0, 5, 40, 100]] = True
    sd = scenes.subdivide(pt, split)
    assert sd.n_tri == pt.n_tri + 3 * 4
    # children cover their parent's area and inherit its truth and start
    a0, a1 = tri_areas(pt), tri_areas(sd)
    for t in range(pt.n_tri):
        kids = np.nonzero(sd.parent == t)[0]
        assert len(kids) == (4 if split[t] else 1)
        assert np.isclose(a1[kids].sum(), a0[t], rtol=1e-6)
        assert np.all(sd.gt_params[kids] == pt.gt_params[t]) and np.all(sd.start_params[kids] == pt.start_params[t])
    # same winding (geometric normal direction) as the parent
    def normal(s, i):
        p = np.asarray(s.positions, np.float64)[np.asarray(s.indices, np.int64)[i]]
        n = np.cross(p[1] - p[0], p[2] - p[0])
        return n / np.linalg.norm(n)
    for t in np.nonzero(split)[0]:
        for k in np.nonzero(sd.parent == t)[0]:
            assert np.dot(normal(sd, k), normal(pt, t)) > 0.999
