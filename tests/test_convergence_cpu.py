"""Host logic of the time-to-error driver: which parameters are free and
which the error scores (SURVEY's parameter error: diffuse and specular
albedo and emission of seen segments, roughness where the true specular
albedo has luminance >= 0.05)."""
import numpy as np
import pytest

from paper_1903_07145_gb300 import convergence, metrics, scenes


def test_unknowns_masks():
    sc = scenes.cornell_box(1000, 8, 8)
    kd_e = convergence.unknowns_mask(sc, "kd_e")
    kd = convergence.unknowns_mask(sc, "kd")
    mat = convergence.unknowns_mask(sc, "material")
    assert kd_e[:, [0, 1, 2, 7, 8, 9]].all() and not kd_e[:, 3:7].any()
    assert kd[:, 0:3].all() and not kd[:, 3:].any()
    assert mat[:, 0:7].all() and not mat[:, 7:].any()
    with pytest.raises(ValueError):
        convergence.unknowns_mask(sc, "all")


def test_survey_score_is_the_identifiable_set_among_the_unknowns():
    sc = scenes.cornell_box(1000, 8, 8)
    gt = np.asarray(sc.gt_params, np.float64).copy()
    gt[2, 3:6] = 0.01          # a dim specular lobe: its roughness is not scored
    gt[3, 3:6] = 0.2
    sc.gt_params = gt.astype(np.float32)
    visible = np.ones(sc.n_segments, bool)
    visible[5] = False
    free = convergence.unknowns_mask(sc, "material")
    m = convergence.scored_mask(sc, free, visible, "survey")
    assert np.array_equal(m, metrics.identifiable_mask(sc.gt_params, visible) & free)
    assert not m[5].any()                  # unseen segment
    assert not m[2, 6] and m[3, 6]         # roughness only where lum(ks) >= 0.05
    assert not m[:, 7:].any()              # emission held, so not scored
    # the legacy score leaves the lights' diffuse albedo out
    leg = convergence.scored_mask(sc, convergence.unknowns_mask(sc, "kd_e"), visible)
    assert not leg[np.asarray(sc.light_segments, int), 0:3].any()
