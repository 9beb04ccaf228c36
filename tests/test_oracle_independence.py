"""Pins for the oracle's independent residual and derivative sample sets
(Sec. 3.3: the L2 gradient 2 (I_R - I_C) dI_R/dtheta, estimated as a product
of two Monte Carlo estimates, is unbiased only when the two estimates are
independent).

* Set 0 x set 1 (``oracle.loss_grad``): its mean over many iterations equals
  the gradient of the expected image's loss, 2/N sum_j (Ibar_j - I_C,j)
  dIbar_j/dtheta, taken from high-spp renders with their own independent
  sets.
* Set 0 x set 0 (``same_set=True``): biased by the covariance of the two
  factors.  For a segment that is the only emitter, the image is exactly
  linear in its emission (I = e X with X free of e, sampling held at theta_s),
  so dI/de = I / e and Cov(I, dI/de) = Var(I) / e: the bias of the emission
  gradient is 2/N sum_j Var_j / (e spp), with Var_j the per-sample variance of
  pixel j, which a high-spp render gives independently.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_07145_gb300 import scenes

D = 2          # scattering events
K = 1000       # iterations averaged (spp 1 + 1 each)
HI = 2048      # samples per reference batch
NB = 8         # independent reference batches


@pytest.fixture(scope="module")
def setup():
    sc = scenes.cornell_box(1000, 8, 8)
    osc = O.OracleScene(sc)
    p = np.asarray(sc.gt_params, np.float64)
    light = int(np.argmax(p[:, 7:10].sum(1)))
    assert np.count_nonzero(p[:, 7:10].sum(1)) == 1
    # captured image: a high-spp render at other diffuse albedos, so the
    # residual is not zero
    q = p.copy()
    q[:, 0:3] = np.clip(q[:, 0:3] * 0.8 + 0.05, 0.0, 1.0)
    tgt, _ = osc.render(q, spp=4096, max_depth=D, set_id=O.SET_TARGET, seed=5)
    n = tgt.size
    # reference gradient of the expected image's loss: NB batches, each the
    # product of a set-0 image and a set-1 Jacobian at iterations no test
    # iteration uses
    refs, var = [], np.zeros_like(tgt)
    for b in range(NB):
        it = (1 << 23) + b
        img, msq = osc.render(p, spp=HI, max_depth=D, set_id=O.SET_RESIDUAL, iteration=it, seed=3)
        var += np.maximum(msq - img * img, 0.0) / NB
        w = 2.0 * (img - tgt) / n
        refs.append(osc.gradient(p, w, spp=HI, max_depth=D, set_id=O.SET_DERIVATIVE, iteration=it, seed=3))
    refs = np.array(refs)
    g_ref = refs.mean(0)
    se_ref = refs.std(0, ddof=1) / np.sqrt(NB)
    return osc, p, tgt, light, g_ref, se_ref, var, n


def _mean_grad(osc, p, tgt, same_set):
    gs = np.array([O.loss_grad(osc, p, [tgt], 1, 1, D, iteration=it, seed=11, same_set=same_set)[1]
                   for it in range(K)])
    return gs.mean(0), gs.std(0, ddof=1) / np.sqrt(K)


def test_independent_sets_unbiased(setup):
    osc, p, tgt, light, g_ref, se_ref, _, _ = setup
    m, se = _mean_grad(osc, p, tgt, same_set=False)
    z = (m - g_ref) / np.sqrt(se * se + se_ref * se_ref + 1e-30)
    # 70 components at 4.5 sigma: a chance failure is below 1e-3
    assert np.max(np.abs(z)) < 4.5, np.max(np.abs(z))
    # the check has power: the light's emission gradient is far from zero
    assert np.all(np.abs(g_ref[light, 7:10]) > 4 * se_ref[light, 7:10])


def test_same_set_biased_by_the_covariance(setup):
    osc, p, tgt, light, g_ref, se_ref, var, n = setup
    m, se = _mean_grad(osc, p, tgt, same_set=True)
    e = p[light, 7:10]
    bias_pred = 2.0 / n * var.sum(0) / e          # spp 1: Cov = Var / e
    d = m[light, 7:10] - g_ref[light, 7:10]
    s = np.sqrt(se[light, 7:10] ** 2 + se_ref[light, 7:10] ** 2)
    # measurably biased ...
    assert np.all(d > 20 * s), d / s
    # ... by the predicted covariance (the variance estimate from NB x HI
    # samples carries a few tenths of a percent of error)
    assert np.all(np.abs(d - bias_pred) < 4.5 * s + 0.01 * bias_pred), (d, bias_pred, s)
