"""Pins for the oracle's stochastic pixel batches (Sec. 4.5: B pixels drawn
uniformly from all pixels of all images per step): the integer pixel map,
uniformity of the draw, the per-entry sample offsets, the batch gradient
against central differences of the batch loss, and the batch loss as an
unbiased estimate of the full-image loss."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_07145_gb300 import scenes


def cornell(w, h, views=1):
    sc = scenes.cornell_box(1000, w, h)
    if views > 1:
        cam = sc.cameras[0]
        sc.cameras = [cam] * views
    return sc


def test_pick_map_is_the_top_bits_for_a_power_of_two():
    """floor(x * 2^k / 2^32) is the top k bits of x: the map is the
    multiply-shift of the full 32-bit word (not a 24-bit uniform, not x mod n)."""
    for k in (1, 5, 12, 20):
        ids = O.pick_pixels(1 << k, 64, iteration=3, seed=99, scene_id=2)
        for b in range(64):
            x = int(O.philox4x32_10([b, 0, (4 << 24) | 3, 0], [99, 2])[0])
            assert ids[b] == x >> (32 - k)


def test_pick_is_uniform_over_all_pixels():
    """Chi-square of 37 pixel counts over 20,000 draws (36 degrees of freedom;
    the 1e-6 tail is at 84)."""
    n, counts = 37, np.zeros(37)
    for it in range(40):
        ids = O.pick_pixels(n, 500, iteration=it, seed=5)
        assert ids.max() < n
        counts += np.bincount(ids, minlength=n)
    e = counts.sum() / n
    chi2 = float(((counts - e) ** 2 / e).sum())
    assert chi2 < 84.0, chi2


def test_pick_depends_on_iteration_seed_and_scene():
    a = O.pick_pixels(10**6, 256, iteration=0, seed=1)
    assert not np.array_equal(a, O.pick_pixels(10**6, 256, iteration=1, seed=1))
    assert not np.array_equal(a, O.pick_pixels(10**6, 256, iteration=0, seed=2))
    assert not np.array_equal(a, O.pick_pixels(10**6, 256, iteration=0, seed=1, scene_id=1))


def test_sample_base_selects_the_sample_range():
    """Sum over samples [k*s, (k+1)*s) = sum over [0, (k+1)*s) - sum over [0, k*s):
    an entry with sample base k*s integrates exactly those samples."""
    sc = cornell(8, 8)
    osc = O.OracleScene(sc)
    p = sc.gt_params.astype(np.float64)
    px = np.array([0, 9, 27, 63, 27], np.uint32)
    s, k = 3, 2
    kw = dict(max_depth=3, seed=4, set_id=1, iteration=7)
    part, _ = osc.render(p, pixels=px, sample_base=np.full(5, k * s, np.uint32), spp=s, **kw)
    hi, _ = osc.render(p, pixels=px, spp=(k + 1) * s, **kw)
    lo, _ = osc.render(p, pixels=px, spp=k * s, **kw)
    assert np.allclose(part * s, hi * (k + 1) * s - lo * k * s, rtol=1e-12, atol=1e-12)
    # and the gradient of those samples likewise
    rng = np.random.default_rng(3)
    w = rng.normal(size=(5, 3))
    gp = osc.gradient(p, w, pixels=px, sample_base=np.full(5, k * s, np.uint32), spp=s, **kw)
    gh = osc.gradient(p, w, pixels=px, spp=(k + 1) * s, **kw)
    gl = osc.gradient(p, w, pixels=px, spp=k * s, **kw)
    assert np.allclose(gp * s, gh * (k + 1) * s - gl * k * s, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("loss", ["l2", "l1"])
def test_batch_gradient_matches_central_differences(loss):
    """With the residual and derivative drawing the same samples (same_set,
    spp_r = spp_d) and sampling frozen, the batch gradient is the exact
    derivative of the batch loss: central differences over 12 parameters."""
    sc = cornell(10, 10, views=2)
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(8)
    p0 = sc.gt_params.astype(np.float64).copy()
    p0[:, 7:10] += rng.uniform(0.0, 0.2, (sc.n_segments, 3))
    targets = [rng.uniform(0.0, 1.0, (100, 3)) for _ in range(2)]
    kw = dict(batch=24, spp_r=3, spp_d=3, max_depth=3, iteration=5, seed=17, loss=loss, same_set=True,
              sparams=p0)
    _, grad, ids = O.loss_grad_batch(osc, p0, targets, **kw)
    h = 1e-6
    for k in rng.choice(sc.n_segments * 10, 12, replace=False):
        pp = p0.copy().reshape(-1)
        pm = p0.copy().reshape(-1)
        pp[k] += h
        pm[k] -= h
        lp, _, _ = O.loss_grad_batch(osc, pp.reshape(p0.shape), targets, **kw)
        lm, _, _ = O.loss_grad_batch(osc, pm.reshape(p0.shape), targets, **kw)
        fd = (lp - lm) / (2 * h)
        g = grad.reshape(-1)[k]
        assert abs(fd - g) <= 1e-5 * max(abs(g), 1e-3 * np.abs(grad).max()), (k, fd, g)


def test_batch_loss_is_an_unbiased_estimate_of_the_full_loss():
    """The mean over many draws of the batch loss (normalised by its 3B
    entry-channels) approaches the mean of the full-image loss at the same
    spp (normalised by the 3N pixel-channels): both estimate
    (1/3N) sum_p E[(I_p - T_p)^2]."""
    sc = cornell(8, 8, views=2)
    osc = O.OracleScene(sc)
    p = sc.gt_params.astype(np.float64) * 0.7
    rng = np.random.default_rng(1)
    targets = [rng.uniform(0.0, 0.6, (64, 3)) for _ in range(2)]
    batch = [O.loss_grad_batch(osc, p, targets, 32, 2, 1, 3, iteration=it, seed=3)[0] for it in range(300)]
    full = [O.loss_grad(osc, p, targets, 2, 1, 3, iteration=it, seed=3)[0] for it in range(30)]
    mb, mf = np.mean(batch), np.mean(full)
    se = np.std(batch) / np.sqrt(len(batch)) + np.std(full) / np.sqrt(len(full))
    assert abs(mb - mf) < 4 * se + 1e-3 * mf, (mb, mf, se)
