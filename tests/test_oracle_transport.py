"""Pins for the oracle's light transport (Eq. 1-2), its gradient (Eq. 5-6)
and its optimiser, against closed forms, quadrature, exact linearity, finite
differences and torch.optim.Adam."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_07145_gb300 import scenes


# ----------------------------------------------------------------------------
# Furnace: closed box, Lambertian rho, uniform emission E on every face.
# Radiance truncated after D scattering events is E * sum_{k=0..D} rho^k.
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("D", [0, 1, 2, 3, 5])
def test_furnace_exact_with_bsdf_sampling(D):
    sc = scenes.furnace_box(rho=0.6, emission=0.25)
    osc = O.OracleScene(sc)
    m, msq = osc.render(sc.gt_params, spp=64, max_depth=D, nee=False, mis=False, profile=1)
    rho = float(np.float32(0.6))
    expect = 32 * 0.25 * sum(rho ** k for k in range(D + 1))
    # cosine-weighted sampling of a Lambertian surface has weight rho exactly,
    # so every sample equals the closed form
    assert np.max(np.abs(m - expect)) < 1e-10 * expect
    assert np.max(np.abs(msq - expect * expect)) < 1e-9 * expect * expect


@pytest.mark.parametrize("nee,mis", [(True, True), (True, False)])
def test_furnace_in_expectation_with_light_sampling(nee, mis):
    sc = scenes.furnace_box(rho=0.6, emission=0.25, width=8, height=8)
    osc = O.OracleScene(sc)
    D = 3
    spp = 4096
    m, msq = osc.render(sc.gt_params, spp=spp, max_depth=D, nee=nee, mis=mis, profile=1, seed=99)
    expect = 32 * 0.25 * sum(float(np.float32(0.6)) ** k for k in range(D + 1))
    var = np.maximum(msq - m * m, 0)[:, 0]
    se = math.sqrt(var.sum() / spp) / var.size
    assert abs(m[:, 0].mean() - expect) < 4 * se
    if mis:
        # per pixel too (64 pixels: 5 sigma).  Light sampling alone is heavy
        # tailed near the box corners (1/r^2), so only the mean is checked there.
        assert np.all(np.abs(m[:, 0] - expect) < 5 * np.sqrt(var / spp) + 1e-9)


# ----------------------------------------------------------------------------
# Direct light from one triangle onto a Lambertian plane (D = 1).
# ----------------------------------------------------------------------------

def plane_and_triangle_light(x, cam_pos, light):
    pos = np.array([[-20, 0, -20], [20, 0, -20], [20, 0, 20], [-20, 0, 20]] + list(light),
                   np.float64)
    idx = np.array([[0, 3, 2], [0, 2, 1], [4, 5, 6]], np.uint32)   # floor normal +y
    seg = np.array([0, 0, 1], np.uint32)
    f = np.asarray(x, np.float64) - np.asarray(cam_pos, np.float64)
    f /= np.linalg.norm(f)
    right = np.cross(f, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, f)
    cam = scenes.Camera(np.stack([right, up, -f, cam_pos], 1).astype(np.float32), 0.02, 4, 4)
    gt = np.zeros((2, 10), np.float32)
    gt[0, 0:3] = [0.5, 0.4, 0.3]
    gt[:, 6] = 0.5
    gt[1, 7:10] = [0.5, 0.5, 0.5]
    return scenes.Scene("plane_light", pos.astype(np.float32), idx, seg, 2, [cam], gt,
                        light_segments=[1])


LIGHT = [[-0.3, 1.0, -0.2], [0.4, 1.0, -0.1], [0.1, 1.0, 0.5]]   # faces -y


def lambert_polygon_irradiance(x, n, verts):
    """Irradiance from a uniform unit-radiance polygon (Lambert's formula, as in
    Arvo 1995): E = 1/2 sum_k Theta_k (Gamma_k . n)."""
    acc = 0.0
    k = len(verts)
    for i in range(k):
        a = verts[i] - x
        b = verts[(i + 1) % k] - x
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        g = np.cross(a, b)
        g /= np.linalg.norm(g)
        acc += math.acos(np.clip(a @ b, -1, 1)) * (g @ n)
    return 0.5 * abs(acc)


def cosine_profile_irradiance(x, n, verts, order=80):
    """int over the triangle of cos_x cos_y^2 / r^2 dA (Gauss-Legendre on the
    square with the Duffy map)."""
    p0, p1, p2 = [np.asarray(v, np.float64) for v in verts]
    nl = np.cross(p1 - p0, p2 - p0)
    A2 = np.linalg.norm(nl)
    nl /= A2
    g, w = np.polynomial.legendre.leggauss(order)
    g = 0.5 * (g + 1)
    w = 0.5 * w
    tot = 0.0
    for ui, wu in zip(g, w):
        for vi, wv in zip(g, w):
            y = p0 + ui * (p1 - p0) + ui * vi * (p2 - p1)
            d = y - x
            r2 = d @ d
            wl = d / math.sqrt(r2)
            cx = max(0.0, wl @ n)
            cy = max(0.0, -(wl @ nl))
            tot += wu * wv * ui * A2 * cx * cy * cy / r2
    return tot


@pytest.mark.parametrize("nee,mis", [(True, True), (False, False), (True, False)])
def test_direct_light_matches_polygon_formula(nee, mis):
    x = np.array([0.2, 0.0, 0.1])
    sc = plane_and_triangle_light(x, np.array([1.5, 0.8, 0.1]), LIGHT)
    osc = O.OracleScene(sc)
    spp = 65536 if nee else 262144
    m, msq = osc.render(sc.gt_params, spp=spp, max_depth=1, nee=nee, mis=mis, profile=1, seed=5)
    E = lambert_polygon_irradiance(x, np.array([0.0, 1.0, 0.0]), [np.array(v) for v in LIGHT])
    Le = 32 * 0.5
    expect = sc.gt_params[0, 0:3].astype(np.float64) / math.pi * Le * E
    var = np.maximum(msq - m * m, 0)
    se = np.sqrt(var.sum(0) / spp) / m.shape[0]
    assert np.all(np.abs(m.mean(0) - expect) < 4.5 * se), (m.mean(0), expect, se)


def test_direct_light_cosine_profile_matches_quadrature():
    x = np.array([0.2, 0.0, 0.1])
    sc = plane_and_triangle_light(x, np.array([1.5, 0.8, 0.1]), LIGHT)
    osc = O.OracleScene(sc)
    spp = 65536
    m, msq = osc.render(sc.gt_params, spp=spp, max_depth=1, profile=0, seed=6)
    E = cosine_profile_irradiance(x, np.array([0.0, 1.0, 0.0]), LIGHT)
    expect = sc.gt_params[0, 0:3].astype(np.float64) / math.pi * 32 * 0.5 * E
    var = np.maximum(msq - m * m, 0)
    se = np.sqrt(var.sum(0) / spp) / m.shape[0]
    assert np.all(np.abs(m.mean(0) - expect) < 4.5 * se), (m.mean(0), expect, se)


def cornell_small(w=16, h=16):
    return scenes.cornell_box(1000, w, h)


def test_linearity_in_emission():
    """With sampling frozen, every sample is linear in the emission vector:
    I_c(e) = sum_s e_{s,c} I_c(e = 1_s)."""
    sc = cornell_small(12, 12)
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(1)
    p = sc.gt_params.astype(np.float64).copy()
    p[:, 7:10] = rng.uniform(0, 0.6, (sc.n_segments, 3))
    kw = dict(spp=8, max_depth=3, sparams=p, seed=3)
    full, _ = osc.render(p, **kw)
    acc = np.zeros_like(full)
    for s in range(sc.n_segments):
        q = p.copy()
        q[:, 7:10] = 0
        q[s, 7:10] = 1.0
        img, _ = osc.render(q, **kw)
        acc += img * p[s, 7:10][None, :]
    assert np.max(np.abs(acc - full)) <= 1e-12 * np.max(np.abs(full))


def test_emission_gradient_equals_unit_emission_image():
    """dI/de_{s,c} = I_c(e = 1_s) (Eq. 5 on a linear function)."""
    sc = cornell_small(10, 10)
    osc = O.OracleScene(sc)
    p = sc.gt_params.astype(np.float64)
    rng = np.random.default_rng(4)
    w = rng.normal(size=(100, 3))
    kw = dict(spp=4, max_depth=3, seed=8)
    grad = osc.gradient(p, w, sparams=p, **kw)
    for s in range(sc.n_segments):
        q = p.copy()
        q[:, 7:10] = 0
        q[s, 7:10] = 1.0
        img, _ = osc.render(q, sparams=p, **kw)
        expect = (w * img).sum(0)
        assert np.allclose(grad[s, 7:10], expect, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("nee,mis,profile", [(True, True, 0), (False, False, 0), (True, False, 1)])
def test_gradient_matches_central_differences(nee, mis, profile):
    """<w, I(p + h e_k) - I(p - h e_k)> / 2h == (J^T w)_k with sampling frozen at p."""
    sc = cornell_small(10, 10)
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(12)
    p = sc.gt_params.astype(np.float64).copy()
    p[:, 7:10] += rng.uniform(0.0, 0.3, (sc.n_segments, 3))
    w = rng.normal(size=(100, 3))
    kw = dict(spp=4, max_depth=3, nee=nee, mis=mis, profile=profile, seed=21)
    grad = osc.gradient(p, w, sparams=p, **kw)
    h = 1e-5
    ks = rng.choice(sc.n_segments * 10, 20, replace=False)
    for k in ks:
        pp = p.copy().reshape(-1)
        pm = p.copy().reshape(-1)
        pp[k] += h
        pm[k] -= h
        ip, _ = osc.render(pp.reshape(p.shape), sparams=p, **kw)
        im, _ = osc.render(pm.reshape(p.shape), sparams=p, **kw)
        fd = float((w * (ip - im)).sum() / (2 * h))
        g = grad.reshape(-1)[k]
        assert abs(fd - g) <= 1e-6 * max(abs(g), 1e-3 * np.abs(grad).max()), (k, fd, g)


def test_gradient_is_sparse_on_untouched_segments():
    """Eq. 6: only segments on the sampled paths get a gradient.  With depth 0
    the camera sees emission only: no material gradient, and no emission
    gradient for invisible segments."""
    sc = cornell_small(8, 8)
    osc = O.OracleScene(sc)
    p = sc.gt_params.astype(np.float64)
    w = np.ones((64, 3))
    g = osc.gradient(p, w, spp=4, max_depth=0)
    assert np.all(g[:, 0:7] == 0)
    assert g[1, 7] > 0  # ceiling visible


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    theta = rng.uniform(0.3, 0.7, (5, 10))
    grads = [rng.normal(scale=0.01, size=(5, 10)) for _ in range(6)]
    t_param = torch.tensor(theta.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t_param], lr=5e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for t, g in enumerate(grads, 1):
        t_param.grad = torch.tensor(g)
        opt.step()
        theta, m, v = O.adam_update(theta, g, m, v, t, l1_emission=0.0)
    assert np.allclose(theta, t_param.detach().numpy(), rtol=0, atol=1e-15)


def test_adam_regulariser_clamps_and_mask():
    theta = np.full((2, 10), 0.5)
    theta[0, 7:10] = 0.001      # small emission pushed to 0 by L1 + clamp
    theta[0, 6] = 0.021
    g = np.zeros((2, 10))
    g[0, 6] = 1.0               # positive gradient on roughness -> decreases, clamps at 0.02
    free = np.ones((2, 10), bool)
    free[1] = False
    th, m, v = O.adam_update(theta, g, np.zeros_like(g), np.zeros_like(g), 1, free=free,
                             lr=5e-3, l1_emission=1e-3)
    # first Adam step moves each coordinate with a non-zero gradient by lr
    assert np.allclose(th[0, 7:10], 0.0)
    assert th[0, 6] == 0.02
    assert np.all(th[1] == 0.5) and np.all(m[1] == 0) and np.all(v[1] == 0)
    assert np.allclose(th[0, 0:6], 0.5)
