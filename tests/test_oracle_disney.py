"""Pins for the oracle's Disney material model (Sec. 4.1): the Jacobian
against central differences, reciprocity, isotropy without anisotropy, the
reduction at normal incidence to the GGX lobe of the Lambert + GGX model and
to a Lambertian lobe, the sampler's density (E[1/pdf] over the upper
hemisphere is its solid angle, 2 pi), energy bounds of the metallic lobe, and
the path gradient (Eq. 5-6 with the Disney Jacobian) against central
differences of the rendered image."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_07145_gb300 import scenes

N = np.array([0.0, 0.0, 1.0])
X = np.array([1.0, 0.3, 0.0])


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def random_dir_up(rng):
    while True:
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        if v[2] > 0.1:
            return v


def random_material(rng):
    m = rng.uniform(0.05, 0.95, 13)
    m[7] = rng.uniform(0.2, 0.9)  # roughness away from the width floor
    return m


def test_jacobian_matches_central_differences():
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(40):
        m = random_material(rng)
        wi, wo = random_dir_up(rng), random_dir_up(rng)
        f, J, ok = O.disney_brdf(m, N, X, wi, wo, jacobian=True)
        assert ok and np.all(f > 0)
        for j in range(13):
            a, b = m.copy(), m.copy()
            a[j] += h
            b[j] -= h
            fd = (O.disney_brdf(a, N, X, wi, wo)[0] - O.disney_brdf(b, N, X, wi, wo)[0]) / (2 * h)
            assert np.allclose(J[:, j], fd, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(f).max())), (j, J[:, j], fd)


def test_reciprocity():
    rng = np.random.default_rng(2)
    for _ in range(100):
        m = random_material(rng)
        wi, wo = random_dir_up(rng), random_dir_up(rng)
        f1, _ = O.disney_brdf(m, N, X, wi, wo)
        f2, _ = O.disney_brdf(m, N, X, wo, wi)
        assert np.allclose(f1, f2, rtol=1e-12, atol=0)


def test_below_horizon_is_zero():
    m = random_material(np.random.default_rng(3))
    f, ok = O.disney_brdf(m, N, X, unit([0.2, 0.1, 0.9]), unit([0.3, 0.0, -0.2]))
    assert not ok and np.all(f == 0)


def test_isotropic_without_anisotropy():
    """anisotropic = 0: f does not depend on the tangent direction."""
    rng = np.random.default_rng(4)
    for _ in range(30):
        m = random_material(rng)
        m[8] = 0.0
        wi, wo = random_dir_up(rng), random_dir_up(rng)
        x2 = np.array([math.cos(1.1), math.sin(1.1), 0.0])
        assert np.allclose(O.disney_brdf(m, N, X, wi, wo)[0], O.disney_brdf(m, N, x2, wi, wo)[0], rtol=1e-12)
        m[8] = 0.8  # and it does with anisotropy
        assert not np.allclose(O.disney_brdf(m, N, X, wi, wo)[0], O.disney_brdf(m, N, x2, wi, wo)[0], rtol=1e-6)


@pytest.mark.parametrize("r", [0.2, 0.45, 0.8])
def test_metallic_at_normal_incidence_is_the_ggx_lobe(r):
    """metallic = 1, no sheen, clearcoat or anisotropy, wi = wo = n: the
    Fresnel term is the base colour and the masking is 1, so f equals the
    Lambert + GGX model's specular lobe (kd = 0, ks = base, same roughness)."""
    base = np.array([0.9, 0.5, 0.2])
    m = np.zeros(13)
    m[0:3] = base
    m[4] = 1.0
    m[7] = r
    f, ok = O.disney_brdf(m, N, X, N, N)
    p10 = np.zeros(10)
    p10[3:6] = base
    p10[6] = r
    g, _, _, ok2 = O.brdf(p10, N, N, N)
    assert ok and ok2
    assert np.allclose(f, g, rtol=1e-12)


def test_diffuse_at_normal_incidence_is_lambertian():
    """Dielectric, no specular, sheen or clearcoat, subsurface 0, both
    directions along n: Burley's diffuse is base / pi for any roughness."""
    for r in (0.0, 0.3, 1.0):
        m = np.zeros(13)
        m[0:3] = [0.7, 0.4, 0.1]
        m[7] = r
        f, _ = O.disney_brdf(m, N, X, N, N)
        assert np.allclose(f, m[0:3] / math.pi, rtol=1e-14)


def _inv_pdf_mean(m, wi, n_samples, seed):
    """E[1{wo above the horizon} / pdf(wo)] over the sampler's directions."""
    rng = np.random.default_rng(seed)
    u = rng.random((n_samples, 3))
    acc = np.zeros(n_samples)
    for i in range(n_samples):
        wo, pdf = O.disney_sample(m, N, X, wi, u[i, 0], u[i, 1], u[i, 2])
        if wo[2] > 0.0 and pdf > 0.0:
            acc[i] = 1.0 / pdf
    return acc.mean(), acc.std() / math.sqrt(n_samples)


@pytest.mark.parametrize("lobe", ["diffuse", "specular", "clearcoat", "mixture"])
def test_sampler_density(lobe):
    """The pdf is the density of the sampled directions: the mean of 1/pdf
    over samples that land above the horizon is the hemisphere's solid angle
    2 pi (a wrong normalisation of D, of the visible-normal pdf or of the
    clearcoat's GTR1 fails this)."""
    m = np.zeros(13)
    m[7] = 0.5
    m[8] = 0.6
    m[12] = 0.3
    if lobe == "diffuse":
        m[0:3] = 0.5
    elif lobe == "specular":
        m[0:3] = 0.5
        m[4] = 1.0
    elif lobe == "clearcoat":
        m[11] = 1.0
    else:
        m[0:3] = 0.5
        m[4] = 0.3
        m[5] = 0.8
        m[11] = 0.7
    p = O.disney_lobes(m)
    assert abs(p.sum() - 1.0) < 1e-15
    wi = unit([0.4, -0.2, 0.8])
    mean, se = _inv_pdf_mean(m, wi, 40000, 7)
    assert abs(mean - 2 * math.pi) <= 4 * se + 1e-3, (lobe, mean, se)


def _albedo(m, wi, n_samples, seed):
    rng = np.random.default_rng(seed)
    u = rng.random((n_samples, 3))
    acc = np.zeros((n_samples, 3))
    for i in range(n_samples):
        wo, pdf = O.disney_sample(m, N, X, wi, u[i, 0], u[i, 1], u[i, 2])
        if wo[2] > 0.0 and pdf > 0.0:
            f, _ = O.disney_brdf(m, N, X, wi, wo)
            acc[i] = f * wo[2] / pdf
    return acc.mean(0), acc.std(0) / math.sqrt(n_samples)


def _ggx_albedo_normal_incidence(alpha, n=20000):
    """Directional albedo at normal incidence of an isotropic GGX lobe with
    Fresnel 1 and separable Smith masking, by 1-D quadrature over the half
    vector's polar angle: at v = n the reflected direction has polar angle
    2 theta_h, so only theta_h < pi / 4 reflects above the horizon, and
    dw_l = 4 (l.h) dw_h with l.h = cos theta_h (textbook GGX: Walter et al.
    2007)."""
    th = (np.arange(n) + 0.5) * (math.pi / 4) / n
    c, t2 = np.cos(th), np.tan(th) ** 2
    D = alpha ** 2 / (math.pi * c ** 4 * (alpha ** 2 + t2) ** 2)
    t2l = np.tan(2 * th) ** 2
    G1l = 2.0 / (1.0 + np.sqrt(1.0 + alpha ** 2 * t2l))
    # f cos_l dw_l = D G1(l) / (4 cos_l) cos_l 4 cos_h dw_h, dw_h = 2 pi sin dtheta
    return float(np.sum(D * G1l * c * np.sin(th)) * 2 * math.pi * (math.pi / 4) / n)


def test_metallic_lobe_energy():
    """A white metal (Fresnel = 1) reflects at most what arrives, and its
    directional albedo at normal incidence equals the quadrature of the
    GGX lobe with separable Smith masking."""
    m = np.zeros(13)
    m[0:3] = 1.0
    m[4] = 1.0
    for r in (0.25, 0.5, 0.8):
        m[7] = r
        a, se = _albedo(m, N, 20000, 11)
        ref = _ggx_albedo_normal_incidence(r * r)
        assert np.all(a <= 1.0 + 4 * se), (r, a, se)
        assert np.all(np.abs(a - ref) <= 4 * se + 1e-4), (r, a, ref, se)


def test_path_gradient_matches_central_differences():
    """<w, I(p + h e_k) - I(p - h e_k)> / 2h == (J^T w)_k for the Disney
    model with sampling frozen at p (Eq. 5 for emission, Eq. 6 with the
    3 x 13 Jacobian for the material values)."""
    sc = scenes.cornell_box(1000, 8, 8)
    osc = O.OracleScene(sc)
    p = scenes.disney_materials(sc, 5).astype(np.float64)
    rng = np.random.default_rng(13)
    w = rng.normal(size=(64, 3))
    kw = dict(spp=4, max_depth=3, seed=21, model=O.MODEL_DISNEY)
    grad = osc.gradient(p, w, sparams=p, **kw)
    assert grad.shape == (sc.n_segments, 16)
    h = 1e-6
    ks = [s * 16 + j for s in range(sc.n_segments) for j in range(16)]
    ks = rng.choice(ks, 40, replace=False)
    for k in ks:
        pp = p.copy().reshape(-1)
        pm = p.copy().reshape(-1)
        pp[k] += h
        pm[k] -= h
        ip, _ = osc.render(pp.reshape(p.shape), sparams=p, **kw)
        im, _ = osc.render(pm.reshape(p.shape), sparams=p, **kw)
        fd = float((w * (ip - im)).sum() / (2 * h))
        g = grad.reshape(-1)[k]
        assert abs(fd - g) <= 1e-5 * max(abs(g), 1e-3 * np.abs(grad).max()), (k, fd, g)


def test_render_is_linear_in_emission():
    sc = scenes.cornell_box(1000, 8, 8)
    osc = O.OracleScene(sc)
    p = scenes.disney_materials(sc, 6).astype(np.float64)
    kw = dict(spp=4, max_depth=3, seed=2, sparams=p.copy(), model=O.MODEL_DISNEY)
    a, _ = osc.render(p, **kw)
    q = p.copy()
    q[:, 13:16] *= 2.5
    b, _ = osc.render(q, **kw)
    assert np.allclose(b, 2.5 * a, rtol=1e-12, atol=0)
    assert a.max() > 0
