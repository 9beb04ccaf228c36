"""Pins for the radiance-cache oracle: spherical-harmonic orthonormality by
quadrature, exactness and partition of unity of the hash-grid encoding,
and finite differences of every gradient."""
import math

import numpy as np
import pytest

from oracle import cache_oracle as K
from oracle import oracle as O
from paper_1903_07145_gb300 import scenes


def test_resolutions_follow_the_geometric_rule():
    r = K.resolutions()
    assert r[0] == 16 and r[-1] == 2048 and len(r) == 16
    assert all(b > a for a, b in zip(r, r[1:]))


def test_sh_is_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform in phi, exact for these degrees
    gx, gw = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(gx, phi, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (gw[:, None] * np.full((1, nphi), 2 * math.pi / nphi)).reshape(-1)
    Y = K.sh4(d)
    G = (Y * w[:, None]).T @ Y
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_hash_encoding_corners_and_partition_of_unity():
    rng = np.random.default_rng(0)
    table = rng.normal(size=(K.LEVELS, 1 << K.LOG2_T, K.FEATURES))
    res = K.resolutions()
    # at a grid vertex of level l the level's feature is the table entry
    for l in [0, 5, 15]:
        n = res[l]
        ijk = np.array([[3, 7, 1], [n, 0, n // 2]])
        x = ijk / n
        h, idx, wts = K.hash_encode(x, table)
        ci = K.corner_index(ijk, n)
        assert np.allclose(h[:, 2 * l:2 * l + 2], table[l, ci], atol=1e-12)
    # trilinear weights sum to one; a constant table gives a constant encoding
    x = rng.random((200, 3))
    _, _, wts = K.hash_encode(x, table)
    assert np.allclose(wts.sum(-1), 1.0)
    h1, _, _ = K.hash_encode(x, np.ones_like(table))
    assert np.allclose(h1, 1.0)
    # dense levels index every vertex once; hashed levels stay in range
    assert (res[0] + 1) ** 3 <= 1 << K.LOG2_T
    big = K.corner_index(np.array([[2048, 2047, 5]]), 2048)
    assert 0 <= big[0] < 1 << K.LOG2_T


def test_spatial_hash_matches_its_definition():
    ijk = np.array([[123, 456, 789]])
    n = 2048
    T = 1 << K.LOG2_T
    expect = ((123 * 1) ^ ((456 * 2654435761) & 0xFFFFFFFF) ^ ((789 * 805459861) & 0xFFFFFFFF)) % T
    assert K.corner_index(ijk, n)[0] == expect


def fd_check(f, x, g, h=1e-6, n=12, seed=0):
    rng = np.random.default_rng(seed)
    flat = x.reshape(-1)
    for k in rng.choice(flat.size, n, replace=False):
        old = flat[k]
        flat[k] = old + h
        fp = f()
        flat[k] = old - h
        fm = f()
        flat[k] = old
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g.reshape(-1)[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g.reshape(-1)[k])


def test_mlp_and_loss_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    W = K.init_weights(3)
    x = rng.normal(size=(20, K.IN_DIM))
    t = rng.uniform(0, 2, (20, 3))

    def loss_of():
        y, _ = K.mlp_forward(x, W)
        return K.rel_l2(y, t)[0]

    def loss_fixed_denominator():
        # the relative L2 holds its denominator constant: evaluate with the
        # denominator of the unperturbed prediction
        y, _ = K.mlp_forward(x, W)
        r = y[:, :3] - t
        return float(np.sum(r * r / den)) / r.size

    y0, acts = K.mlp_forward(x, W)
    den = y0[:, :3] ** 2 + 0.01
    _, d = K.rel_l2(y0, t)
    gw, gx = K.mlp_backward(d, acts, W)
    for i in range(len(W)):
        fd_check(loss_fixed_denominator, W[i], gw[i], seed=i)
    fd_check(loss_fixed_denominator, x, gx, seed=9)
    assert np.isfinite(loss_of())


def test_hash_backward_by_finite_differences():
    rng = np.random.default_rng(2)
    table = rng.normal(size=(K.LEVELS, 1 << 10, K.FEATURES))
    # small table: every level hashed or dense over 2^10 entries
    x = rng.random((30, 3))
    w = rng.normal(size=(30, K.LEVELS * K.FEATURES))

    def enc_dot():
        h, _, _ = K.hash_encode(x, table)
        return float((h * w).sum())

    h, idx, wts = K.hash_encode(x, table)
    g = K.hash_backward(w, idx, wts, table.shape)
    fd_check(enc_dot, table, g, n=20)


# ----------------------------------------------------------------------------
# Paths cut at the cache vertex
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("b_term", [1, 2])
def test_cut_paths_decompose_the_plain_estimate(b_term):
    """Per sample, the plain estimate equals prefix + beta_b * (reflected
    radiance gathered from b on): the cut keeps the emission found at b and
    the training target holds everything after it."""
    sc = scenes.cornell_box(1000, 8, 8)
    osc = O.OracleScene(sc)
    p = sc.gt_params.astype(np.float64)
    kw = dict(spp=6, max_depth=4, seed=5, set_id=0, iteration=3)
    term = osc.cache_terminals(p, b_term, **kw)
    rec = osc.cache_records(p, b_term, **kw)
    plain, _ = osc.render(p, **kw)
    assert np.array_equal(term["seg"], rec["seg"])
    assert np.array_equal(term["x"], rec["x"]) and np.array_equal(term["ns"], rec["ns"])
    m = term["seg"] >= 0
    assert m.mean() > 0.5
    assert np.all(term["beta"][m] > 0) and np.all(term["beta"][~m] == 0)
    assert np.all(rec["target"] >= 0)
    assert np.allclose(np.einsum("ij,ij->i", term["wi"][m], term["ns"][m]) > -1e-12, True)
    comp = K.cached_image(term, 6, rec["target"])
    assert np.allclose(comp, plain, rtol=1e-12, atol=1e-14)
    # with the cut past the last vertex nothing is cached
    none = osc.cache_terminals(p, 4, **kw)
    assert np.all(none["seg"] == -1)
    assert np.allclose(none["prefix"].reshape(-1, 6, 3).mean(1), plain, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("b_term", [1, 2])
def test_cached_gradient_matches_central_differences(b_term):
    """With sampling frozen and a closed-form cache Lc = A theta_7 + c, the
    vector-Jacobian product of the cut estimator matches central differences
    in every parameter kind (earlier vertices' BSDF factors by Eq. 6, the
    terminal segment through the cache)."""
    sc = scenes.cornell_box(1000, 8, 8)
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(3)
    p = sc.gt_params.astype(np.float64).copy()
    p[:, 3:6] = rng.uniform(0.05, 0.3, (sc.n_segments, 3))
    A = rng.normal(size=(3, 7))
    c0 = rng.uniform(0.5, 1.0, 3)
    w = rng.normal(size=(64, 3))
    kw = dict(spp=4, max_depth=3, seed=9, set_id=1)

    def image(q):
        term = osc.cache_terminals(q, b_term, sparams=p, **kw)
        m = term["seg"] >= 0
        cval = np.zeros_like(term["prefix"])
        cval[m] = q[term["seg"][m], :7] @ A.T + c0
        return K.cached_image(term, 4, cval), term, cval

    _, term, cval = image(p)
    cjac = np.zeros((cval.shape[0], 3, 7))
    cjac[term["seg"] >= 0] = A
    grad = osc.cache_gradient(p, w, b_term, cval, cjac, sparams=p, **kw)
    h = 1e-5
    ks = rng.choice(sc.n_segments * 10, 24, replace=False)
    for k in ks:
        pp = p.copy().reshape(-1)
        pm = p.copy().reshape(-1)
        pp[k] += h
        pm[k] -= h
        ip = image(pp.reshape(p.shape))[0]
        im = image(pm.reshape(p.shape))[0]
        fd = float((w * (ip - im)).sum() / (2 * h))
        g = grad.reshape(-1)[k]
        assert abs(fd - g) <= 1e-6 * max(abs(g), 1e-3 * np.abs(grad).max()), (k, fd, g)
    # the terminal segments' material rows move through the cache Jacobian
    assert np.abs(grad[:, :7]).sum() > 0


def test_bf16_rounding_ties_to_even_and_matches_torch():
    one = 1.0
    assert K.bf16(one) == 1.0 and K.bf16(3.0) == 3.0
    assert K.bf16(1 + 2 ** -8) == 1.0                      # halfway, even neighbour below
    assert K.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6          # halfway, even neighbour above
    assert K.bf16(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7   # above halfway
    assert K.bf16(-(1 + 3 * 2 ** -8)) == -(1 + 2 ** -6)
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(size=10000).astype(np.float32) * 10.0 ** np.random.default_rng(1).integers(-6, 6, 10000)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(K.bf16(x), ref)


def test_bf16_storage_changes_only_rounding():
    """With BF16 storage the network is the FP64 one evaluated on rounded
    operands: close to it, every stored activation is a BF16 value, and an
    input that is already BF16 reaches the first layer unchanged."""
    rng = np.random.default_rng(4)
    W = [K.bf16(w) for w in K.init_weights(5)]
    x = rng.normal(size=(50, K.IN_DIM))
    y64, _ = K.mlp_forward(x, W)
    y16, acts = K.mlp_forward(x, W, storage="bf16")
    assert np.linalg.norm(y16 - y64) <= 2e-2 * np.linalg.norm(y64)
    assert all(np.array_equal(a, K.bf16(a)) for a in acts[:-1])
    xe = K.bf16(x)
    _, acts_e = K.mlp_forward(xe, W, storage="bf16")
    assert np.array_equal(acts_e[0], xe)
    assert np.array_equal(acts_e[1], K.bf16(np.maximum(xe @ W[0], 0.0)))
