"""FP64 CPU oracle of the learned radiance cache -- test infrastructure.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module; it shares no code with the CUDA path.  The paper has no
learned component; this follows the cache's specification in plain numpy:

* position: multiresolution hash-grid encoding (Mueller, Evans, Schied,
  Keller, "Instant Neural Graphics Primitives", SIGGRAPH 2022): L levels of
  F features, T entries per level, resolutions N_l = floor(N_min * b^l) with
  b = exp((ln N_max - ln N_min) / (L - 1)); a point x in [0,1]^3 is scaled to
  p = x * N_l, its cell's 8 corners are looked up (dense index
  i + j (N+1) + k (N+1)^2 when (N+1)^3 <= T, else the spatial hash
  (i * 1) xor (j * 2654435761) xor (k * 805459861) mod T) and trilinearly
  interpolated;
* view direction and normal: real spherical harmonics up to degree 3
  (16 coefficients each);
* the terminal segment's 7 material parameters;
* input layout [hash (L*F = 32) | SH(dir) 16 | SH(normal) 16 | params 7 |
  zeros 9] = 80;
* MLP 80 -> 64 -> 64 -> 64 -> 64 -> 16 (first 3 outputs used), ReLU on the
  hidden layers, no biases;
* loss: relative L2, mean over records and channels of
  (y - t)^2 / (sg(y)^2 + 0.01), sg = stop-gradient.

The network's operands are specified as BF16 (tensor-core inputs with FP32
accumulation).  Where that precision decides a discrete branch -- a ReLU
mask, a unit's activation at zero -- the oracle takes the decision the same
way: with storage="bf16" the input and each hidden activation are rounded
to BF16 (round to nearest, ties to even) where the network stores them,
while every sum and product stays FP64.  The default (storage=None) is the
plain FP64 network.

Parity status: pinned (SH orthonormality by quadrature, exact corner values
and partition of unity of the hash encoding, finite differences of every
gradient, see tests/test_oracle_cache.py).
"""
from __future__ import annotations

import math

import numpy as np

LEVELS, FEATURES, LOG2_T, N_MIN, N_MAX = 16, 2, 19, 16, 2048
IN_DIM, HIDDEN, OUT_DIM, N_HIDDEN = 80, 64, 16, 4
PRIMES = (1, 2654435761, 805459861)


def bf16(a):
    """Round to the nearest bfloat16 (8 significant bits, ties to even); the
    result is returned as float64."""
    b = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32)).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def resolutions(levels=LEVELS, n_min=N_MIN, n_max=N_MAX):
    b = math.exp((math.log(n_max) - math.log(n_min)) / (levels - 1))
    return [int(math.floor(n_min * b ** l)) for l in range(levels)]


def corner_index(ijk, n, T=1 << LOG2_T):
    """Table index of integer grid vertices ijk (..., 3) at resolution n in a
    table of T entries (a power of two)."""
    ijk = np.asarray(ijk, np.uint64)
    if (n + 1) ** 3 <= T:
        return (ijk[..., 0] + ijk[..., 1] * (n + 1) + ijk[..., 2] * (n + 1) * (n + 1)).astype(np.int64)
    h = (ijk[..., 0] * np.uint64(PRIMES[0])) & np.uint64(0xFFFFFFFF)
    h ^= (ijk[..., 1] * np.uint64(PRIMES[1])) & np.uint64(0xFFFFFFFF)
    h ^= (ijk[..., 2] * np.uint64(PRIMES[2])) & np.uint64(0xFFFFFFFF)
    return (h & np.uint64(T - 1)).astype(np.int64)


def hash_encode(x, table, levels=LEVELS, features=FEATURES):
    """x: (N, 3) in [0,1]; table: (L, T, F).  Returns (N, L*F) features and
    the corner indices / weights needed for the backward pass."""
    x = np.asarray(x, np.float64)
    T = table.shape[1]
    res = resolutions(levels)
    out = np.zeros((x.shape[0], levels * features))
    idx = np.zeros((x.shape[0], levels, 8), np.int64)
    wts = np.zeros((x.shape[0], levels, 8))
    for l, n in enumerate(res):
        p = x * n
        i0 = np.floor(p)
        f = p - i0
        i0 = i0.astype(np.int64)
        for c in range(8):
            o = np.array([(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1])
            w = np.prod(np.where(o[None, :] == 1, f, 1.0 - f), axis=1)
            ci = corner_index(np.clip(i0 + o[None, :], 0, n), n, T)
            idx[:, l, c] = ci
            wts[:, l, c] = w
            out[:, l * features:(l + 1) * features] += w[:, None] * table[l, ci, :]
    return out, idx, wts


def hash_backward(d_out, idx, wts, table_shape, features=FEATURES):
    g = np.zeros(table_shape)
    levels = idx.shape[1]
    for l in range(levels):
        for c in range(8):
            np.add.at(g[l], idx[:, l, c], wts[:, l, c][:, None] * d_out[:, l * features:(l + 1) * features])
    return g


def sh4(d):
    """Real spherical harmonics of degrees 0..3 (16 values) of unit vectors."""
    d = np.asarray(d, np.float64)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = math.pi
    c0 = 0.5 / math.sqrt(pi)
    c1 = math.sqrt(3.0 / (4.0 * pi))
    out = np.stack([
        np.full_like(x, c0),
        -c1 * y, c1 * z, -c1 * x,
        0.5 * math.sqrt(15.0 / pi) * x * y,
        -0.5 * math.sqrt(15.0 / pi) * y * z,
        0.25 * math.sqrt(5.0 / pi) * (3 * z * z - 1),
        -0.5 * math.sqrt(15.0 / pi) * x * z,
        0.25 * math.sqrt(15.0 / pi) * (x * x - y * y),
        -0.25 * math.sqrt(35.0 / (2 * pi)) * y * (3 * x * x - y * y),
        0.5 * math.sqrt(105.0 / pi) * x * y * z,
        -0.25 * math.sqrt(21.0 / (2 * pi)) * y * (5 * z * z - 1),
        0.25 * math.sqrt(7.0 / pi) * z * (5 * z * z - 3),
        -0.25 * math.sqrt(21.0 / (2 * pi)) * x * (5 * z * z - 1),
        0.25 * math.sqrt(105.0 / pi) * z * (x * x - y * y),
        -0.25 * math.sqrt(35.0 / (2 * pi)) * x * (x * x - 3 * y * y),
    ], axis=1)
    return out


def encode(x, d, n, params7, table):
    """Cache input (N, 80) from positions in [0,1]^3, unit directions, unit
    normals and the terminal segments' 7 material parameters."""
    h, idx, wts = hash_encode(x, table)
    N = h.shape[0]
    inp = np.zeros((N, IN_DIM))
    inp[:, 0:32] = h
    inp[:, 32:48] = sh4(d)
    inp[:, 48:64] = sh4(n)
    inp[:, 64:71] = params7
    return inp, (idx, wts)


def init_weights(seed=0):
    """He-uniform weights: [W1 (80x64), W2, W3, W4 (64x64), W5 (64x16)]."""
    rng = np.random.default_rng(seed)
    dims = [IN_DIM] + [HIDDEN] * N_HIDDEN + [OUT_DIM]
    return [rng.uniform(-1, 1, (dims[i], dims[i + 1])) * math.sqrt(6.0 / dims[i]) for i in range(len(dims) - 1)]


def mlp_forward(inp, weights, storage=None):
    """Forward pass; storage="bf16" rounds the input and the hidden
    activations to BF16 where the network stores them."""
    rnd = bf16 if storage == "bf16" else (lambda a: a)
    acts = [rnd(np.asarray(inp, np.float64))]
    z = acts[0]
    for i, W in enumerate(weights):
        z = z @ W
        if i < len(weights) - 1:
            z = rnd(np.maximum(z, 0.0))
        acts.append(z)
    return z, acts


def mlp_backward(d_out, acts, weights):
    """Returns (weight gradients, input gradient) for d_out = dL/dy (N, 16)."""
    grads = [None] * len(weights)
    d = np.asarray(d_out, np.float64)
    for i in reversed(range(len(weights))):
        grads[i] = acts[i].T @ d
        d = d @ weights[i].T
        if i > 0:
            d = d * (acts[i] > 0.0)
    return grads, d


def rel_l2(y, target, eps=0.01):
    """Loss and dL/dy (denominator held constant), over the first 3 outputs."""
    y3 = y[:, :3]
    denom = y3 * y3 + eps
    r = y3 - target
    n = r.size
    loss = float(np.sum(r * r / denom)) / n
    d = np.zeros_like(y)
    d[:, :3] = 2.0 * r / denom / n
    return loss, d


def unit_coords(x, lo, hi):
    """World positions to the grid's unit cube (the scene's bounding box),
    clamped to [0, 1]."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return np.clip((np.asarray(x, np.float64) - lo) / (hi - lo), 0.0, 1.0)


def cache_eval(x01, wi, ns, p7, weights, table, storage=None):
    """Cache prediction Lc (N, 3) and its Jacobian (N, 3, 7) with respect to
    the 7 material parameters in the input."""
    inp, _ = encode(x01, wi, ns, p7, table)
    y, acts = mlp_forward(inp, weights, storage)
    J = np.zeros((inp.shape[0], 3, 7))
    for c in range(3):
        d = np.zeros((inp.shape[0], OUT_DIM))
        d[:, c] = 1.0
        _, dx = mlp_backward(d, acts, weights)
        J[:, c, :] = dx[:, 64:71]
    return y[:, :3], J


def cached_values(term, params, weights, table, lo, hi, storage=None):
    """Cache value and Jacobian per path row of oracle terminals (zeros on
    rows without a terminal vertex)."""
    rows = term["seg"].shape[0]
    cval = np.zeros((rows, 3))
    cjac = np.zeros((rows, 3, 7))
    m = term["seg"] >= 0
    if m.any():
        p7 = np.asarray(params, np.float64)[term["seg"][m], :7]
        y, J = cache_eval(unit_coords(term["x"][m], lo, hi), term["wi"][m], term["ns"][m], p7,
                          weights, table, storage)
        cval[m] = y
        cjac[m] = J
    return cval, cjac


def cached_image(term, spp, cval):
    """Pixel means of prefix + beta_b * Lc over each pixel's spp rows."""
    v = term["prefix"] + term["beta"] * cval
    return v.reshape(-1, spp, 3).mean(1)
