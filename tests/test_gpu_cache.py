"""GPU parity of the radiance cache, through the C ABI, against the FP64
cache oracle (network) and the cut-path oracle (tracer).

The network runs on BF16 operands with FP32 accumulation.  The tests round
the weights to BF16 on both sides, and the oracle stores the input and the
hidden activations as BF16 too (storage="bf16"), so that both sides take the
ReLU decisions on the same values; what remains is FP32 vs FP64
accumulation and the BF16 rounding of the backward signals (relative 2^-9
each, over 5 layers):
  * predictions: relative L2 <= 1e-2;
  * input vector-Jacobian products and training gradients (every weight
    layer on its own and the table): relative L2 <= 1e-2 and cosine >=
    0.999 (measured: 0.4-0.6% for the VJP, under 0.2% per weight layer,
    0.4% for the table);
  * cached images and gradients (same Philox streams, FP32 vs FP64 paths):
    relative L2 <= 1e-2 and gradient cosine >= 0.999;
  * training records: the same paths reach the cache vertex, and their
    positions, directions, normals and targets agree as plain paths do.

A ReLU decision is discontinuous in its gradient.  FP32 accumulation (in
the tensor cores' order) and FP64 round an activation to different BF16
neighbours now and then (~1% of rows), which moves later pre-activations
by ~5e-4; a unit that close to its kink then switches on one side only and
that row's gradient changes by 10-20%.  Gradient parity of the network
kernels therefore uses rows whose every hidden pre-activation, in the
oracle, is at least 2e-3 from zero ("decided" rows, picked from the oracle
alone); predictions, which are continuous there, use any rows.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import cache_oracle as K  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1903_07145_gb300 import scenes  # noqa: E402
from paper_1903_07145_gb300.tracer import CacheOptions, TraceOptions, Tracer  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 4321


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def cosine(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b)))


bf16 = K.bf16
BF = "bf16"


def network(seed, out_scale=1.0, table_scale=0.5, log2_t=K.LOG2_T):
    W = K.init_weights(seed)
    W[-1] = W[-1] * out_scale
    W = [bf16(w) for w in W]
    rng = np.random.default_rng(seed + 100)
    table = rng.uniform(-table_scale, table_scale, (K.LEVELS, 1 << log2_t, K.FEATURES)).astype(np.float32)
    return W, table.astype(np.float64)


def flat(W):
    return np.concatenate([w.reshape(-1) for w in W]).astype(np.float32)


def unit(v):
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def f32(a):
    """The float32 values the C ABI receives, as float64: both sides see the
    same inputs (a float64 position moves the finest grid level's weights by
    ~1e-4, enough to change BF16-rounded features)."""
    return np.asarray(a, np.float32).astype(np.float64)


def rows(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3))
    x[: min(n, 4)] = [[0, 0, 0], [1, 1, 1], [0, 1, 0.5], [1, 0, 0.25]][: min(n, 4)]
    d = unit(rng.normal(size=(n, 3)))
    nr = unit(rng.normal(size=(n, 3)))
    p7 = rng.random((n, 7))
    return f32(x), f32(d), f32(nr), f32(p7)


def decided_rows(n, seed, W, table, margin=2e-3):
    """n rows whose hidden pre-activations (oracle, BF16 storage) all keep
    |z| >= margin."""
    out = [[], [], [], []]
    got, s = 0, seed
    while got < n:
        cand = rows(4 * n, s)
        inp, _ = K.encode(*cand, table)
        a = bf16(inp)
        ok = np.ones(a.shape[0], bool)
        for w in W[:4]:
            z = a @ w
            ok &= np.min(np.abs(z), axis=1) >= margin
            a = bf16(np.maximum(z, 0.0))
        for k in range(4):
            out[k].append(cand[k][ok])
        got += int(ok.sum())
        s += 7919
    return tuple(np.concatenate(o)[:n] for o in out)


def cache_tracer(sc, opts=None, seed=SEED):
    tr = Tracer(sc, seed=seed)
    tr.configure_cache(opts or CacheOptions(enabled=False))
    return tr


# ---------------------------------------------------------------------------
# Network kernels against the cache oracle
# ---------------------------------------------------------------------------

def test_grid_matches_oracle(built):
    tr = cache_tracer(scenes.cornell_box(1000, 8, 8))
    st = tr.cache_status()
    assert st["res"] == K.resolutions()
    assert np.allclose(st["lo"], tr.scene.positions.min(0)) and np.allclose(st["hi"], tr.scene.positions.max(0))


@pytest.mark.parametrize("n", [1, 17, 1000, 4099])
def test_prediction_matches_oracle(built, n):
    tr = cache_tracer(scenes.cornell_box(1000, 8, 8))
    W, table = network(7)
    tr.set_cache_weights(flat(W), table)
    x, d, nr, p7 = rows(n, n)
    got = tr.cache_eval(x, d, nr, p7).cpu().numpy().astype(np.float64)
    ref, _ = K.cache_eval(x, d, nr, p7, W, table, BF)
    assert got.shape == (n, 3)
    assert rel(got, ref) <= 1e-2, rel(got, ref)


@pytest.mark.parametrize("n", [16, 1000])
def test_input_vjp_matches_oracle(built, n):
    tr = cache_tracer(scenes.cornell_box(1000, 8, 8))
    W, table = network(8)
    tr.set_cache_weights(flat(W), table)
    x, d, nr, p7 = decided_rows(n, 3 * n, W, table)
    u = f32(np.random.default_rng(5).normal(size=(n, 3)))
    rgb, dp = tr.cache_eval(x, d, nr, p7, upstream=u)
    ref_y, J = K.cache_eval(x, d, nr, p7, W, table, BF)
    ref = np.einsum("nc,ncj->nj", u, J)
    got = dp.cpu().numpy().astype(np.float64)
    assert rel(rgb.cpu().numpy(), ref_y) <= 1e-2
    assert rel(got, ref) <= 1e-2, rel(got, ref)
    assert cosine(got, ref) >= 0.999


@pytest.mark.parametrize("n", [64, 2000, 20000])
def test_training_gradients_match_oracle(built, n):
    """n = 20000: 313 tiles of 64 rows (the last one ragged) over at most one
    block per SM, so blocks accumulate the weight gradients of several tiles
    in tensor memory before adding them to the global gradient."""
    tr = cache_tracer(scenes.cornell_box(1000, 8, 8))
    W, table = network(9)
    tr.set_cache_weights(flat(W), table)
    x, d, nr, p7 = decided_rows(n, 11 * n, W, table)
    target = f32(np.random.default_rng(6).uniform(0.0, 2.0, (n, 3)))
    loss, gw, gt = tr.cache_grad(x, d, nr, p7, target)
    inp, (idx, wts) = K.encode(x, d, nr, p7, table)
    y, acts = K.mlp_forward(inp, W, BF)
    ref_loss, dy = K.rel_l2(y, target)
    ref_gw, dx = K.mlp_backward(dy, acts, W)
    ref_gt = K.hash_backward(dx[:, :32], idx, wts, table.shape)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    got_w = gw.cpu().numpy().astype(np.float64)
    ref_w = np.concatenate([g.reshape(-1) for g in ref_gw])
    assert rel(got_w, ref_w) <= 1e-2 and cosine(got_w, ref_w) >= 0.999, (rel(got_w, ref_w), cosine(got_w, ref_w))
    # every layer on its own (W1 80 x 64, W2..W4 64 x 64, W5 64 x 16)
    off = 0
    for g in ref_gw:
        a, b = got_w[off:off + g.size], g.reshape(-1)
        assert rel(a, b) <= 1e-2 and cosine(a, b) >= 0.999, (off, rel(a, b), cosine(a, b))
        off += g.size
    got_t = gt.cpu().numpy().astype(np.float64)
    ref_t = ref_gt.reshape(-1)
    assert rel(got_t, ref_t) <= 1e-2 and cosine(got_t, ref_t) >= 0.999, (rel(got_t, ref_t), cosine(got_t, ref_t))
    # entries no row touches stay exactly zero
    assert np.all(got_t[ref_t == 0] == 0)


def test_weights_round_trip_and_adam_moves_them(built):
    sc = scenes.cornell_box(1000, 16, 16)
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=1, train_spp=2, train_steps=2))
    W, table = network(10)
    tr.set_cache_weights(flat(W), table)
    w0, t0 = tr.cache_weights(table=True)
    assert np.array_equal(w0, flat(W)) and np.array_equal(t0, table.astype(np.float32).reshape(-1))
    tr.set_params(sc.gt_params)
    tr.cache_train(TraceOptions(spp_r=16, max_depth=3), iteration=0)
    w1, t1 = tr.cache_weights(table=True)
    st = tr.cache_status()
    assert st["train_steps"] == 2 and st["records"] > 0 and np.isfinite(st["last_loss"])
    # each Adam step moves a weight by at most about lr (the bias-corrected
    # ratio m / sqrt(v) can exceed 1 slightly when successive gradients grow)
    moved = np.abs(w1 - w0)
    assert moved.max() <= 2.1 * 1e-2 and np.mean(moved > 0) > 0.5
    assert np.any(t1 != t0)


# ---------------------------------------------------------------------------
# The cached estimator against the cut-path oracle
# ---------------------------------------------------------------------------

def cached_setup(b_term, w=16, h=16, seed_net=12):
    sc = scenes.cornell_box(1000, w, h)
    rng = np.random.default_rng(3)
    p = sc.gt_params.astype(np.float32).copy()
    p[:, 7:10] += rng.uniform(0.0, 0.15, (sc.n_segments, 3)).astype(np.float32)
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=b_term))
    tr.set_params(p)
    W, table = network(seed_net, out_scale=30.0)
    tr.set_cache_weights(flat(W), table)
    st = tr.cache_status()
    return sc, p.astype(np.float64), tr, W, table, np.array(st["lo"], np.float64), np.array(st["hi"], np.float64)


@pytest.mark.parametrize("b_term,D", [(1, 3), (2, 3), (1, 5)])
def test_cached_image_matches_oracle(built, b_term, D):
    sc, p, tr, W, table, lo, hi = cached_setup(b_term)
    spp = 8
    opts = TraceOptions(spp_r=spp, max_depth=D)
    img = tr.render(opts, view=0, set_id=0, spp=spp, iteration=2).cpu().numpy().astype(np.float64)
    osc = O.OracleScene(sc)
    term = osc.cache_terminals(p, b_term, spp=spp, max_depth=D, set_id=0, iteration=2, seed=SEED)
    cval, _ = K.cached_values(term, p, W, table, lo, hi, BF)
    ref = K.cached_image(term, spp, cval)
    cache_part = (term["beta"] * cval).reshape(-1, spp, 3).mean(1)
    assert np.linalg.norm(cache_part) > 0.1 * np.linalg.norm(ref)  # the cache term matters here
    assert rel(img, ref) <= 1e-2, rel(img, ref)


def test_cached_image_full_size_room_sampled_pixels(built):
    """The 61k-triangle room at its benchmark size (8 views of 320x240, 32
    spp, depth 5) with the cache at vertex 1 and a random network: 24 pixels
    sampled across the views, recomputed one by one by the cut-path oracle
    composed with the oracle network (the queries read the table's FP16
    copy, the oracle the FP32 table)."""
    sc = scenes.room_60k()
    rng = np.random.default_rng(5)
    p = sc.gt_params.astype(np.float32).copy()
    p[:, 7:10] += rng.uniform(0.0, 0.05, (sc.n_segments, 3)).astype(np.float32)
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=1))
    tr.set_params(p)
    W, table = network(14, out_scale=30.0)
    tr.set_cache_weights(flat(W), table)
    st = tr.cache_status()
    lo, hi = np.array(st["lo"], np.float64), np.array(st["hi"], np.float64)
    spp = 32
    img = tr.render(TraceOptions(spp_r=spp, max_depth=5), view=-1, set_id=0, spp=spp,
                    iteration=1).cpu().numpy().astype(np.float64)
    osc = O.OracleScene(sc)
    p64 = p.astype(np.float64)
    got, ref, part = [], [], []
    for v in range(len(sc.cameras)):
        px = rng.choice(320 * 240, 3, replace=False).astype(np.uint32)
        term = osc.cache_terminals(p64, 1, view=v, pixels=px, spp=spp, max_depth=5, set_id=0, iteration=1,
                                   seed=SEED)
        cval, _ = K.cached_values(term, p64, W, table, lo, hi, BF)
        ref.append(K.cached_image(term, spp, cval))
        part.append((term["beta"] * cval).reshape(-1, spp, 3).mean(1))
        got.append(img[tr.offsets[v] + px.astype(np.int64)])
    got, ref, part = np.concatenate(got), np.concatenate(ref), np.concatenate(part)
    assert np.linalg.norm(part) > 0.1 * np.linalg.norm(ref)  # the cache term matters here
    assert rel(got, ref) <= 1e-2, rel(got, ref)
    tr.close()


@pytest.mark.parametrize("b_term", [1, 2])
def test_cached_gradient_matches_oracle(built, b_term):
    sc, p, tr, W, table, lo, hi = cached_setup(b_term)
    spp, D = 8, 3
    opts = TraceOptions(spp_r=spp, spp_d=spp, max_depth=D)
    wimg = np.random.default_rng(9).normal(size=(tr.n_pix, 3)).astype(np.float32)
    g = tr.backward(torch.from_numpy(wimg).cuda(), opts, set_id=1, iteration=4).cpu().numpy().astype(np.float64)
    osc = O.OracleScene(sc)
    term = osc.cache_terminals(p, b_term, spp=spp, max_depth=D, set_id=1, iteration=4, seed=SEED)
    cval, cjac = K.cached_values(term, p, W, table, lo, hi, BF)
    ref = osc.cache_gradient(p, wimg, b_term, cval, cjac, spp=spp, max_depth=D, set_id=1, iteration=4,
                             seed=SEED)
    assert cosine(g, ref) >= 0.999, cosine(g, ref)
    assert rel(g, ref) <= 1e-2, rel(g, ref)


@pytest.mark.parametrize("b_term", [1, 2])
def test_training_records_match_oracle(built, b_term):
    sc = scenes.cornell_box(1000, 24, 24)
    p = sc.gt_params.astype(np.float32)
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=b_term, train_spp=3, train_steps=1,
                                       record_capacity=1 << 16))
    tr.set_params(p)
    D = 4
    tr.cache_train(TraceOptions(spp_r=16, max_depth=D), iteration=7)
    rec = tr.cache_records(1 << 16)
    osc = O.OracleScene(sc)
    ref = osc.cache_records(p.astype(np.float64), b_term, spp=3, max_depth=D, set_id=3, iteration=7, seed=SEED)
    ids_gpu = rec[:, 0].astype(np.int64)
    assert len(np.unique(ids_gpu)) == len(ids_gpu)
    ids_ref = np.nonzero(ref["seg"] >= 0)[0]
    common = np.intersect1d(ids_gpu, ids_ref)
    assert len(common) >= 0.995 * max(len(ids_gpu), len(ids_ref))
    order = np.argsort(ids_gpu)
    rec = rec[order][np.searchsorted(ids_gpu[order], common)]
    assert np.array_equal(rec[:, 1].astype(np.int64), ref["seg"][common])
    diam = float(np.linalg.norm(sc.positions.max(0) - sc.positions.min(0)))
    assert np.max(np.abs(rec[:, 2:5] - ref["x"][common])) <= 1e-4 * diam
    assert np.max(np.abs(rec[:, 5:8] - ref["wi"][common])) <= 1e-3
    assert np.max(np.abs(rec[:, 8:11] - ref["ns"][common])) <= 1e-3
    t_gpu, t_ref = rec[:, 11:14].astype(np.float64), ref["target"][common]
    assert rel(t_gpu, t_ref) <= 2e-3, rel(t_gpu, t_ref)
    per = np.linalg.norm(t_gpu - t_ref, axis=1) / np.maximum(np.linalg.norm(t_ref, axis=1), 1e-6)
    assert np.mean(per <= 1e-3) >= 0.99


# ---------------------------------------------------------------------------
# Switches, fallback and training
# ---------------------------------------------------------------------------

def test_disabled_or_out_of_range_cache_is_the_plain_tracer(built):
    sc = scenes.cornell_box(1000, 32, 32)
    p = sc.gt_params
    opts = TraceOptions(spp_r=8, max_depth=3)
    plain = Tracer(sc, seed=SEED)
    plain.configure("wavefront")
    plain.set_params(p)
    ref = plain.render(opts, view=0, set_id=0, spp=8).cpu().numpy()
    for co in [CacheOptions(enabled=False, b_term=1), CacheOptions(enabled=True, b_term=3)]:
        tr = cache_tracer(sc, co)
        tr.set_params(p)
        assert np.array_equal(tr.render(opts, view=0, set_id=0, spp=8).cpu().numpy(), ref)


def test_bias_monitor_falls_back_to_the_plain_tracer(built):
    sc = scenes.cornell_box(1000, 32, 32)
    p = sc.gt_params
    opts = TraceOptions(spp_r=8, spp_d=8, max_depth=3)
    plain = Tracer(sc, seed=SEED)
    plain.configure("wavefront")
    plain.set_params(p)
    target = plain.render(TraceOptions(spp_r=64, max_depth=3), set_id=2, spp=64)
    ref = plain.render(opts, view=0, set_id=0, spp=8).cpu().numpy()
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=1, bias_threshold=1e-6))
    tr.set_params(p)
    tr.set_targets(target)
    ib, gb = tr.cache_bias(opts, spp=8)
    assert ib > 1e-6 and gb > 1e-6
    st = tr.cache_status()
    assert st["fell_back"] and not st["active"]
    assert st["image_bias"] == ib and st["grad_bias"] == gb
    assert np.array_equal(tr.render(opts, view=0, set_id=0, spp=8).cpu().numpy(), ref)


def test_training_lowers_the_loss_and_the_bias(built):
    sc = scenes.cornell_box(1000, 32, 32)
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=1, train_spp=4, train_steps=4))
    tr.set_params(sc.gt_params)
    opts = TraceOptions(spp_r=64, spp_d=8, max_depth=3)
    bias0, _ = tr.cache_bias(opts, spp=64)
    losses = []
    for it in range(150):
        tr.cache_train(opts, iteration=it)
        if it < 5 or it >= 140:
            losses.append(tr.cache_status()["last_loss"])
    bias1, _ = tr.cache_bias(opts, spp=64)
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5]), losses
    assert bias1 < 0.5 * bias0, (bias0, bias1)


def test_cached_optimisation_steps(built):
    """ipt_step with the cache: forward and adjoint use it, the training pass
    follows, and the loss goes down as in the plain optimisation."""
    sc = scenes.cornell_box(1000, 32, 32)
    plain = Tracer(sc, seed=SEED)
    plain.set_params(sc.gt_params)
    target = plain.render(TraceOptions(spp_r=256, max_depth=3), set_id=2, spp=256)
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=1, train_spp=2, train_steps=2))
    tr.set_targets(target)
    p0 = sc.gt_params.copy()
    p0[:, 0:3] = 0.5
    tr.set_params(p0)
    from paper_1903_07145_gb300.tracer import AdamOptions
    opts = TraceOptions(spp_r=4, spp_d=4, max_depth=3)
    losses = [tr.step(opts, AdamOptions(lr=2e-2)) for _ in range(200)]
    st = tr.cache_status()
    assert st["active"] and st["train_steps"] == 400
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5]), (losses[:5], losses[-20:])


def test_trained_cache_gains_over_the_plain_estimator(built):
    """What the trained network gains: at 4 samples per pixel, the cached
    image is closer to the converged image (plain tracer, 4096 spp) than the
    plain estimator's, because the cache replaces the noisy tail of every
    path by its learned mean (and costs fewer traced rays); an untrained
    cache is worse than the plain estimator, so the gain is the training's."""
    sc = scenes.cornell_box(1000, 64, 64)
    plain = Tracer(sc, seed=SEED)
    plain.configure("wavefront")
    plain.set_params(sc.gt_params)
    D = 3
    ref = plain.render(TraceOptions(spp_r=4096, max_depth=D), set_id=2, spp=4096).cpu().numpy()
    opts = TraceOptions(spp_r=4, spp_d=4, max_depth=D)
    err_plain = rel(plain.render(opts, set_id=0, spp=4).cpu().numpy(), ref)
    tr = cache_tracer(sc, CacheOptions(enabled=True, b_term=1, train_spp=4, train_steps=4))
    tr.set_params(sc.gt_params)
    err_untrained = rel(tr.render(opts, set_id=0, spp=4).cpu().numpy(), ref)
    train = TraceOptions(spp_r=64, max_depth=D)
    for it in range(400):
        tr.cache_train(train, iteration=it)
    err_cached = rel(tr.render(opts, set_id=0, spp=4).cpu().numpy(), ref)
    print(f"image error at 4 spp: plain {err_plain:.4f}, untrained cache {err_untrained:.4f}, "
          f"trained cache {err_cached:.4f}")
    assert err_untrained > err_plain
    assert err_cached < 0.9 * err_plain
