"""Disney material model (Sec. 4.1) on the CUDA path, through the C ABI, on
both integrators: images match the FP64 oracle on the same sample set
(relative L2 <= 1e-3, several depths) and with independent sample sets at
4096 spp (per pixel within 3 combined standard errors but for the chance
fraction); loss and gradient match it on the same sample sets (whole images
and stochastic pixel batches); the gradient equals central differences of
the GPU's own forward (h = 1e-3, 20 random values); and Adam on the Disney
parameters recovers the base colour and emission of a Cornell box."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_1903_07145_gb300 import _lib as L  # noqa: E402
from paper_1903_07145_gb300 import scenes  # noqa: E402
from paper_1903_07145_gb300.tracer import AdamOptions, TraceOptions, Tracer  # noqa: E402

pytestmark = pytest.mark.gpu
SEED = 0x5EED_D15E


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


INTEGRATORS = ["megakernel", "wavefront"]


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("depth", [1, 3, 5])
def test_image_matches_oracle(built, depth, integrator):
    """Same sample set: FP32 and FP64 paths part only at rare grazing or edge
    decisions (the bar of the Lambert + GGX images)."""
    sc = scenes.cornell_box(1000, 64, 64)
    p = scenes.disney_materials(sc, 3)
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator)
    tr.disney_set_params(p)
    opts = TraceOptions(max_depth=depth)
    img = tr.disney_render(opts, view=0, set_id=0, spp=32, iteration=5).cpu().numpy()
    osc = O.OracleScene(sc)
    ref, _ = osc.render(p.astype(np.float64), spp=32, max_depth=depth, set_id=0, iteration=5, seed=SEED,
                        model=O.MODEL_DISNEY)
    assert rel(img, ref) <= 1e-3, rel(img, ref)
    tr.close()


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_full_size_room_sampled_pixels(built, integrator):
    """The 61k-triangle room at its benchmark size (8 views of 320x240, 32
    spp, depth 5) with random Disney materials: 16 pixels sampled across the
    views, recomputed one by one by the oracle's Disney model with the same
    key."""
    sc = scenes.room_60k()
    p = scenes.disney_materials(sc, 7)
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator)
    tr.disney_set_params(p)
    img = tr.disney_render(TraceOptions(max_depth=5), view=-1, set_id=0, spp=32, iteration=3).cpu().numpy()
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(9)
    got, ref = [], []
    for v in range(len(sc.cameras)):
        px = rng.choice(320 * 240, 2, replace=False).astype(np.uint32)
        m, _ = osc.render(p.astype(np.float64), view=v, pixels=px, spp=32, max_depth=5, set_id=0, iteration=3,
                          seed=SEED, model=O.MODEL_DISNEY)
        ref.append(m)
        got.append(img[tr.offsets[v] + px.astype(np.int64)])
    assert rel(np.concatenate(got), np.concatenate(ref)) <= 1e-3, rel(np.concatenate(got), np.concatenate(ref))
    tr.close()


def test_image_independent_keys_4096spp(built):
    """Independent Philox keys on the two sides: the difference is Monte Carlo
    noise, so at most 0.5% of pixel-channels lie beyond 3 combined standard
    errors (0.27% by chance) and the image difference matches the combined
    noise (a bias would add to it)."""
    sc = scenes.cornell_box(1000, 48, 48)
    p = scenes.disney_materials(sc, 3)
    spp = 4096
    tr = Tracer(sc, seed=101)
    tr.disney_set_params(p)
    g, gm2 = tr.disney_render(TraceOptions(max_depth=3), view=0, set_id=2, spp=spp, with_msq=True)
    g = g.cpu().numpy().astype(np.float64)
    gm2 = gm2.cpu().numpy().astype(np.float64)
    tr.close()
    osc = O.OracleScene(sc)
    o, om2 = osc.render(p.astype(np.float64), spp=spp, max_depth=3, set_id=2, seed=202,
                        model=O.MODEL_DISNEY)
    se2 = (np.maximum(gm2 - g * g, 0) + np.maximum(om2 - o * o, 0)) / spp
    z = np.abs(g - o) / np.sqrt(se2 + 1e-30)
    frac = np.mean(z > 3.0)
    assert frac <= 0.005, frac
    floor = math.sqrt(se2.sum()) / np.linalg.norm(o)
    assert rel(g, o) <= 1.2 * floor + 1e-3, (rel(g, o), floor)


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_gradient_central_differences(built, integrator):
    """(E(p + h e_k) - E(p - h e_k)) / 2h of the L2 loss of the GPU's own
    images (same sample set, sampling frozen at p) against the loss gradient
    of ipt_disney_loss_grad with the residual's samples as derivative
    samples, on 20 random material and emission values (h = 1e-3)."""
    sc = scenes.cornell_box(1000, 32, 32)
    p = scenes.disney_materials(sc, 5).astype(np.float32)
    rng = np.random.default_rng(6)
    target = rng.uniform(0.0, 0.8, (32 * 32, 3)).astype(np.float32)
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator)
    tr.disney_set_params(p)
    tr.set_targets(torch.from_numpy(target).cuda())
    it = 3
    opts = TraceOptions(spp_r=16, spp_d=16, max_depth=3, gradcheck_same_set=True)
    _, g = tr.disney_loss_grad(opts, iteration=it)
    g = g.cpu().numpy().astype(np.float64).reshape(-1)
    pt = torch.from_numpy(p).cuda()
    tgt = target.astype(np.float64)
    n = tgt.size

    def loss_at(q):
        tr.disney_set_params(q)
        img = tr.disney_render(opts, view=0, set_id=0, spp=16, iteration=it, sampling_params=pt)
        r = img.cpu().numpy().astype(np.float64) - tgt
        return float((r * r).sum() / n)

    h = 1e-3
    # values inside (h, 1 - h), where no clamp or floor is active
    cand = [k for k in range(p.size) if h < p.reshape(-1)[k] < 1 - h]
    ks = rng.choice(cand, 20, replace=False)
    scale = np.abs(g).max()
    for k in ks:
        qp = p.copy().reshape(-1)
        qm = p.copy().reshape(-1)
        qp[k] += h
        qm[k] -= h
        fd = (loss_at(qp.reshape(p.shape)) - loss_at(qm.reshape(p.shape))) / (2 * h)
        assert abs(fd - g[k]) <= 1e-2 * max(abs(g[k]), 1e-2 * scale), (k, fd, g[k])
    tr.close()


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("batch,loss", [(0, "l2"), (0, "l1"), (300, "l2")])
def test_loss_and_gradient_match_oracle(built, batch, loss, integrator):
    sc = scenes.cornell_box(1000, 24, 20)
    rng = np.random.default_rng(8)
    p = scenes.disney_materials(sc, 4).astype(np.float64)
    targets = [rng.uniform(0.0, 0.8, (24 * 20, 3))]
    spp_r, spp_d, D, it = 16, 8, 3, 7
    osc = O.OracleScene(sc)
    if batch:
        lo, go, _ = _oracle_batch(osc, p, targets, batch, spp_r, spp_d, D, it, loss)
    else:
        lo, go = O.loss_grad(osc, p, targets, spp_r, spp_d, D, iteration=it, seed=SEED, loss=loss,
                             model=O.MODEL_DISNEY)
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator)
    tr.disney_set_params(p.astype(np.float32))
    tr.set_targets(torch.from_numpy(targets[0].astype(np.float32)).cuda())
    lg, gg = tr.disney_loss_grad(TraceOptions(spp_r=spp_r, spp_d=spp_d, max_depth=D, loss=loss,
                                              pixel_batch=batch), iteration=it)
    gg = gg.cpu().numpy().astype(np.float64)
    assert gg.shape == (sc.n_segments, 16)
    assert abs(lg - lo) <= 1e-3 * abs(lo), (lg, lo)
    cos = float((gg * go).sum() / (np.linalg.norm(gg) * np.linalg.norm(go)))
    assert cos >= 0.999 and rel(gg, go) <= 1e-2, (cos, rel(gg, go))
    # every material value of a visible wall gets a gradient
    assert np.count_nonzero(go[0, 0:13]) == 13
    tr.close()


def _oracle_batch(osc, p, targets, batch, spp_r, spp_d, D, it, loss):
    """Pixel-batch loss and gradient of the Disney model: the draw, sample
    counters and 3B normalisation of oracle.loss_grad_batch."""
    n_pix = osc.cams[0].width * osc.cams[0].height
    ids = O.pick_pixels(n_pix, batch, it, seed=SEED, scene_id=0)
    ent = np.arange(batch, dtype=np.uint32)
    img, _ = osc.render(p, pixels=ids, sample_base=ent * np.uint32(spp_r), spp=spp_r, max_depth=D,
                        set_id=O.SET_RESIDUAL, iteration=it, seed=SEED, model=O.MODEL_DISNEY)
    g, lo = O.residual(img, targets[0][ids], 3 * batch, loss)
    go = osc.gradient(p, g, pixels=ids, sample_base=ent * np.uint32(spp_d), spp=spp_d, max_depth=D,
                      set_id=O.SET_DERIVATIVE, iteration=it, seed=SEED, model=O.MODEL_DISNEY)
    return lo, go, ids


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_optimisation_recovers_base_colour_and_emission(built, integrator):
    """From grey walls and no light, Adam on base colour and emission (other
    material values held at the truth) brings the parameters within a few
    per cent of the truth on the segments the camera sees."""
    sc = scenes.cornell_box(1000, 48, 48)
    truth = scenes.disney_materials(sc, 9)
    truth[:, 4] = 0.0  # dielectric walls, so that the base colour shows
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator)
    tr.disney_set_params(truth)
    tr.set_targets(tr.disney_render(TraceOptions(max_depth=3), set_id=L.IPT_SET_TARGET, spp=1024))
    free = np.zeros((sc.n_segments, 16), np.uint8)
    free[:, 0:3] = 1
    free[:, 13:16] = 1
    p0 = truth.copy()
    p0[:, 0:3] = 0.5
    p0[:, 13:16] = 0.0
    tr.disney_set_params(p0, free_mask=free)
    opts = TraceOptions(spp_r=16, spp_d=4, max_depth=3)
    first = tr.disney_loss_grad(opts, iteration=1 << 20)[0]
    for it in range(1500):
        tr.disney_step(opts, AdamOptions(lr=1e-2 * 0.5 ** (it // 500)), want_loss=False)
    last = tr.disney_loss_grad(opts, iteration=1 << 20)[0]
    got = tr.disney_params()
    assert last < 0.05 * first, (first, last)
    e, g = got[1, 13:16], truth[1, 13:16]
    assert np.all(np.abs(e / g - 1.0) <= 0.1), (e, g)
    for s in (0, 2, 3, 4):  # floor, back, left, right walls
        assert np.all(np.abs(got[s, 0:3] - truth[s, 0:3]) <= 0.05), (s, got[s, 0:3], truth[s, 0:3])
    tr.close()


def test_argument_checks(built):
    sc = scenes.cornell_box(1000, 8, 8)
    tr = Tracer(sc, seed=1)
    with pytest.raises(L.IptError):  # nothing set yet
        tr.disney_render(TraceOptions(), set_id=0, spp=4)
    p = scenes.disney_materials(sc, 1)
    p[2, 5] = np.nan
    with pytest.raises(L.IptError):
        tr.disney_set_params(p)
    tr.close()
