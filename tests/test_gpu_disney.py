"""Disney material model (Sec. 4.1) on the CUDA path, through the C ABI, on
both integrators: images, loss and gradient match the FP64 oracle on the
same sample sets (whole images and stochastic pixel batches, several depths),
and Adam on the Disney parameters recovers the base colour and emission of a
Cornell box."""
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
    sc = scenes.cornell_box(1000, 24, 20)
    p = scenes.disney_materials(sc, 3)
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator)
    tr.disney_set_params(p)
    opts = TraceOptions(max_depth=depth)
    img = tr.disney_render(opts, view=0, set_id=0, spp=16, iteration=5).cpu().numpy()
    osc = O.OracleScene(sc)
    ref, _ = osc.render(p.astype(np.float64), spp=16, max_depth=depth, set_id=0, iteration=5, seed=SEED,
                        model=O.MODEL_DISNEY)
    assert rel(img, ref) <= 2e-3, rel(img, ref)
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
