"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances:
  * Philox: bit-exact.
  * ray hits: identical triangle ids on >= 99.99% of a fixed ray set, t within
    1e-5 relative on those;
  * images: same Philox key -> image relative L2 <= 1e-3 (FP32 vs FP64 paths
    only diverge at rare grazing/edge decisions); independent keys at 4096 spp
    -> at most 0.5% of pixels beyond 3 combined standard errors and image
    relative L2 <= 1e-3 plus the Monte Carlo floor;
  * gradients: cosine >= 0.999 and relative L2 <= 1e-2 against the oracle;
    central differences (h = 1e-3) of the GPU's own forward on 20 random
    parameters, relative error <= 1e-2.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_1903_07145_gb300 import scenes  # noqa: E402
from paper_1903_07145_gb300 import _lib  # noqa: E402
from paper_1903_07145_gb300.tracer import (AdamOptions, TraceOptions, Tracer,  # noqa: E402
                                           render)

pytestmark = pytest.mark.gpu

SEED = 1234


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def cosine(a, b):
    return float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return True


INTEGRATORS = ["megakernel", "wavefront"]


def tracer(sc, seed, integrator="wavefront", **kw):
    tr = Tracer(sc, seed=seed, **kw)
    tr.configure(integrator)
    return tr


def perturbed(scene, seed=3, emission=0.15):
    """Parameters away from the initial guess: random materials, some
    emission on every segment (so light sampling covers many segments)."""
    rng = np.random.default_rng(seed)
    p = scene.gt_params.astype(np.float32).copy()
    p[:, 7:10] += rng.uniform(0.0, emission, (scene.n_segments, 3)).astype(np.float32)
    return p


# ---------------------------------------------------------------------------
def test_philox_bit_exact(built):
    sc = scenes.cornell_box(1000, 8, 8)
    tr = Tracer(sc, seed=1)
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = [0, 0, 0, 0]
    key[0] = [0, 0]
    out = tr.philox(torch.from_numpy(ctr.view(np.int32)), torch.from_numpy(key.view(np.int32)))
    got = out.cpu().numpy().view(np.uint32)
    for i in range(0, n, 97):
        assert list(got[i]) == list(O.philox4x32_10(ctr[i], key[i]))
    assert list(got[0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bvh_width", [2, 4, 8])
@pytest.mark.parametrize("which", ["cornell", "room_small", "room_61k", "room_516k"])
def test_ray_hits_match_oracle(built, which, bvh_width):
    if which == "cornell":
        sc = scenes.cornell_box(1000)
    elif which == "room_small":
        sc = scenes.indoor_room(7, n_cuboids=6, cuboid_sub=3, room_sub=4, n_lights=2, n_views=1,
                                width=16, height=12)
    elif which == "room_61k":
        sc = scenes.room_60k()
    else:
        sc = scenes.room_500k()
        sc.cameras = sc.cameras[:1]
    tr = Tracer(sc, seed=1)
    tr.configure("wavefront", bvh_width=bvh_width)
    o, d = scenes.random_rays(sc, 100000, seed=5)
    tri, t, u, v = [x.cpu().numpy() for x in tr.trace_rays(torch.from_numpy(o), torch.from_numpy(d))]
    osc = O.OracleScene(sc)
    otri, ot, ou, ov = osc.intersect(o, d, brute=(which == "cornell"))
    same = tri == otri
    assert same.mean() >= 0.9999, same.mean()
    hit = same & (otri >= 0)
    # t within 1e-5 relative; for short hits the FP32 floor is the absolute
    # precision of the coordinates (1e-5 of 1% of the scene diameter)
    floor = 1e-2 * osc.diameter
    t_ok = np.abs(t[hit] - ot[hit]) <= 1e-5 * np.maximum(ot[hit], floor)
    assert t_ok.mean() >= 0.9999, (t_ok.mean(), np.sort(np.abs(t[hit] - ot[hit]) / ot[hit])[-5:])
    # barycentrics on every hit that passes the t bound: the hit point they
    # give differs from the oracle's by at most 1e-5 of max(t, floor), the
    # precision of t itself.  FP32 edge functions carry a relative error of a
    # few ulps of t / triangle size, so the point error is ~1e-7 of t; a
    # dropped or swapped barycentric moves it by a triangle's size.
    tri_o = otri[hit][t_ok]
    P = sc.positions.astype(np.float64)[sc.indices[tri_o]]          # (n, 3 vertices, 3)
    ug, vg = u[hit][t_ok].astype(np.float64), v[hit][t_ok].astype(np.float64)
    uo, vo = ou[hit][t_ok], ov[hit][t_ok]
    pg = (1 - ug - vg)[:, None] * P[:, 0] + ug[:, None] * P[:, 1] + vg[:, None] * P[:, 2]
    po = (1 - uo - vo)[:, None] * P[:, 0] + uo[:, None] * P[:, 1] + vo[:, None] * P[:, 2]
    dp = np.linalg.norm(pg - po, axis=1) / np.maximum(ot[hit][t_ok], floor)
    assert dp.max() <= 1e-5, np.sort(dp)[-5:]
    if which in ("cornell", "room_small"):
        # triangles of the scene's own size: the barycentrics themselves
        assert np.max(np.abs(ug - uo)) < 1e-3 and np.max(np.abs(vg - vo)) < 1e-3
    assert np.median(np.abs(ug - uo)) < 1e-5
    # skipping the hit triangle never returns it again
    skip = torch.from_numpy(otri.astype(np.int32))
    tri2 = tr.trace_rays(torch.from_numpy(o), torch.from_numpy(d), skip)[0].cpu().numpy()
    assert not np.any((tri2 == otri) & (otri >= 0))


# ---------------------------------------------------------------------------
def render_both(sc, params, spp, D, seed_gpu, seed_ora, view=0, set_id=2, nee=True, mis=True, profile=0,
                sparams=None, integrator="wavefront"):
    tr = tracer(sc, seed_gpu, integrator)
    tr.set_params(params)
    opts = TraceOptions(spp_r=spp, max_depth=D, nee=nee, mis=mis,
                        emission_profile="cosine" if profile == 0 else "uniform")
    sp = None if sparams is None else torch.from_numpy(np.asarray(sparams, np.float32)).cuda()
    pp = torch.from_numpy(np.asarray(params, np.float32)).cuda()
    img, msq = tr.render(opts, view=view, set_id=set_id, spp=spp, params=pp, sampling_params=sp,
                         with_msq=True)
    osc = O.OracleScene(sc)
    om, omsq = osc.render(params, view=view, spp=spp, max_depth=D, nee=nee, mis=mis, profile=profile,
                          set_id=set_id, seed=seed_ora, sparams=sparams)
    return img.cpu().numpy().astype(np.float64), msq.cpu().numpy().astype(np.float64), om, omsq


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("nee,mis,profile,D", [(True, True, 0, 3), (False, False, 0, 3),
                                               (True, False, 1, 2), (True, True, 0, 0),
                                               (True, True, 1, 6)])
def test_image_same_key(built, nee, mis, profile, D, integrator):
    sc = scenes.cornell_box(1000, 64, 64)
    p = perturbed(sc)
    g, _, o, _ = render_both(sc, p, 32, D, SEED, SEED, nee=nee, mis=mis, profile=profile,
                             integrator=integrator)
    assert rel(g, o) <= 1e-3, rel(g, o)


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_image_same_key_ragged_spp_and_views(built, integrator):
    """spp = 12 (3 samples per lane over 4 lanes), several views of
    different sizes, with the whole-image (view = -1) render; the wavefront
    runs with chunks of 1024 slots, so chunks end inside views."""
    sc = scenes.indoor_room(11, n_cuboids=8, cuboid_sub=3, room_sub=4, n_lights=2, n_views=3,
                            width=37, height=23)
    sc.cameras[1] = scenes.Camera(sc.cameras[1].cam_to_world, 50.0, 19, 31)
    p = perturbed(sc)
    tr = Tracer(sc, seed=SEED)
    tr.configure(integrator, wavefront_slots=1024)
    tr.set_params(p)
    opts = TraceOptions(spp_r=12, max_depth=4)
    img = tr.render(opts, view=-1, set_id=2, spp=12).cpu().numpy()
    osc = O.OracleScene(sc)
    ref = np.concatenate([osc.render(p, view=v, spp=12, max_depth=4, set_id=2, seed=SEED)[0]
                          for v in range(3)])
    assert img.shape == ref.shape
    # 12 spp on 2291 pixels: a few paths diverge between FP32 and FP64 at
    # grazing or edge decisions; they dominate the small image's error
    assert rel(img, ref) <= 2e-3
    per_pixel = np.linalg.norm(img - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-6)
    assert np.mean(per_pixel <= 1e-3) >= 0.99


def test_image_independent_keys_4096spp(built):
    sc = scenes.cornell_box(1000, 64, 64)
    p = sc.gt_params
    spp = 4096
    g, gm2, o, om2 = render_both(sc, p, spp, 3, 101, 202)
    se2 = (np.maximum(gm2 - g * g, 0) + np.maximum(om2 - o * o, 0)) / spp
    z = np.abs(g - o) / np.sqrt(se2 + 1e-30)
    frac = np.mean(z > 3.0)          # per pixel-channel; 0.27% expected by chance
    assert frac <= 0.005, frac
    # with independent keys the difference is Monte Carlo noise: its size must
    # match the combined standard errors (a bias would add to it)
    floor = math.sqrt(se2.sum()) / np.linalg.norm(o)
    assert rel(g, o) <= 1.2 * floor + 1e-3, (rel(g, o), floor)


def test_image_with_vertex_normals(built):
    sc = scenes.cornell_box(1000, 32, 32)
    rng = np.random.default_rng(2)
    # per-vertex normals tilted from the face normals (interpolated shading)
    P = sc.positions.astype(np.float64)
    nrm = np.zeros_like(P)
    for t in sc.indices:
        a, b, c = P[t]
        n = np.cross(b - a, c - a)
        nrm[t] += n / np.linalg.norm(n)
    nrm += rng.normal(scale=0.05, size=nrm.shape)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    sc.normals = nrm.astype(np.float32)
    p = perturbed(sc)
    g, _, o, _ = render_both(sc, p, 32, 3, SEED, SEED)
    assert rel(g, o) <= 1e-3


# ---------------------------------------------------------------------------
def backward_both(sc, p, spp, D, set_id=1, nee=True, mis=True, profile=0, pixels_mask=None, seed=SEED,
                  integrator="wavefront"):
    tr = tracer(sc, seed, integrator)
    tr.set_params(p)
    rng = np.random.default_rng(9)
    w = rng.normal(size=(tr.n_pix, 3)).astype(np.float32)
    if pixels_mask is not None:
        w[~pixels_mask] = 0
    opts = TraceOptions(spp_r=spp, spp_d=spp, max_depth=D, nee=nee, mis=mis,
                        emission_profile="cosine" if profile == 0 else "uniform")
    g = tr.backward(torch.from_numpy(w).cuda(), opts, set_id=set_id).cpu().numpy().astype(np.float64)
    osc = O.OracleScene(sc)
    ref = np.zeros((sc.n_segments, 10))
    for v in range(len(sc.cameras)):
        a, b = tr.offsets[v], tr.offsets[v + 1]
        px = None
        wv = w[a:b]
        if pixels_mask is not None:
            px = np.nonzero(pixels_mask[a:b])[0].astype(np.uint32)
            if px.size == 0:
                continue
            wv = wv[px]
        ref += osc.gradient(p, wv, view=v, pixels=px, spp=spp, max_depth=D, nee=nee, mis=mis,
                            profile=profile, set_id=set_id, seed=seed)
    return g, ref


@pytest.mark.parametrize("integrator", INTEGRATORS)
@pytest.mark.parametrize("nee,mis,profile,D", [(True, True, 0, 3), (False, False, 0, 3),
                                               (True, False, 1, 2), (True, True, 0, 6), (True, True, 0, 1)])
def test_gradient_matches_oracle_cornell(built, nee, mis, profile, D, integrator):
    sc = scenes.cornell_box(1000, 64, 64)
    p = perturbed(sc)
    g, ref = backward_both(sc, p, 16, D, nee=nee, mis=mis, profile=profile, integrator=integrator)
    assert cosine(g, ref) >= 0.999, cosine(g, ref)
    assert rel(g, ref) <= 1e-2, rel(g, ref)


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_gradient_matches_oracle_large_room_crop(built, integrator):
    """~516k triangles, 150 segments: a 64x48 crop of view 0 (the other
    pixels get a zero upstream gradient and are skipped)."""
    sc = scenes.room_500k()
    sc.cameras = sc.cameras[:2]
    p = perturbed(sc, emission=0.05)
    W, H = sc.cameras[0].width, sc.cameras[0].height
    mask = np.zeros(sum(c.width * c.height for c in sc.cameras), bool)
    for y in range(200, 248):
        mask[y * W + 300: y * W + 364] = True
    g, ref = backward_both(sc, p, 16, 6, pixels_mask=mask, integrator=integrator)
    assert cosine(g, ref) >= 0.999, cosine(g, ref)
    assert rel(g, ref) <= 1e-2, rel(g, ref)


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_gradient_central_differences(built, integrator):
    """<w, I(p+h e_k) - I(p-h e_k)>/2h against J^T w on 20 random parameters,
    same sample set on both sides and sampling frozen at p (h = 1e-3)."""
    sc = scenes.cornell_box(1000, 32, 32)
    p = perturbed(sc)
    tr = tracer(sc, SEED, integrator)
    tr.set_params(p)
    opts = TraceOptions(spp_r=16, spp_d=16, max_depth=3, gradcheck_same_set=True)
    rng = np.random.default_rng(4)
    w = torch.from_numpy(rng.normal(size=(tr.n_pix, 3)).astype(np.float32)).cuda()
    pt = torch.from_numpy(p).cuda()
    g = tr.backward(w, opts, set_id=0, params=pt, sampling_params=pt).cpu().numpy().reshape(-1)
    h = 1e-3
    ks = rng.choice(sc.n_segments * 10, 20, replace=False)
    scale = np.abs(g).max()
    for k in ks:
        pp = p.copy().reshape(-1)
        pm = p.copy().reshape(-1)
        pp[k] += h
        pm[k] -= h
        ip = tr.render(opts, set_id=0, spp=16, params=torch.from_numpy(pp.reshape(p.shape)).cuda(),
                       sampling_params=pt)
        im = tr.render(opts, set_id=0, spp=16, params=torch.from_numpy(pm.reshape(p.shape)).cuda(),
                       sampling_params=pt)
        fd = float((w.double() * (ip.double() - im.double())).sum() / (2 * h))
        assert abs(fd - g[k]) <= 1e-2 * max(abs(g[k]), 1e-2 * scale), (k, fd, g[k])


def test_gradient_central_differences_large_room(built):
    """The ~516k-triangle, 150-segment room at 640x480: central differences
    (h = 1e-3, same sample set on both sides, sampling frozen at p) of
    <w, I> against J^T w on 20 random parameters among those the weights
    reach, w nonzero on a 64x48 crop."""
    sc = scenes.room_500k()
    sc.cameras = sc.cameras[:1]
    p = perturbed(sc, emission=0.05)
    tr = tracer(sc, SEED, "wavefront")
    tr.set_params(p)
    opts = TraceOptions(spp_r=8, spp_d=8, max_depth=4, gradcheck_same_set=True)
    W = sc.cameras[0].width
    rng = np.random.default_rng(6)
    w_np = np.zeros((tr.n_pix, 3), np.float32)
    for y in range(200, 248):
        w_np[y * W + 300: y * W + 364] = rng.normal(size=(64, 3))
    w = torch.from_numpy(w_np).cuda()
    pt = torch.from_numpy(p).cuda()
    g = tr.backward(w, opts, set_id=0, params=pt, sampling_params=pt).cpu().numpy().reshape(-1)
    scale = np.abs(g).max()
    reached = np.flatnonzero(np.abs(g) > 1e-3 * scale)
    assert len(reached) >= 20
    h = 1e-3
    for k in rng.choice(reached, 20, replace=False):
        pp = p.copy().reshape(-1)
        pm = p.copy().reshape(-1)
        pp[k] += h
        pm[k] -= h
        ip = tr.render(opts, set_id=0, spp=8, params=torch.from_numpy(pp.reshape(p.shape)).cuda(),
                       sampling_params=pt)
        im = tr.render(opts, set_id=0, spp=8, params=torch.from_numpy(pm.reshape(p.shape)).cuda(),
                       sampling_params=pt)
        fd = float((w.double() * (ip.double() - im.double())).sum() / (2 * h))
        assert abs(fd - g[k]) <= 1e-2 * max(abs(g[k]), 1e-2 * scale), (k, fd, g[k])
    tr.close()


def test_autograd_function(built):
    sc = scenes.cornell_box(1000, 16, 16)
    tr = Tracer(sc, seed=SEED)
    p = torch.from_numpy(perturbed(sc)).cuda().requires_grad_(True)
    opts = TraceOptions(spp_r=16, spp_d=16, max_depth=3, gradcheck_same_set=True)
    img = render(p, tr, opts, set_id=0)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    direct = tr.backward(w, opts, set_id=0, params=p.detach(), sampling_params=p.detach())
    # same paths; only the order of the float gradient sums differs
    assert float(torch.linalg.norm(p.grad - direct) / torch.linalg.norm(direct)) <= 1e-5


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_loss_grad_and_adam_match_oracle(built, integrator):
    sc = scenes.cornell_box(1000, 32, 32)
    gt = sc.gt_params
    osc = O.OracleScene(sc)
    target, _ = osc.render(gt, spp=64, max_depth=3, set_id=2, seed=77)
    tr = tracer(sc, SEED, integrator)
    p0 = scenes.initial_params(sc, 0.5)
    tr.set_params(p0)
    tr.set_targets(torch.from_numpy(target.astype(np.float32)).cuda())
    opts = TraceOptions(spp_r=16, spp_d=16, max_depth=3)
    loss, grad = tr.loss_grad(opts, iteration=5)
    oloss, ograd = O.loss_grad(osc, p0, [target], 16, 16, 3, iteration=5, seed=SEED)
    assert abs(loss - oloss) <= 1e-4 * abs(oloss)
    g = grad.cpu().numpy()
    assert cosine(g, ograd) >= 0.999 and rel(g, ograd) <= 1e-2
    # one Adam step with the oracle's gradient
    adam = AdamOptions()
    tr.set_params(p0)
    tr.adam_step(adam, torch.from_numpy(ograd.astype(np.float32)).cuda())
    newp = tr.get_params()
    ref, _, _ = O.adam_update(p0, ograd, np.zeros_like(ograd), np.zeros_like(ograd), 1)
    assert np.max(np.abs(newp - ref)) < 1e-6


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_full_size_room_sampled_pixels(built, integrator):
    """The 61k-triangle room at its benchmark size (8 views of 320x240, 32
    spp, depth 5): 24 pixels sampled across the views, recomputed one by one
    by the oracle with the same key."""
    sc = scenes.room_60k()
    p = perturbed(sc, emission=0.02)
    tr = tracer(sc, SEED, integrator)
    tr.set_params(p)
    opts = TraceOptions(spp_r=32, max_depth=5)
    img = tr.render(opts, view=-1, set_id=0, spp=32).cpu().numpy()
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(3)
    got, ref = [], []
    for v in range(len(sc.cameras)):
        px = rng.choice(320 * 240, 3, replace=False).astype(np.uint32)
        m, _ = osc.render(p, view=v, pixels=px, spp=32, max_depth=5, set_id=0, seed=SEED)
        ref.append(m)
        got.append(img[tr.offsets[v] + px.astype(np.int64)])
    got = np.concatenate(got)
    ref = np.concatenate(ref)
    assert rel(got, ref) <= 1e-3, rel(got, ref)


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_full_size_large_room_sampled_pixels(built, integrator):
    """~516k triangles, 16 views of 640x480, 16 spp, depth 6: 16 sampled pixels."""
    sc = scenes.room_500k()
    p = perturbed(sc, emission=0.02)
    tr = tracer(sc, SEED, integrator)
    tr.set_params(p)
    opts = TraceOptions(spp_r=16, max_depth=6)
    img = tr.render(opts, view=-1, set_id=0, spp=16).cpu().numpy()
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(4)
    got, ref = [], []
    for v in range(len(sc.cameras)):
        px = rng.choice(640 * 480, 1, replace=False).astype(np.uint32)
        m, _ = osc.render(p, view=v, pixels=px, spp=16, max_depth=6, set_id=0, seed=SEED)
        ref.append(m)
        got.append(img[tr.offsets[v] + px.astype(np.int64)])
    assert rel(np.concatenate(got), np.concatenate(ref)) <= 1e-3


# ---------------------------------------------------------------------------
def test_degenerate_cases(built):
    # depth 0: only directly visible emission; no material gradient
    sc = scenes.cornell_box(1000, 16, 16)
    p = perturbed(sc)
    g, ref = backward_both(sc, p, 4, 0)
    assert np.all(g[:, 0:7] == 0) and np.allclose(g, ref, rtol=1e-4, atol=1e-7)
    # all-zero emission: black image, zero gradient
    q = p.copy()
    q[:, 7:10] = 0
    tr = Tracer(sc, seed=1)
    tr.set_params(q)
    opts = TraceOptions(spp_r=4, spp_d=4, max_depth=3)
    assert float(tr.render(opts, spp=4).abs().max()) == 0.0
    # single-pixel, single-sample view
    sc1 = scenes.cornell_box(1000, 1, 1)
    a, _, b, _ = render_both(sc1, p, 1, 3, SEED, SEED)
    assert rel(a, b) <= 1e-3 or np.allclose(a, b, atol=1e-5)


def test_invalid_arguments_rejected(built):
    sc = scenes.cornell_box(1000, 8, 8)
    tr = Tracer(sc, seed=1)
    ctx = tr.ctx
    import ctypes as C
    bad = sc.positions.copy()
    bad[3, 1] = np.nan
    idx = np.ascontiguousarray(sc.indices)
    seg = np.ascontiguousarray(sc.tri_segment)
    with pytest.raises(_lib.IptError) as e:
        _lib.ipt_scene_upload(ctx, C.c_void_p(bad.ctypes.data), bad.shape[0], None,
                              C.c_void_p(idx.ctypes.data), idx.shape[0], C.c_void_p(seg.ctypes.data), 7, 32.0)
    assert e.value.status == 1
    seg2 = seg.copy()
    seg2[0] = 99
    with pytest.raises(_lib.IptError):
        _lib.ipt_scene_upload(ctx, C.c_void_p(sc.positions.ctypes.data), sc.positions.shape[0], None,
                              C.c_void_p(idx.ctypes.data), idx.shape[0], C.c_void_p(seg2.ctypes.data), 7,
                              32.0)
    with pytest.raises(_lib.IptError):
        _lib.ipt_scene_upload(ctx, C.c_void_p(sc.positions.ctypes.data), sc.positions.shape[0], None,
                              C.c_void_p(idx.ctypes.data), 0, C.c_void_p(seg.ctypes.data), 7, 32.0)
    with pytest.raises(_lib.IptError):
        tr.render(TraceOptions(max_depth=65), spp=4)
    with pytest.raises(_lib.IptError):
        tr.backward(torch.zeros(64, 3, device="cuda"), TraceOptions(max_depth=9))
    with pytest.raises(_lib.IptError):
        tr.loss_grad(TraceOptions())            # no targets
    with pytest.raises(_lib.IptError):
        tr.render(TraceOptions(), spp=0)
    tr.synchronize()


@pytest.mark.parametrize("integrator", INTEGRATORS)
def test_loss_grad_shards_add_up(built, integrator):
    """ipt_loss_grad_shard over 3 pixel ranges sums to ipt_loss_grad (the
    random numbers are keyed by global pixel id, so each pixel's samples are
    the same whichever shard traces them)."""
    from paper_1903_07145_gb300.parallel import shard_range
    sc = scenes.cornell_box(1000, 32, 32)
    osc = O.OracleScene(sc)
    target, _ = osc.render(sc.gt_params, spp=16, max_depth=3, set_id=2, seed=5)
    tr = tracer(sc, SEED, integrator)
    tr.set_params(scenes.initial_params(sc, 0.5))
    tr.set_targets(torch.from_numpy(target.astype(np.float32)).cuda())
    opts = TraceOptions(spp_r=8, spp_d=8, max_depth=3)
    loss, grad = tr.loss_grad(opts, iteration=3)
    n = tr.n_pix
    tot_l, tot_g = 0.0, torch.zeros_like(grad)
    for r in range(3):
        b, c = shard_range(n, 3, r)
        l, g = tr.loss_grad_shard(opts, 3, b, c, n)
        tot_l += l
        tot_g += g
    assert abs(tot_l - loss) <= 1e-9 * abs(loss)
    assert rel(tot_g.cpu().numpy(), grad.cpu().numpy()) <= 1e-5
    with pytest.raises(_lib.IptError):
        tr.loss_grad_shard(opts, 3, n - 1, 2, n)


@pytest.mark.parametrize("spp,slots,bvh_width", [(32, 1 << 20, 4), (12, 4096, 4), (1, 1024, 4), (8, 4096, 2),
                                                  (16, 4096, 8)])
def test_wavefront_equals_megakernel(built, spp, slots, bvh_width):
    """Both integrators draw the same numbers at the same slots: images agree
    to float rounding, gradients to the order of the float sums."""
    sc = scenes.indoor_room(13, n_cuboids=10, cuboid_sub=3, room_sub=4, n_lights=3, n_views=2,
                            width=40, height=30)
    p = perturbed(sc, emission=0.05)
    out = {}
    for integ in INTEGRATORS:
        tr = Tracer(sc, seed=SEED)
        tr.configure(integ, wavefront_slots=slots, bvh_width=bvh_width)
        tr.set_params(p)
        opts = TraceOptions(spp_r=spp, spp_d=spp, max_depth=5)
        img = tr.render(opts, set_id=0, spp=spp).cpu().numpy()
        w = torch.from_numpy(np.random.default_rng(1).normal(size=(tr.n_pix, 3)).astype(np.float32)).cuda()
        g = tr.backward(w, opts, set_id=1).cpu().numpy()
        out[integ] = (img, g)
        tr.close()
    assert rel(out["wavefront"][0], out["megakernel"][0]) <= 1e-5
    assert rel(out["wavefront"][1], out["megakernel"][1]) <= 1e-4


def test_bvh_widths_give_the_same_images(built):
    """The binary, 4-wide and 8-wide BVHs find the same closest hits (up to
    exact ties), so images agree to float rounding."""
    sc = scenes.room_60k()
    sc.cameras = sc.cameras[:2]
    p = perturbed(sc, emission=0.02)
    imgs = []
    for width in (2, 4, 8):
        tr = Tracer(sc, seed=SEED)
        tr.configure("wavefront", bvh_width=width)
        tr.set_params(p)
        imgs.append(tr.render(TraceOptions(max_depth=5), set_id=0, spp=8).cpu().numpy())
        tr.close()
    assert rel(imgs[1], imgs[0]) <= 1e-4
    assert rel(imgs[2], imgs[0]) <= 1e-4


@pytest.mark.parametrize("bvh_width", [2, 4, 8])
def test_refill_points_give_the_same_results(built, bvh_width):
    """The traversal's refill point (trace_steps) only changes which lanes
    run which ray when: every ray's closest hit and occlusion stay the same,
    so images agree to float rounding and gradients to the order of the
    float sums, with a refill after every lane (1), at 8 and 16 idle lanes
    (16: the default), only when the whole warp is idle (32) and beyond it
    (100)."""
    sc = scenes.indoor_room(17, n_cuboids=10, cuboid_sub=3, room_sub=4, n_lights=3, n_views=2,
                            width=40, height=30)
    p = perturbed(sc, emission=0.05)
    opts = TraceOptions(spp_r=8, spp_d=8, max_depth=5)
    w = torch.from_numpy(np.random.default_rng(2).normal(size=(2 * 40 * 30, 3)).astype(np.float32)).cuda()
    out = []
    for steps in (1, 8, 16, 32, 100):
        tr = Tracer(sc, seed=SEED)
        tr.configure("wavefront", wavefront_slots=4096, trace_steps=steps, bvh_width=bvh_width)
        tr.set_params(p)
        out.append((tr.render(opts, set_id=0, spp=8).cpu().numpy(), tr.backward(w, opts, set_id=1).cpu().numpy()))
        tr.close()
    for img, g in out[1:]:
        assert rel(img, out[0][0]) <= 1e-6
        assert rel(g, out[0][1]) <= 1e-5


@pytest.mark.parametrize("bvh_width", [4, 8])
def test_ray_reordering_gives_the_same_results(built, bvh_width):
    """Reordering the secondary closest-hit queues by origin and direction
    cell only changes the order in which the traversal takes the rays: images
    and gradients equal those traced in queue order (gradients up to the
    order of the float sums), for coarse and fine bin grids, with chunks that
    end inside a view."""
    sc = scenes.indoor_room(17, n_cuboids=10, cuboid_sub=3, room_sub=4, n_lights=3, n_views=2,
                            width=40, height=30)
    p = perturbed(sc, emission=0.05)
    opts = TraceOptions(spp_r=8, spp_d=8, max_depth=5)
    w = torch.from_numpy(np.random.default_rng(2).normal(size=(2 * 40 * 30, 3)).astype(np.float32)).cuda()
    out = []
    for cells, dirs in ((0, 0), (1, 1), (4, 2), (4, 4), (2, 8), (16, 0)):
        tr = Tracer(sc, seed=SEED)
        tr.configure("wavefront", wavefront_slots=4096, bvh_width=bvh_width, sort_cells=cells, sort_dirs=dirs)
        assert tr.config()["sort_cells"] == cells
        tr.set_params(p)
        out.append((tr.render(opts, set_id=0, spp=8).cpu().numpy(), tr.backward(w, opts, set_id=1).cpu().numpy()))
        tr.close()
    for img, g in out[1:]:
        assert np.array_equal(img, out[0][0])
        assert rel(g, out[0][1]) <= 1e-5


@pytest.mark.parametrize("path", ["disney", "pixel_batch", "cache"])
def test_ray_reordering_other_paths(built, path):
    """The reordering under the Disney model's loss and gradient, under
    stochastic pixel batches and with the radiance cache ending paths: the
    same results as queue order (gradients up to the order of the float
    sums)."""
    from paper_1903_07145_gb300.tracer import CacheOptions
    sc = scenes.indoor_room(23, n_cuboids=8, cuboid_sub=3, room_sub=4, n_lights=2, n_views=2,
                            width=40, height=30)
    p = perturbed(sc, emission=0.05)
    out = []
    for cells in (0, 6):
        tr = Tracer(sc, seed=SEED)
        tr.configure("wavefront", wavefront_slots=8192, sort_cells=cells, sort_dirs=2 if cells else 0)
        if path == "disney":
            dp = scenes.disney_materials(sc, 5)
            tr.disney_set_params(dp)
            tr.set_targets(tr.disney_render(TraceOptions(max_depth=4), set_id=_lib.IPT_SET_TARGET, spp=16))
            dp[:, 0:3] = 0.5
            tr.disney_set_params(dp)
            loss, g = tr.disney_loss_grad(TraceOptions(spp_r=8, spp_d=8, max_depth=4), iteration=2)
            out.append((loss, g.cpu().numpy(), None))
        elif path == "pixel_batch":
            tr.set_params(sc.gt_params)
            tr.set_targets(tr.render(TraceOptions(max_depth=4), set_id=_lib.IPT_SET_TARGET, spp=16))
            tr.set_params(p)
            loss, g = tr.loss_grad(TraceOptions(spp_r=16, spp_d=2, max_depth=4, pixel_batch=256), iteration=3)
            out.append((loss, g.cpu().numpy(), None))
        else:
            tr.configure_cache(CacheOptions(enabled=True, b_term=1))
            rng = np.random.default_rng(8)  # a random network, so the cache's term is not zero
            tr.set_cache_weights(rng.normal(0.0, 0.2, _lib.IPT_CACHE_WEIGHTS).astype(np.float32),
                                 rng.normal(0.0, 0.5, _lib.IPT_CACHE_TABLE_FLOATS).astype(np.float32))
            tr.set_params(p)
            img = tr.render(TraceOptions(spp_r=8, max_depth=4), view=-1, set_id=0, spp=8).cpu().numpy()
            out.append((0.0, None, img))
        tr.close()
    (l0, g0, i0), (l1, g1, i1) = out
    if i0 is not None:
        assert np.array_equal(i0, i1)
    else:
        assert abs(l1 - l0) <= 1e-6 * abs(l0), (l0, l1)
        assert rel(g1, g0) <= 1e-5, rel(g1, g0)


def test_ray_reordering_rejects_too_many_bins(built):
    sc = scenes.cornell_box(1000, 16, 16)
    tr = Tracer(sc, seed=SEED)
    for cells, dirs in ((8, 2), (17, 0), (1, 17)):
        with pytest.raises(_lib.IptError):
            tr.configure("wavefront", sort_cells=cells, sort_dirs=dirs)
    tr.configure("wavefront", sort_cells=8, sort_dirs=1)
    tr.close()


def test_kernels_run_from_an_sm103a_binary(built):
    """The device loads the library's kernels from the sm_103a cubin, not a
    JIT-compiled PTX fallback."""
    binary, ptx = _lib.ipt_build_info(0)
    assert binary == 103, (binary, ptx)
