"""FP64 CPU oracle for Inverse Path Tracing -- test infrastructure.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module.  It wraps ``libipt_oracle.so`` (built from ``ipt_oracle.cpp`` with
g++) and adds the loss, residual and Adam steps as plain numpy in float64.
It shares no code with the CUDA path.

Loss (Sec. 3.2, Eq. 3 uses L1; the L2 form is the default here):
    L2: E = (1/N) sum_j,c (I_R^A - I_C)^2,  dE/dI = 2 (I_R^A - I_C) / N
    L1: E = (1/N) sum_j,c |I_R^A - I_C|,    dE/dI = sgn(I_R^A - I_C) / N
N is the number of pixel-channels over all views.  The printed sign of Eq. 4
is that of the gradient of -E; the descent direction uses sgn(I_R - I_C).
Residual and derivative use independent sample sets (Sec. 3.3): set 0 for
the residual image, set 1 for the derivative paths.

Parity status: pinned (see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ipt_oracle.cpp")
LIB = os.path.join(HERE, "libipt_oracle.so")

SET_RESIDUAL, SET_DERIVATIVE, SET_TARGET, SET_CACHE, SET_PICK = 0, 1, 2, 3, 4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-pthread", "-o", LIB + ".tmp", SRC]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class Camera(C.Structure):
    _fields_ = [("cam_to_world", C.c_double * 12), ("fov_y_deg", C.c_double),
                ("width", C.c_uint32), ("height", C.c_uint32)]


class Opts(C.Structure):
    _fields_ = [("spp", C.c_uint32), ("max_depth", C.c_uint32), ("nee", C.c_int32),
                ("mis", C.c_int32), ("profile", C.c_int32), ("set", C.c_uint32),
                ("iteration", C.c_uint32), ("scene_id", C.c_uint32), ("seed", C.c_uint64),
                ("emission_scale", C.c_double), ("pixel_offset", C.c_uint32), ("model", C.c_uint32)]


MODEL_LAMBERT_GGX, MODEL_DISNEY = 0, 1
STRIDE = {MODEL_LAMBERT_GGX: 10, MODEL_DISNEY: 16}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.ora_scene_create.restype = P
            L.ora_scene_create.argtypes = [P, C.c_uint32, P, P, C.c_uint32, P, C.c_uint32]
            L.ora_scene_destroy.argtypes = [P]
            L.ora_scene_diameter.restype = C.c_double
            L.ora_scene_diameter.argtypes = [P]
            L.ora_scene_areas.argtypes = [P, P, P]
            L.ora_philox4x32_10.argtypes = [P, P, P]
            L.ora_intersect.argtypes = [P, C.c_uint32, P, P, P, C.c_double, C.c_int32,
                                        P, P, P, P, C.c_int32]
            L.ora_brdf.argtypes = [P, P, P, P, P, dp, dp]
            L.ora_brdf.restype = C.c_int
            L.ora_ggx_D.restype = C.c_double
            L.ora_ggx_D.argtypes = [C.c_double, C.c_double]
            L.ora_smith_lambda.restype = C.c_double
            L.ora_smith_lambda.argtypes = [C.c_double, C.c_double]
            L.ora_bsdf_sample.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, P, dp]
            L.ora_bsdf_pdf.restype = C.c_double
            L.ora_bsdf_pdf.argtypes = [P, P, P, P]
            L.ora_disney_brdf.argtypes = [P, P, P, P, P, P, P]
            L.ora_disney_brdf.restype = C.c_int
            L.ora_disney_pdf.argtypes = [P, P, P, P, P]
            L.ora_disney_pdf.restype = C.c_double
            L.ora_disney_sample.argtypes = [P, P, P, P, C.c_double, C.c_double, C.c_double, P, dp]
            L.ora_disney_lobes.argtypes = [P, P]
            L.ora_light_sample.argtypes = [P, P, C.c_uint32, P, P, P, P]
            L.ora_light_sample.restype = C.c_int
            L.ora_render.argtypes = [P, C.POINTER(Camera), P, P, C.POINTER(Opts), P, P,
                                     C.c_uint32, P, P, C.c_int32]
            L.ora_gradient.argtypes = [P, C.POINTER(Camera), P, P, C.POINTER(Opts), P, P,
                                       C.c_uint32, P, P, C.c_int32]
            L.ora_count_rays.argtypes = [P, C.POINTER(Camera), P, P, C.POINTER(Opts), P,
                                         C.c_uint32, P, P]
            L.ora_cache_terminals.argtypes = [P, C.POINTER(Camera), P, P, C.POINTER(Opts),
                                              C.c_uint32, P, C.c_uint32, P, P, P, P, P, P,
                                              C.c_int32]
            L.ora_cache_gradient.argtypes = [P, C.POINTER(Camera), P, P, C.POINTER(Opts),
                                             C.c_uint32, P, C.c_uint32, P, P, P, P, C.c_int32]
            L.ora_cache_records.argtypes = [P, C.POINTER(Camera), P, P, C.POINTER(Opts),
                                            C.c_uint32, P, C.c_uint32, P, P, P, P, P, C.c_int32]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().ora_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def camera_struct(cam) -> Camera:
    c = Camera()
    m = np.asarray(cam.cam_to_world, np.float64).reshape(12)
    for i in range(12):
        c.cam_to_world[i] = float(m[i])
    c.fov_y_deg = float(cam.fov_y_deg)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


class OracleScene:
    """FP64 copy of a scene (from the float32 arrays the generator returns)."""

    def __init__(self, scene):
        self.scene = scene
        self.pos = np.ascontiguousarray(scene.positions, np.float32)
        self.nrm = None if scene.normals is None else np.ascontiguousarray(scene.normals, np.float32)
        self.idx = np.ascontiguousarray(scene.indices, np.uint32)
        self.seg = np.ascontiguousarray(scene.tri_segment, np.uint32)
        self.n_seg = int(scene.n_segments)
        self.h = lib().ora_scene_create(_p(self.pos), self.pos.shape[0], _p(self.nrm),
                                        _p(self.idx), self.idx.shape[0], _p(self.seg),
                                        self.n_seg)
        self.cams = [camera_struct(c) for c in scene.cameras]
        self.offsets = np.concatenate([[0], np.cumsum([c.width * c.height for c in scene.cameras])])

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.ora_scene_destroy(h)
            self.h = None

    @property
    def diameter(self) -> float:
        return lib().ora_scene_diameter(self.h)

    def areas(self):
        ta = np.zeros(self.idx.shape[0])
        sa = np.zeros(self.n_seg)
        lib().ora_scene_areas(self.h, _p(ta), _p(sa))
        return ta, sa

    def intersect(self, orig, dirs, skip=None, tmin=0.0, brute=False, threads=None):
        o = np.ascontiguousarray(orig, np.float64)
        d = np.ascontiguousarray(dirs, np.float64)
        n = o.shape[0]
        sk = None if skip is None else np.ascontiguousarray(skip, np.int32)
        tri = np.zeros(n, np.int32)
        t = np.zeros(n)
        u = np.zeros(n)
        v = np.zeros(n)
        lib().ora_intersect(self.h, n, _p(o), _p(d), _p(sk), float(tmin), int(brute),
                            _p(tri), _p(t), _p(u), _p(v), threads or default_threads())
        return tri, t, u, v

    def opts(self, view=0, spp=16, max_depth=3, nee=True, mis=True, profile=0, set_id=0,
             iteration=0, seed=0, scene_id=0, model=MODEL_LAMBERT_GGX):
        o = Opts()
        o.model = model
        o.spp = spp
        o.max_depth = max_depth
        o.nee = int(nee)
        o.mis = int(mis)
        o.profile = profile
        o.set = set_id
        o.iteration = iteration
        o.scene_id = scene_id
        o.seed = seed
        o.emission_scale = float(self.scene.emission_scale)
        o.pixel_offset = int(self.offsets[view])
        return o

    def render(self, params, view=0, pixels=None, sparams=None, threads=None, sample_base=None, **kw):
        """Mean and mean-of-squares images (npix, 3) for one view.
        sample_base: per listed pixel, the counter of its first sample."""
        cam = self.cams[view]
        p = np.ascontiguousarray(params, np.float64)
        sp = None if sparams is None else np.ascontiguousarray(sparams, np.float64)
        px = None if pixels is None else np.ascontiguousarray(pixels, np.uint32)
        n = cam.width * cam.height if px is None else px.shape[0]
        sb = None if sample_base is None else np.ascontiguousarray(sample_base, np.uint32).reshape(n)
        mean = np.zeros((n, 3))
        msq = np.zeros((n, 3))
        o = self.opts(view=view, **kw)
        lib().ora_render(self.h, C.byref(cam), _p(p), _p(sp), C.byref(o), _p(px), _p(sb), n,
                         _p(mean), _p(msq), threads or default_threads())
        return mean, msq

    def gradient(self, params, g, view=0, pixels=None, sparams=None, threads=None, sample_base=None, **kw):
        """J^T g for one view: g is (npix, 3); returns (S, 10), or (S, 16) for
        the Disney model."""
        cam = self.cams[view]
        p = np.ascontiguousarray(params, np.float64)
        sp = None if sparams is None else np.ascontiguousarray(sparams, np.float64)
        px = None if pixels is None else np.ascontiguousarray(pixels, np.uint32)
        n = cam.width * cam.height if px is None else px.shape[0]
        sb = None if sample_base is None else np.ascontiguousarray(sample_base, np.uint32).reshape(n)
        gg = np.ascontiguousarray(g, np.float64).reshape(n, 3)
        o = self.opts(view=view, **kw)
        out = np.zeros((self.n_seg, STRIDE[o.model]))
        lib().ora_gradient(self.h, C.byref(cam), _p(p), _p(sp), C.byref(o), _p(px), _p(sb), n,
                           _p(gg), _p(out), threads or default_threads())
        return out

    def count_rays(self, params, view=0, pixels=None, **kw):
        cam = self.cams[view]
        p = np.ascontiguousarray(params, np.float64)
        px = None if pixels is None else np.ascontiguousarray(pixels, np.uint32)
        n = cam.width * cam.height if px is None else px.shape[0]
        nv = np.zeros(1, np.uint64)
        nn = np.zeros(1, np.uint64)
        o = self.opts(view=view, **kw)
        lib().ora_count_rays(self.h, C.byref(cam), _p(p), None, C.byref(o), _p(px), n,
                             _p(nv), _p(nn))
        return int(nv[0]), int(nn[0])

    def _npix(self, view, pixels):
        cam = self.cams[view]
        px = None if pixels is None else np.ascontiguousarray(pixels, np.uint32)
        return cam, px, (cam.width * cam.height if px is None else px.shape[0])

    def cache_terminals(self, params, b_term, view=0, pixels=None, sparams=None, threads=None, **kw):
        """Per path row (pixel i, sample k -> i * spp + k) of the cached
        estimator: prefix value, beta_b, x, wi, ns and segment (-1: no
        terminal vertex)."""
        cam, px, n = self._npix(view, pixels)
        o = self.opts(view=view, **kw)
        rows = n * o.spp
        p = np.ascontiguousarray(params, np.float64)
        sp = None if sparams is None else np.ascontiguousarray(sparams, np.float64)
        out = {k: np.zeros((rows, 3)) for k in ("prefix", "beta", "x", "wi", "ns")}
        seg = np.zeros(rows, np.int32)
        lib().ora_cache_terminals(self.h, C.byref(cam), _p(p), _p(sp), C.byref(o), int(b_term), _p(px), n,
                                  _p(out["prefix"]), _p(out["beta"]), _p(out["x"]), _p(out["wi"]),
                                  _p(out["ns"]), _p(seg), threads or default_threads())
        out["seg"] = seg
        return out

    def cache_gradient(self, params, g, b_term, cval, cjac, view=0, pixels=None, sparams=None,
                       threads=None, **kw):
        """J^T g of the cached estimator given per-row cache values (rows, 3)
        and Jacobians (rows, 3, 7) with respect to (kd, ks, r)."""
        cam, px, n = self._npix(view, pixels)
        o = self.opts(view=view, **kw)
        p = np.ascontiguousarray(params, np.float64)
        sp = None if sparams is None else np.ascontiguousarray(sparams, np.float64)
        gg = np.ascontiguousarray(g, np.float64).reshape(n, 3)
        cv = np.ascontiguousarray(cval, np.float64).reshape(n * o.spp, 3)
        cj = np.ascontiguousarray(cjac, np.float64).reshape(n * o.spp, 21)
        out = np.zeros((self.n_seg, 10))
        lib().ora_cache_gradient(self.h, C.byref(cam), _p(p), _p(sp), C.byref(o), int(b_term), _p(px), n,
                                 _p(gg), _p(cv), _p(cj), _p(out), threads or default_threads())
        return out

    def cache_records(self, params, b_term, view=0, pixels=None, sparams=None, threads=None, **kw):
        """Training records of full-length paths: x, wi, ns, segment (-1: the
        path ends before b_term) and the reflected-radiance target at b_term."""
        cam, px, n = self._npix(view, pixels)
        o = self.opts(view=view, **kw)
        rows = n * o.spp
        p = np.ascontiguousarray(params, np.float64)
        sp = None if sparams is None else np.ascontiguousarray(sparams, np.float64)
        out = {k: np.zeros((rows, 3)) for k in ("x", "wi", "ns", "target")}
        seg = np.zeros(rows, np.int32)
        lib().ora_cache_records(self.h, C.byref(cam), _p(p), _p(sp), C.byref(o), int(b_term), _p(px), n,
                                _p(out["x"]), _p(out["wi"]), _p(out["ns"]), _p(seg), _p(out["target"]),
                                threads or default_threads())
        out["seg"] = seg
        return out

    def light_sample(self, sparams, u):
        u = np.ascontiguousarray(u, np.float64).reshape(-1, 4)
        n = u.shape[0]
        tri = np.zeros(n, np.int32)
        y = np.zeros((n, 3))
        pa = np.zeros(n)
        sp = np.ascontiguousarray(sparams, np.float64)
        rc = lib().ora_light_sample(self.h, _p(sp), n, _p(u), _p(tri), _p(y), _p(pa))
        if rc != 0:
            raise ValueError("no emitting segment")
        return tri, y, pa


def brdf(params10, n, wi, wo):
    p = np.ascontiguousarray(params10, np.float64)
    f = np.zeros(3)
    s = C.c_double()
    ds = C.c_double()
    ok = lib().ora_brdf(_p(p), _p(np.asarray(n, np.float64)), _p(np.asarray(wi, np.float64)),
                        _p(np.asarray(wo, np.float64)), _p(f), C.byref(s), C.byref(ds))
    return f, s.value, ds.value, bool(ok)


def ggx_D(nh, alpha):
    return lib().ora_ggx_D(float(nh), float(alpha))


def smith_lambda(c, alpha):
    return lib().ora_smith_lambda(float(c), float(alpha))


def bsdf_sample(params10, n, wi, u_lobe, u1, u2):
    p = np.ascontiguousarray(params10, np.float64)
    wo = np.zeros(3)
    pdf = C.c_double()
    lib().ora_bsdf_sample(_p(p), _p(np.asarray(n, np.float64)), _p(np.asarray(wi, np.float64)),
                          float(u_lobe), float(u1), float(u2), _p(wo), C.byref(pdf))
    return wo, pdf.value


def bsdf_pdf(params10, n, wi, wo):
    p = np.ascontiguousarray(params10, np.float64)
    return lib().ora_bsdf_pdf(_p(p), _p(np.asarray(n, np.float64)),
                              _p(np.asarray(wi, np.float64)), _p(np.asarray(wo, np.float64)))


def _vec3s(*vs):
    """float64 copies kept alive by the caller for the duration of a call."""
    return [np.ascontiguousarray(v, np.float64).reshape(3) for v in vs]


def disney_brdf(m13, n, x, wi, wo, jacobian=False):
    """Disney model (Sec. 4.1) at one configuration: f_r (3,), and with
    jacobian the (3, 13) derivatives with respect to the material values."""
    m = np.ascontiguousarray(m13, np.float64)
    n, x, wi, wo = _vec3s(n, x, wi, wo)
    f = np.zeros(3)
    J = np.zeros((3, 13)) if jacobian else None
    ok = lib().ora_disney_brdf(_p(m), _p(n), _p(x), _p(wi), _p(wo), _p(f), _p(J))
    return (f, J, bool(ok)) if jacobian else (f, bool(ok))


def disney_pdf(m13, n, x, wi, wo):
    m = np.ascontiguousarray(m13, np.float64)
    n, x, wi, wo = _vec3s(n, x, wi, wo)
    return lib().ora_disney_pdf(_p(m), _p(n), _p(x), _p(wi), _p(wo))


def disney_sample(m13, n, x, wi, u_lobe, u1, u2):
    m = np.ascontiguousarray(m13, np.float64)
    n, x, wi = _vec3s(n, x, wi)
    wo = np.zeros(3)
    pdf = C.c_double()
    lib().ora_disney_sample(_p(m), _p(n), _p(x), _p(wi), float(u_lobe), float(u1), float(u2), _p(wo),
                            C.byref(pdf))
    return wo, pdf.value


def disney_lobes(m13):
    m = np.ascontiguousarray(m13, np.float64)
    p = np.zeros(3)
    lib().ora_disney_lobes(_p(m), _p(p))
    return p


# ---------------------------------------------------------------------------
# Loss, residual and optimiser (plain numpy, float64)
# ---------------------------------------------------------------------------

def residual(image, target, n_total, loss="l2"):
    """Upstream gradient dE/dI and the loss contribution of these pixels."""
    r = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    if loss == "l2":
        return 2.0 * r / n_total, float(np.sum(r * r)) / n_total
    return np.sign(r) / n_total, float(np.sum(np.abs(r))) / n_total


def adam_update(theta, grad, m, v, t, free=None, lr=5e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                l1_emission=1e-3):
    """One Adam step (Kingma & Ba 2015) on (S, 10) parameters with an L1
    regulariser on emission (Sec. 4.4) added to the gradient, then the
    clamps kd, ks in [0,1], roughness in [0.02,1], emission >= 0.
    Parameters whose free mask is 0 keep their value and moments."""
    theta = np.array(theta, np.float64)
    g = np.array(grad, np.float64)
    g[:, 7:10] += l1_emission * np.sign(theta[:, 7:10])
    m = np.array(m, np.float64)
    v = np.array(v, np.float64)
    fm = np.ones_like(theta, bool) if free is None else np.asarray(free, bool)
    m_new = beta1 * m + (1 - beta1) * g
    v_new = beta2 * v + (1 - beta2) * g * g
    mh = m_new / (1 - beta1 ** t)
    vh = v_new / (1 - beta2 ** t)
    th_new = theta - lr * mh / (np.sqrt(vh) + eps)
    th_new[:, 0:6] = np.clip(th_new[:, 0:6], 0.0, 1.0)
    th_new[:, 6] = np.clip(th_new[:, 6], 0.02, 1.0)
    th_new[:, 7:10] = np.maximum(th_new[:, 7:10], 0.0)
    theta = np.where(fm, th_new, theta)
    m = np.where(fm, m_new, m)
    v = np.where(fm, v_new, v)
    return theta, m, v


def adam_update_disney(theta, grad, m, v, t, free=None, lr=5e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                       l1_emission=1e-3):
    """adam_update for the Disney model's (S, 16) parameters: the 13
    material values clamped to [0, 1] (roughness to [0.02, 1]), emission
    (13-15) >= 0 with the L1 regulariser."""
    theta = np.array(theta, np.float64)
    g = np.array(grad, np.float64)
    g[:, 13:16] += l1_emission * np.sign(theta[:, 13:16])
    m = np.array(m, np.float64)
    v = np.array(v, np.float64)
    fm = np.ones_like(theta, bool) if free is None else np.asarray(free, bool)
    m_new = beta1 * m + (1 - beta1) * g
    v_new = beta2 * v + (1 - beta2) * g * g
    mh = m_new / (1 - beta1 ** t)
    vh = v_new / (1 - beta2 ** t)
    th_new = theta - lr * mh / (np.sqrt(vh) + eps)
    th_new[:, 0:13] = np.clip(th_new[:, 0:13], 0.0, 1.0)
    th_new[:, 7] = np.clip(th_new[:, 7], 0.02, 1.0)
    th_new[:, 13:16] = np.maximum(th_new[:, 13:16], 0.0)
    theta = np.where(fm, th_new, theta)
    m = np.where(fm, m_new, m)
    v = np.where(fm, v_new, v)
    return theta, m, v


def loss_grad(osc: OracleScene, params, targets, spp_r, spp_d, max_depth, iteration=0, seed=0,
              loss="l2", nee=True, mis=True, profile=0, same_set=False, pixels=None,
              threads=None, model=MODEL_LAMBERT_GGX):
    """One nested-SGD gradient evaluation over all views (or a pixel subset per
    view): render set 0, residual against targets, J^T g with set 1."""
    n_total = sum(c.width * c.height * 3 for c in osc.cams) if pixels is None else \
        sum(len(p) * 3 for p in pixels)
    grad = np.zeros((osc.n_seg, STRIDE[model]))
    total = 0.0
    for v in range(len(osc.cams)):
        px = None if pixels is None else pixels[v]
        img, _ = osc.render(params, view=v, pixels=px, spp=spp_r, max_depth=max_depth,
                            nee=nee, mis=mis, profile=profile, set_id=SET_RESIDUAL,
                            iteration=iteration, seed=seed, threads=threads, model=model)
        tgt = targets[v] if px is None else targets[v][px]
        g, l_v = residual(img, tgt.reshape(-1, 3), n_total, loss)
        total += l_v
        grad += osc.gradient(params, g, view=v, pixels=px, spp=spp_d, max_depth=max_depth,
                             nee=nee, mis=mis, profile=profile,
                             set_id=SET_RESIDUAL if same_set else SET_DERIVATIVE,
                             iteration=iteration, seed=seed, threads=threads, model=model)
    return total, grad


# ---------------------------------------------------------------------------
# Stochastic pixel batches (Sec. 4.5: B pixels drawn uniformly from all pixels
# of all images per step)
# ---------------------------------------------------------------------------

def pick_pixels(n_pixels, batch, iteration, seed=0, scene_id=0):
    """Global pixel ids (over all views, view-major) of the B batch entries of
    one iteration, drawn uniformly with replacement.  Entry b takes the first
    word x of Philox4x32-10 at key (seed_lo, seed_hi ^ scene_id) and counter
    (b, 0, (4 << 24) | iteration, 0); its pixel is floor(x * n / 2^32), an
    integer map both sides evaluate exactly."""
    key = [seed & 0xFFFFFFFF, ((seed >> 32) & 0xFFFFFFFF) ^ scene_id]
    out = np.zeros(batch, np.uint32)
    for b in range(batch):
        x = int(philox4x32_10([b, 0, (SET_PICK << 24) | (iteration & 0xFFFFFF), 0], key)[0])
        out[b] = (x * int(n_pixels)) >> 32
    return out


def loss_grad_batch(osc: OracleScene, params, targets, batch, spp_r, spp_d, max_depth, iteration=0,
                    seed=0, loss="l2", nee=True, mis=True, profile=0, same_set=False, scene_id=0,
                    sparams=None, threads=None):
    """One nested-SGD gradient evaluation on a stochastic pixel batch: the B
    entries of pick_pixels; entry b renders spp_r samples of set 0 from sample
    counter b*spp_r and differentiates spp_d samples of set 1 from b*spp_d; the
    loss is normalised by the 3B entry-channels, so its expectation over the
    draw is the full-image loss.  Returns (loss, grad, picked ids)."""
    offs = np.asarray(osc.offsets, np.int64)
    n_pix = int(sum(c.width * c.height for c in osc.cams))
    ids = pick_pixels(n_pix, batch, iteration, seed, scene_id)
    views = np.searchsorted(offs, ids.astype(np.int64), side="right") - 1
    n_total = 3 * batch
    grad = np.zeros((osc.n_seg, 10))
    total = 0.0
    for v in range(len(osc.cams)):
        ent = np.nonzero(views == v)[0].astype(np.uint32)
        if ent.size == 0:
            continue
        px = (ids[ent].astype(np.int64) - offs[v]).astype(np.uint32)
        img, _ = osc.render(params, view=v, pixels=px, sparams=sparams, sample_base=ent * np.uint32(spp_r),
                            spp=spp_r,
                            max_depth=max_depth, nee=nee, mis=mis, profile=profile,
                            set_id=SET_RESIDUAL, iteration=iteration, seed=seed, scene_id=scene_id,
                            threads=threads)
        g, l_v = residual(img, np.asarray(targets[v]).reshape(-1, 3)[px], n_total, loss)
        total += l_v
        grad += osc.gradient(params, g, view=v, pixels=px, sparams=sparams, spp=spp_d,
                             sample_base=ent * np.uint32(spp_r if same_set else spp_d),
                             max_depth=max_depth, nee=nee, mis=mis, profile=profile,
                             set_id=SET_RESIDUAL if same_set else SET_DERIVATIVE,
                             iteration=iteration, seed=seed, scene_id=scene_id, threads=threads)
    return total, grad, ids
