"""Torch-facing wrapper of the C ABI: one context plus one uploaded scene.

PyTorch provides device memory and the stream; every computation runs in
libipt.so's kernels.  The context is created on the current torch stream of
its device, so torch ops and the library's kernels are ordered.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .scenes import Scene


@dataclass
class TraceOptions:
    spp_r: int = 16
    spp_d: int = 16
    max_depth: int = 3
    loss: str = "l2"
    nee: bool = True
    mis: bool = True
    emission_profile: str = "cosine"
    gradcheck_same_set: bool = False
    pixel_batch: int = 0  # 0: every pixel; B: B pixels drawn per iteration (Sec. 4.5)

    def c(self) -> L.ipt_trace_opts:
        return L.ipt_trace_opts(self.spp_r, self.spp_d, self.max_depth,
                                0 if self.loss == "l2" else 1, int(self.nee), int(self.mis),
                                0 if self.emission_profile == "cosine" else 1,
                                int(self.gradcheck_same_set), int(self.pixel_batch))


@dataclass
class AdamOptions:
    lr: float = 5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    l1_emission: float = 1e-3

    def c(self) -> L.ipt_adam_opts:
        return L.ipt_adam_opts(self.lr, self.beta1, self.beta2, self.eps, self.l1_emission)


@dataclass
class CacheOptions:
    """Radiance-cache options (see ipt_cache_opts in include/ipt.h)."""
    enabled: bool = True
    b_term: int = 1
    train_spp: int = 0
    train_steps: int = 4
    record_capacity: int = 1 << 21
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.99
    eps: float = 1e-15
    bias_threshold: float = 0.0
    init_seed: int = 1

    def c(self) -> L.ipt_cache_opts:
        return L.ipt_cache_opts(int(self.enabled), self.b_term, self.train_spp, self.train_steps,
                                self.record_capacity, self.lr, self.beta1, self.beta2, self.eps,
                                self.bias_threshold, self.init_seed)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def cameras_c(cams):
    arr = (L.ipt_camera * len(cams))()
    for i, c in enumerate(cams):
        m = np.asarray(c.cam_to_world, np.float32).reshape(12)
        for k in range(12):
            arr[i].cam_to_world[k] = float(m[k])
        arr[i].fov_y_deg = float(c.fov_y_deg)
        arr[i].width = int(c.width)
        arr[i].height = int(c.height)
    return arr


class Tracer:
    def __init__(self, scene: Scene, device: int = 0, seed: int = 0, targets=None, flags: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("the inverse path tracer needs a CUDA device")
        self.scene = scene
        self.device = torch.device("cuda", device)
        # the library queues its work on torch's current stream, so torch ops
        # and the kernels stay ordered
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = L.ipt_create(device, stream, seed, flags & ~L.IPT_FLAG_OWN_STREAM)
        pos = np.ascontiguousarray(scene.positions, np.float32)
        nrm = None if scene.normals is None else np.ascontiguousarray(scene.normals, np.float32)
        idx = np.ascontiguousarray(scene.indices, np.uint32)
        seg = np.ascontiguousarray(scene.tri_segment, np.uint32)
        self.sid = L.ipt_scene_upload(self.ctx, _np_ptr(pos), pos.shape[0], _np_ptr(nrm),
                                      _np_ptr(idx), idx.shape[0], _np_ptr(seg), scene.n_segments,
                                      float(scene.emission_scale))
        self._cams = cameras_c(scene.cameras)
        L.ipt_views_set(self.ctx, self.sid, self._cams, len(scene.cameras), None, 0)
        self.n_seg = scene.n_segments
        self.sizes = [(c.height, c.width) for c in scene.cameras]
        self.offsets = np.concatenate([[0], np.cumsum([h * w for h, w in self.sizes])]).astype(np.int64)
        self.n_pix = int(self.offsets[-1])
        if targets is not None:
            self.set_targets(targets)

    def close(self):
        if getattr(self, "ctx", None):
            L.ipt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters ---------------------------------------------------------
    def set_params(self, params, free_mask=None):
        p = np.ascontiguousarray(np.asarray(params, np.float32).reshape(self.n_seg, 10))
        fm = None if free_mask is None else np.ascontiguousarray(np.asarray(free_mask, np.uint8))
        L.ipt_params_set(self.ctx, self.sid, _np_ptr(p), _np_ptr(fm))

    def get_params(self) -> np.ndarray:
        out = np.zeros((self.n_seg, 10), np.float32)
        L.ipt_params_get(self.ctx, self.sid, _np_ptr(out))
        return out

    def set_targets(self, targets):
        """targets: (n_pix, 3) float32 torch tensor on the device, or numpy."""
        if isinstance(targets, torch.Tensor):
            t = targets.to(self.device, torch.float32).contiguous()
            assert t.numel() == 3 * self.n_pix
            L.ipt_targets_set(self.ctx, self.sid, _ptr(t), 1)
            self._targets = t
        else:
            a = np.ascontiguousarray(np.asarray(targets, np.float32))
            assert a.size == 3 * self.n_pix
            L.ipt_targets_set(self.ctx, self.sid, _np_ptr(a), 0)
            self.synchronize()

    # -- path tracing -------------------------------------------------------
    def render(self, opts: TraceOptions, view: int = -1, set_id: int = L.IPT_SET_TARGET,
               spp: int | None = None, iteration: int = 0, params=None, sampling_params=None,
               with_msq: bool = False):
        n = self.n_pix if view < 0 else self.sizes[view][0] * self.sizes[view][1]
        img = torch.empty((n, 3), device=self.device, dtype=torch.float32)
        msq = torch.empty_like(img) if with_msq else None
        L.ipt_render(self.ctx, self.sid, view, opts.c(), set_id, opts.spp_r if spp is None else spp,
                     iteration,
                     _ptr(params), _ptr(sampling_params), _ptr(img), _ptr(msq))
        return (img, msq) if with_msq else img

    def backward(self, grad_image, opts: TraceOptions, set_id: int = L.IPT_SET_DERIVATIVE,
                 iteration: int = 0, params=None, sampling_params=None):
        g = grad_image.to(self.device, torch.float32).contiguous()
        assert g.numel() == 3 * self.n_pix
        out = torch.empty((self.n_seg, 10), device=self.device, dtype=torch.float32)
        L.ipt_backward(self.ctx, self.sid, opts.c(), set_id, iteration, _ptr(params),
                       _ptr(sampling_params), _ptr(g), _ptr(out))
        return out

    def loss_grad(self, opts: TraceOptions, iteration: int = 0):
        grad = torch.empty((self.n_seg, 10), device=self.device, dtype=torch.float32)
        loss = L.ipt_loss_grad(self.ctx, self.sid, opts.c(), iteration, True, _ptr(grad))
        return loss, grad

    def loss_grad_shard(self, opts: TraceOptions, iteration: int, pix_begin: int, pix_count: int,
                        n_total: int):
        grad = torch.empty((self.n_seg, 10), device=self.device, dtype=torch.float32)
        loss = L.ipt_loss_grad_shard(self.ctx, self.sid, opts.c(), iteration, pix_begin, pix_count,
                                     n_total, _ptr(grad))
        return loss, grad

    # -- Disney material model (Sec. 4.1; megakernel integrator) -------------
    def disney_set_params(self, params, free_mask=None):
        """(S, 16) blocks: base colour, subsurface, metallic, specular,
        specular tint, roughness, anisotropic, sheen, sheen tint, clearcoat,
        clearcoat gloss, emission."""
        p = np.ascontiguousarray(np.asarray(params, np.float32).reshape(self.n_seg, 16))
        fm = None if free_mask is None else np.ascontiguousarray(np.asarray(free_mask, np.uint8))
        L.ipt_disney_params_set(self.ctx, self.sid, _np_ptr(p), _np_ptr(fm))

    def disney_params(self) -> np.ndarray:
        out = np.zeros((self.n_seg, 16), np.float32)
        L.ipt_disney_params_get(self.ctx, self.sid, _np_ptr(out))
        return out

    def disney_render(self, opts: TraceOptions, view: int = -1, set_id: int = L.IPT_SET_TARGET,
                      spp: int | None = None, iteration: int = 0, sampling_params=None, with_msq: bool = False):
        n = self.n_pix if view < 0 else self.sizes[view][0] * self.sizes[view][1]
        img = torch.empty((n, 3), device=self.device, dtype=torch.float32)
        msq = torch.empty_like(img) if with_msq else None
        L.ipt_disney_render(self.ctx, self.sid, view, opts.c(), set_id, opts.spp_r if spp is None else spp,
                            iteration, _ptr(sampling_params), _ptr(img), _ptr(msq))
        return (img, msq) if with_msq else img

    def disney_loss_grad(self, opts: TraceOptions, iteration: int = 0):
        grad = torch.empty((self.n_seg, 16), device=self.device, dtype=torch.float32)
        loss = L.ipt_disney_loss_grad(self.ctx, self.sid, opts.c(), iteration, True, _ptr(grad))
        return loss, grad

    def disney_step(self, opts: TraceOptions, adam: AdamOptions, want_loss: bool = True):
        return L.ipt_disney_step(self.ctx, self.sid, opts.c(), adam.c(), want_loss)

    def adam_step(self, adam: AdamOptions, grad=None):
        L.ipt_adam_step(self.ctx, self.sid, _ptr(grad), adam.c())

    def step(self, opts: TraceOptions, adam: AdamOptions, want_loss: bool = True):
        return L.ipt_step(self.ctx, self.sid, opts.c(), adam.c(), want_loss)

    def trace_rays(self, orig, dirs, skip=None):
        o = orig.to(self.device, torch.float32).contiguous()
        d = dirs.to(self.device, torch.float32).contiguous()
        n = o.shape[0]
        sk = None if skip is None else skip.to(self.device, torch.int32).contiguous()
        tri = torch.empty(n, device=self.device, dtype=torch.int32)
        t = torch.empty(n, device=self.device, dtype=torch.float32)
        u = torch.empty_like(t)
        v = torch.empty_like(t)
        L.ipt_trace_rays(self.ctx, self.sid, n, _ptr(o), _ptr(d), _ptr(sk), _ptr(tri), _ptr(t),
                         _ptr(u), _ptr(v))
        return tri, t, u, v

    def checkpoint(self) -> bytes:
        """The scene's optimisation state (parameters, Adam state, iteration,
        radiance cache) as bytes."""
        return L.ipt_checkpoint_save(self.ctx, self.sid)

    def restore(self, data: bytes):
        L.ipt_checkpoint_load(self.ctx, self.sid, data)

    def pick_pixels(self, batch: int, iteration: int):
        """Global pixel ids of the pixel batch of `iteration` (int32 tensor)."""
        out = torch.empty(max(batch, 1), dtype=torch.int32, device=self.device)
        L.ipt_pick_pixels(self.ctx, self.sid, batch, iteration, _ptr(out))
        return out[:batch]

    def philox(self, ctr, key):
        c = ctr.to(self.device, torch.int32).contiguous()
        k = key.to(self.device, torch.int32).contiguous()
        out = torch.empty_like(c)
        L.ipt_philox(self.ctx, c.shape[0], _ptr(c), _ptr(k), _ptr(out))
        return out

    def synchronize(self):
        L.ipt_synchronize(self.ctx)

    def info(self):
        return L.ipt_scene_info(self.ctx, self.sid)

    def configure(self, integrator="wavefront", wavefront_slots=0, trace_steps=0, blocks_per_sm=0,
                  bvh_width=0, sort_cells=0, sort_dirs=0):
        if isinstance(integrator, int):
            integrator = "wavefront" if integrator == 1 else "megakernel"
        L.ipt_config_set(self.ctx, 1 if integrator == "wavefront" else 0, wavefront_slots,
                         trace_steps, blocks_per_sm, bvh_width, sort_cells, sort_dirs)

    def config(self):
        return L.ipt_config_get(self.ctx)

    def kernel_times(self, reset=False):
        return L.ipt_kernel_times(self.ctx, reset)

    # --- radiance cache ---------------------------------------------------
    def configure_cache(self, opts: CacheOptions):
        L.ipt_cache_configure(self.ctx, self.sid, opts.c())

    def cache_weights(self, table: bool = False):
        w = np.zeros(L.IPT_CACHE_WEIGHTS, np.float32)
        t = np.zeros(L.IPT_CACHE_TABLE_FLOATS, np.float32) if table else None
        L.ipt_cache_weights_get(self.ctx, self.sid, _np_ptr(w), _np_ptr(t))
        return (w, t) if table else w

    def set_cache_weights(self, weights=None, table=None):
        w = None if weights is None else np.ascontiguousarray(weights, np.float32).reshape(-1)
        t = None if table is None else np.ascontiguousarray(table, np.float32).reshape(-1)
        if w is not None and w.size != L.IPT_CACHE_WEIGHTS:
            raise ValueError("weights must hold IPT_CACHE_WEIGHTS floats")
        if t is not None and t.size != L.IPT_CACHE_TABLE_FLOATS:
            raise ValueError("table must hold IPT_CACHE_TABLE_FLOATS floats")
        L.ipt_cache_weights_set(self.ctx, self.sid, _np_ptr(w), _np_ptr(t))

    def cache_eval(self, x01, dirs, nrm, params7, upstream=None):
        """Prediction (n, 3) and, with upstream, d(upstream . prediction) / d params7 (n, 7)."""
        dev = self.device
        f = lambda a, k: torch.as_tensor(a, dtype=torch.float32, device=dev).reshape(-1, k).contiguous()
        x, d, nn, p7 = f(x01, 3), f(dirs, 3), f(nrm, 3), f(params7, 7)
        n = x.shape[0]
        rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
        up = None if upstream is None else f(upstream, 3)
        dp = None if upstream is None else torch.empty((n, 7), dtype=torch.float32, device=dev)
        L.ipt_cache_eval(self.ctx, self.sid, n, _ptr(x), _ptr(d), _ptr(nn), _ptr(p7), _ptr(up),
                         _ptr(rgb), _ptr(dp))
        self.synchronize()
        return rgb if dp is None else (rgb, dp)

    def cache_grad(self, x01, dirs, nrm, params7, target, table=True):
        """Relative-L2 loss of the rows and its gradients (weights, table)."""
        dev = self.device
        f = lambda a, k: torch.as_tensor(a, dtype=torch.float32, device=dev).reshape(-1, k).contiguous()
        x, d, nn, p7, tg = f(x01, 3), f(dirs, 3), f(nrm, 3), f(params7, 7), f(target, 3)
        gw = torch.empty(L.IPT_CACHE_WEIGHTS, dtype=torch.float32, device=dev)
        gt = torch.empty(L.IPT_CACHE_TABLE_FLOATS, dtype=torch.float32, device=dev) if table else None
        loss = L.ipt_cache_grad(self.ctx, self.sid, x.shape[0], _ptr(x), _ptr(d), _ptr(nn), _ptr(p7),
                                _ptr(tg), _ptr(gw), _ptr(gt))
        return loss, gw, gt

    def cache_train(self, opts: TraceOptions, iteration: int = 0):
        L.ipt_cache_train(self.ctx, self.sid, opts.c(), iteration)

    def cache_records(self, capacity: int):
        out = np.zeros((capacity, 16), np.float32)
        n = L.ipt_cache_records(self.ctx, self.sid, _np_ptr(out))
        return out[:n]

    def cache_status(self):
        return L.ipt_cache_status(self.ctx, self.sid)

    def cache_bias(self, opts: TraceOptions, spp: int, iteration: int = 0):
        return L.ipt_cache_bias(self.ctx, self.sid, opts.c(), spp, iteration)

    def counters(self, reset=False):
        return L.ipt_counters_read(self.ctx, reset)


class RenderFunction(torch.autograd.Function):
    """images = render(params); backward = the adjoint kernel's J^T g.

    forward renders all views (n_pix x 3) with ``spp_r`` samples of the
    forward set; backward traces ``spp_d`` samples of an independent set
    (Sec. 3.3), or of the same set when ``gradcheck_same_set`` is on, with
    sampling held at the forward's parameters."""

    @staticmethod
    def forward(ctx, params, tracer: Tracer, opts: TraceOptions, set_id: int, iteration: int,
                sampling_params=None):
        p = params.detach().contiguous()
        sp = p if sampling_params is None else sampling_params.detach().contiguous()
        img = tracer.render(opts, -1, set_id, opts.spp_r, iteration, params=p, sampling_params=sp)
        ctx.tracer = tracer
        ctx.opts = opts
        ctx.set_id = set_id
        ctx.iteration = iteration
        ctx.save_for_backward(p, sp)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        p, sp = ctx.saved_tensors
        dset = ctx.set_id if ctx.opts.gradcheck_same_set else L.IPT_SET_DERIVATIVE
        spp_opts = TraceOptions(**{**ctx.opts.__dict__})
        if ctx.opts.gradcheck_same_set:
            spp_opts.spp_d = ctx.opts.spp_r
        g = ctx.tracer.backward(grad_img, spp_opts, dset, ctx.iteration, params=p, sampling_params=sp)
        return g, None, None, None, None, None


def render(params, tracer: Tracer, opts: TraceOptions, set_id: int = L.IPT_SET_RESIDUAL,
           iteration: int = 0, sampling_params=None):
    return RenderFunction.apply(params, tracer, opts, set_id, iteration, sampling_params)
