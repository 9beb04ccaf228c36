"""ctypes binding of libipt.so (include/ipt.h): argument marshalling only.

Every function here has the name of the C entry point it calls and raises
IptError on a non-zero status.  Device buffers are passed as integer device
pointers (e.g. ``tensor.data_ptr()``); nothing here computes any part of the
path.  If the shared library is missing the import of a call fails loudly:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libipt.so")

IPT_OK = 0
IPT_SET_RESIDUAL, IPT_SET_DERIVATIVE, IPT_SET_TARGET, IPT_SET_CACHE = 0, 1, 2, 3
IPT_CACHE_WEIGHTS = 18432
IPT_CACHE_TABLE_FLOATS = 16 * 524288 * 2

EXPORTED = [
    "ipt_create", "ipt_destroy", "ipt_status_string", "ipt_last_error_detail",
    "ipt_scene_upload", "ipt_views_set", "ipt_targets_set", "ipt_params_set",
    "ipt_params_get", "ipt_params_device", "ipt_render", "ipt_backward", "ipt_loss_grad",
    "ipt_adam_step", "ipt_step", "ipt_trace_rays", "ipt_pick_pixels", "ipt_philox", "ipt_synchronize",
    "ipt_scene_info", "ipt_kernel_times", "ipt_counters_read", "ipt_loss_grad_shard",
    "ipt_backward_noalloc", "ipt_config_set", "ipt_config_get",
    "ipt_batch_create", "ipt_batch_step", "ipt_batch_params_get", "ipt_batch_destroy", "ipt_batch_set_active",
    "ipt_cache_configure", "ipt_cache_weights_set", "ipt_cache_weights_get", "ipt_cache_eval",
    "ipt_cache_grad", "ipt_cache_train", "ipt_cache_records", "ipt_cache_status", "ipt_cache_bias",
    "ipt_probe_gather", "ipt_build_info", "ipt_checkpoint_save", "ipt_checkpoint_load",
    "ipt_disney_params_set", "ipt_disney_params_get", "ipt_disney_render", "ipt_disney_loss_grad",
    "ipt_disney_step",
]
IPT_DISNEY_VALUES = 16
IPT_FLAG_KERNEL_TIMING, IPT_FLAG_COUNTERS, IPT_FLAG_OWN_STREAM = 1, 2, 4
KERNEL_NAMES = ["prepare", "forward", "adjoint", "finalize", "adam", "trace_rays", "philox",
                "wf_camera", "wf_closest", "wf_shadow", "wf_shade", "wf_adj_a", "wf_adj_connect",
                "wf_adj_b", "wf_reduce", "batch_step", "cache_infer", "cache_vjp", "cache_records",
                "cache_grad", "cache_adam", "wf_sort"]


class IptError(RuntimeError):
    def __init__(self, status, detail=""):
        self.status = status
        super().__init__(f"ipt status {status}: {detail}")


class ipt_options(C.Structure):
    _fields_ = [("device", C.c_int32), ("stream", C.c_void_p), ("seed", C.c_uint64),
                ("flags", C.c_int32)]


class ipt_camera(C.Structure):
    _fields_ = [("cam_to_world", C.c_float * 12), ("fov_y_deg", C.c_float),
                ("width", C.c_uint32), ("height", C.c_uint32)]


class ipt_config(C.Structure):
    _fields_ = [("integrator", C.c_int32), ("wavefront_slots", C.c_uint32),
                ("trace_steps", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("bvh_width", C.c_uint32), ("sort_cells", C.c_uint32), ("sort_dirs", C.c_uint32)]


class ipt_trace_opts(C.Structure):
    _fields_ = [("spp_r", C.c_uint32), ("spp_d", C.c_uint32), ("max_depth", C.c_uint32),
                ("loss", C.c_int32), ("nee", C.c_int32), ("mis", C.c_int32),
                ("emission_profile", C.c_int32), ("gradcheck_same_set", C.c_int32),
                ("pixel_batch", C.c_uint32)]


class ipt_adam_opts(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("l1_emission", C.c_float)]


class ipt_cache_opts(C.Structure):
    _fields_ = [("enabled", C.c_int32), ("b_term", C.c_uint32), ("train_spp", C.c_uint32),
                ("train_steps", C.c_uint32), ("record_capacity", C.c_uint32), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("bias_threshold", C.c_float), ("init_seed", C.c_uint64)]


class ipt_cache_stats(C.Structure):
    _fields_ = [("active", C.c_int32), ("fell_back", C.c_int32), ("records", C.c_uint32),
                ("pad", C.c_uint32), ("train_steps", C.c_uint64), ("last_loss", C.c_double),
                ("image_bias", C.c_double), ("grad_bias", C.c_double), ("lo", C.c_float * 3),
                ("hi", C.c_float * 3), ("res", C.c_int32 * 16)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libipt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run paper_1903_07145_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            P, U32, I32, U64 = C.c_void_p, C.c_uint32, C.c_int32, C.c_uint64
            sig = {
                "ipt_create": [C.POINTER(P), C.POINTER(ipt_options)],
                "ipt_destroy": [P],
                "ipt_last_error_detail": [P, C.c_char_p, C.c_size_t],
                "ipt_scene_upload": [P, P, U32, P, P, U32, P, U32, C.c_float, C.POINTER(I32)],
                "ipt_views_set": [P, I32, C.POINTER(ipt_camera), U32, P, I32],
                "ipt_targets_set": [P, I32, P, I32],
                "ipt_params_set": [P, I32, P, P],
                "ipt_params_get": [P, I32, P],
                "ipt_params_device": [P, I32, C.POINTER(P)],
                "ipt_render": [P, I32, I32, C.POINTER(ipt_trace_opts), U32, U32, U64, P, P, P, P],
                "ipt_backward": [P, I32, C.POINTER(ipt_trace_opts), U32, U64, P, P, P, P],
                "ipt_backward_noalloc": [P, I32, C.POINTER(ipt_trace_opts), U32, U64, P, P, P, P],
                "ipt_loss_grad": [P, I32, C.POINTER(ipt_trace_opts), U64, C.POINTER(C.c_double), P],
                "ipt_adam_step": [P, I32, P, C.POINTER(ipt_adam_opts)],
                "ipt_step": [P, I32, C.POINTER(ipt_trace_opts), C.POINTER(ipt_adam_opts),
                             C.POINTER(C.c_double)],
                "ipt_trace_rays": [P, I32, U32, P, P, P, P, P, P, P],
                "ipt_philox": [P, U32, P, P, P],
                "ipt_pick_pixels": [P, I32, U32, U64, P],
                "ipt_checkpoint_save": [P, I32, P, C.POINTER(C.c_size_t)],
                "ipt_checkpoint_load": [P, I32, P, C.c_size_t],
                "ipt_synchronize": [P],
                "ipt_scene_info": [P, I32, C.POINTER(U32), C.POINTER(U32), C.POINTER(U32),
                                   C.POINTER(U32), C.POINTER(U32), C.POINTER(U64)],
                "ipt_kernel_times": [P, C.POINTER(C.c_double), C.POINTER(U64), I32],
                "ipt_counters_read": [P, C.POINTER(U64), I32],
                "ipt_batch_set_active": [P, I32, P],
                "ipt_batch_create": [P, P, U32, C.POINTER(I32)],
                "ipt_batch_step": [P, I32, C.POINTER(ipt_trace_opts), C.POINTER(ipt_adam_opts), P],
                "ipt_batch_params_get": [P, I32, U32, P],
                "ipt_batch_destroy": [P, I32],
                "ipt_config_set": [P, C.POINTER(ipt_config)],
                "ipt_config_get": [P, C.POINTER(ipt_config)],
                "ipt_loss_grad_shard": [P, I32, C.POINTER(ipt_trace_opts), U64, U64, U64, U64,
                                        C.POINTER(C.c_double), P],
                "ipt_cache_configure": [P, I32, C.POINTER(ipt_cache_opts)],
                "ipt_cache_weights_set": [P, I32, P, P],
                "ipt_cache_weights_get": [P, I32, P, P],
                "ipt_cache_eval": [P, I32, U32, P, P, P, P, P, P, P],
                "ipt_cache_grad": [P, I32, U32, P, P, P, P, P, C.POINTER(C.c_double), P, P],
                "ipt_cache_train": [P, I32, C.POINTER(ipt_trace_opts), U64],
                "ipt_cache_records": [P, I32, C.POINTER(U32), P],
                "ipt_cache_status": [P, I32, C.POINTER(ipt_cache_stats)],
                "ipt_cache_bias": [P, I32, C.POINTER(ipt_trace_opts), U32, U64, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)],
                "ipt_probe_gather": [I32, U64, C.POINTER(C.c_double)],
                "ipt_build_info": [I32, C.POINTER(I32), C.POINTER(I32)],
                "ipt_disney_params_set": [P, I32, P, P],
                "ipt_disney_params_get": [P, I32, P],
                "ipt_disney_render": [P, I32, I32, C.POINTER(ipt_trace_opts), U32, U32, U64, P, P, P],
                "ipt_disney_loss_grad": [P, I32, C.POINTER(ipt_trace_opts), U64, C.POINTER(C.c_double), P],
                "ipt_disney_step": [P, I32, C.POINTER(ipt_trace_opts), C.POINTER(ipt_adam_opts),
                                    C.POINTER(C.c_double)],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.ipt_status_string.argtypes = [C.c_int]
            L.ipt_status_string.restype = C.c_char_p
            _lib = L
    return _lib


def _check(ctx, status):
    if status != IPT_OK:
        buf = C.create_string_buffer(512)
        if ctx:
            lib().ipt_last_error_detail(ctx, buf, 512)
        msg = lib().ipt_status_string(status).decode()
        raise IptError(status, f"{msg}: {buf.value.decode()}")


def ipt_create(device=0, stream=0, seed=0, flags=0):
    o = ipt_options(device, stream or None, seed, flags)
    h = C.c_void_p()
    _check(None, lib().ipt_create(C.byref(h), C.byref(o)))
    return h


def ipt_destroy(ctx):
    _check(None, lib().ipt_destroy(ctx))


def ipt_scene_upload(ctx, pos, n_vert, nrm, idx, n_tri, tri_seg, n_seg, emission_scale):
    sid = C.c_int32()
    _check(ctx, lib().ipt_scene_upload(ctx, pos, n_vert, nrm, idx, n_tri, tri_seg, n_seg,
                                       emission_scale, C.byref(sid)))
    return sid.value


def ipt_views_set(ctx, scene, cams, n_views, target, target_on_device):
    _check(ctx, lib().ipt_views_set(ctx, scene, cams, n_views, target, target_on_device))


def ipt_targets_set(ctx, scene, target, target_on_device):
    _check(ctx, lib().ipt_targets_set(ctx, scene, target, target_on_device))


def ipt_params_set(ctx, scene, params, free_mask):
    _check(ctx, lib().ipt_params_set(ctx, scene, params, free_mask))


def ipt_params_get(ctx, scene, out):
    _check(ctx, lib().ipt_params_get(ctx, scene, out))


def ipt_params_device(ctx, scene):
    p = C.c_void_p()
    _check(ctx, lib().ipt_params_device(ctx, scene, C.byref(p)))
    return p.value


def ipt_render(ctx, scene, view, opts, set_id, spp, iteration, params, sparams, rgb, msq):
    _check(ctx, lib().ipt_render(ctx, scene, view, C.byref(opts), set_id, spp, iteration,
                                 params, sparams, rgb, msq))


def ipt_backward(ctx, scene, opts, set_id, iteration, params, sparams, grad_image, grad_out):
    _check(ctx, lib().ipt_backward(ctx, scene, C.byref(opts), set_id, iteration, params, sparams,
                                   grad_image, grad_out))


def ipt_backward_noalloc(ctx, scene, opts, set_id, iteration, params, sparams, grad_image, grad_out):
    _check(ctx, lib().ipt_backward_noalloc(ctx, scene, C.byref(opts), set_id, iteration, params,
                                           sparams, grad_image, grad_out))


def ipt_loss_grad(ctx, scene, opts, iteration, want_loss, grad_out):
    loss = C.c_double()
    _check(ctx, lib().ipt_loss_grad(ctx, scene, C.byref(opts), iteration,
                                    C.byref(loss) if want_loss else None, grad_out))
    return loss.value if want_loss else None


def ipt_adam_step(ctx, scene, grad, adam):
    _check(ctx, lib().ipt_adam_step(ctx, scene, grad, C.byref(adam)))


def ipt_step(ctx, scene, opts, adam, want_loss):
    loss = C.c_double()
    _check(ctx, lib().ipt_step(ctx, scene, C.byref(opts), C.byref(adam),
                               C.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def ipt_disney_params_set(ctx, scene, params, free_mask):
    _check(ctx, lib().ipt_disney_params_set(ctx, scene, params, free_mask))


def ipt_disney_params_get(ctx, scene, out):
    _check(ctx, lib().ipt_disney_params_get(ctx, scene, out))


def ipt_disney_render(ctx, scene, view, opts, set_id, spp, iteration, sparams, rgb, msq):
    _check(ctx, lib().ipt_disney_render(ctx, scene, view, C.byref(opts), set_id, spp, iteration, sparams, rgb, msq))


def ipt_disney_loss_grad(ctx, scene, opts, iteration, want_loss, grad_out):
    loss = C.c_double()
    _check(ctx, lib().ipt_disney_loss_grad(ctx, scene, C.byref(opts), iteration,
                                           C.byref(loss) if want_loss else None, grad_out))
    return loss.value if want_loss else None


def ipt_disney_step(ctx, scene, opts, adam, want_loss):
    loss = C.c_double()
    _check(ctx, lib().ipt_disney_step(ctx, scene, C.byref(opts), C.byref(adam),
                                      C.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def ipt_trace_rays(ctx, scene, n, orig, dirs, skip, tri, t, u, v):
    _check(ctx, lib().ipt_trace_rays(ctx, scene, n, orig, dirs, skip, tri, t, u, v))


def ipt_checkpoint_save(ctx, scene) -> bytes:
    n = C.c_size_t(0)
    _check(ctx, lib().ipt_checkpoint_save(ctx, scene, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(ctx, lib().ipt_checkpoint_save(ctx, scene, buf, C.byref(n)))
    return buf.raw[:n.value]


def ipt_checkpoint_load(ctx, scene, data: bytes):
    buf = C.create_string_buffer(data, len(data))
    _check(ctx, lib().ipt_checkpoint_load(ctx, scene, buf, len(data)))


def ipt_pick_pixels(ctx, scene, batch, iteration, out):
    _check(ctx, lib().ipt_pick_pixels(ctx, scene, batch, iteration, out))


def ipt_philox(ctx, n, ctr, key, out):
    _check(ctx, lib().ipt_philox(ctx, n, ctr, key, out))


def ipt_synchronize(ctx):
    _check(ctx, lib().ipt_synchronize(ctx))


def ipt_scene_info(ctx, scene):
    a = [C.c_uint32() for _ in range(5)]
    npx = C.c_uint64()
    _check(ctx, lib().ipt_scene_info(ctx, scene, *[C.byref(x) for x in a], C.byref(npx)))
    return dict(n_tri=a[0].value, n_seg=a[1].value, n_nodes=a[2].value, bvh_depth=a[3].value,
                n_views=a[4].value, n_pixels=npx.value)


def ipt_kernel_times(ctx, reset=False):
    ms = (C.c_double * len(KERNEL_NAMES))()
    n = (C.c_uint64 * len(KERNEL_NAMES))()
    _check(ctx, lib().ipt_kernel_times(ctx, ms, n, int(reset)))
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_NAMES)}


def ipt_counters_read(ctx, reset=False):
    out = (C.c_uint64 * 6)()
    _check(ctx, lib().ipt_counters_read(ctx, out, int(reset)))
    return dict(closest_rays=out[0], shadow_rays=out[1], closest_node_visits=out[2],
                closest_tri_tests=out[3], shadow_node_visits=out[4], shadow_tri_tests=out[5])


def ipt_loss_grad_shard(ctx, scene, opts, iteration, pix_begin, pix_count, n_total, grad_out):
    loss = C.c_double()
    _check(ctx, lib().ipt_loss_grad_shard(ctx, scene, C.byref(opts), iteration, pix_begin, pix_count,
                                          n_total, C.byref(loss), grad_out))
    return loss.value


def ipt_config_set(ctx, integrator=1, wavefront_slots=0, trace_steps=0, blocks_per_sm=0, bvh_width=0,
                   sort_cells=0, sort_dirs=0):
    c = ipt_config(integrator, wavefront_slots, trace_steps, blocks_per_sm, bvh_width, sort_cells, sort_dirs)
    _check(ctx, lib().ipt_config_set(ctx, C.byref(c)))


def ipt_config_get(ctx):
    c = ipt_config()
    _check(ctx, lib().ipt_config_get(ctx, C.byref(c)))
    return dict(integrator=c.integrator, wavefront_slots=c.wavefront_slots,
                trace_steps=c.trace_steps, blocks_per_sm=c.blocks_per_sm, bvh_width=c.bvh_width,
                sort_cells=c.sort_cells, sort_dirs=c.sort_dirs)


def ipt_batch_create(ctx, scene_ids):
    arr = (C.c_int32 * len(scene_ids))(*scene_ids)
    bid = C.c_int32()
    _check(ctx, lib().ipt_batch_create(ctx, arr, len(scene_ids), C.byref(bid)))
    return bid.value


def ipt_batch_step(ctx, batch, opts, adam, losses_out):
    _check(ctx, lib().ipt_batch_step(ctx, batch, C.byref(opts), C.byref(adam), losses_out))


def ipt_batch_params_get(ctx, batch, member, out):
    _check(ctx, lib().ipt_batch_params_get(ctx, batch, member, out))


def ipt_batch_set_active(ctx, batch, active):
    flags = [1 if int(x) else 0 for x in active]
    buf = (C.c_uint8 * len(flags))(*flags)
    _check(ctx, lib().ipt_batch_set_active(ctx, batch, C.cast(buf, C.c_void_p)))


def ipt_batch_destroy(ctx, batch):
    _check(ctx, lib().ipt_batch_destroy(ctx, batch))


def ipt_cache_configure(ctx, scene, opts):
    _check(ctx, lib().ipt_cache_configure(ctx, scene, C.byref(opts)))


def ipt_cache_weights_set(ctx, scene, weights, table):
    _check(ctx, lib().ipt_cache_weights_set(ctx, scene, weights, table))


def ipt_cache_weights_get(ctx, scene, weights, table):
    _check(ctx, lib().ipt_cache_weights_get(ctx, scene, weights, table))


def ipt_cache_eval(ctx, scene, n, x01, dirs, nrm, params7, upstream, rgb_out, dparams_out):
    _check(ctx, lib().ipt_cache_eval(ctx, scene, n, x01, dirs, nrm, params7, upstream, rgb_out,
                                     dparams_out))


def ipt_cache_grad(ctx, scene, n, x01, dirs, nrm, params7, target, grad_weights, grad_table):
    loss = C.c_double()
    _check(ctx, lib().ipt_cache_grad(ctx, scene, n, x01, dirs, nrm, params7, target, C.byref(loss),
                                     grad_weights, grad_table))
    return loss.value


def ipt_cache_train(ctx, scene, opts, iteration):
    _check(ctx, lib().ipt_cache_train(ctx, scene, C.byref(opts), iteration))


def ipt_cache_records(ctx, scene, out):
    n = C.c_uint32()
    _check(ctx, lib().ipt_cache_records(ctx, scene, C.byref(n), out))
    return n.value


def ipt_cache_status(ctx, scene):
    st = ipt_cache_stats()
    _check(ctx, lib().ipt_cache_status(ctx, scene, C.byref(st)))
    return dict(active=bool(st.active), fell_back=bool(st.fell_back), records=st.records,
                train_steps=st.train_steps, last_loss=st.last_loss, image_bias=st.image_bias,
                grad_bias=st.grad_bias, lo=list(st.lo), hi=list(st.hi), res=list(st.res))


def ipt_cache_bias(ctx, scene, opts, spp, iteration):
    ib = C.c_double()
    gb = C.c_double()
    _check(ctx, lib().ipt_cache_bias(ctx, scene, C.byref(opts), spp, iteration, C.byref(ib),
                                     C.byref(gb)))
    return ib.value, gb.value


def ipt_probe_gather(device, nbytes):
    gbs = C.c_double()
    _check(None, lib().ipt_probe_gather(device, nbytes, C.byref(gbs)))
    return gbs.value


def ipt_build_info(device):
    """(binary version, PTX version) of the library's kernels on `device`."""
    b = C.c_int32()
    p = C.c_int32()
    _check(None, lib().ipt_build_info(device, C.byref(b), C.byref(p)))
    return b.value, p.value
