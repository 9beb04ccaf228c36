"""Several scenes in one context, optimised together as a batch.

Each scene keeps its own parameters, Adam state and loss; every stage of an
iteration is one launch over all of their pixels, and the iteration is
replayed as a CUDA graph (ipt_batch_step).  The same calls also drive the
scenes one at a time (ipt_step), which the tests use as the reference.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .scenes import Scene
from .tracer import AdamOptions, TraceOptions, _np_ptr, _ptr, cameras_c


class SceneSet:
    def __init__(self, scenes: list[Scene], device: int = 0, seed: int = 0, flags: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("the inverse path tracer needs a CUDA device")
        self.device = torch.device("cuda", device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = L.ipt_create(device, stream, seed, flags & ~L.IPT_FLAG_OWN_STREAM)
        self.scenes = scenes
        self.sids = []
        self._cams = []
        for sc in scenes:
            pos = np.ascontiguousarray(sc.positions, np.float32)
            nrm = None if sc.normals is None else np.ascontiguousarray(sc.normals, np.float32)
            idx = np.ascontiguousarray(sc.indices, np.uint32)
            seg = np.ascontiguousarray(sc.tri_segment, np.uint32)
            sid = L.ipt_scene_upload(self.ctx, _np_ptr(pos), pos.shape[0], _np_ptr(nrm), _np_ptr(idx),
                                     idx.shape[0], _np_ptr(seg), sc.n_segments, float(sc.emission_scale))
            cams = cameras_c(sc.cameras)
            L.ipt_views_set(self.ctx, sid, cams, len(sc.cameras), None, 0)
            self._cams.append(cams)
            self.sids.append(sid)
        self.n_pix = [sum(c.width * c.height for c in sc.cameras) for sc in scenes]
        self.batch = None

    def close(self):
        if getattr(self, "ctx", None):
            L.ipt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, integrator="wavefront", wavefront_slots=0, trace_steps=0, blocks_per_sm=0,
                  bvh_width=0, sort_cells=0, sort_dirs=0):
        L.ipt_config_set(self.ctx, 1 if integrator == "wavefront" else 0, wavefront_slots, trace_steps,
                         blocks_per_sm, bvh_width, sort_cells, sort_dirs)

    def set_params(self, i, params, free_mask=None):
        p = np.ascontiguousarray(np.asarray(params, np.float32).reshape(-1, 10))
        fm = None if free_mask is None else np.ascontiguousarray(np.asarray(free_mask, np.uint8))
        L.ipt_params_set(self.ctx, self.sids[i], _np_ptr(p), _np_ptr(fm))

    def params(self, i):
        out = np.zeros((self.scenes[i].n_segments, 10), np.float32)
        L.ipt_params_get(self.ctx, self.sids[i], _np_ptr(out))
        return out

    def set_targets(self, i, targets: torch.Tensor):
        t = targets.to(self.device, torch.float32).contiguous()
        assert t.numel() == 3 * self.n_pix[i]
        L.ipt_targets_set(self.ctx, self.sids[i], _ptr(t), 1)
        L.ipt_synchronize(self.ctx)

    def render(self, i, opts: TraceOptions, set_id=L.IPT_SET_TARGET, spp=None, iteration=0):
        img = torch.empty((self.n_pix[i], 3), device=self.device, dtype=torch.float32)
        L.ipt_render(self.ctx, self.sids[i], -1, opts.c(), set_id, opts.spp_r if spp is None else spp,
                     iteration, None, None, _ptr(img), None)
        return img

    def step(self, i, opts: TraceOptions, adam: AdamOptions, want_loss=True):
        """One eager iteration of scene i alone."""
        return L.ipt_step(self.ctx, self.sids[i], opts.c(), adam.c(), want_loss)

    # -- batch ----------------------------------------------------------------
    def make_batch(self):
        """Batch of every scene, from their current parameters."""
        if self.batch is not None:
            L.ipt_batch_destroy(self.ctx, self.batch)
        self.batch = L.ipt_batch_create(self.ctx, self.sids)
        return self.batch

    def set_active(self, active):
        """Members that take part in the next batch steps (inactive ones keep
        their parameters and Adam state)."""
        L.ipt_batch_set_active(self.ctx, self.batch, np.asarray(active, np.uint8))

    def batch_step(self, opts: TraceOptions, adam: AdamOptions, want_losses=True):
        out = np.zeros(len(self.sids), np.float64) if want_losses else None
        L.ipt_batch_step(self.ctx, self.batch, opts.c(), adam.c(),
                         None if out is None else C.c_void_p(out.ctypes.data))
        return out

    def batch_params(self, i):
        out = np.zeros((self.scenes[i].n_segments, 10), np.float32)
        L.ipt_batch_params_get(self.ctx, self.batch, i, _np_ptr(out))
        return out

    def synchronize(self):
        L.ipt_synchronize(self.ctx)

    def kernel_times(self, reset=False):
        return L.ipt_kernel_times(self.ctx, reset)
