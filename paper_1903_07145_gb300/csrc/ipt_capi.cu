// C ABI of the GB300 inverse path tracer: context, scenes, views, parameters
// and the calls of one nested-SGD iteration (the other groups of entry
// points live in ipt_capi_*.cu).  See include/ipt.h.
#include "ipt_capi_internal.h"

using namespace ipt_capi;

namespace ipt_capi {

ipt_status fail(ipt_ctx* c, ipt_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

ipt_status cuda_fail(ipt_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? IPT_ERR_OUT_OF_MEMORY : IPT_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}



void free_scene(DeviceScene* s) {
  if (!s) return;
  free_cache(s->cache);
  free_disney(s->disney);
  for (void* p : s->owned) cudaFree(p);
  cudaFree(s->pick);
  cudaFree(s->g_pick);
  delete s;
}

// Resolves recorded event pairs into per-kernel totals (waits for them).
void resolve_timings(ipt_ctx* c) {
  for (const PendingTiming& p : c->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->kernel_ms[p.id] += ms;
      c->kernel_n[p.id] += (uint64_t)p.launches;
    }
    c->spare_events.push_back(p.a);
    c->spare_events.push_back(p.b);
  }
  c->pending.clear();
}

cudaEvent_t take_event(ipt_ctx* c) {
  if (!c->spare_events.empty()) {
    cudaEvent_t e = c->spare_events.back();
    c->spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}



void stage_begin(void* user, int id) {
  StageTimer* t = static_cast<StageTimer*>(user);
  if (t->c->pending.size() > 8192) resolve_timings(t->c);
  t->id = id;
  t->a = take_event(t->c);
  if (t->a) cudaEventRecord(t->a, t->c->stream);
}

void stage_end(void* user) {
  StageTimer* t = static_cast<StageTimer*>(user);
  if (!t->a) return;
  cudaEvent_t b = take_event(t->c);
  if (!b) return;
  cudaEventRecord(b, t->c->stream);
  t->c->pending.push_back({t->id, t->a, b, 1});
  t->a = nullptr;
}

ipt::SceneBuffers buffers(const ipt_ctx* ctx, const DeviceScene* s) {
  ipt::SceneBuffers b;
  b.counters = ctx->counters_dev;
  b.wide = ctx->cfg.bvh_width == 2 ? 0 : (ctx->cfg.bvh_width == 8 ? 2 : 1);
  b.nodes = s->nodes;
  b.nodes4 = s->nodes4;
  b.nodes8 = s->nodes8;
  b.tris = s->tris;
  b.vnrm = s->vnrm;
  b.seg_tris = s->seg_tris;
  b.seg_begin = s->seg_begin;
  b.tri_cdf = s->tri_cdf;
  b.seg_area = s->seg_area;
  b.orig_to_internal = s->orig_to_internal;
  b.n_seg = s->n_seg;
  b.n_tri = s->n_tri;
  b.eps = s->eps;
  b.emission_scale = s->emission_scale;
  return b;
}

ipt_status get_scene(ipt_ctx* ctx, int32_t id, DeviceScene** out) {
  if (!ctx) return IPT_ERR_INVALID_ARG;
  if (id < 0 || (size_t)id >= ctx->scenes.size() || !ctx->scenes[id])
    return fail(ctx, IPT_ERR_INVALID_ARG, "unknown scene id " + std::to_string(id));
  *out = ctx->scenes[id];
  return IPT_OK;
}

ipt_status check_opts(ipt_ctx* ctx, const ipt_trace_opts* o, bool adjoint, bool batch_ok) {
  if (!o) return fail(ctx, IPT_ERR_INVALID_ARG, "null trace options");
  if (o->pixel_batch && !batch_ok) return fail(ctx, IPT_ERR_INVALID_ARG, "pixel_batch must be 0 for this call");
  if ((uint64_t)o->pixel_batch * std::max(o->spp_r, o->spp_d) >= (1ull << 32))
    return fail(ctx, IPT_ERR_INVALID_ARG, "pixel_batch * spp must stay below 2^32");
  const uint32_t maxd = adjoint ? ipt::kMaxAdjointDepth : ipt::kMaxForwardDepth;
  if (o->max_depth > maxd)
    return fail(ctx, IPT_ERR_INVALID_ARG, "max_depth " + std::to_string(o->max_depth) + " above limit " +
                                              std::to_string(maxd));
  if (o->loss != 0 && o->loss != 1) return fail(ctx, IPT_ERR_INVALID_ARG, "loss must be 0 (L2) or 1 (L1)");
  if (o->emission_profile != 0 && o->emission_profile != 1)
    return fail(ctx, IPT_ERR_INVALID_ARG, "emission_profile must be 0 or 1");
  return IPT_OK;
}

ipt::TraceParams trace_params(const ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* o, uint32_t set,
                              uint32_t spp, uint64_t it) {
  ipt::TraceParams tp;
  tp.seed = ctx->seed;
  tp.scene_id = (uint32_t)scene;
  tp.set = set;
  tp.iteration = it;
  tp.spp = spp;
  tp.max_depth = o->max_depth;
  tp.nee = o->nee;
  tp.mis = o->mis;
  tp.profile = o->emission_profile;
  return tp;
}

// Device buffers of a pixel batch of `batch` entries (grown, never shrunk).
ipt_status ensure_pick(ipt_ctx* ctx, DeviceScene* s, uint32_t batch) {
  if (s->pick_cap >= batch) return IPT_OK;
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  ++ctx->alloc_gen;
  cudaFree(s->pick);
  cudaFree(s->g_pick);
  s->pick = nullptr;
  s->g_pick = nullptr;
  s->pick_cap = 0;
  IPT_CK(cudaMalloc(&s->pick, batch * sizeof(uint32_t)));
  IPT_CK(cudaMalloc(&s->g_pick, 3 * (size_t)batch * sizeof(float)));
  s->pick_cap = batch;
  return IPT_OK;
}

ipt_status ensure_tables(ipt_ctx* ctx, DeviceScene* s, const float* params, const float* sparams) {
  const bool is_ctx = (params == s->params) && (sparams == nullptr || sparams == s->params);
  if (is_ctx && s->tab_is_ctx) return IPT_OK;
  Timed tm(ctx, IPT_KERNEL_PREPARE);
  IPT_CK(ipt::launch_prepare(buffers(ctx, s), s->tab, params, sparams ? sparams : params, ctx->stream));
  s->tab_is_ctx = is_ctx;
  s->tab_batch = -1;
  return IPT_OK;
}

void wf_release(ipt_ctx* c) {
  for (void* p : c->wf_owned) cudaFree(p);
  c->wf_owned.clear();
  c->wf = ipt::WfBuffers();
  c->wf_adjoint = false;
  c->wf_disney = false;
}

// Wavefront buffers for `cap` slots (plus the adjoint's carry when asked),
// allocated on first use and kept by the context.
ipt_status ensure_wf(ipt_ctx* ctx, bool adjoint, uint32_t n_params, bool disney, uint32_t depth) {
  const uint32_t cap = ctx->cfg.wavefront_slots ? ctx->cfg.wavefront_slots : (1u << 20);
  if (adjoint && (depth == 0 || depth > (uint32_t)ipt::kMaxAdjointDepth)) depth = ipt::kMaxAdjointDepth;
  const bool fits = ctx->wf.cap == cap &&
                    (!adjoint || (ctx->wf_adjoint && ctx->wf.blk_params >= n_params && ctx->wf.depth_cap >= depth)) &&
                    (!disney || ctx->wf_disney);
  if (fits) return IPT_OK;
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  ++ctx->alloc_gen;
  const uint32_t keep_params = std::max(n_params, ctx->wf.blk_params);
  const uint32_t keep_depth = std::max(adjoint ? depth : 0u, ctx->wf_adjoint ? ctx->wf.depth_cap : 0u);
  const bool want_adj = adjoint || ctx->wf_adjoint;
  const bool want_disney = want_adj && (disney || ctx->wf_disney);
  wf_release(ctx);
  ipt::WfBuffers& w = ctx->wf;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t n) {
    if (e != cudaSuccess) return;
    void* q = nullptr;
    e = cudaMalloc(&q, n * sizeof(**p));
    if (e == cudaSuccess) {
      ctx->wf_owned.push_back(q);
      *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    }
  };
  A(&w.ray_o, cap);
  A(&w.ray_d, cap);
  A(&w.hit, cap);
  A(&w.beta, cap);
  A(&w.rad, cap);
  A(&w.q0, cap);
  A(&w.q1, cap);
  A(&w.cnt, 8);
  A(&w.sh_o, cap);
  A(&w.sh_d, cap);
  A(&w.sh_meta, cap);
  A(&w.sh_c, cap);
  A(&w.sh_vis, cap);
  A(&w.qs, cap);
  A(&w.keys, (size_t)cap + 16);  // padded: the sort reads whole groups of 8
  A(&w.bins, ipt::kSortMaxBins);
  if (want_adj) {
    A(&w.aT, (size_t)keep_depth * cap);
    A(&w.aU, (size_t)keep_depth * cap);
    A(&w.aR, (size_t)keep_depth * cap);
    A(&w.nv, cap);
    A(&w.sh_ge, cap);
    A(&w.sh_gm, cap);
    A(&w.sh_n, cap);
    if (want_disney) {
      A(&w.aWi, (size_t)keep_depth * cap);
      A(&w.aWo, (size_t)keep_depth * cap);
      A(&w.sh_dv, 4 * (size_t)cap);
    }
    // block-private rows for chunks whose accumulators fit in shared memory;
    // a wider chunk accumulates in one row in global memory
    const size_t shared_params = std::min<size_t>(keep_params, 10u * ipt::wf_max_segments());
    A(&w.blk, std::max((size_t)ipt::wf_max_blocks(ctx->L) * shared_params, (size_t)keep_params));
  }
  if (e != cudaSuccess) {
    wf_release(ctx);
    return cuda_fail(ctx, e, "wavefront buffers");
  }
  w.cap = cap;
  w.blk_params = want_adj ? keep_params : 0;
  w.depth_cap = want_adj ? keep_depth : 0;
  ctx->wf_adjoint = want_adj;
  ctx->wf_disney = want_disney;
  return IPT_OK;
}

bool use_wavefront_cap(const ipt_ctx* ctx, uint32_t spp) {
  const uint32_t cap = ctx->cfg.wavefront_slots ? ctx->cfg.wavefront_slots : (1u << 20);
  return spp <= cap;
}

bool use_wavefront(const ipt_ctx* ctx, uint32_t spp) {
  const uint32_t cap = ctx->cfg.wavefront_slots ? ctx->cfg.wavefront_slots : (1u << 20);
  return ctx->cfg.integrator == 1 && spp <= cap;
}

// Scene-table entry of one scene for a launch over its pixels
// [pix_base, pix_base + n) (launch pixels 0..n-1).
ipt::WfScene wf_entry(const ipt_ctx* ctx, int32_t scene_id, const DeviceScene* s, uint32_t pix_base, uint32_t n) {
  ipt::WfScene e{};
  e.s = ipt::scene_dev(buffers(ctx, s));
  e.t = ipt::seg_dev(s->tab);
  e.views = reinterpret_cast<const ipt::ViewDev*>(s->views_dev);
  e.n_views = (uint32_t)s->views.size();
  e.pix_begin = 0;
  e.n_pix = n;
  e.pix_base = pix_base;
  e.seg_offset = 0;
  e.n_seg = s->n_seg;
  e.key = make_uint2((uint32_t)(ctx->seed & 0xFFFFFFFFu), (uint32_t)(ctx->seed >> 32) ^ (uint32_t)scene_id);
  e.es = s->emission_scale;
  e.bb_lo = make_float3(s->bb_lo[0], s->bb_lo[1], s->bb_lo[2]);
  const float ex = s->bb_hi[0] - s->bb_lo[0], ey = s->bb_hi[1] - s->bb_lo[1], ez = s->bb_hi[2] - s->bb_lo[2];
  e.bb_inv = make_float3(ex > 0.f ? 1.f / ex : 0.f, ey > 0.f ? 1.f / ey : 0.f, ez > 0.f ? 1.f / ez : 0.f);
  return e;
}

ipt_status upload_entry(ipt_ctx* ctx, const ipt::WfScene& e) {
  if (!ctx->wf_tab) IPT_CK(cudaMalloc(&ctx->wf_tab, sizeof(ipt::WfScene)));
  IPT_CK(cudaMemcpyAsync(ctx->wf_tab, &e, sizeof(e), cudaMemcpyHostToDevice, ctx->stream));
  return IPT_OK;
}

// Pixel batch of one iteration into out[0..B-1] (device).
ipt_status draw_picks(ipt_ctx* ctx, int32_t scene_id, const DeviceScene* s, uint32_t B, uint64_t iteration,
                      uint32_t* out) {
  if (s->n_pix >= (1ull << 32)) return fail(ctx, IPT_ERR_INVALID_ARG, "pixel batches need fewer than 2^32 pixels");
  ipt::WfScene e = wf_entry(ctx, scene_id, s, 0, B);
  e.pick = out;
  e.n_all = (uint32_t)s->n_pix;
  ipt_status st = upload_entry(ctx, e);
  if (st != IPT_OK) return st;
  IPT_CK(ipt::wf_pick(ctx->wf_tab, std::vector<ipt::WfScene>{e}, nullptr, (uint32_t)iteration, ctx->stream));
  return IPT_OK;
}

// Forward pass through the configured integrator.  Launch pixel i is scene
// pixel begin + i; img/msq are indexed by launch pixel, target and g_out by
// scene pixel.
ipt_status run_forward(ipt_ctx* ctx, int32_t scene_id, DeviceScene* s, uint32_t begin, uint32_t n,
                       const ipt::TraceParams& tp, float* img, float* msq, const float* target, float* g_out,
                       double* partials, float g_scale, int loss_kind, const ipt::CachePass* cache,
                       uint32_t* pick) {
  if (cache && !use_wavefront_cap(ctx, tp.spp))
    return fail(ctx, IPT_ERR_INVALID_ARG, "cached passes need spp <= wavefront_slots");
  if (cache || use_wavefront(ctx, tp.spp)) {
    ipt_status st = ensure_wf(ctx, false, 10u * s->n_seg);
    if (st != IPT_OK) return st;
    ipt::WfScene e = wf_entry(ctx, scene_id, s, begin, n);
    e.pick = pick;  // batch entries 0..n-1 (begin is 0)
    e.n_all = (uint32_t)s->n_pix;
    e.g_scale = g_scale;
    e.target = target;
    e.g_img = g_out;
    e.img = img;
    e.msq = msq;
    if ((st = upload_entry(ctx, e)) != IPT_OK) return st;
    StageTimer timer{ctx};
    const ipt::WfHook hook{stage_begin, stage_end, &timer};
    IPT_CK(ipt::wf_forward(ctx->L, ctx->wf_tab, std::vector<ipt::WfScene>{e}, tp, loss_kind, nullptr, ctx->wf,
                           partials, ctx->err_dev, ctx->stream,
                           (ctx->flags & IPT_FLAG_KERNEL_TIMING) ? &hook : nullptr, cache));
  } else {
    // a pixel batch (begin 0) keeps the whole target: the kernel reads the
    // drawn pixel's value
    if (target && !pick) {
      target += 3 * (size_t)begin;
      g_out += 3 * (size_t)begin;
    }
    ipt::TraceParams tpk = tp;
    tpk.pick = pick;
    Timed tm(ctx, IPT_KERNEL_FORWARD);
    IPT_CK(ipt::launch_forward(ctx->L, buffers(ctx, s), s->tab, s->views_dev, (uint32_t)s->views.size(), begin, n,
                               tpk, img, msq, target, g_out, partials, g_scale, loss_kind, ctx->err_dev,
                               ctx->stream));
  }
  return IPT_OK;
}

// Adjoint pass over scene pixels [begin, begin + n) (accumulates into
// grad_acc, which the caller zeroes).  g_img is indexed by scene pixel.
ipt_status run_adjoint(ipt_ctx* ctx, int32_t scene_id, DeviceScene* s, uint32_t begin, uint32_t n,
                       const ipt::TraceParams& tp, const float* g_img, double* grad_acc,
                       const ipt::CachePass* cache, uint32_t* pick) {
  if (cache && !use_wavefront_cap(ctx, tp.spp))
    return fail(ctx, IPT_ERR_INVALID_ARG, "cached passes need spp <= wavefront_slots");
  if (cache || use_wavefront(ctx, tp.spp)) {
    ipt_status st = ensure_wf(ctx, true, 10u * s->n_seg, false, tp.max_depth);
    if (st != IPT_OK) return st;
    ipt::WfScene e = wf_entry(ctx, scene_id, s, begin, n);
    e.pick = pick;
    e.n_all = (uint32_t)s->n_pix;
    e.g_img = const_cast<float*>(g_img);
    if ((st = upload_entry(ctx, e)) != IPT_OK) return st;
    StageTimer timer{ctx};
    const ipt::WfHook hook{stage_begin, stage_end, &timer};
    IPT_CK(ipt::wf_adjoint(ctx->L, ctx->wf_tab, std::vector<ipt::WfScene>{e}, tp, nullptr, ctx->wf, grad_acc,
                           ctx->err_dev, ctx->stream, (ctx->flags & IPT_FLAG_KERNEL_TIMING) ? &hook : nullptr,
                           cache));
  } else {
    ipt::TraceParams tpk = tp;
    tpk.pick = pick;
    Timed tm(ctx, IPT_KERNEL_ADJOINT);
    IPT_CK(ipt::launch_adjoint(ctx->L, buffers(ctx, s), s->tab, s->views_dev, (uint32_t)s->views.size(), begin, n,
                               tpk, pick ? g_img : g_img + 3 * (size_t)begin, grad_acc, s->grad_f, ctx->err_dev,
                               ctx->stream));
  }
  return IPT_OK;
}

// --- radiance cache helpers -------------------------------------------------

bool cache_on(const DeviceScene* s) { return s->cache && s->cache->active; }

ipt::CacheNet cache_net(const DeviceScene* s, bool unit_inputs) {
  const CacheState* c = s->cache;
  ipt::CacheNet n{};
  n.wt = c->wt;
  n.table = reinterpret_cast<const float2*>(c->table);
  n.table_h = c->table_h;
  for (int l = 0; l < ipt::kCacheLevels; ++l) n.res[l] = c->res[l];
  n.dense = c->dense;
  if (unit_inputs) {
    n.lo = make_float3(0.f, 0.f, 0.f);
    n.inv_ext = make_float3(1.f, 1.f, 1.f);
  } else {
    const float ex = s->bb_hi[0] - s->bb_lo[0], ey = s->bb_hi[1] - s->bb_lo[1], ez = s->bb_hi[2] - s->bb_lo[2];
    n.lo = make_float3(s->bb_lo[0], s->bb_lo[1], s->bb_lo[2]);
    n.inv_ext = make_float3(ex > 0.f ? 1.f / ex : 1.f, ey > 0.f ? 1.f / ey : 1.f, ez > 0.f ? 1.f / ez : 1.f);
  }
  return n;
}

// Query buffers for the context's wavefront capacity (reallocated when the
// capacity grew).
ipt_status cache_query_buffers(ipt_ctx* ctx, CacheState* c) {
  const uint32_t cap = ctx->cfg.wavefront_slots ? ctx->cfg.wavefront_slots : (1u << 20);
  if (c->buf.q_cap >= cap) return IPT_OK;
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  void* ptrs[6] = {c->buf.q.x, c->buf.q.d, c->buf.q.n, c->buf.q.u, c->buf.qc, c->buf.qdp};
  for (void* q : ptrs) {
    if (!q) continue;
    cudaFree(q);
    c->owned.erase(std::remove(c->owned.begin(), c->owned.end(), q), c->owned.end());
  }
  c->buf.q_cap = 0;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t n) {
    void* q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, n * sizeof(**p));
    if (e == cudaSuccess) {
      c->owned.push_back(q);
      *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    }
  };
  A(&c->buf.q.x, cap);
  A(&c->buf.q.d, cap);
  A(&c->buf.q.n, cap);
  A(&c->buf.q.u, cap);
  A(&c->buf.qc, cap);
  A(&c->buf.qdp, 8 * (size_t)cap);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cache query buffers");
  c->buf.q_cap = cap;
  return IPT_OK;
}

// The cache's part of a pass over scene s (query or record mode).
ipt_status cache_pass(ipt_ctx* ctx, DeviceScene* s, bool record, ipt::CachePass* out) {
  ipt_status st = cache_query_buffers(ctx, s->cache);
  if (st != IPT_OK) return st;
  out->net = cache_net(s, false);
  out->buf = s->cache->buf;
  out->b_term = s->cache->opts.b_term;
  out->record = record ? 1 : 0;
  return IPT_OK;
}

// Training pass: record the set-3 paths of `iteration`, then train_steps
// Adam steps over the records.
ipt_status cache_train_pass(ipt_ctx* ctx, int32_t scene, DeviceScene* s, const ipt_trace_opts* opts,
                            uint64_t iteration) {
  CacheState* c = s->cache;
  const uint32_t spp = c->opts.train_spp ? c->opts.train_spp : std::max(1u, opts->spp_r / 16u);
  ipt::CachePass cp;
  ipt_status st = cache_pass(ctx, s, true, &cp);
  if (st != IPT_OK) return st;
  IPT_CK(cudaMemsetAsync(c->buf.counts, 0, 4 * sizeof(uint32_t), ctx->stream));
  st = run_forward(ctx, scene, s, 0, (uint32_t)s->n_pix, trace_params(ctx, scene, opts, IPT_SET_CACHE, spp, iteration),
                   nullptr, nullptr, nullptr, nullptr, nullptr, 0.f, 0, &cp);
  if (st != IPT_OK) return st;
  const uint32_t steps = c->opts.train_steps;
  IPT_CK(cudaMemsetAsync(c->loss_dev, 0, steps * sizeof(double), ctx->stream));
  const ipt::CacheNet net = cache_net(s, false);
  for (uint32_t i = 0; i < steps; ++i) {
    {
      Timed tm(ctx, IPT_KERNEL_CACHE_GRAD);
      ipt::CacheOut o{};
      o.gw = c->gw;
      o.gt = reinterpret_cast<float2*>(c->gt);
      o.loss = c->loss_dev + i;
      o.err = ctx->err_dev;
      IPT_CK(ipt::cache_grad(net, c->buf.r, s->tab.mat_a, s->tab.mat_b, c->buf.counts + 1, c->buf.r_cap, i, steps, o,
                             ctx->L.num_sms, ctx->stream));
    }
    Timed tm(ctx, IPT_KERNEL_CACHE_ADAM);
    const double t = (double)(++c->steps_done);
    const float bc1 = (float)(1.0 - std::pow((double)c->opts.beta1, t));
    const float bc2 = (float)(1.0 - std::pow((double)c->opts.beta2, t));
    IPT_CK(ipt::cache_adam(c->w, c->mw, c->vw, c->gw, c->table, c->mt, c->vt, c->gt, c->wt, c->table_h,
                           c->opts.lr, c->opts.beta1, c->opts.beta2, c->opts.eps, bc1, bc2, ctx->L.num_sms,
                           ctx->stream));
  }
  c->last_pass_steps = steps;
  return IPT_OK;
}


// Forward + residual + adjoint over pixels [begin, begin + count), with the
// loss normalised by n_total pixels (all shards together).
ipt_status loss_grad_async(ipt_ctx* ctx, int32_t scene, DeviceScene* s, const ipt_trace_opts* opts,
                           uint64_t iteration, float* grad_out, uint64_t begin, uint64_t count, uint64_t n_total) {
  ipt_status st;
  const bool whole = begin == 0 && count == s->n_pix && n_total == s->n_pix;
  if ((st = check_opts(ctx, opts, true, whole)) != IPT_OK) return st;
  if (s->views.empty() || !s->target) return fail(ctx, IPT_ERR_INVALID_ARG, "loss needs views and targets");
  if (opts->spp_r == 0 || opts->spp_d == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp_r and spp_d must be positive");
  if (begin + count > s->n_pix || count == 0 || n_total < count)
    return fail(ctx, IPT_ERR_INVALID_ARG, "pixel range outside the views");
  const uint32_t B = opts->pixel_batch;
  if (B && cache_on(s)) return fail(ctx, IPT_ERR_INVALID_ARG, "pixel batches do not run with the radiance cache");
  IPT_CK(cudaSetDevice(ctx->device));
  if ((st = ensure_tables(ctx, s, s->params, nullptr)) != IPT_OK) return st;
  const uint32_t np = 10u * s->n_seg;
  // a pixel batch traces entries 0..B-1 of the drawn pixels
  if (B && ((st = ensure_pick(ctx, s, B)) != IPT_OK || (st = draw_picks(ctx, scene, s, B, iteration, s->pick)) != IPT_OK))
    return st;
  const uint32_t lb = B ? 0u : (uint32_t)begin, ln = B ? B : (uint32_t)count;
  float* g_buf = B ? s->g_pick : s->g_img;
  uint32_t* pick = B ? s->pick : nullptr;
  const float g_scale = (float)(1.0 / (3.0 * (double)(B ? B : n_total)));
  ipt::CachePass cp;
  if (cache_on(s) && (st = cache_pass(ctx, s, false, &cp)) != IPT_OK) return st;
  const ipt::CachePass* cpp = cache_on(s) ? &cp : nullptr;
  st = run_forward(ctx, scene, s, lb, ln, trace_params(ctx, scene, opts, IPT_SET_RESIDUAL, opts->spp_r, iteration),
                   nullptr, nullptr, s->target, g_buf, s->loss_partials, g_scale, opts->loss, cpp, pick);
  if (st != IPT_OK) return st;
  IPT_CK(cudaMemsetAsync(s->grad_acc, 0, np * sizeof(double), ctx->stream));
  const uint32_t set = opts->gradcheck_same_set ? IPT_SET_RESIDUAL : IPT_SET_DERIVATIVE;
  ipt::TraceParams tpd = trace_params(ctx, scene, opts, set, opts->spp_d, iteration);
  if (opts->gradcheck_same_set) tpd.sample_stride = opts->spp_r;
  st = run_adjoint(ctx, scene, s, lb, ln, tpd, g_buf, s->grad_acc, cpp, pick);
  if (st != IPT_OK) return st;
  Timed tm(ctx, IPT_KERNEL_FINALIZE);
  IPT_CK(ipt::launch_finalize(s->loss_partials, ipt::loss_partials_capacity(ctx->L), s->loss_dev, s->grad_acc,
                              grad_out, np, ctx->stream));
  s->loss_fresh = true;
  return IPT_OK;
}

ipt_status read_loss(ipt_ctx* ctx, DeviceScene* s, double* loss_out, uint64_t n_total) {
  IPT_CK(cudaMemcpyAsync(ctx->loss_host, s->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  ipt_status st = ipt_synchronize(ctx);
  if (st != IPT_OK) return st;
  *loss_out = *ctx->loss_host / (3.0 * (double)n_total);
  return IPT_OK;
}

ipt::AdamHost adam_host(const ipt_adam_opts* a) {
  ipt::AdamHost h;
  h.lr = a->lr;
  h.beta1 = a->beta1;
  h.beta2 = a->beta2;
  h.eps = a->eps;
  h.l1 = a->l1_emission;
  return h;
}

}  // namespace ipt_capi

extern "C" {

const char* ipt_status_string(ipt_status s) {
  switch (s) {
    case IPT_OK: return "ok";
    case IPT_ERR_INVALID_ARG: return "invalid argument";
    case IPT_ERR_OUT_OF_MEMORY: return "out of device memory";
    case IPT_ERR_CUDA: return "CUDA error";
    case IPT_ERR_TIMEOUT: return "timeout";
    case IPT_ERR_NONFINITE: return "non-finite value";
    case IPT_ERR_NOT_READY: return "not ready";
  }
  return "unknown status";
}

ipt_status ipt_last_error_detail(const ipt_ctx* ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return IPT_ERR_INVALID_ARG;
  std::snprintf(buf, n, "%s", ctx->last_error.c_str());
  return IPT_OK;
}

ipt_status ipt_create(ipt_ctx** out, const ipt_options* opt) {
  if (!out || !opt) return IPT_ERR_INVALID_ARG;
  *out = nullptr;
  ipt_ctx* ctx = new (std::nothrow) ipt_ctx();
  if (!ctx) return IPT_ERR_OUT_OF_MEMORY;
  ctx->device = opt->device;
  ctx->seed = opt->seed;
  ctx->flags = opt->flags;
  cudaError_t e = cudaSetDevice(opt->device);
  if (e == cudaSuccess && (opt->flags & IPT_FLAG_OWN_STREAM)) {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    ctx->own_stream = e == cudaSuccess;
  } else {
    ctx->stream = static_cast<cudaStream_t>(opt->stream);  // NULL: legacy default stream
  }
  if (e == cudaSuccess) e = ipt::init_launcher(&ctx->L, opt->device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->err_dev, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(ctx->err_dev, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->loss_host, sizeof(double));
  if (e == cudaSuccess && (opt->flags & IPT_FLAG_COUNTERS)) {
    e = cudaMalloc(&ctx->counters_dev, 6 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->counters_dev, 0, 6 * sizeof(unsigned long long));
  }
  if (e != cudaSuccess) {
    ipt_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? IPT_ERR_OUT_OF_MEMORY : IPT_ERR_CUDA;
  }
  *out = ctx;
  return IPT_OK;
}

ipt_status ipt_destroy(ipt_ctx* ctx) {
  if (!ctx) return IPT_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (Batch* b : ctx->batches)
    if (b) {
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      for (void* p : b->owned) cudaFree(p);
      if (b->losses_host) cudaFreeHost(b->losses_host);
      delete b;
    }
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (DeviceScene* s : ctx->scenes) free_scene(s);
  wf_release(ctx);
  if (ctx->wf_tab) cudaFree(ctx->wf_tab);
  resolve_timings(ctx);
  for (cudaEvent_t e : ctx->spare_events) cudaEventDestroy(e);
  if (ctx->counters_dev) cudaFree(ctx->counters_dev);
  if (ctx->err_dev) cudaFree(ctx->err_dev);
  if (ctx->loss_host) cudaFreeHost(ctx->loss_host);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return IPT_OK;
}

ipt_status ipt_scene_upload(ipt_ctx* ctx, const float* pos, uint32_t n_vert, const float* nrm,
                            const uint32_t* idx, uint32_t n_tri, const uint32_t* tri_seg,
                            uint32_t n_seg, float emission_scale, int32_t* scene_id) {
  if (!ctx || !scene_id) return IPT_ERR_INVALID_ARG;
  if (!(emission_scale > 0.0f) || !std::isfinite(emission_scale))
    return fail(ctx, IPT_ERR_INVALID_ARG, "emission_scale must be positive and finite");
  HostScene hs;
  std::string err;
  if (!ipt::build_scene(pos, n_vert, nrm, idx, n_tri, tri_seg, n_seg, &hs, &err))
    return fail(ctx, IPT_ERR_INVALID_ARG, err);
  IPT_CK(cudaSetDevice(ctx->device));
  DeviceScene* s = new (std::nothrow) DeviceScene();
  if (!s) return IPT_ERR_OUT_OF_MEMORY;
  s->n_tri = hs.n_tri;
  s->n_seg = hs.n_seg;
  s->n_nodes = hs.n_nodes;
  s->depth = hs.depth;
  s->eps = (float)(1e-5 * hs.diameter);
  s->emission_scale = emission_scale;
  for (int a = 0; a < 3; ++a) {
    s->bb_lo[a] = pos[a];
    s->bb_hi[a] = pos[a];
  }
  for (uint32_t i = 1; i < n_vert; ++i)
    for (int a = 0; a < 3; ++a) {
      s->bb_lo[a] = std::min(s->bb_lo[a], pos[3 * i + a]);
      s->bb_hi[a] = std::max(s->bb_hi[a], pos[3 * i + a]);
    }
  const uint32_t S = n_seg;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t n) {
    if (e == cudaSuccess) e = dev_alloc(s, p, n);
  };
  A(&s->nodes, 4 * (size_t)hs.n_nodes);
  A(&s->nodes4, 4 * (size_t)hs.n_nodes4);
  A(&s->nodes8, 6 * (size_t)hs.n_nodes8);
  A(&s->tris, 3 * (size_t)n_tri);
  if (!hs.vnrm.empty()) A(&s->vnrm, 3 * (size_t)n_tri);
  A(&s->seg_tris, n_tri);
  A(&s->seg_begin, S + 1);
  A(&s->tri_cdf, n_tri);
  A(&s->seg_area, S);
  A(&s->orig_to_internal, n_tri);
  A(&s->tab.mat_a, S);
  A(&s->tab.mat_b, S);
  A(&s->tab.emis, S);
  A(&s->tab.samp, S);
  A(&s->tab.pspec, S);
  A(&s->tab.cdf, S);
  A(&s->tab.lum, S);
  A(&s->tab.W, 1);
  A(&s->params, 10 * (size_t)S);
  A(&s->adam_m, 10 * (size_t)S);
  A(&s->adam_v, 10 * (size_t)S);
  A(&s->free_mask, 10 * (size_t)S);
  A(&s->step_dev, 1);
  A(&s->grad_acc, 10 * (size_t)S);
  A(&s->grad_f, 10 * (size_t)S);
  A(&s->loss_partials, (size_t)ipt::loss_partials_capacity(ctx->L));
  A(&s->loss_dev, 1);
  A(&s->guard_dev, 1);
  auto H = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  H(s->nodes, hs.nodes.data(), hs.nodes.size() * sizeof(float));
  H(s->nodes4, hs.nodes4.data(), hs.nodes4.size() * sizeof(uint32_t));
  H(s->nodes8, hs.nodes8.data(), hs.nodes8.size() * sizeof(uint32_t));
  H(s->tris, hs.tris.data(), hs.tris.size() * sizeof(float));
  if (s->vnrm) H(s->vnrm, hs.vnrm.data(), hs.vnrm.size() * sizeof(float));
  H(s->seg_tris, hs.seg_tris.data(), hs.seg_tris.size() * sizeof(uint32_t));
  H(s->seg_begin, hs.seg_begin.data(), hs.seg_begin.size() * sizeof(uint32_t));
  H(s->tri_cdf, hs.tri_cdf.data(), hs.tri_cdf.size() * sizeof(double));
  H(s->seg_area, hs.seg_area.data(), hs.seg_area.size() * sizeof(double));
  H(s->orig_to_internal, hs.orig_to_internal.data(), hs.orig_to_internal.size() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(s->params, 0, 10 * sizeof(float) * S);
  if (e == cudaSuccess) e = cudaMemset(s->adam_m, 0, 10 * sizeof(float) * S);
  if (e == cudaSuccess) e = cudaMemset(s->adam_v, 0, 10 * sizeof(float) * S);
  if (e == cudaSuccess) e = cudaMemset(s->free_mask, 1, 10 * S);
  if (e == cudaSuccess) e = cudaMemset(s->step_dev, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_scene(s);
    return cuda_fail(ctx, e, "scene upload");
  }
  ctx->scenes.push_back(s);
  *scene_id = (int32_t)ctx->scenes.size() - 1;
  return IPT_OK;
}

ipt_status ipt_views_set(ipt_ctx* ctx, int32_t scene, const ipt_camera* cams, uint32_t n_views,
                         const float* target_rgb, int32_t target_on_device) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!cams || n_views == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "need at least one view");
  std::vector<ipt::ViewHost> v(n_views);
  uint64_t off = 0;
  for (uint32_t i = 0; i < n_views; ++i) {
    const ipt_camera& c = cams[i];
    if (c.width == 0 || c.height == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "view with zero width or height");
    if (!(c.fov_y_deg > 0.0f && c.fov_y_deg < 180.0f))
      return fail(ctx, IPT_ERR_INVALID_ARG, "fov_y_deg must be in (0, 180)");
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(c.cam_to_world[k])) return fail(ctx, IPT_ERR_INVALID_ARG, "non-finite camera matrix");
    std::memcpy(v[i].m, c.cam_to_world, sizeof(v[i].m));
    const double th = std::tan(0.5 * (double)c.fov_y_deg * 3.14159265358979323846 / 180.0);
    v[i].ty = (float)th;
    v[i].tx = (float)(th * (double)c.width / (double)c.height);
    v[i].w = c.width;
    v[i].h = c.height;
    v[i].offset = (uint32_t)off;
    off += (uint64_t)c.width * c.height;
    if (off >= (1ull << 32)) return fail(ctx, IPT_ERR_INVALID_ARG, "more than 2^32 pixels");
  }
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  if (s->views_dev) cudaFree(s->views_dev), s->views_dev = nullptr;
  if (s->target) cudaFree(s->target), s->target = nullptr;
  if (s->g_img) cudaFree(s->g_img), s->g_img = nullptr;
  IPT_CK(cudaMalloc(&s->views_dev, n_views * sizeof(ipt::ViewHost)));
  IPT_CK(cudaMemcpy(s->views_dev, v.data(), n_views * sizeof(ipt::ViewHost), cudaMemcpyHostToDevice));
  IPT_CK(cudaMalloc(&s->g_img, off * 3 * sizeof(float)));
  s->views = v;
  s->n_pix = off;
  if (target_rgb) return ipt_targets_set(ctx, scene, target_rgb, target_on_device);
  return IPT_OK;
}

ipt_status ipt_targets_set(ipt_ctx* ctx, int32_t scene, const float* target_rgb, int32_t target_on_device) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!target_rgb || s->n_pix == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "targets need views and data");
  IPT_CK(cudaSetDevice(ctx->device));
  if (!s->target) IPT_CK(cudaMalloc(&s->target, s->n_pix * 3 * sizeof(float)));
  IPT_CK(cudaMemcpyAsync(s->target, target_rgb, s->n_pix * 3 * sizeof(float),
                         target_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  return IPT_OK;
}

ipt_status ipt_params_set(ipt_ctx* ctx, int32_t scene, const float* params, const uint8_t* free_mask) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!params) return fail(ctx, IPT_ERR_INVALID_ARG, "null params");
  const size_t n = 10 * (size_t)s->n_seg;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(params[i])) return fail(ctx, IPT_ERR_NONFINITE, "non-finite parameter " + std::to_string(i));
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaMemcpyAsync(s->params, params, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  IPT_CK(cudaMemsetAsync(s->adam_m, 0, n * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(s->adam_v, 0, n * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(s->step_dev, 0, sizeof(int), ctx->stream));
  if (free_mask) {
    IPT_CK(cudaMemcpyAsync(s->free_mask, free_mask, n, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    IPT_CK(cudaMemsetAsync(s->free_mask, 1, n, ctx->stream));
  }
  IPT_CK(cudaStreamSynchronize(ctx->stream));  // host buffers may be released on return
  s->tab_is_ctx = false;
  s->params_set = true;
  s->iteration = 0;
  return IPT_OK;
}

ipt_status ipt_params_get(ipt_ctx* ctx, int32_t scene, float* params_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!params_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null output");
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaMemcpyAsync(params_out, s->params, 10 * sizeof(float) * s->n_seg, cudaMemcpyDeviceToHost,
                         ctx->stream));
  return ipt_synchronize(ctx);
}

ipt_status ipt_params_device(ipt_ctx* ctx, int32_t scene, float** params_dev) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!params_dev) return IPT_ERR_INVALID_ARG;
  *params_dev = s->params;
  s->tab_is_ctx = false;  // the caller may write through the pointer
  return IPT_OK;
}

ipt_status ipt_render(ipt_ctx* ctx, int32_t scene, int32_t view, const ipt_trace_opts* opts, uint32_t set,
                      uint32_t spp, uint64_t iteration, const float* params, const float* sampling_params,
                      float* rgb_out, float* msq_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, false)) != IPT_OK) return st;
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "no views set");
  if (view < -1 || view >= (int32_t)s->views.size()) return fail(ctx, IPT_ERR_INVALID_ARG, "view out of range");
  if (spp == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp must be positive");
  if (!rgb_out && !msq_out) return fail(ctx, IPT_ERR_INVALID_ARG, "no output");
  IPT_CK(cudaSetDevice(ctx->device));
  const float* p = params ? params : s->params;
  if ((st = ensure_tables(ctx, s, p, sampling_params)) != IPT_OK) return st;
  const uint32_t begin = view < 0 ? 0u : s->views[view].offset;
  const uint32_t n = view < 0 ? (uint32_t)s->n_pix : s->views[view].w * s->views[view].h;
  ipt::CachePass cp;
  if (cache_on(s) && (st = cache_pass(ctx, s, false, &cp)) != IPT_OK) return st;
  return run_forward(ctx, scene, s, begin, n, trace_params(ctx, scene, opts, set, spp, iteration), rgb_out, msq_out,
                     nullptr, nullptr, nullptr, 0.f, 0, cache_on(s) ? &cp : nullptr);
}

ipt_status ipt_backward(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint32_t set, uint64_t iteration,
                        const float* params, const float* sampling_params, const float* grad_image,
                        float* grad_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, true)) != IPT_OK) return st;
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "no views set");
  if (!grad_image || !grad_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null grad_image or grad_out");
  if (opts->spp_d == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp_d must be positive");
  IPT_CK(cudaSetDevice(ctx->device));
  const float* p = params ? params : s->params;
  if ((st = ensure_tables(ctx, s, p, sampling_params)) != IPT_OK) return st;
  const uint32_t np = 10u * s->n_seg;
  IPT_CK(cudaMemsetAsync(s->grad_acc, 0, np * sizeof(double), ctx->stream));
  s->loss_fresh = false;  // grad_acc now holds a vector-Jacobian product, not a loss gradient
  ipt::CachePass cp;
  if (cache_on(s) && (st = cache_pass(ctx, s, false, &cp)) != IPT_OK) return st;
  st = run_adjoint(ctx, scene, s, 0, (uint32_t)s->n_pix,
                   trace_params(ctx, scene, opts, set, opts->spp_d, iteration), grad_image, s->grad_acc,
                   cache_on(s) ? &cp : nullptr);
  if (st != IPT_OK) return st;
  Timed tm(ctx, IPT_KERNEL_FINALIZE);
  IPT_CK(ipt::launch_finalize(nullptr, 0, nullptr, s->grad_acc, grad_out, np, ctx->stream));
  return IPT_OK;
}



ipt_status ipt_loss_grad(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint64_t iteration,
                         double* loss_out, float* grad_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = loss_grad_async(ctx, scene, s, opts, iteration, grad_out, 0, s->n_pix, s->n_pix)) != IPT_OK) return st;
  if (loss_out) return read_loss(ctx, s, loss_out, opts->pixel_batch ? opts->pixel_batch : s->n_pix);
  return IPT_OK;
}

ipt_status ipt_loss_grad_shard(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint64_t iteration,
                               uint64_t pix_begin, uint64_t pix_count, uint64_t n_total_pixels,
                               double* loss_out, float* grad_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!grad_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null grad_out");
  if ((st = loss_grad_async(ctx, scene, s, opts, iteration, grad_out, pix_begin, pix_count, n_total_pixels)) !=
      IPT_OK)
    return st;
  if (loss_out) return read_loss(ctx, s, loss_out, n_total_pixels);
  return IPT_OK;
}


ipt_status ipt_adam_step(ipt_ctx* ctx, int32_t scene, const float* grad, const ipt_adam_opts* adam) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!adam) return fail(ctx, IPT_ERR_INVALID_ARG, "null adam options");
  if (!(adam->lr >= 0.0f) || !(adam->beta1 >= 0.0f && adam->beta1 < 1.0f) ||
      !(adam->beta2 >= 0.0f && adam->beta2 < 1.0f) || !(adam->eps > 0.0f) || !(adam->l1_emission >= 0.0f))
    return fail(ctx, IPT_ERR_INVALID_ARG, "invalid adam options");
  IPT_CK(cudaSetDevice(ctx->device));
  Timed tm(ctx, IPT_KERNEL_ADAM);
  // the loss is checked with the context's own gradient (the one it belongs to)
  const double* loss = (grad == nullptr && s->loss_fresh) ? s->loss_dev : nullptr;
  IPT_CK(ipt::launch_adam(buffers(ctx, s), s->tab, s->params, s->adam_m, s->adam_v, s->free_mask, s->grad_acc, grad,
                          s->step_dev, adam_host(adam), loss, s->guard_dev, ctx->err_dev, ctx->stream));
  s->tab_is_ctx = true;  // the Adam kernel rebuilt the tables from the new parameters
  s->tab_batch = -1;
  return IPT_OK;
}

ipt_status ipt_step(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, const ipt_adam_opts* adam,
                    double* loss_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = loss_grad_async(ctx, scene, s, opts, s->iteration, nullptr, 0, s->n_pix, s->n_pix)) != IPT_OK) return st;
  if (cache_on(s) && (st = cache_train_pass(ctx, scene, s, opts, s->iteration)) != IPT_OK) return st;
  if ((st = ipt_adam_step(ctx, scene, nullptr, adam)) != IPT_OK) return st;
  s->iteration++;
  if (loss_out) return read_loss(ctx, s, loss_out, opts->pixel_batch ? opts->pixel_batch : s->n_pix);
  return IPT_OK;
}

ipt_status ipt_trace_rays(ipt_ctx* ctx, int32_t scene, uint32_t n, const float* orig, const float* dir,
                          const int32_t* skip, int32_t* tri_out, float* t_out, float* u_out, float* v_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (n && (!orig || !dir || !tri_out)) return fail(ctx, IPT_ERR_INVALID_ARG, "null ray buffers");
  IPT_CK(cudaSetDevice(ctx->device));
  Timed tm(ctx, IPT_KERNEL_TRACE);
  IPT_CK(ipt::launch_trace_rays(buffers(ctx, s), n, orig, dir, skip, tri_out, t_out, u_out, v_out, ctx->err_dev,
                                ctx->stream));
  return IPT_OK;
}

ipt_status ipt_pick_pixels(ipt_ctx* ctx, int32_t scene, uint32_t batch, uint64_t iteration, uint32_t* ids_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (batch == 0) return IPT_OK;
  if (!ids_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null ids_out");
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "pixel batches need views");
  IPT_CK(cudaSetDevice(ctx->device));
  return draw_picks(ctx, scene, s, batch, iteration, ids_out);
}

ipt_status ipt_philox(ipt_ctx* ctx, uint32_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  if (!ctx) return IPT_ERR_INVALID_ARG;
  if (n && (!ctr || !key || !out)) return fail(ctx, IPT_ERR_INVALID_ARG, "null philox buffers");
  IPT_CK(cudaSetDevice(ctx->device));
  Timed tm(ctx, IPT_KERNEL_PHILOX);
  IPT_CK(ipt::launch_philox(n, ctr, key, out, ctx->stream));
  return IPT_OK;
}

ipt_status ipt_synchronize(ipt_ctx* ctx) {
  if (!ctx) return IPT_ERR_INVALID_ARG;
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  uint32_t err = 0;
  IPT_CK(cudaMemcpy(&err, ctx->err_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (err) {
    cudaMemset(ctx->err_dev, 0, sizeof(uint32_t));
    if (err & ipt::kErrStack)
      return fail(ctx, IPT_ERR_CUDA, "device error word " + std::to_string(err) + " (traversal stack overflow)");
    if (err & ipt::kErrTimeout)
      return fail(ctx, IPT_ERR_TIMEOUT,
                  "a bounded wait for the tensor cores gave up in the radiance cache's training pass; its "
                  "gradients are incomplete");
    return fail(ctx, IPT_ERR_NONFINITE,
                "non-finite loss or gradient: the Adam step was skipped, parameters and Adam state are those of "
                "the last good step");
  }
  return IPT_OK;
}

ipt_status ipt_scene_info(ipt_ctx* ctx, int32_t scene, uint32_t* n_tri, uint32_t* n_seg, uint32_t* n_nodes,
                          uint32_t* bvh_depth, uint32_t* n_views, uint64_t* n_pixels) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (n_tri) *n_tri = s->n_tri;
  if (n_seg) *n_seg = s->n_seg;
  if (n_nodes) *n_nodes = s->n_nodes;
  if (bvh_depth) *bvh_depth = s->depth;
  if (n_views) *n_views = (uint32_t)s->views.size();
  if (n_pixels) *n_pixels = s->n_pix;
  return IPT_OK;
}

ipt_status ipt_config_set(ipt_ctx* ctx, const ipt_config* cfg) {
  if (!ctx || !cfg) return IPT_ERR_INVALID_ARG;
  if (cfg->integrator != 0 && cfg->integrator != 1)
    return fail(ctx, IPT_ERR_INVALID_ARG, "integrator must be 0 (megakernel) or 1 (wavefront)");
  if (cfg->wavefront_slots && cfg->wavefront_slots < 1024)
    return fail(ctx, IPT_ERR_INVALID_ARG, "wavefront_slots must be 0 or at least 1024");
  if (cfg->trace_steps > 4096) return fail(ctx, IPT_ERR_INVALID_ARG, "trace_steps above 4096");
  if (cfg->bvh_width != 0 && cfg->bvh_width != 2 && cfg->bvh_width != 4 && cfg->bvh_width != 8)
    return fail(ctx, IPT_ERR_INVALID_ARG, "bvh_width must be 0, 2, 4 or 8");
  if (cfg->sort_cells > 16 || cfg->sort_dirs > 16)
    return fail(ctx, IPT_ERR_INVALID_ARG, "sort_cells and sort_dirs must be at most 16");
  {
    const uint64_t d = cfg->sort_dirs, c = cfg->sort_cells;
    if ((d ? 6u * d * d : 1u) * c * c * c > ipt::kSortMaxBins)
      return fail(ctx, IPT_ERR_INVALID_ARG, "6 sort_dirs^2 sort_cells^3 above 8192");
  }
  IPT_CK(cudaSetDevice(ctx->device));
  const uint32_t old_cap = ctx->cfg.wavefront_slots ? ctx->cfg.wavefront_slots : (1u << 20);
  const uint32_t new_cap = cfg->wavefront_slots ? cfg->wavefront_slots : (1u << 20);
  if (old_cap != new_cap || cfg->blocks_per_sm != ctx->cfg.blocks_per_sm) {
    IPT_CK(cudaStreamSynchronize(ctx->stream));
    wf_release(ctx);
  }
  ctx->cfg = *cfg;
  ctx->L.wf_steps = cfg->trace_steps ? (int)cfg->trace_steps : 16;
  ctx->L.wf_fixed_blocks = (int)cfg->blocks_per_sm;
  ctx->L.sort_cells = (int)cfg->sort_cells;
  ctx->L.sort_dirs = (int)cfg->sort_dirs;
  IPT_CK(ipt::wf_init(&ctx->L));
  return IPT_OK;
}

ipt_status ipt_config_get(const ipt_ctx* ctx, ipt_config* cfg) {
  if (!ctx || !cfg) return IPT_ERR_INVALID_ARG;
  *cfg = ctx->cfg;
  return IPT_OK;
}

ipt_status ipt_kernel_times(ipt_ctx* ctx, double* total_ms, uint64_t* launches, int32_t reset) {
  if (!ctx) return IPT_ERR_INVALID_ARG;
  if (!(ctx->flags & IPT_FLAG_KERNEL_TIMING))
    return fail(ctx, IPT_ERR_INVALID_ARG, "context created without IPT_FLAG_KERNEL_TIMING");
  IPT_CK(cudaSetDevice(ctx->device));
  resolve_timings(ctx);
  for (int k = 0; k < IPT_KERNEL_COUNT; ++k) {
    if (total_ms) total_ms[k] = ctx->kernel_ms[k];
    if (launches) launches[k] = ctx->kernel_n[k];
    if (reset) {
      ctx->kernel_ms[k] = 0.0;
      ctx->kernel_n[k] = 0;
    }
  }
  return IPT_OK;
}

ipt_status ipt_counters_read(ipt_ctx* ctx, uint64_t* out, int32_t reset) {
  if (!ctx || !out) return IPT_ERR_INVALID_ARG;
  if (!ctx->counters_dev) return fail(ctx, IPT_ERR_INVALID_ARG, "context created without IPT_FLAG_COUNTERS");
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  unsigned long long v[6];
  IPT_CK(cudaMemcpy(v, ctx->counters_dev, sizeof(v), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 6; ++k) out[k] = v[k];
  if (reset) IPT_CK(cudaMemset(ctx->counters_dev, 0, sizeof(v)));
  return IPT_OK;
}

}  // extern "C"
