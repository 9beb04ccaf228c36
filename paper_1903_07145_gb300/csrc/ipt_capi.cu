// C ABI of the GB300 inverse path tracer: context, scenes, views, parameters
// and the calls of one nested-SGD iteration.  See include/ipt.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ipt.h"
#include "ipt_cache.h"
#include "ipt_internal.h"
#include "ipt_path.cuh"
#include "ipt_wavefront.h"

using ipt::HostScene;

namespace {

// Radiance cache of one scene: network, Adam state, query and record buffers.
struct CacheState {
  ipt_cache_opts opts{};
  bool active = false;     // enabled and not turned off by the bias monitor
  bool fell_back = false;
  int res[ipt::kCacheLevels] = {0};
  uint32_t dense = 0;
  float* w = nullptr;      // FP32 master weights
  float* mw = nullptr;
  float* vw = nullptr;
  float* gw = nullptr;
  uint4* wt = nullptr;     // BF16 image
  float* table = nullptr;
  float* mt = nullptr;
  float* vt = nullptr;
  float* gt = nullptr;
  double* loss_dev = nullptr;   // per training step
  double* host = nullptr;       // pinned scratch (loss sums, counts)
  uint64_t steps_done = 0;
  uint32_t last_pass_steps = 0;
  ipt::CacheBuffers buf{};
  // rows of the evaluation entry points
  ipt::CacheRows api{};
  float4* api_ma = nullptr;
  float4* api_mb = nullptr;
  float4* api_c = nullptr;
  float* api_dp = nullptr;
  uint32_t api_cap = 0;
  std::vector<void*> api_owned;
  std::vector<void*> owned;
  double image_bias = -1.0, grad_bias = -1.0;
};

void free_cache(CacheState* c) {
  if (!c) return;
  for (void* p : c->owned) cudaFree(p);
  for (void* p : c->api_owned) cudaFree(p);
  if (c->host) cudaFreeHost(c->host);
  delete c;
}

// Disney material model of one scene (Sec. 4.1): its own 16-value
// parameter blocks, optimiser state and tables, next to the scene's
// Lambert + GGX parameters.
struct DisneyState {
  float* params = nullptr;   // S x 16
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  uint8_t* free_mask = nullptr;
  int* step_dev = nullptr;
  double* grad_acc = nullptr;
  float* gacc = nullptr;     // global accumulators when shared memory is too small
  ipt::SegBuffers tab{};     // emission, light selection (mat_a, mat_b, pspec unused)
  ipt::DisneyBuffers dt{};
  bool tab_is_ctx = false;
  uint64_t iteration = 0;
  std::vector<void*> owned;
};

void free_disney(DisneyState* d) {
  if (!d) return;
  for (void* p : d->owned) cudaFree(p);
  delete d;
}

struct DeviceScene;
// The scene's Disney state, allocated on first use.
ipt_status disney_state(ipt_ctx* ctx, DeviceScene* s, DisneyState** out);

struct DeviceScene {
  uint32_t n_tri = 0, n_seg = 0, n_nodes = 0, depth = 0;
  float eps = 0.f, emission_scale = 1.f;
  // geometry
  float4* nodes = nullptr;
  uint4* nodes4 = nullptr;
  float4* tris = nullptr;
  float4* vnrm = nullptr;
  uint32_t* seg_tris = nullptr;
  uint32_t* seg_begin = nullptr;
  double* tri_cdf = nullptr;
  double* seg_area = nullptr;
  uint32_t* orig_to_internal = nullptr;
  // parameter tables
  ipt::SegBuffers tab{};
  bool tab_is_ctx = false;  // tables were built from the context's own parameters
  // parameters and optimiser state
  float* params = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  uint8_t* free_mask = nullptr;
  int* step_dev = nullptr;
  bool params_set = false;
  // views and per-pixel buffers
  std::vector<ipt::ViewHost> views;
  ipt::ViewHost* views_dev = nullptr;
  uint64_t n_pix = 0;
  float* target = nullptr;
  float* g_img = nullptr;
  // stochastic pixel batch: drawn pixel ids and upstream gradient per entry
  uint32_t* pick = nullptr;
  float* g_pick = nullptr;
  uint32_t pick_cap = 0;
  // reductions
  double* grad_acc = nullptr;
  float* grad_f = nullptr;
  double* loss_partials = nullptr;
  double* loss_dev = nullptr;
  uint32_t* guard_dev = nullptr;  // the Adam step's finiteness decision (scenes over a grid)
  bool loss_fresh = false;        // loss_dev holds the loss of the gradient in grad_acc
  uint64_t iteration = 0;
  float bb_lo[3] = {0.f, 0.f, 0.f}, bb_hi[3] = {1.f, 1.f, 1.f};  // vertex bounding box
  CacheState* cache = nullptr;
  DisneyState* disney = nullptr;
  std::vector<void*> owned;
};

}  // namespace

struct Batch {
  std::vector<int32_t> members;
  uint32_t n_seg_total = 0;
  uint64_t n_pix_total = 0;
  std::vector<ipt::WfScene> tab_host;
  ipt::WfScene* tab_dev = nullptr;
  std::vector<ipt::BatchMember> mem_host;
  ipt::BatchMember* mem_dev = nullptr;
  std::vector<uint8_t> active;  // members that take part in the steps
  float* params = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  uint8_t* free_mask = nullptr;
  double* grad_acc = nullptr;
  float* gacc = nullptr;  // megakernel: global FP32 accumulators when shared memory is too small
  uint32_t* iter_dev = nullptr;
  double* loss_rows = nullptr;
  double* losses_dev = nullptr;
  double* losses_host = nullptr;  // pinned
  std::vector<void*> owned;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ipt_trace_opts g_opts{};
  ipt_adam_opts g_adam{};
  ipt_config g_cfg{};
};

struct PendingTiming {
  int id;
  cudaEvent_t a, b;
  int launches;
};

struct ipt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t seed = 0;
  int flags = 0;
  ipt::Launcher L;
  std::vector<DeviceScene*> scenes;
  std::string last_error;
  uint32_t* err_dev = nullptr;
  double* loss_host = nullptr;  // pinned
  unsigned long long* counters_dev = nullptr;
  std::vector<PendingTiming> pending;
  std::vector<cudaEvent_t> spare_events;
  double kernel_ms[IPT_KERNEL_COUNT] = {0};
  uint64_t kernel_n[IPT_KERNEL_COUNT] = {0};
  ipt_config cfg = {1, 1u << 20, 32, 0, 4};
  ipt::WfBuffers wf;
  std::vector<void*> wf_owned;
  bool wf_adjoint = false;
  bool wf_disney = false;          // the adjoint buffers include the Disney model's records
  ipt::WfScene* wf_tab = nullptr;  // one-entry scene table of single-scene launches
  std::vector<Batch*> batches;
  cudaStream_t cap_stream = nullptr;  // stream the batch graphs are captured on
  double* noalloc_acc = nullptr;      // device address of ipt_backward_noalloc's array on this device
};

namespace {

ipt_status fail(ipt_ctx* c, ipt_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

ipt_status cuda_fail(ipt_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? IPT_ERR_OUT_OF_MEMORY : IPT_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define IPT_CK(expr)                                          \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr);  \
  } while (0)

template <class T>
cudaError_t dev_alloc(DeviceScene* s, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
  if (e == cudaSuccess) {
    s->owned.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
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

// Brackets one launch with CUDA events on the context stream when kernel
// timing is on.
struct Timed {
  ipt_ctx* c;
  int id;
  int launches = 1;  // kernels launched inside the bracket
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(ipt_ctx* ctx, int kernel) : c(ctx), id(kernel) {
    if (c->flags & IPT_FLAG_KERNEL_TIMING) {
      if (c->pending.size() > 8192) resolve_timings(c);
      a = take_event(c);
      b = take_event(c);
      if (a && b) cudaEventRecord(a, c->stream);
    }
  }
  ~Timed() {
    if (a && b) {
      cudaEventRecord(b, c->stream);
      c->pending.push_back({id, a, b, launches});
    }
  }
};

// Stage hook for the wavefront launchers: one event pair per launch.
struct StageTimer {
  ipt_ctx* c;
  int id = 0;
  cudaEvent_t a = nullptr;
};

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
  b.wide = ctx->cfg.bvh_width != 2 ? 1 : 0;
  b.nodes = s->nodes;
  b.nodes4 = s->nodes4;
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

ipt_status check_opts(ipt_ctx* ctx, const ipt_trace_opts* o, bool adjoint, bool batch_ok = false) {
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
ipt_status ensure_wf(ipt_ctx* ctx, bool adjoint, uint32_t n_params, bool disney = false) {
  const uint32_t cap = ctx->cfg.wavefront_slots ? ctx->cfg.wavefront_slots : (1u << 20);
  const bool fits = ctx->wf.cap == cap && (!adjoint || (ctx->wf_adjoint && ctx->wf.blk_params >= n_params)) &&
                    (!disney || ctx->wf_disney);
  if (fits) return IPT_OK;
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  const uint32_t keep_params = std::max(n_params, ctx->wf.blk_params);
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
  if (want_adj) {
    A(&w.aT, (size_t)ipt::kMaxAdjointDepth * cap);
    A(&w.aU, (size_t)ipt::kMaxAdjointDepth * cap);
    A(&w.aR, (size_t)ipt::kMaxAdjointDepth * cap);
    A(&w.nv, cap);
    A(&w.sh_ge, cap);
    A(&w.sh_gm, cap);
    A(&w.sh_n, cap);
    if (want_disney) {
      A(&w.aWi, (size_t)ipt::kMaxAdjointDepth * cap);
      A(&w.aWo, (size_t)ipt::kMaxAdjointDepth * cap);
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
                       double* partials, float g_scale, int loss_kind, const ipt::CachePass* cache = nullptr,
                       uint32_t* pick = nullptr) {
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
                       const ipt::CachePass* cache = nullptr, uint32_t* pick = nullptr) {
  if (cache && !use_wavefront_cap(ctx, tp.spp))
    return fail(ctx, IPT_ERR_INVALID_ARG, "cached passes need spp <= wavefront_slots");
  if (cache || use_wavefront(ctx, tp.spp)) {
    ipt_status st = ensure_wf(ctx, true, 10u * s->n_seg);
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
    IPT_CK(ipt::cache_adam(c->w, c->mw, c->vw, c->gw, c->table, c->mt, c->vt, c->gt, c->wt, c->opts.lr,
                           c->opts.beta1, c->opts.beta2, c->opts.eps, bc1, bc2, ctx->L.num_sms, ctx->stream));
  }
  c->last_pass_steps = steps;
  return IPT_OK;
}

}  // namespace

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

// Forward + residual + adjoint over pixels [begin, begin + count), with the
// loss normalised by n_total pixels (all shards together).
static ipt_status loss_grad_async(ipt_ctx* ctx, int32_t scene, DeviceScene* s, const ipt_trace_opts* opts,
                                  uint64_t iteration, float* grad_out, uint64_t begin, uint64_t count,
                                  uint64_t n_total) {
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

static ipt_status read_loss(ipt_ctx* ctx, DeviceScene* s, double* loss_out, uint64_t n_total) {
  IPT_CK(cudaMemcpyAsync(ctx->loss_host, s->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  ipt_status st = ipt_synchronize(ctx);
  if (st != IPT_OK) return st;
  *loss_out = *ctx->loss_host / (3.0 * (double)n_total);
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

static ipt::AdamHost adam_host(const ipt_adam_opts* a) {
  ipt::AdamHost h;
  h.lr = a->lr;
  h.beta1 = a->beta1;
  h.beta2 = a->beta2;
  h.eps = a->eps;
  h.l1 = a->l1_emission;
  return h;
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
  if (cfg->bvh_width != 0 && cfg->bvh_width != 2 && cfg->bvh_width != 4)
    return fail(ctx, IPT_ERR_INVALID_ARG, "bvh_width must be 0, 2 or 4");
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
  IPT_CK(ipt::wf_init(&ctx->L));
  return IPT_OK;
}

ipt_status ipt_config_get(const ipt_ctx* ctx, ipt_config* cfg) {
  if (!ctx || !cfg) return IPT_ERR_INVALID_ARG;
  *cfg = ctx->cfg;
  return IPT_OK;
}

static ipt_status get_batch(ipt_ctx* ctx, int32_t id, Batch** out) {
  if (!ctx) return IPT_ERR_INVALID_ARG;
  if (id < 0 || (size_t)id >= ctx->batches.size() || !ctx->batches[id])
    return fail(ctx, IPT_ERR_INVALID_ARG, "unknown batch id " + std::to_string(id));
  *out = ctx->batches[id];
  return IPT_OK;
}

// Scene table of a batch for the context's current configuration.
// Scene table of a batch: every member's pixels, or B batch entries per
// member when the step uses pixel batches (batch > 0; the members' pick
// buffers must hold B entries).  Also sets each member's loss normalisation.
static void batch_table(ipt_ctx* ctx, Batch* b, uint32_t batch) {
  b->tab_host.clear();
  uint32_t pix = 0, seg = 0;
  for (size_t k = 0; k < b->members.size(); ++k) {
    const int32_t id = b->members[k];
    DeviceScene* s = ctx->scenes[id];
    b->mem_host[k].active = b->active[k];
    b->mem_host[k].slot = (uint32_t)b->tab_host.size();
    b->mem_host[k].grad_offset = seg;
    if (!b->active[k]) continue;  // no pixels in the launch; its segment range stays unused
    const uint32_t n = batch ? batch : (uint32_t)s->n_pix;
    ipt::WfScene e = wf_entry(ctx, id, s, 0, n);
    e.pix_begin = pix;
    e.seg_offset = seg;
    e.g_scale = (float)(1.0 / (3.0 * (double)n));
    e.target = s->target;
    e.g_img = batch ? s->g_pick : s->g_img;
    e.pick = batch ? s->pick : nullptr;
    e.n_all = (uint32_t)s->n_pix;
    b->tab_host.push_back(e);
    b->mem_host[k].inv_n = e.g_scale;
    pix += n;
    seg += s->n_seg;
  }
}

ipt_status ipt_batch_create(ipt_ctx* ctx, const int32_t* scenes, uint32_t n, int32_t* batch_id) {
  if (!ctx || !scenes || !batch_id) return IPT_ERR_INVALID_ARG;
  if (n == 0 || n > 4096) return fail(ctx, IPT_ERR_INVALID_ARG, "a batch needs 1 to 4096 scenes");
  std::vector<int32_t> ids(scenes, scenes + n);
  {
    std::vector<int32_t> sorted = ids;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(ctx, IPT_ERR_INVALID_ARG, "a scene appears twice in the batch");
  }
  uint64_t pix = 0;
  uint32_t segs = 0;
  for (int32_t id : ids) {
    DeviceScene* s;
    ipt_status st = get_scene(ctx, id, &s);
    if (st != IPT_OK) return st;
    if (s->views.empty() || !s->target)
      return fail(ctx, IPT_ERR_INVALID_ARG, "batch member " + std::to_string(id) + " has no views or targets");
    pix += s->n_pix;
    segs += s->n_seg;
  }
  if (pix >= (1ull << 32)) return fail(ctx, IPT_ERR_INVALID_ARG, "batch above 2^32 pixels");
  IPT_CK(cudaSetDevice(ctx->device));
  Batch* b = new (std::nothrow) Batch();
  if (!b) return IPT_ERR_OUT_OF_MEMORY;
  b->members = ids;
  b->active.assign(ids.size(), 1);
  b->n_seg_total = segs;
  b->n_pix_total = pix;
  const size_t np = 10 * (size_t)segs;
  const int rows = ipt::loss_partials_capacity(ctx->L);
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t count) {
    if (e != cudaSuccess) return;
    void* q = nullptr;
    e = cudaMalloc(&q, count * sizeof(**p));
    if (e == cudaSuccess) {
      b->owned.push_back(q);
      *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    }
  };
  A(&b->tab_dev, n);
  A(&b->mem_dev, n);
  A(&b->params, np);
  A(&b->adam_m, np);
  A(&b->adam_v, np);
  A(&b->free_mask, np);
  A(&b->grad_acc, np);
  if (np > ipt::batch_shared_params()) A(&b->gacc, np);
  A(&b->iter_dev, 1);
  A(&b->loss_rows, (size_t)rows * n);
  A(&b->losses_dev, n);
  if (e == cudaSuccess) e = cudaMallocHost(&b->losses_host, n * sizeof(double));
  uint32_t off = 0;
  for (int32_t id : ids) {
    DeviceScene* s = ctx->scenes[id];
    const size_t k = 10 * (size_t)s->n_seg;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->params + 10 * (size_t)off, s->params, k * sizeof(float), cudaMemcpyDeviceToDevice,
                          ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->free_mask + 10 * (size_t)off, s->free_mask, k, cudaMemcpyDeviceToDevice, ctx->stream);
    ipt::BatchMember m;
    m.tab = s->tab;
    m.seg_area = s->seg_area;
    m.seg_offset = off;
    m.n_seg = s->n_seg;
    m.es = s->emission_scale;
    m.inv_n = (float)(1.0 / (3.0 * (double)s->n_pix));
    m.active = 1;
    m.slot = (uint32_t)b->mem_host.size();
    m.grad_offset = off;
    b->mem_host.push_back(m);
    s->tab_is_ctx = false;  // the batch owns the member's tables from now on
    off += s->n_seg;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->adam_m, 0, np * sizeof(float), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->adam_v, 0, np * sizeof(float), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->iter_dev, 0, sizeof(uint32_t), ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->mem_dev, b->mem_host.data(), n * sizeof(ipt::BatchMember), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess) e = ipt::launch_prepare_batch(b->mem_dev, n, b->params, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    for (void* p : b->owned) cudaFree(p);
    if (b->losses_host) cudaFreeHost(b->losses_host);
    delete b;
    return cuda_fail(ctx, e, "batch create");
  }
  ctx->batches.push_back(b);
  *batch_id = (int32_t)ctx->batches.size() - 1;
  return IPT_OK;
}

static bool same_opts(const ipt_trace_opts& a, const ipt_trace_opts& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }
static bool same_adam(const ipt_adam_opts& a, const ipt_adam_opts& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }
static bool same_cfg(const ipt_config& a, const ipt_config& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

// The iteration of a batch, queued on stream `st` (captured into the graph).
static ipt_status batch_enqueue(ipt_ctx* ctx, Batch* b, const ipt_trace_opts* opts, const ipt_adam_opts* adam,
                                cudaStream_t st) {
  const uint32_t n = (uint32_t)b->members.size();
  const size_t np = 10 * (size_t)b->n_seg_total;
  ipt::TraceParams tp{};
  tp.seed = ctx->seed;
  tp.set = IPT_SET_RESIDUAL;
  tp.iteration = 0;
  tp.spp = opts->spp_r;
  tp.max_depth = opts->max_depth;
  tp.nee = opts->nee;
  tp.mis = opts->mis;
  tp.profile = opts->emission_profile;
  if (opts->pixel_batch) IPT_CK(ipt::wf_pick(b->tab_dev, b->tab_host, b->iter_dev, 0u, st));
  // the megakernel runs each pass as one launch over the whole table
  const bool mk = ctx->cfg.integrator == 0;
  const uint32_t ns = (uint32_t)b->tab_host.size();
  const uint32_t total = ns ? b->tab_host.back().pix_begin + b->tab_host.back().n_pix : 0u;
  uint32_t n_seg_active = 0;
  for (const ipt::WfScene& e : b->tab_host) n_seg_active = std::max(n_seg_active, e.seg_offset + e.n_seg);
  if (mk)
    IPT_CK(ipt::launch_forward_batch(ctx->L, b->tab_dev, ns, total, tp, b->iter_dev, opts->loss, b->loss_rows,
                                     ctx->err_dev, st));
  else
    IPT_CK(ipt::wf_forward(ctx->L, b->tab_dev, b->tab_host, tp, opts->loss, b->iter_dev, ctx->wf, b->loss_rows,
                           ctx->err_dev, st, nullptr));
  IPT_CK(cudaMemsetAsync(b->grad_acc, 0, np * sizeof(double), st));
  tp.set = opts->gradcheck_same_set ? IPT_SET_RESIDUAL : IPT_SET_DERIVATIVE;
  tp.spp = opts->spp_d;
  if (opts->gradcheck_same_set) tp.sample_stride = opts->spp_r;
  if (mk)
    IPT_CK(ipt::launch_adjoint_batch(ctx->L, b->tab_dev, ns, total, n_seg_active, tp, b->iter_dev, b->grad_acc,
                                     b->gacc, ctx->err_dev, st));
  else
    IPT_CK(ipt::wf_adjoint(ctx->L, b->tab_dev, b->tab_host, tp, b->iter_dev, ctx->wf, b->grad_acc, ctx->err_dev,
                           st, nullptr));
  IPT_CK(ipt::launch_batch_losses(b->loss_rows, ipt::loss_partials_capacity(ctx->L), b->mem_dev, n,
                                  (uint32_t)b->tab_host.size(), b->losses_dev, st));
  IPT_CK(ipt::launch_adam_batch(b->mem_dev, n, b->params, b->adam_m, b->adam_v, b->free_mask, b->grad_acc,
                                b->iter_dev, adam_host(adam), b->losses_dev, ctx->err_dev, st));
  IPT_CK(ipt::launch_tick(b->iter_dev, st));
  return IPT_OK;
}

ipt_status ipt_batch_step(ipt_ctx* ctx, int32_t batch, const ipt_trace_opts* opts, const ipt_adam_opts* adam,
                          double* losses_out) {
  Batch* b;
  ipt_status st = get_batch(ctx, batch, &b);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, true, true)) != IPT_OK) return st;
  if (!adam) return fail(ctx, IPT_ERR_INVALID_ARG, "null adam options");
  if (opts->spp_r == 0 || opts->spp_d == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp_r and spp_d must be positive");
  const uint32_t cap = ctx->cfg.wavefront_slots ? ctx->cfg.wavefront_slots : (1u << 20);
  if (std::max(opts->spp_r, opts->spp_d) > cap)
    return fail(ctx, IPT_ERR_INVALID_ARG, "spp above the wavefront chunk size");
  IPT_CK(cudaSetDevice(ctx->device));
  if (std::find(b->active.begin(), b->active.end(), (uint8_t)1) == b->active.end()) {
    // no member takes part: nothing to trace or update
    if (losses_out) std::fill(losses_out, losses_out + b->members.size(), 0.0);
    return IPT_OK;
  }
  if (!b->exec || !same_opts(*opts, b->g_opts) || !same_adam(*adam, b->g_adam) || !same_cfg(ctx->cfg, b->g_cfg)) {
    // everything the graph touches is allocated before the capture
    if (opts->pixel_batch)
      for (int32_t id : b->members)
        if ((st = ensure_pick(ctx, ctx->scenes[id], opts->pixel_batch)) != IPT_OK) return st;
    batch_table(ctx, b, opts->pixel_batch);
    IPT_CK(cudaMemcpyAsync(b->mem_dev, b->mem_host.data(), b->mem_host.size() * sizeof(ipt::BatchMember),
                           cudaMemcpyHostToDevice, ctx->stream));
    uint32_t max_seg = 0;
    for (const ipt::WfChunk& c : ipt::wf_plan(b->tab_host, cap, opts->spp_d, ipt::wf_max_segments()))
      max_seg = std::max(max_seg, c.seg_n);
    if ((st = ensure_wf(ctx, true, 10u * max_seg)) != IPT_OK) return st;
    IPT_CK(cudaMemcpyAsync(b->tab_dev, b->tab_host.data(), b->tab_host.size() * sizeof(ipt::WfScene),
                           cudaMemcpyHostToDevice, ctx->stream));
    IPT_CK(cudaStreamSynchronize(ctx->stream));
    if (!ctx->cap_stream) IPT_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
    if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
    IPT_CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    st = batch_enqueue(ctx, b, opts, adam, ctx->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (st != IPT_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    IPT_CK(ce);
    b->graph = g;
    IPT_CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->g_opts = *opts;
    b->g_adam = *adam;
    b->g_cfg = ctx->cfg;
  }
  {
    Timed tm(ctx, IPT_KERNEL_BATCH_STEP);
    IPT_CK(cudaGraphLaunch(b->exec, ctx->stream));
  }
  if (losses_out) {
    const size_t n = b->members.size();
    IPT_CK(cudaMemcpyAsync(b->losses_host, b->losses_dev, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if ((st = ipt_synchronize(ctx)) != IPT_OK) return st;
    std::memcpy(losses_out, b->losses_host, n * sizeof(double));
  }
  return IPT_OK;
}

ipt_status ipt_batch_set_active(ipt_ctx* ctx, int32_t batch, const uint8_t* active) {
  Batch* b;
  ipt_status st = get_batch(ctx, batch, &b);
  if (st != IPT_OK) return st;
  if (!active) return fail(ctx, IPT_ERR_INVALID_ARG, "null active flags");
  bool changed = false;
  for (size_t k = 0; k < b->members.size(); ++k) {
    const uint8_t a = active[k] ? 1 : 0;
    changed |= a != b->active[k];
    b->active[k] = a;
  }
  if (changed && b->exec) {  // the next step recaptures with the new launch table
    IPT_CK(cudaSetDevice(ctx->device));
    IPT_CK(cudaStreamSynchronize(ctx->stream));
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
  }
  return IPT_OK;
}

ipt_status ipt_batch_params_get(ipt_ctx* ctx, int32_t batch, uint32_t member, float* params_out) {
  Batch* b;
  ipt_status st = get_batch(ctx, batch, &b);
  if (st != IPT_OK) return st;
  if (member >= b->members.size() || !params_out) return fail(ctx, IPT_ERR_INVALID_ARG, "bad member or output");
  const ipt::BatchMember& m = b->mem_host[member];
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaMemcpyAsync(params_out, b->params + 10 * (size_t)m.seg_offset, 10 * sizeof(float) * m.n_seg,
                         cudaMemcpyDeviceToHost, ctx->stream));
  return ipt_synchronize(ctx);
}

ipt_status ipt_batch_destroy(ipt_ctx* ctx, int32_t batch) {
  Batch* b;
  ipt_status st = get_batch(ctx, batch, &b);
  if (st != IPT_OK) return st;
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (void* p : b->owned) cudaFree(p);
  if (b->losses_host) cudaFreeHost(b->losses_host);
  for (int32_t id : b->members) ctx->scenes[id]->tab_is_ctx = false;
  delete b;
  ctx->batches[batch] = nullptr;
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

// ---------------------------------------------------------------------------
// ipt_backward_noalloc: ipt_backward for callers that may not allocate device
// memory.  Its only scratch, the FP64 gradient accumulator, is this file-scope
// array: 10 * kNoAllocMaxSegments doubles (80 KiB) that every device which
// loads the library keeps until the process exits.  Host code only sees a
// stand-in for the array; the device address is looked up by the first call
// with each context, with the context's device current, kept in the context
// (a device reset ends every context, so no address outlives one) and
// handed to the kernels.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kNoAllocMaxSegments = 1024;

static __device__ __align__(256) double g_noalloc_grad[10 * kNoAllocMaxSegments];

// Device address of g_noalloc_grad on the context's device (current).
cudaError_t noalloc_scratch(ipt_ctx* ctx, double** out) {
  if (!ctx->noalloc_acc) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_grad);
    if (e != cudaSuccess) return e;
    ctx->noalloc_acc = static_cast<double*>(p);
  }
  *out = ctx->noalloc_acc;
  return cudaSuccess;
}

}  // namespace

extern "C" ipt_status ipt_backward_noalloc(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts,
                                           uint32_t set, uint64_t iteration, const float* params,
                                           const float* sampling_params, const float* grad_image,
                                           float* grad_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, true)) != IPT_OK) return st;
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "no views set");
  if (!grad_image || !grad_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null grad_image or grad_out");
  if (opts->spp_d == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp_d must be positive");
  if (s->n_seg > kNoAllocMaxSegments)
    return fail(ctx, IPT_ERR_INVALID_ARG, "ipt_backward_noalloc supports at most " +
                                              std::to_string(kNoAllocMaxSegments) + " segments, scene has " +
                                              std::to_string(s->n_seg));
  IPT_CK(cudaSetDevice(ctx->device));
  double* acc = nullptr;
  IPT_CK(noalloc_scratch(ctx, &acc));
  const float* p = params ? params : s->params;
  const bool is_ctx = (p == s->params) && (sampling_params == nullptr || sampling_params == s->params);
  if (!(is_ctx && s->tab_is_ctx)) {
    Timed tm(ctx, IPT_KERNEL_PREPARE);
    IPT_CK(ipt::launch_prepare(buffers(ctx, s), s->tab, p, sampling_params ? sampling_params : p, ctx->stream));
    s->tab_is_ctx = is_ctx;
  }
  const uint32_t np = 10u * s->n_seg;
  IPT_CK(cudaMemsetAsync(acc, 0, np * sizeof(double), ctx->stream));
  {
    Timed tm(ctx, IPT_KERNEL_ADJOINT);
    IPT_CK(ipt::launch_adjoint(ctx->L, buffers(ctx, s), s->tab, s->views_dev, (uint32_t)s->views.size(), 0,
                               (uint32_t)s->n_pix, trace_params(ctx, scene, opts, set, opts->spp_d, iteration),
                               grad_image, acc, nullptr, ctx->err_dev, ctx->stream));
  }
  Timed tm(ctx, IPT_KERNEL_FINALIZE);
  IPT_CK(ipt::launch_finalize(nullptr, 0, nullptr, acc, grad_out, np, ctx->stream));
  return IPT_OK;
}

// ---------------------------------------------------------------------------
// Radiance cache entry points
// ---------------------------------------------------------------------------
namespace {

// splitmix64 (Steele, Lea, Flood 2014): the initialisation's random stream.
struct SplitMix {
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
};

ipt_status check_cache_opts(ipt_ctx* ctx, const ipt_cache_opts* o) {
  if (!o) return fail(ctx, IPT_ERR_INVALID_ARG, "null cache options");
  if (o->b_term == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "b_term must be at least 1");
  if (o->train_steps == 0 || o->train_steps > 64) return fail(ctx, IPT_ERR_INVALID_ARG, "train_steps must be 1..64");
  if (o->record_capacity == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "record_capacity must be positive");
  if (!(o->lr > 0.0f) || !(o->eps > 0.0f) || !(o->beta1 >= 0.0f && o->beta1 < 1.0f) ||
      !(o->beta2 >= 0.0f && o->beta2 < 1.0f) || !(o->bias_threshold >= 0.0f))
    return fail(ctx, IPT_ERR_INVALID_ARG, "invalid cache optimizer options");
  return IPT_OK;
}

ipt_status get_cache(ipt_ctx* ctx, int32_t scene, DeviceScene** s) {
  ipt_status st = get_scene(ctx, scene, s);
  if (st != IPT_OK) return st;
  if (!(*s)->cache) return fail(ctx, IPT_ERR_INVALID_ARG, "scene has no cache (ipt_cache_configure)");
  return IPT_OK;
}

// Record buffers for `cap` records.
ipt_status cache_record_buffers(ipt_ctx* ctx, CacheState* c, uint32_t cap) {
  if (c->buf.r_cap == cap) return IPT_OK;
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  void* ptrs[4] = {c->buf.r.x, c->buf.r.d, c->buf.r.n, c->buf.r.u};
  for (void* q : ptrs) {
    if (!q) continue;
    cudaFree(q);
    c->owned.erase(std::remove(c->owned.begin(), c->owned.end(), q), c->owned.end());
  }
  c->buf.r_cap = 0;
  cudaError_t e = cudaSuccess;
  float4** arr[4] = {&c->buf.r.x, &c->buf.r.d, &c->buf.r.n, &c->buf.r.u};
  for (float4** p : arr) {
    void* q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, (size_t)cap * sizeof(float4));
    if (e == cudaSuccess) {
      c->owned.push_back(q);
      *p = static_cast<float4*>(q);
    }
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cache record buffers");
  c->buf.r_cap = cap;
  return IPT_OK;
}

// Network, Adam state and counters of a new cache, initialised from seed.
ipt_status cache_create(ipt_ctx* ctx, DeviceScene* s, const ipt_cache_opts* o) {
  CacheState* c = new (std::nothrow) CacheState();
  if (!c) return IPT_ERR_OUT_OF_MEMORY;
  ipt::cache_grid(c->res, &c->dense);
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t n) {
    void* q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, n * sizeof(**p));
    if (e == cudaSuccess) {
      c->owned.push_back(q);
      *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    }
  };
  const size_t nw = ipt::kCacheWeights, nt = ipt::kCacheTableFloats;
  A(&c->w, nw);
  A(&c->mw, nw);
  A(&c->vw, nw);
  A(&c->gw, nw);
  A(&c->wt, ipt::kCacheWtElems / 8);
  A(&c->table, nt);
  A(&c->mt, nt);
  A(&c->vt, nt);
  A(&c->gt, nt);
  A(&c->loss_dev, 64);
  A(&c->buf.counts, 4);
  if (e == cudaSuccess) e = cudaMallocHost(&c->host, 128 * sizeof(double));
  std::vector<float> w(nw), t(nt);
  SplitMix rng{o->init_seed};
  const uint32_t fan_in[5] = {80, 64, 64, 64, 64};
  const uint32_t off[6] = {0, 5120, 9216, 13312, 17408, 18432};
  for (int L = 0; L < 5; ++L) {
    const double a = std::sqrt(6.0 / fan_in[L]);
    for (uint32_t i = off[L]; i < off[L + 1]; ++i) w[i] = (float)((2.0 * rng.uniform() - 1.0) * a);
  }
  for (size_t i = 0; i < nt; ++i) t[i] = (float)((2.0 * rng.uniform() - 1.0) * 1e-4);
  if (e == cudaSuccess) e = cudaMemcpy(c->w, w.data(), nw * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->table, t.data(), nt * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->mw, 0, nw * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->vw, 0, nw * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->gw, 0, nw * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->mt, 0, nt * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->vt, 0, nt * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->gt, 0, nt * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->wt, 0, ipt::kCacheWtElems * 2);
  if (e == cudaSuccess) e = cudaMemset(c->buf.counts, 0, 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = ipt::cache_pack_weights(c->w, c->wt, ctx->stream);
  if (e != cudaSuccess) {
    free_cache(c);
    return cuda_fail(ctx, e, "cache allocation");
  }
  s->cache = c;
  return IPT_OK;
}

// Evaluation rows for n inputs.
ipt_status cache_api_rows(ipt_ctx* ctx, CacheState* c, uint32_t n) {
  if (c->api_cap >= n) return IPT_OK;
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  for (void* p : c->api_owned) cudaFree(p);
  c->api_owned.clear();
  c->api_cap = 0;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t k) {
    void* q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, k * sizeof(**p));
    if (e == cudaSuccess) {
      c->api_owned.push_back(q);
      *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    }
  };
  A(&c->api.x, n);
  A(&c->api.d, n);
  A(&c->api.n, n);
  A(&c->api.u, n);
  A(&c->api_ma, n);
  A(&c->api_mb, n);
  A(&c->api_c, n);
  A(&c->api_dp, 8 * (size_t)n);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cache evaluation rows");
  c->api_cap = n;
  return IPT_OK;
}

}  // namespace

extern "C" {

ipt_status ipt_cache_configure(ipt_ctx* ctx, int32_t scene, const ipt_cache_opts* opts) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = check_cache_opts(ctx, opts)) != IPT_OK) return st;
  IPT_CK(cudaSetDevice(ctx->device));
  if (!s->cache && (st = cache_create(ctx, s, opts)) != IPT_OK) return st;
  CacheState* c = s->cache;
  if ((st = cache_record_buffers(ctx, c, opts->record_capacity)) != IPT_OK) return st;
  if ((st = cache_query_buffers(ctx, c)) != IPT_OK) return st;
  c->opts = *opts;
  c->active = opts->enabled != 0;
  c->fell_back = false;
  return IPT_OK;
}

ipt_status ipt_cache_weights_set(ipt_ctx* ctx, int32_t scene, const float* weights, const float* table) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  CacheState* c = s->cache;
  IPT_CK(cudaSetDevice(ctx->device));
  const size_t nw = ipt::kCacheWeights, nt = ipt::kCacheTableFloats;
  if (weights) {
    IPT_CK(cudaMemcpyAsync(c->w, weights, nw * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    IPT_CK(ipt::cache_pack_weights(c->w, c->wt, ctx->stream));
  }
  if (table) IPT_CK(cudaMemcpyAsync(c->table, table, nt * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  IPT_CK(cudaMemsetAsync(c->mw, 0, nw * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(c->vw, 0, nw * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(c->mt, 0, nt * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(c->vt, 0, nt * sizeof(float), ctx->stream));
  c->steps_done = 0;
  return ipt_synchronize(ctx);
}

ipt_status ipt_cache_weights_get(ipt_ctx* ctx, int32_t scene, float* weights, float* table) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  CacheState* c = s->cache;
  IPT_CK(cudaSetDevice(ctx->device));
  if (weights)
    IPT_CK(cudaMemcpyAsync(weights, c->w, ipt::kCacheWeights * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (table)
    IPT_CK(cudaMemcpyAsync(table, c->table, ipt::kCacheTableFloats * sizeof(float), cudaMemcpyDeviceToHost,
                           ctx->stream));
  return ipt_synchronize(ctx);
}

ipt_status ipt_cache_eval(ipt_ctx* ctx, int32_t scene, uint32_t n, const float* x01, const float* dir,
                          const float* nrm, const float* params7, const float* upstream, float* rgb_out,
                          float* dparams_out) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (n == 0) return IPT_OK;
  if (!x01 || !dir || !nrm || !params7 || !rgb_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null input or output");
  CacheState* c = s->cache;
  IPT_CK(cudaSetDevice(ctx->device));
  if ((st = cache_api_rows(ctx, c, n)) != IPT_OK) return st;
  IPT_CK(ipt::cache_pack_rows(n, x01, dir, nrm, params7, upstream, c->api, c->api_ma, c->api_mb, ctx->stream));
  const bool vjp = upstream && dparams_out;
  ipt::CacheOut o{};
  o.c = c->api_c;
  o.dp = vjp ? c->api_dp : nullptr;
  {
    Timed tm(ctx, vjp ? IPT_KERNEL_CACHE_VJP : IPT_KERNEL_CACHE_INFER);
    IPT_CK(ipt::cache_infer(cache_net(s, true), c->api, c->api_ma, c->api_mb, nullptr, n, o, vjp, ctx->L.num_sms,
                            ctx->stream));
  }
  IPT_CK(ipt::cache_unpack_out(n, c->api_c, c->api_dp, rgb_out, vjp ? dparams_out : nullptr, ctx->stream));
  return IPT_OK;
}

ipt_status ipt_cache_grad(ipt_ctx* ctx, int32_t scene, uint32_t n, const float* x01, const float* dir,
                          const float* nrm, const float* params7, const float* target, double* loss_out,
                          float* grad_weights, float* grad_table) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (n == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "no rows");
  if (!x01 || !dir || !nrm || !params7 || !target) return fail(ctx, IPT_ERR_INVALID_ARG, "null input");
  CacheState* c = s->cache;
  IPT_CK(cudaSetDevice(ctx->device));
  if ((st = cache_api_rows(ctx, c, n)) != IPT_OK) return st;
  IPT_CK(ipt::cache_pack_rows(n, x01, dir, nrm, params7, target, c->api, c->api_ma, c->api_mb, ctx->stream));
  const size_t nw = ipt::kCacheWeights, nt = ipt::kCacheTableFloats;
  IPT_CK(cudaMemsetAsync(c->gw, 0, nw * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(c->gt, 0, nt * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(c->loss_dev, 0, sizeof(double), ctx->stream));
  ipt::CacheOut o{};
  o.gw = c->gw;
  o.gt = reinterpret_cast<float2*>(c->gt);
  o.loss = c->loss_dev;
  o.err = ctx->err_dev;
  {
    Timed tm(ctx, IPT_KERNEL_CACHE_GRAD);
    IPT_CK(ipt::cache_grad(cache_net(s, true), c->api, c->api_ma, c->api_mb, nullptr, n, 0, 1, o, ctx->L.num_sms,
                           ctx->stream));
  }
  if (grad_weights)
    IPT_CK(cudaMemcpyAsync(grad_weights, c->gw, nw * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  if (grad_table)
    IPT_CK(cudaMemcpyAsync(grad_table, c->gt, nt * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  IPT_CK(cudaMemsetAsync(c->gw, 0, nw * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(c->gt, 0, nt * sizeof(float), ctx->stream));
  if (loss_out) {
    IPT_CK(cudaMemcpyAsync(c->host, c->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if ((st = ipt_synchronize(ctx)) != IPT_OK) return st;
    *loss_out = c->host[0] / (3.0 * (double)n);
  }
  return IPT_OK;
}

ipt_status ipt_cache_train(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint64_t iteration) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, false)) != IPT_OK) return st;
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "no views set");
  IPT_CK(cudaSetDevice(ctx->device));
  if ((st = ensure_tables(ctx, s, s->params, nullptr)) != IPT_OK) return st;
  return cache_train_pass(ctx, scene, s, opts, iteration);
}

ipt_status ipt_cache_records(ipt_ctx* ctx, int32_t scene, uint32_t* n_out, float* records) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!n_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null n_out");
  CacheState* c = s->cache;
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaMemcpyAsync(c->host, c->buf.counts, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  if ((st = ipt_synchronize(ctx)) != IPT_OK) return st;
  const uint32_t n = std::min(reinterpret_cast<const uint32_t*>(c->host)[1], c->buf.r_cap);
  *n_out = n;
  if (!records || n == 0) return IPT_OK;
  std::vector<float4> x(n), d(n), nr(n), u(n);
  IPT_CK(cudaMemcpy(x.data(), c->buf.r.x, n * sizeof(float4), cudaMemcpyDeviceToHost));
  IPT_CK(cudaMemcpy(d.data(), c->buf.r.d, n * sizeof(float4), cudaMemcpyDeviceToHost));
  IPT_CK(cudaMemcpy(nr.data(), c->buf.r.n, n * sizeof(float4), cudaMemcpyDeviceToHost));
  IPT_CK(cudaMemcpy(u.data(), c->buf.r.u, n * sizeof(float4), cudaMemcpyDeviceToHost));
  for (uint32_t i = 0; i < n; ++i) {
    float* r = records + 16 * (size_t)i;
    uint32_t pid;
    int32_t seg;
    std::memcpy(&pid, &nr[i].w, 4);
    std::memcpy(&seg, &x[i].w, 4);
    r[0] = (float)pid;
    r[1] = (float)seg;
    const float v[12] = {x[i].x, x[i].y, x[i].z, d[i].x, d[i].y, d[i].z, nr[i].x, nr[i].y, nr[i].z, u[i].x, u[i].y,
                         u[i].z};
    for (int k = 0; k < 12; ++k) r[2 + k] = v[k];
    r[14] = r[15] = 0.0f;
  }
  return IPT_OK;
}

ipt_status ipt_cache_status(ipt_ctx* ctx, int32_t scene, ipt_cache_stats* out) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!out) return fail(ctx, IPT_ERR_INVALID_ARG, "null output");
  CacheState* c = s->cache;
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaMemcpyAsync(c->host, c->loss_dev, 64 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  IPT_CK(cudaMemcpyAsync(c->host + 64, c->buf.counts, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  if ((st = ipt_synchronize(ctx)) != IPT_OK) return st;
  std::memset(out, 0, sizeof(*out));
  out->active = c->active ? 1 : 0;
  out->fell_back = c->fell_back ? 1 : 0;
  out->records = reinterpret_cast<const uint32_t*>(c->host + 64)[1];
  out->train_steps = c->steps_done;
  const uint32_t kept = std::min(out->records, c->buf.r_cap);
  double sum = 0.0;
  for (uint32_t i = 0; i < c->last_pass_steps; ++i) sum += c->host[i];
  out->last_loss = kept ? sum / (3.0 * (double)kept) : 0.0;
  out->image_bias = c->image_bias;
  out->grad_bias = c->grad_bias;
  for (int a = 0; a < 3; ++a) {
    out->lo[a] = s->bb_lo[a];
    out->hi[a] = s->bb_hi[a];
  }
  for (int l = 0; l < ipt::kCacheLevels; ++l) out->res[l] = c->res[l];
  return IPT_OK;
}

ipt_status ipt_cache_bias(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint32_t spp,
                          uint64_t iteration, double* image_bias, double* grad_bias) {
  DeviceScene* s;
  ipt_status st = get_cache(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, true)) != IPT_OK) return st;
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "no views set");
  if (spp == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp must be positive");
  CacheState* c = s->cache;
  IPT_CK(cudaSetDevice(ctx->device));
  const size_t npx = 3 * (size_t)s->n_pix, np = 10u * (size_t)s->n_seg;
  float *img = nullptr, *grad = nullptr;
  IPT_CK(cudaMalloc(&img, 2 * npx * sizeof(float)));
  if (cudaMalloc(&grad, 2 * np * sizeof(float)) != cudaSuccess) {
    cudaFree(img);
    return fail(ctx, IPT_ERR_OUT_OF_MEMORY, "bias buffers");
  }
  const bool was = c->active;
  const bool with_grad = s->target != nullptr;
  ipt_trace_opts go = *opts;  // gradients at the monitor's sample count too
  go.spp_r = spp;
  go.spp_d = spp;
  for (int k = 0; k < 2 && st == IPT_OK; ++k) {
    c->active = k == 1;
    st = ipt_render(ctx, scene, -1, opts, IPT_SET_RESIDUAL, spp, iteration, nullptr, nullptr, img + k * npx, nullptr);
    if (st == IPT_OK && with_grad)
      st = loss_grad_async(ctx, scene, s, &go, iteration, grad + k * np, 0, s->n_pix, s->n_pix);
  }
  c->active = was;
  std::vector<float> hi(2 * npx), hg(2 * np);
  if (st == IPT_OK && cudaMemcpy(hi.data(), img, 2 * npx * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = fail(ctx, IPT_ERR_CUDA, "bias image copy");
  if (st == IPT_OK && with_grad &&
      cudaMemcpy(hg.data(), grad, 2 * np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = fail(ctx, IPT_ERR_CUDA, "bias gradient copy");
  cudaFree(img);
  cudaFree(grad);
  if (st != IPT_OK) return st;
  if ((st = ipt_synchronize(ctx)) != IPT_OK) return st;
  auto rel = [](const float* a, const float* b, size_t n) {
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < n; ++i) {
      const double d = (double)b[i] - (double)a[i];
      num += d * d;
      den += (double)a[i] * (double)a[i];
    }
    return den > 0.0 ? std::sqrt(num / den) : 0.0;
  };
  c->image_bias = rel(hi.data(), hi.data() + npx, npx);
  c->grad_bias = with_grad ? rel(hg.data(), hg.data() + np, np) : -1.0;
  if (image_bias) *image_bias = c->image_bias;
  if (grad_bias) *grad_bias = c->grad_bias;
  const double thr = c->opts.bias_threshold;
  if (thr > 0.0 && c->active && (c->image_bias > thr || c->grad_bias > thr)) {
    c->active = false;
    c->fell_back = true;
  }
  return IPT_OK;
}


}  // extern "C"

// --- checkpoints --------------------------------------------------------------

namespace {

struct CkptHeader {           // 64 bytes
  char magic[8];              // "IPTCKPT1"
  uint32_t version;           // 1
  uint32_t n_seg;
  uint64_t iteration;
  int32_t adam_step;
  uint32_t has_cache;
  uint64_t cache_steps;
  uint32_t cache_active;
  uint32_t cache_fell_back;
  uint32_t has_disney;        // Disney-model parameters and optimiser state follow
  int32_t disney_step;
  uint64_t disney_iteration;
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header layout");

constexpr uint32_t kCkptVersion = 1;

// Byte layout after the header: params, adam_m, adam_v (10 S floats each),
// free mask (10 S bytes, padded to 8); with a cache: weights, their Adam m
// and v (kCacheWeights floats each), table, its Adam m and v
// (kCacheTableFloats floats each); with Disney-model state: its params,
// adam_m, adam_v (16 S floats each) and free mask (16 S bytes, padded to 8).
size_t ckpt_bytes(uint32_t n_seg, bool cache, bool disney) {
  const size_t np = 10 * (size_t)n_seg, nd = 16 * (size_t)n_seg;
  size_t n = sizeof(CkptHeader) + 3 * np * sizeof(float) + ((np + 7) & ~(size_t)7);
  if (cache) n += 3 * (size_t)ipt::kCacheWeights * sizeof(float) + 3 * (size_t)ipt::kCacheTableFloats * sizeof(float);
  if (disney) n += 3 * nd * sizeof(float) + ((nd + 7) & ~(size_t)7);
  return n;
}

}  // namespace

extern "C" {

ipt_status ipt_checkpoint_save(ipt_ctx* ctx, int32_t scene, void* buf, size_t* n) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!n) return fail(ctx, IPT_ERR_INVALID_ARG, "null size");
  const bool cache = s->cache != nullptr;
  const bool disney = s->disney != nullptr;
  const size_t need = ckpt_bytes(s->n_seg, cache, disney);
  if (!buf) {
    *n = need;
    return IPT_OK;
  }
  if (*n < need) return fail(ctx, IPT_ERR_INVALID_ARG, "checkpoint buffer of " + std::to_string(*n) +
                                                           " bytes, need " + std::to_string(need));
  IPT_CK(cudaSetDevice(ctx->device));
  CkptHeader h{};
  std::memcpy(h.magic, "IPTCKPT1", 8);
  h.version = kCkptVersion;
  h.n_seg = s->n_seg;
  h.iteration = s->iteration;
  IPT_CK(cudaMemcpyAsync(&h.adam_step, s->step_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  h.has_cache = cache ? 1u : 0u;
  if (cache) {
    h.cache_steps = s->cache->steps_done;
    h.cache_active = s->cache->active ? 1u : 0u;
    h.cache_fell_back = s->cache->fell_back ? 1u : 0u;
  }
  h.has_disney = disney ? 1u : 0u;
  if (disney) {
    IPT_CK(cudaMemcpyAsync(&h.disney_step, s->disney->step_dev, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           ctx->stream));
    h.disney_iteration = s->disney->iteration;
  }
  const size_t np = 10 * (size_t)s->n_seg;
  char* p = static_cast<char*>(buf) + sizeof(CkptHeader);
  auto D2H = [&](const void* src, size_t bytes) -> cudaError_t {
    const cudaError_t e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    p += bytes;
    return e;
  };
  IPT_CK(D2H(s->params, np * sizeof(float)));
  IPT_CK(D2H(s->adam_m, np * sizeof(float)));
  IPT_CK(D2H(s->adam_v, np * sizeof(float)));
  IPT_CK(D2H(s->free_mask, np));
  p += ((np + 7) & ~(size_t)7) - np;
  if (cache) {
    const CacheState* c = s->cache;
    const size_t nw = ipt::kCacheWeights * sizeof(float), nt = ipt::kCacheTableFloats * sizeof(float);
    IPT_CK(D2H(c->w, nw));
    IPT_CK(D2H(c->mw, nw));
    IPT_CK(D2H(c->vw, nw));
    IPT_CK(D2H(c->table, nt));
    IPT_CK(D2H(c->mt, nt));
    IPT_CK(D2H(c->vt, nt));
  }
  if (disney) {
    const DisneyState* d = s->disney;
    const size_t nd = 16 * (size_t)s->n_seg;
    IPT_CK(D2H(d->params, nd * sizeof(float)));
    IPT_CK(D2H(d->adam_m, nd * sizeof(float)));
    IPT_CK(D2H(d->adam_v, nd * sizeof(float)));
    IPT_CK(D2H(d->free_mask, nd));
  }
  IPT_CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(buf, &h, sizeof(h));
  *n = need;
  return IPT_OK;
}

ipt_status ipt_checkpoint_load(ipt_ctx* ctx, int32_t scene, const void* buf, size_t n) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!buf || n < sizeof(CkptHeader)) return fail(ctx, IPT_ERR_INVALID_ARG, "checkpoint shorter than its header");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, "IPTCKPT1", 8) != 0) return fail(ctx, IPT_ERR_INVALID_ARG, "not a checkpoint");
  if (h.version != kCkptVersion)
    return fail(ctx, IPT_ERR_INVALID_ARG, "checkpoint version " + std::to_string(h.version));
  if (h.n_seg != s->n_seg)
    return fail(ctx, IPT_ERR_INVALID_ARG, "checkpoint of " + std::to_string(h.n_seg) + " segments, scene has " +
                                              std::to_string(s->n_seg));
  if (h.has_cache > 1 || (h.has_cache && !s->cache))
    return fail(ctx, IPT_ERR_INVALID_ARG, "checkpoint carries cache state: configure the scene's cache first");
  if (h.has_disney > 1) return fail(ctx, IPT_ERR_INVALID_ARG, "bad Disney flag");
  const size_t expect = ckpt_bytes(h.n_seg, h.has_cache != 0, h.has_disney != 0);
  if (n != expect)
    return fail(ctx, IPT_ERR_INVALID_ARG, "checkpoint of " + std::to_string(n) + " bytes, expected " +
                                              std::to_string(expect));
  const size_t np = 10 * (size_t)s->n_seg;
  const float* pf = reinterpret_cast<const float*>(static_cast<const char*>(buf) + sizeof(CkptHeader));
  for (size_t i = 0; i < np; ++i)
    if (!std::isfinite(pf[i])) return fail(ctx, IPT_ERR_NONFINITE, "non-finite parameter " + std::to_string(i));
  IPT_CK(cudaSetDevice(ctx->device));
  const char* p = static_cast<const char*>(buf) + sizeof(CkptHeader);
  auto H2D = [&](void* dst, size_t bytes) -> cudaError_t {
    const cudaError_t e = cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, ctx->stream);
    p += bytes;
    return e;
  };
  IPT_CK(H2D(s->params, np * sizeof(float)));
  IPT_CK(H2D(s->adam_m, np * sizeof(float)));
  IPT_CK(H2D(s->adam_v, np * sizeof(float)));
  IPT_CK(H2D(s->free_mask, np));
  p += ((np + 7) & ~(size_t)7) - np;
  IPT_CK(cudaMemcpyAsync(s->step_dev, &h.adam_step, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  if (h.has_cache) {
    CacheState* c = s->cache;
    const size_t nw = ipt::kCacheWeights * sizeof(float), nt = ipt::kCacheTableFloats * sizeof(float);
    IPT_CK(H2D(c->w, nw));
    IPT_CK(H2D(c->mw, nw));
    IPT_CK(H2D(c->vw, nw));
    IPT_CK(H2D(c->table, nt));
    IPT_CK(H2D(c->mt, nt));
    IPT_CK(H2D(c->vt, nt));
    IPT_CK(ipt::cache_pack_weights(c->w, c->wt, ctx->stream));
    c->steps_done = h.cache_steps;
    c->active = h.cache_active != 0;
    c->fell_back = h.cache_fell_back != 0;
  }
  if (h.has_disney) {
    DisneyState* d;
    if ((st = disney_state(ctx, s, &d)) != IPT_OK) return st;
    const size_t nd = 16 * (size_t)s->n_seg;
    IPT_CK(H2D(d->params, nd * sizeof(float)));
    IPT_CK(H2D(d->adam_m, nd * sizeof(float)));
    IPT_CK(H2D(d->adam_v, nd * sizeof(float)));
    IPT_CK(H2D(d->free_mask, nd));
    IPT_CK(cudaMemcpyAsync(d->step_dev, &h.disney_step, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    d->iteration = h.disney_iteration;
    d->tab_is_ctx = false;
  }
  IPT_CK(cudaStreamSynchronize(ctx->stream));  // the caller may release buf on return
  s->iteration = h.iteration;
  s->tab_is_ctx = false;  // tables are rebuilt from the loaded parameters
  s->params_set = true;
  return IPT_OK;
}

}  // extern "C"

// --- Disney material model (megakernel integrator) -------------------------

namespace {

constexpr uint32_t kDisneyValues = 16;

ipt_status disney_state(ipt_ctx* ctx, DeviceScene* s, DisneyState** out) {
  if (s->disney) {
    *out = s->disney;
    return IPT_OK;
  }
  DisneyState* d = new (std::nothrow) DisneyState();
  if (!d) return IPT_ERR_OUT_OF_MEMORY;
  const size_t S = s->n_seg, np = kDisneyValues * S;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t count) {
    if (e != cudaSuccess) return;
    void* q = nullptr;
    e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(**p));
    if (e == cudaSuccess) {
      d->owned.push_back(q);
      *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    }
  };
  A(&d->params, np);
  A(&d->adam_m, np);
  A(&d->adam_v, np);
  A(&d->free_mask, np);
  A(&d->step_dev, 1);
  A(&d->grad_acc, np);
  if (S > ipt::disney_max_shared_segments()) A(&d->gacc, np);
  A(&d->tab.emis, S);
  A(&d->tab.samp, S);
  A(&d->tab.cdf, S);
  A(&d->tab.lum, S);
  A(&d->tab.W, 1);
  A(&d->dt.mat, 4 * S);
  A(&d->dt.lobe, S);
  A(&d->dt.samp, 2 * S);
  if (e != cudaSuccess) {
    free_disney(d);
    return cuda_fail(ctx, e, "Disney state");
  }
  s->disney = d;
  *out = d;
  return IPT_OK;
}

ipt_status get_disney(ipt_ctx* ctx, int32_t scene, DeviceScene** s, DisneyState** d) {
  ipt_status st = get_scene(ctx, scene, s);
  if (st != IPT_OK) return st;
  if (!(*s)->disney) return fail(ctx, IPT_ERR_INVALID_ARG, "no Disney parameters set (ipt_disney_params_set)");
  *d = (*s)->disney;
  return IPT_OK;
}

// Scene-table entry of a Disney-model launch over scene pixels [begin, begin + n).
ipt::WfScene disney_entry(const ipt_ctx* ctx, int32_t scene, const DeviceScene* s, const DisneyState* d,
                          uint32_t begin, uint32_t n) {
  ipt::WfScene e = wf_entry(ctx, scene, s, begin, n);
  e.t = ipt::seg_dev(d->tab);
  e.dis = ipt::DisneyDev{d->dt.mat, d->dt.lobe, d->dt.samp};
  e.n_all = (uint32_t)s->n_pix;
  return e;
}

ipt_status disney_tables(ipt_ctx* ctx, DeviceScene* s, DisneyState* d, const float* sparams) {
  if (!sparams && d->tab_is_ctx) return IPT_OK;
  Timed tm(ctx, IPT_KERNEL_PREPARE);
  IPT_CK(ipt::launch_disney_tables(buffers(ctx, s), d->tab, d->dt, d->params, sparams, ctx->stream));
  d->tab_is_ctx = sparams == nullptr;
  return IPT_OK;
}

}  // namespace

extern "C" {

ipt_status ipt_disney_params_set(ipt_ctx* ctx, int32_t scene, const float* params, const uint8_t* free_mask) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if (!params) return fail(ctx, IPT_ERR_INVALID_ARG, "null params");
  const size_t n = kDisneyValues * (size_t)s->n_seg;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(params[i])) return fail(ctx, IPT_ERR_NONFINITE, "non-finite parameter " + std::to_string(i));
  IPT_CK(cudaSetDevice(ctx->device));
  DisneyState* d;
  if ((st = disney_state(ctx, s, &d)) != IPT_OK) return st;
  IPT_CK(cudaMemcpyAsync(d->params, params, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  IPT_CK(cudaMemsetAsync(d->adam_m, 0, n * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(d->adam_v, 0, n * sizeof(float), ctx->stream));
  IPT_CK(cudaMemsetAsync(d->step_dev, 0, sizeof(int), ctx->stream));
  if (free_mask) {
    IPT_CK(cudaMemcpyAsync(d->free_mask, free_mask, n, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    IPT_CK(cudaMemsetAsync(d->free_mask, 1, n, ctx->stream));
  }
  IPT_CK(cudaStreamSynchronize(ctx->stream));  // host buffers may be released on return
  d->tab_is_ctx = false;
  d->iteration = 0;
  return IPT_OK;
}

ipt_status ipt_disney_params_get(ipt_ctx* ctx, int32_t scene, float* params_out) {
  DeviceScene* s;
  DisneyState* d;
  ipt_status st = get_disney(ctx, scene, &s, &d);
  if (st != IPT_OK) return st;
  if (!params_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null output");
  IPT_CK(cudaSetDevice(ctx->device));
  IPT_CK(cudaMemcpyAsync(params_out, d->params, kDisneyValues * sizeof(float) * s->n_seg, cudaMemcpyDeviceToHost,
                         ctx->stream));
  return ipt_synchronize(ctx);
}

ipt_status ipt_disney_render(ipt_ctx* ctx, int32_t scene, int32_t view, const ipt_trace_opts* opts, uint32_t set,
                             uint32_t spp, uint64_t iteration, const float* sampling_params, float* rgb_out,
                             float* msq_out) {
  DeviceScene* s;
  DisneyState* d;
  ipt_status st = get_disney(ctx, scene, &s, &d);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, false)) != IPT_OK) return st;
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "no views set");
  if (view < -1 || view >= (int32_t)s->views.size()) return fail(ctx, IPT_ERR_INVALID_ARG, "view out of range");
  if (spp == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp must be positive");
  if (!rgb_out && !msq_out) return fail(ctx, IPT_ERR_INVALID_ARG, "no output");
  IPT_CK(cudaSetDevice(ctx->device));
  if ((st = disney_tables(ctx, s, d, sampling_params)) != IPT_OK) return st;
  const uint32_t begin = view < 0 ? 0u : s->views[view].offset;
  const uint32_t n = view < 0 ? (uint32_t)s->n_pix : s->views[view].w * s->views[view].h;
  const ipt::TraceParams tp = trace_params(ctx, scene, opts, set, spp, iteration);
  if (use_wavefront(ctx, spp)) {
    if ((st = ensure_wf(ctx, false, kDisneyValues * s->n_seg)) != IPT_OK) return st;
    ipt::WfScene e = disney_entry(ctx, scene, s, d, begin, n);
    e.img = rgb_out;
    e.msq = msq_out;
    if ((st = upload_entry(ctx, e)) != IPT_OK) return st;
    StageTimer timer{ctx};
    const ipt::WfHook hook{stage_begin, stage_end, &timer};
    IPT_CK(ipt::wf_forward(ctx->L, ctx->wf_tab, std::vector<ipt::WfScene>{e}, tp, 0, nullptr, ctx->wf, nullptr,
                           ctx->err_dev, ctx->stream, (ctx->flags & IPT_FLAG_KERNEL_TIMING) ? &hook : nullptr,
                           nullptr, true));
    return IPT_OK;
  }
  Timed tm(ctx, IPT_KERNEL_FORWARD);
  IPT_CK(ipt::launch_disney_forward(ctx->L, buffers(ctx, s), d->tab, d->dt, s->views_dev,
                                    (uint32_t)s->views.size(), begin, n, tp, rgb_out, msq_out, nullptr, nullptr,
                                    nullptr, 0.f, 0, ctx->err_dev, ctx->stream));
  return IPT_OK;
}

// Forward + residual + adjoint of the Disney parameters, all pixels or a
// stochastic pixel batch; grad_out (device, S x 16) nullable.
static ipt_status disney_loss_grad_async(ipt_ctx* ctx, int32_t scene, DeviceScene* s, DisneyState* d,
                                         const ipt_trace_opts* opts, uint64_t iteration, float* grad_out) {
  ipt_status st;
  if ((st = check_opts(ctx, opts, true, true)) != IPT_OK) return st;
  if (s->views.empty() || !s->target) return fail(ctx, IPT_ERR_INVALID_ARG, "loss needs views and targets");
  if (opts->spp_r == 0 || opts->spp_d == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp_r and spp_d must be positive");
  IPT_CK(cudaSetDevice(ctx->device));
  if ((st = disney_tables(ctx, s, d, nullptr)) != IPT_OK) return st;
  const uint32_t B = opts->pixel_batch;
  if (B && ((st = ensure_pick(ctx, s, B)) != IPT_OK || (st = draw_picks(ctx, scene, s, B, iteration, s->pick)) != IPT_OK))
    return st;
  const uint32_t n = B ? B : (uint32_t)s->n_pix;
  float* g_buf = B ? s->g_pick : s->g_img;
  const uint32_t* pick = B ? s->pick : nullptr;
  const float g_scale = (float)(1.0 / (3.0 * (double)n));
  const ipt::SceneBuffers sb = buffers(ctx, s);
  const uint32_t np = kDisneyValues * s->n_seg;
  ipt::TraceParams tpr = trace_params(ctx, scene, opts, IPT_SET_RESIDUAL, opts->spp_r, iteration);
  const uint32_t set = opts->gradcheck_same_set ? IPT_SET_RESIDUAL : IPT_SET_DERIVATIVE;
  ipt::TraceParams tpd = trace_params(ctx, scene, opts, set, opts->spp_d, iteration);
  if (opts->gradcheck_same_set) tpd.sample_stride = opts->spp_r;
  if (use_wavefront(ctx, std::max(opts->spp_r, opts->spp_d))) {
    StageTimer timer{ctx};
    const ipt::WfHook hook{stage_begin, stage_end, &timer};
    const ipt::WfHook* hp = (ctx->flags & IPT_FLAG_KERNEL_TIMING) ? &hook : nullptr;
    if ((st = ensure_wf(ctx, true, np, true)) != IPT_OK) return st;
    ipt::WfScene e = disney_entry(ctx, scene, s, d, 0u, n);
    e.pick = const_cast<uint32_t*>(pick);
    e.g_scale = g_scale;
    e.target = s->target;
    e.g_img = g_buf;
    if ((st = upload_entry(ctx, e)) != IPT_OK) return st;
    IPT_CK(ipt::wf_forward(ctx->L, ctx->wf_tab, std::vector<ipt::WfScene>{e}, tpr, opts->loss, nullptr, ctx->wf,
                           s->loss_partials, ctx->err_dev, ctx->stream, hp, nullptr, true));
    IPT_CK(cudaMemsetAsync(d->grad_acc, 0, np * sizeof(double), ctx->stream));
    IPT_CK(ipt::wf_adjoint(ctx->L, ctx->wf_tab, std::vector<ipt::WfScene>{e}, tpd, nullptr, ctx->wf, d->grad_acc,
                           ctx->err_dev, ctx->stream, hp, nullptr, true));
  } else {
    tpr.pick = pick;
    tpd.pick = pick;
    {
      Timed tm(ctx, IPT_KERNEL_FORWARD);
      IPT_CK(ipt::launch_disney_forward(ctx->L, sb, d->tab, d->dt, s->views_dev, (uint32_t)s->views.size(), 0, n,
                                        tpr, nullptr, nullptr, s->target, g_buf, s->loss_partials, g_scale,
                                        opts->loss, ctx->err_dev, ctx->stream));
    }
    IPT_CK(cudaMemsetAsync(d->grad_acc, 0, np * sizeof(double), ctx->stream));
    {
      Timed tm(ctx, IPT_KERNEL_ADJOINT);
      IPT_CK(ipt::launch_disney_adjoint(ctx->L, sb, d->tab, d->dt, s->views_dev, (uint32_t)s->views.size(), 0, n,
                                        tpd, g_buf, d->grad_acc, d->gacc, ctx->err_dev, ctx->stream));
    }
  }
  Timed tm(ctx, IPT_KERNEL_FINALIZE);
  IPT_CK(ipt::launch_finalize(s->loss_partials, ipt::loss_partials_capacity(ctx->L), s->loss_dev, d->grad_acc,
                              grad_out, np, ctx->stream));
  return IPT_OK;
}


ipt_status ipt_disney_loss_grad(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint64_t iteration,
                                double* loss_out, float* grad_out) {
  DeviceScene* s;
  DisneyState* d;
  ipt_status st = get_disney(ctx, scene, &s, &d);
  if (st != IPT_OK) return st;
  if ((st = disney_loss_grad_async(ctx, scene, s, d, opts, iteration, grad_out)) != IPT_OK) return st;
  if (loss_out) return read_loss(ctx, s, loss_out, opts->pixel_batch ? opts->pixel_batch : s->n_pix);
  return IPT_OK;
}

ipt_status ipt_disney_step(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, const ipt_adam_opts* adam,
                           double* loss_out) {
  DeviceScene* s;
  DisneyState* d;
  ipt_status st = get_disney(ctx, scene, &s, &d);
  if (st != IPT_OK) return st;
  if (!adam) return fail(ctx, IPT_ERR_INVALID_ARG, "null adam options");
  if (!(adam->lr >= 0.0f) || !(adam->beta1 >= 0.0f && adam->beta1 < 1.0f) ||
      !(adam->beta2 >= 0.0f && adam->beta2 < 1.0f) || !(adam->eps > 0.0f) || !(adam->l1_emission >= 0.0f))
    return fail(ctx, IPT_ERR_INVALID_ARG, "invalid adam options");
  if ((st = disney_loss_grad_async(ctx, scene, s, d, opts, d->iteration, nullptr)) != IPT_OK) return st;
  {
    Timed tm(ctx, IPT_KERNEL_ADAM);
    IPT_CK(ipt::launch_disney_adam(buffers(ctx, s), d->tab, d->dt, d->params, d->adam_m, d->adam_v, d->free_mask,
                                   d->grad_acc, nullptr, d->step_dev, adam_host(adam), s->loss_dev, ctx->err_dev,
                                   ctx->stream));
  }
  d->tab_is_ctx = true;  // the Adam kernel rebuilt the tables from the new parameters
  d->iteration++;
  if (loss_out) return read_loss(ctx, s, loss_out, opts->pixel_batch ? opts->pixel_batch : s->n_pix);
  return IPT_OK;
}

}  // extern "C"
