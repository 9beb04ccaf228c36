// C ABI: batches of scenes optimised together, one launch per stage over
// all members and one CUDA graph per iteration (include/ipt.h, ipt_batch_*).
#include "ipt_capi_internal.h"

using namespace ipt_capi;

extern "C" {

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
  for (int32_t id : b->members) ctx->scenes[id]->tab_batch = *batch_id;
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
  if (!b->exec || !same_opts(*opts, b->g_opts) || !same_adam(*adam, b->g_adam) || !same_cfg(ctx->cfg, b->g_cfg) ||
      b->g_alloc_gen != ctx->alloc_gen) {
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
    if ((st = ensure_wf(ctx, true, 10u * max_seg, false, opts->max_depth)) != IPT_OK) return st;
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
    b->g_alloc_gen = ctx->alloc_gen;
  }
  // the members' parameter tables (shared with the single-scene calls) hold
  // the batch's parameters unless a single-scene call rebuilt them since
  bool stale = false;
  for (int32_t id : b->members) stale = stale || ctx->scenes[id]->tab_batch != batch;
  if (stale) {
    IPT_CK(ipt::launch_prepare_batch(b->mem_dev, (uint32_t)b->members.size(), b->params, ctx->stream));
    for (int32_t id : b->members) ctx->scenes[id]->tab_batch = batch;
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
  for (int32_t id : b->members) {
    ctx->scenes[id]->tab_is_ctx = false;
    ctx->scenes[id]->tab_batch = -1;
  }
  delete b;
  ctx->batches[batch] = nullptr;
  return IPT_OK;
}

}  // extern "C"
