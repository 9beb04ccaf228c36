// C ABI: the Disney material model's entry points (include/ipt.h,
// ipt_disney_*).
#include "ipt_capi_internal.h"

using namespace ipt_capi;

// --- Disney material model (megakernel integrator) -------------------------

namespace {

constexpr uint32_t kDisneyValues = 16;

}  // namespace

// The scene's Disney state, allocated on first use.
ipt_status ipt_capi::disney_state(ipt_ctx* ctx, DeviceScene* s, DisneyState** out) {
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

namespace {

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
    if ((st = ensure_wf(ctx, true, np, true, opts->max_depth)) != IPT_OK) return st;
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
