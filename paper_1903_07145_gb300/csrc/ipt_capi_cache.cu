// C ABI: the learned radiance cache's entry points (include/ipt.h,
// ipt_cache_*).
#include "ipt_capi_internal.h"

using namespace ipt_capi;

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
  A(&c->table_h, nt / 2);
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
  if (e == cudaSuccess) e = ipt::cache_pack_table(c->table, c->table_h, ctx->stream);
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
  if (table) {
    IPT_CK(cudaMemcpyAsync(c->table, table, nt * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    IPT_CK(ipt::cache_pack_table(c->table, c->table_h, ctx->stream));
  }
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
