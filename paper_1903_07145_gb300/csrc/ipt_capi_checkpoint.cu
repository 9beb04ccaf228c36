// C ABI: checkpoints of a scene's optimisation (include/ipt.h,
// ipt_checkpoint_*).
#include "ipt_capi_internal.h"

using namespace ipt_capi;

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
    IPT_CK(ipt::cache_pack_table(c->table, c->table_h, ctx->stream));
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
