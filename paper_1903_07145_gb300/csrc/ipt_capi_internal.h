// Private to the C ABI's translation units (ipt_capi*.cu): the structures
// behind the opaque handles of include/ipt.h -- context, scenes, batches, a
// scene's radiance cache and Disney-model state -- and the helpers the entry
// points share.  ipt_capi.cu defines the helpers and the context, scene and
// iteration calls; ipt_capi_batch.cu, ipt_capi_cache.cu,
// ipt_capi_checkpoint.cu, ipt_capi_disney.cu and ipt_capi_noalloc.cu hold the
// other groups of entry points.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ipt.h"
#include "ipt_cache.h"
#include "ipt_internal.h"
#include "ipt_path.cuh"
#include "ipt_wavefront.h"

namespace ipt_capi {

using ipt::HostScene;

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
  float* table = nullptr;       // FP32 master
  uint32_t* table_h = nullptr;  // FP16 pairs read by queries
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

inline void free_cache(CacheState* c) {
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

inline void free_disney(DisneyState* d) {
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
  uint4* nodes8 = nullptr;
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
  int32_t tab_batch = -1;   // batch whose parameters built the tables (-1: a single-scene call did)
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
  uint64_t g_alloc_gen = 0;  // the context's alloc_gen when the graph was captured
};

struct PendingTiming {
  int id;
  cudaEvent_t a, b;
  int launches;
};

}  // namespace ipt_capi

struct ipt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t seed = 0;
  int flags = 0;
  ipt::Launcher L;
  std::vector<ipt_capi::DeviceScene*> scenes;
  std::string last_error;
  uint32_t* err_dev = nullptr;
  double* loss_host = nullptr;  // pinned
  unsigned long long* counters_dev = nullptr;
  std::vector<ipt_capi::PendingTiming> pending;
  std::vector<cudaEvent_t> spare_events;
  double kernel_ms[IPT_KERNEL_COUNT] = {0};
  uint64_t kernel_n[IPT_KERNEL_COUNT] = {0};
  ipt_config cfg = {1, 1u << 20, 32, 0, 4};
  ipt::WfBuffers wf;
  std::vector<void*> wf_owned;
  bool wf_adjoint = false;
  // bumped whenever device buffers that a captured batch graph may use are
  // reallocated (wavefront state, pixel-batch buffers): a batch whose graph
  // was captured at an older value recaptures before its next replay
  uint64_t alloc_gen = 0;
  bool wf_disney = false;          // the adjoint buffers include the Disney model's records
  ipt::WfScene* wf_tab = nullptr;  // one-entry scene table of single-scene launches
  std::vector<ipt_capi::Batch*> batches;
  cudaStream_t cap_stream = nullptr;  // stream the batch graphs are captured on
  double* noalloc_acc = nullptr;      // device address of ipt_backward_noalloc's array on this device
};

namespace ipt_capi {

ipt_status fail(ipt_ctx* c, ipt_status s, const std::string& msg);
ipt_status cuda_fail(ipt_ctx* c, cudaError_t e, const char* where);
void free_scene(DeviceScene* s);
void resolve_timings(ipt_ctx* c);
cudaEvent_t take_event(ipt_ctx* c);
void stage_begin(void* user, int id);
void stage_end(void* user);
ipt::SceneBuffers buffers(const ipt_ctx* ctx, const DeviceScene* s);
ipt_status get_scene(ipt_ctx* ctx, int32_t id, DeviceScene** out);
ipt_status check_opts(ipt_ctx* ctx, const ipt_trace_opts* o, bool adjoint, bool batch_ok = false);
ipt::TraceParams trace_params(const ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* o, uint32_t set,
                              uint32_t spp, uint64_t it);
ipt_status ensure_pick(ipt_ctx* ctx, DeviceScene* s, uint32_t batch);
ipt_status ensure_tables(ipt_ctx* ctx, DeviceScene* s, const float* params, const float* sparams);
void wf_release(ipt_ctx* c);
// Wavefront state for the context's chunk size; an adjoint caller passes
// the trace's max_depth (the per-vertex carry holds that many vertices) and
// the S x 10 (or S x 16) parameters of its widest chunk.  Capacities only
// grow.
ipt_status ensure_wf(ipt_ctx* ctx, bool adjoint, uint32_t n_params, bool disney = false, uint32_t depth = 0);
bool use_wavefront_cap(const ipt_ctx* ctx, uint32_t spp);
bool use_wavefront(const ipt_ctx* ctx, uint32_t spp);
ipt::WfScene wf_entry(const ipt_ctx* ctx, int32_t scene_id, const DeviceScene* s, uint32_t pix_base, uint32_t n);
ipt_status upload_entry(ipt_ctx* ctx, const ipt::WfScene& e);
ipt_status draw_picks(ipt_ctx* ctx, int32_t scene_id, const DeviceScene* s, uint32_t B, uint64_t iteration,
                      uint32_t* out);
ipt_status run_forward(ipt_ctx* ctx, int32_t scene_id, DeviceScene* s, uint32_t begin, uint32_t n,
                       const ipt::TraceParams& tp, float* img, float* msq, const float* target, float* g_out,
                       double* partials, float g_scale, int loss_kind, const ipt::CachePass* cache = nullptr,
                       uint32_t* pick = nullptr);
ipt_status run_adjoint(ipt_ctx* ctx, int32_t scene_id, DeviceScene* s, uint32_t begin, uint32_t n,
                       const ipt::TraceParams& tp, const float* g_img, double* grad_acc,
                       const ipt::CachePass* cache = nullptr, uint32_t* pick = nullptr);
bool cache_on(const DeviceScene* s);
ipt::CacheNet cache_net(const DeviceScene* s, bool unit_inputs);
ipt_status cache_query_buffers(ipt_ctx* ctx, CacheState* c);
ipt_status cache_pass(ipt_ctx* ctx, DeviceScene* s, bool record, ipt::CachePass* out);
ipt_status cache_train_pass(ipt_ctx* ctx, int32_t scene, DeviceScene* s, const ipt_trace_opts* opts,
                            uint64_t iteration);
// Forward + residual + adjoint over pixels [begin, begin + count), the loss
// normalised by n_total pixels (all shards together).
ipt_status loss_grad_async(ipt_ctx* ctx, int32_t scene, DeviceScene* s, const ipt_trace_opts* opts,
                           uint64_t iteration, float* grad_out, uint64_t begin, uint64_t count, uint64_t n_total);
ipt_status read_loss(ipt_ctx* ctx, DeviceScene* s, double* loss_out, uint64_t n_total);
ipt::AdamHost adam_host(const ipt_adam_opts* a);

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

}  // namespace ipt_capi
