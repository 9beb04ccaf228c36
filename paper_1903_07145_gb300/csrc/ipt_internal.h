// Host-side declarations shared by the C ABI and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace ipt {

// Result of the host scene build: BVH, triangle layout and light tables.
struct HostScene {
  uint32_t n_tri = 0, n_seg = 0, n_nodes = 0, depth = 0;
  std::vector<float> nodes;      // 16 floats per inner node
  std::vector<uint32_t> nodes4;  // 16 words per 4-wide quantized node
  uint32_t n_nodes4 = 0;
  std::vector<uint32_t> nodes8;  // 24 words per 8-wide quantized node
  uint32_t n_nodes8 = 0;
  std::vector<float> tris;       // 12 floats per triangle (leaf order)
  std::vector<float> vnrm;       // 12 floats per triangle, empty if no normals
  std::vector<uint32_t> orig_to_internal;
  std::vector<uint32_t> seg_tris;
  std::vector<uint32_t> seg_begin;
  std::vector<double> tri_cdf;
  std::vector<double> seg_area;
  double diameter = 0.0;
};

// Validates the input and builds the scene; returns false with a message.
bool build_scene(const float* pos, uint32_t n_vert, const float* nrm, const uint32_t* idx,
                 uint32_t n_tri, const uint32_t* tri_seg, uint32_t n_seg, HostScene* out,
                 std::string* err);

// Device pointers of one scene, passed to the launchers.
struct SceneBuffers {
  const float4* nodes;
  const uint4* nodes4;
  const uint4* nodes8;
  const float4* tris;
  const float4* vnrm;
  const uint32_t* seg_tris;
  const uint32_t* seg_begin;
  const double* tri_cdf;
  const double* seg_area;
  const uint32_t* orig_to_internal;
  uint32_t n_seg, n_tri;
  float eps;
  float emission_scale;
  unsigned long long* counters;  // nullptr unless counting
  int wide;                      // 0: binary BVH, 1: 4-wide, 2: 8-wide quantized BVH
};

// Per-segment parameter tables (device).
struct SegBuffers {
  float4* mat_a;
  float4* mat_b;
  float4* emis;
  float4* samp;
  double* pspec;
  double* cdf;
  double* lum;
  double* W;
};

struct ViewHost {
  float m[12];
  float tx, ty;
  uint32_t w, h;
  uint32_t offset;
  uint32_t pad[3];
};

struct TraceParams {
  uint64_t seed;
  uint32_t scene_id;
  uint32_t set;
  uint64_t iteration;
  uint32_t spp;
  uint32_t max_depth;
  int nee, mis, profile;
  // pixel batches: entry b's samples start at counter b * sample_stride
  // (0 = spp; the derivative pass of a same-set gradient check uses the
  // residual's spp so that its samples are the residual's first ones)
  uint32_t sample_stride = 0;
  // megakernel: the pixel batch's drawn pixels (entries 0..n-1), or nullptr
  const uint32_t* pick = nullptr;
};

struct Launcher {
  int num_sms = 0;
  int fwd_blocks_per_sm = 0;
  int adj_blocks_per_sm[4] = {0, 0, 0, 0};
  int wf_blocks_per_sm = 0;  // traversal kernels
  int wf_fixed_blocks = 0;   // configured blocks per SM for every wavefront kernel (0: by occupancy)
  int wf_max_rows = 0;       // gradient rows any adjoint stage may use (blocks of its widest grid)
  int wf_steps = 16;  // refill point of the persistent traversal (idle lanes; binary BVH: steps)
  int sort_cells = 0; // secondary closest-hit rays reordered by origin cell (cells per axis; 0: off)
  int sort_dirs = 0;  //   and direction (divisions of each cube-map face side; 0: none)
};

// Wavefront state (device), sized for `cap` path slots per chunk.
struct WfBuffers {
  float4 *ray_o = nullptr, *ray_d = nullptr, *hit = nullptr, *beta = nullptr, *rad = nullptr;
  uint32_t *q0 = nullptr, *q1 = nullptr, *cnt = nullptr;
  float4 *sh_o = nullptr, *sh_d = nullptr;
  uint4* sh_meta = nullptr;
  float4* sh_c = nullptr;
  uint32_t* sh_vis = nullptr;
  float4 *aT = nullptr, *aU = nullptr;
  float2* aR = nullptr;
  uint32_t* nv = nullptr;
  float4 *sh_ge = nullptr, *sh_gm = nullptr, *sh_n = nullptr;
  // Disney model adjoint: per-vertex directions and hit, and the shadow
  // records' material derivatives (4 float4 = 13 values per record)
  float4 *aWi = nullptr, *aWo = nullptr, *sh_dv = nullptr;
  float* blk = nullptr;
  // reordering of secondary closest-hit rays: the queue's slots by bin, the
  // bin of each queue entry, and per-bin counts / offsets
  uint32_t* qs = nullptr;
  uint16_t* keys = nullptr;
  uint32_t* bins = nullptr;
  uint32_t cap = 0;
  uint32_t blk_params = 0;  // S x 10 capacity of each block row
  uint32_t depth_cap = 0;   // vertices the per-vertex carry holds (adjoint max_depth)
};

constexpr int kMaxAdjointDepth = 8;
constexpr uint32_t kSortMaxBins = 8192;  // bins of the ray reordering (6 dirs^2 cells^3 at most)
constexpr int kMaxForwardDepth = 64;
constexpr int kBlockThreads = 128;

int loss_partials_capacity(const Launcher& L);

cudaError_t launch_prepare(const SceneBuffers& s, const SegBuffers& t, const float* params,
                           const float* sparams, cudaStream_t st);

cudaError_t launch_forward(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                           const ViewHost* views_dev, uint32_t n_views, uint32_t pix_begin,
                           uint32_t n_pix, const TraceParams& tp, float* img, float* msq,
                           const float* target, float* g_out, double* loss_partials,
                           float g_scale, int loss_kind, uint32_t* err, cudaStream_t st);

// gacc_scratch: 10 * n_seg floats, used (and required) when the scene has
// more than wf_max_segments() segments; may be null otherwise.
cudaError_t launch_adjoint(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                           const ViewHost* views_dev, uint32_t n_views, uint32_t pix_begin, uint32_t n_pix,
                           const TraceParams& tp, const float* g_img, double* grad_acc,
                           float* gacc_scratch, uint32_t* err, cudaStream_t st);

// Segments whose gradient accumulators fit a block's shared memory; chunks
// (or scenes) with more accumulate in global memory.
uint32_t wf_max_segments();

cudaError_t launch_finalize(const double* loss_partials, int n_partials, double* loss_dev,
                            const double* grad_acc, float* grad_out, uint32_t n_params,
                            cudaStream_t st);

struct AdamHost {
  float lr, beta1, beta2, eps, l1;
};

// Adam on a scene's parameters.  loss (device, nullable) and the gradient are
// checked first: if either is not finite the step is skipped (parameters,
// moments and step count unchanged) and kErrNonFinite is set in *err.  guard:
// a device word the check of scenes above kWideSegments segments writes.
cudaError_t launch_adam(const SceneBuffers& s, const SegBuffers& t, float* params, float* m,
                        float* v, const uint8_t* free_mask, const double* grad_acc,
                        const float* grad_f, int* step_dev, const AdamHost& a, const double* loss,
                        uint32_t* guard, uint32_t* err, cudaStream_t st);

// One member scene of a batch: where its parameters sit in the batch's
// concatenated vector, and its parameter tables.
struct BatchMember {
  SegBuffers tab;
  const double* seg_area;
  uint32_t seg_offset, n_seg;
  float es;
  float inv_n;      // 1 / (3 N) of its loss
  uint32_t active;  // 0: takes no part in the batch's steps (parameters and Adam state frozen)
  uint32_t slot;         // its entry in the launch table when active
  uint32_t grad_offset;  // its first segment in the step's gradient accumulators (active members, packed)
};

// Adam over the whole batch (block b updates member b, then rebuilds its
// tables); step t = *iter_dev + 1.  A member whose loss (losses[b]) or
// gradient is not finite is skipped and kErrNonFinite is set in *err.
cudaError_t launch_adam_batch(const BatchMember* members, uint32_t n_members, float* params, float* m, float* v,
                              const uint8_t* free_mask, const double* grad_acc, const uint32_t* iter_dev,
                              const AdamHost& a, const double* losses, uint32_t* err, cudaStream_t st);
// Tables of every member from the batch parameters.
cudaError_t launch_prepare_batch(const BatchMember* members, uint32_t n_members, const float* params,
                                 cudaStream_t st);
// loss[b] = sum over rows of rows[r * n_tab + slot_b], scaled by the member's
// 1 / (3 N); 0 for members that are not active.
cudaError_t launch_batch_losses(const double* rows, int n_rows, const BatchMember* members, uint32_t n,
                                uint32_t n_tab, double* loss, cudaStream_t st);
cudaError_t launch_tick(uint32_t* counter, cudaStream_t st);

cudaError_t launch_trace_rays(const SceneBuffers& s, uint32_t n, const float* orig,
                              const float* dir, const int32_t* skip, int32_t* tri_out,
                              float* t_out, float* u_out, float* v_out, uint32_t* err,
                              cudaStream_t st);

cudaError_t launch_philox(uint32_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t st);

cudaError_t init_launcher(Launcher* L, int device);

// Optional per-stage timing hook of the wavefront launchers.
struct WfHook {
  void (*begin)(void* user, int kernel_id);
  void (*end)(void* user);
  void* user;
};

cudaError_t wf_init(Launcher* L);
int wf_max_blocks(const Launcher& L);

// Disney material model (megakernel integrator): per-segment tables built
// from the 16-value parameter blocks, next to the shared light-selection
// tables in SegBuffers (emis, samp.z = p_A, cdf, lum, W).
struct DisneyBuffers {
  float4* mat;    // 4 per segment: the 13 material values, then zeros
  double2* lobe;  // cumulative lobe probabilities (P_d, P_d + P_s), FP64
  float4* samp;   // 2 per segment: (a_x, a_y, a_c, 0), (P_d, P_s, P_c, 0)
};

cudaError_t launch_disney_tables(const SceneBuffers& s, const SegBuffers& t, const DisneyBuffers& d,
                                 const float* params, const float* sparams, cudaStream_t st);
cudaError_t launch_disney_forward(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                                  const DisneyBuffers& d, const ViewHost* views_dev, uint32_t n_views,
                                  uint32_t pix_begin, uint32_t n_pix, const TraceParams& tp, float* img, float* msq,
                                  const float* target, float* g_out, double* loss_partials, float g_scale,
                                  int loss_kind, uint32_t* err, cudaStream_t st);
// Accumulates into grad_acc (16 per segment); scenes whose accumulators do
// not fit a block's shared memory use gacc_scratch (16 S floats).
cudaError_t launch_disney_adjoint(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                                  const DisneyBuffers& d, const ViewHost* views_dev, uint32_t n_views,
                                  uint32_t pix_begin, uint32_t n_pix, const TraceParams& tp, const float* g_img,
                                  double* grad_acc, float* gacc_scratch, uint32_t* err, cudaStream_t st);
// Adam with the Disney clamps (material values in [0, 1], roughness in
// [0.02, 1], emission >= 0 with the L1 term), then the tables.
// As launch_adam (the same check of loss and gradient), for the Disney blocks.
cudaError_t launch_disney_adam(const SceneBuffers& s, const SegBuffers& t, const DisneyBuffers& d, float* params,
                               float* m, float* v, const uint8_t* free_mask, const double* grad_acc,
                               const float* grad_f, int* step_dev, const AdamHost& a, const double* loss,
                               uint32_t* err, cudaStream_t st);
uint32_t disney_max_shared_segments();

}  // namespace ipt
