// Scene table of the wavefront integrator (shared by the launchers and the
// C ABI).  A launch traces the concatenated pixels of the table's scenes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ipt_cache.h"
#include "ipt_device.cuh"
#include "ipt_internal.h"

namespace ipt {

struct WfScene {
  SceneDev s;                // geometry
  SegDev t;                  // parameter tables (emission and light selection for either model)
  DisneyDev dis;             // Disney material tables, or null pointers (Lambert + GGX)
  const ViewDev* views;
  uint32_t n_views;
  uint32_t pix_begin;        // first launch pixel of this scene
  uint32_t n_pix;            // pixels of this scene in the launch
  uint32_t pix_base;         // scene pixel id of its first launch pixel
  uint32_t seg_offset;       // first segment of this scene in the launch's segment space
  uint32_t n_seg;
  uint2 key;                 // Philox key: (seed_lo, seed_hi ^ scene id)
  float es;                  // emission scale
  float g_scale;             // 1 / (3 N) of this scene's loss
  const float* target;       // indexed by scene pixel id (residual mode), or nullptr
  float* g_img;              // dE/dI, indexed by entry
  float* img;                // optional outputs, indexed by entry - pix_base
  float* msq;
  // Stochastic pixel batch (Sec. 4.5), or nullptr: the scene's launch pixels
  // are then batch entries 0..n_pix-1 (pix_base 0); entry b traces scene
  // pixel pick[b] with sample counters b*spp .. b*spp+spp-1.  Without a batch
  // the entry of a launch pixel is its scene pixel id.
  uint32_t* pick;
  uint32_t n_all;            // pixels of the scene the batch draws from
  float3 bb_lo, bb_inv;      // vertex bounding box: lower corner, 1 / extent per axis (0 if flat)
};

// Radiance cache in a pass: query mode ends paths at vertex b_term and adds
// the cache's prediction; record mode (training) traces full paths and
// records, at b_term, the inputs and the reflected radiance gathered after it.
struct CachePass {
  CacheNet net;
  CacheBuffers buf;
  uint32_t b_term;
  int record;
};

struct WfChunk {
  uint32_t p0, n_pix;        // launch pixels of the chunk
  uint32_t seg_lo, seg_n;    // segment range its gradient accumulators cover
};

std::vector<WfChunk> wf_plan(const std::vector<WfScene>& tab, uint32_t cap, uint32_t spp, uint32_t max_seg);
uint32_t wf_max_segments();

// disney: the table's scenes trace with the Disney material model (their
// `dis` tables; gradients of 16 values per segment).
cudaError_t wf_forward(const Launcher& L, const WfScene* tab_dev, const std::vector<WfScene>& tab,
                       const TraceParams& tp, int loss_kind, const uint32_t* iter_dev, const WfBuffers& wb,
                       double* loss_rows, uint32_t* err, cudaStream_t st, const WfHook* hook,
                       const CachePass* cache = nullptr, bool disney = false);

// Draws the pixel batch of every table entry that has one, for the iteration
// *iter_dev (or iter when iter_dev is null).
cudaError_t wf_pick(const WfScene* tab_dev, const std::vector<WfScene>& tab, const uint32_t* iter_dev,
                    uint32_t iter, cudaStream_t st);

cudaError_t wf_adjoint(const Launcher& L, const WfScene* tab_dev, const std::vector<WfScene>& tab,
                       const TraceParams& tp, const uint32_t* iter_dev, const WfBuffers& wb, double* grad_acc,
                       uint32_t* err, cudaStream_t st, const WfHook* hook, const CachePass* cache = nullptr,
                       bool disney = false);

// Batched megakernel over a launch table (Lambert + GGX): the residual pass
// writes each entry's upstream gradient and per-block loss rows
// (loss_partials_capacity(L) rows of n_scenes); the derivative pass adds
// g . dI/dtheta into grad_acc over the table's packed segments (10 n_seg),
// through gacc_scratch (10 n_seg floats) when they exceed a block's shared
// memory (batch_shared_params()).
cudaError_t launch_forward_batch(const Launcher& L, const WfScene* tab_dev, uint32_t n_scenes, uint32_t total,
                                 const TraceParams& tp, const uint32_t* iter_dev, int loss_kind, double* loss_rows,
                                 uint32_t* err, cudaStream_t st);
cudaError_t launch_adjoint_batch(const Launcher& L, const WfScene* tab_dev, uint32_t n_scenes, uint32_t total,
                                 uint32_t n_seg, const TraceParams& tp, const uint32_t* iter_dev, double* grad_acc,
                                 float* gacc_scratch, uint32_t* err, cudaStream_t st);
uint32_t batch_shared_params();

}  // namespace ipt
