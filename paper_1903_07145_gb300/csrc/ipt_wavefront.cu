// Wavefront integrator over a table of scenes: the same paths as the
// megakernel (same random numbers at the same (vertex, call) slots), traced
// stage by stage over chunks of path slots so that every traversal launch
// works on a compacted queue.  A launch covers the concatenated pixels of
// one or more scenes (a batch); every slot carries its scene index, and a
// scene's paths are identical whether it is traced alone or in a batch.
//
// Per chunk (slots are pixel-major: slot = local_pixel * spp + sample):
//   wf_camera                   camera rays, path state, queue 0 = all slots
//   per vertex k = 0..D:
//     wf_trace<closest>         persistent closest-hit traversal; lanes refill
//                               from the queue as their rays finish
//     shading                   emission (MIS), next-event candidate -> shadow
//                               queue, BRDF sample -> next queue
//     wf_trace<any>             persistent shadow-ray traversal
//   wf_reduce                   per-pixel mean / residual / per-scene loss
// The adjoint splits shading in two (before and after the shadow rays), keeps
// each path's per-vertex carry (T_l, U_l, dw/dtheta factors) in SoA global
// memory, and accumulates g . dI/dtheta in per-block shared memory over the
// chunk's segment range, flushed to block-private rows and reduced in FP64.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ipt_device.cuh"
#include "ipt_disney.cuh"
#include "ipt_internal.h"
#include "ipt_path.cuh"
#include "ipt_wavefront.h"

namespace cg = cooperative_groups;

namespace ipt {

constexpr uint32_t kDead = 0x80000000u;  // beta.w: path finished
constexpr uint32_t kSceneShift = 8;      // beta.w: vertex index in bits 0-7, scene in bits 8-23
constexpr int kWfThreads = 128;

__device__ __forceinline__ uint32_t pack_state(uint32_t k, uint32_t scene) { return k | (scene << kSceneShift); }
__device__ __forceinline__ uint32_t state_k(uint32_t w) { return w & 0xffu; }
__device__ __forceinline__ uint32_t state_scene(uint32_t w) { return (w >> kSceneShift) & 0xffffu; }

struct WfDev {
  float4* ray_o;  // origin, w = skip triangle (int bits)
  float4* ray_d;  // direction, w = pdf of this direction (0 for camera rays)
  float4* hit;    // x = triangle (int bits, -1 miss), t, u, v
  float4* beta;   // throughput, w = vertex index | scene << 8 | kDead
  float4* rad;    // path radiance (forward)
  uint32_t* q0;
  uint32_t* q1;
  uint32_t* cnt;  // [0] |q0|, [1] |q1|, [2] |shadow|, [3] closest fetch, [4] shadow fetch
  float4* sh_o;   // origin, w = skip triangle a
  float4* sh_d;   // direction, w = extent
  uint4* sh_meta; // slot, skip triangle b (light), vertex segment, light segment
  float4* sh_c;   // forward: contribution
  uint32_t* sh_vis;
  // adjoint
  float4* aT;     // [l * cap + slot]: T_l.xyz, dw/dkd factor
  float4* aU;     // U_l.xyz, dw/dks factor
  float2* aR;     // dw/dr factor, segment (int bits)
  uint32_t* nv;
  float4* sh_ge;  // g beta f k es (emission gradient of the light segment)
  float4* sh_gm;  // g beta Le k, w = specular factor
  float4* sh_n;   // f Le k (the contribution without beta), w = d spec / d r
  // Disney model: aT.w = cos/pdf, aR = (u, segment); aWi = (wi, triangle),
  // aWo = (wo, v); sh_dv = the vertex material derivative of a shadow record
  float4* aWi;
  float4* aWo;
  float4* sh_dv;
  float* blk;     // per-block rows of the chunk's partial gradients
  uint32_t cap;
};

// Bin grid of the reordering of secondary closest-hit rays (see ray_bin).
struct BinGrid {
  int cells, dirs;     // origin cells per axis of a scene's box; direction cells per cube-map face side
  uint32_t per_scene;  // bins per scene: 6 dirs^2 cells^3 (cells^3 for dirs = 0)
  uint32_t scene0;     // first scene of the chunk (its scenes' bins follow one another)
  uint32_t n_bins;     // per_scene x the chunk's scenes
};

// Per-launch constants.
struct WfParams {
  uint32_t set;
  uint32_t iter;
  const uint32_t* iter_dev;  // iteration counter on the device (overrides iter)
  uint32_t spp;
  uint32_t stride;           // sample counter stride of pixel-batch entries
  uint32_t max_depth;
  int nee, mis, profile, loss_kind;
  uint32_t n_scenes;
  uint32_t seg_lo, seg_n;    // segment range of the chunk's gradient accumulators
  float* gacc;               // accumulators in global memory (chunks too wide for shared memory), or nullptr
  BinGrid bin;               // reordering: bin grid of the rays appended to the next closest-hit queue
  uint16_t* keys;            //   and their bins, by queue position (nullptr: no reordering)
  uint32_t cache_k;          // vertex where the radiance cache ends paths (kNoCache: off)
  int cache_record;          // training pass: record at cache_k, gather only from there on
  CacheBuffers cb;
};

constexpr uint32_t kNoCache = 0xffffffffu;

__device__ __forceinline__ uint32_t set_iter(const WfParams& p) {
  const uint32_t it = p.iter_dev ? *p.iter_dev : p.iter;
  return (p.set << 24) | (it & 0xffffffu);
}

__device__ __forceinline__ uint32_t* queue(const WfDev& w, int which) { return which ? w.q1 : w.q0; }

// Warp-aggregated append: one atomic per group of lanes that arrive together.
__device__ __forceinline__ uint32_t enqueue(uint32_t* counter, bool want) {
  cg::coalesced_group g = cg::coalesced_threads();
  const unsigned m = g.ballot(want);
  if (!m) return 0xffffffffu;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if ((int)g.thread_rank() == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = g.shfl(base, leader);
  return want ? base + (uint32_t)__popc(m & ((1u << g.thread_rank()) - 1u)) : 0xffffffffu;
}

// Scene pixel id, sample counter and entry (the index of its upstream
// gradient and image outputs) of a slot of the chunk starting at launch
// pixel p0.
__device__ __forceinline__ void slot_pixel(const WfScene& e, uint32_t p0, uint32_t slot, uint32_t spp,
                                           uint32_t stride, uint32_t& pid, uint32_t& smp, uint32_t& entry) {
  const uint32_t lp = slot / spp;
  smp = slot - lp * spp;
  entry = p0 + lp - e.pix_begin + e.pix_base;
  pid = entry;
  if (e.pick) {
    pid = e.pick[entry];
    smp += entry * stride;
  }
}

__device__ __forceinline__ PathRng path_rng(const WfScene& e, uint32_t pid, uint32_t smp, uint32_t si) {
  PathRng rng;
  rng.base = make_uint4(pid, smp, si, 0);
  rng.key = e.key;
  return rng;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWfThreads) wf_camera(const WfScene* tab, WfParams lp, uint32_t p0,
                                                        uint32_t n_slots, WfDev w) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    w.cnt[0] = n_slots;
    w.cnt[3] = 0;
    if (lp.cache_k != kNoCache) {
      lp.cb.counts[0] = 0;
      lp.cb.counts[2] = min(lp.cb.counts[1], lp.cb.r_cap);
    }
  }
  const uint32_t si = set_iter(lp);
  for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < n_slots; slot += gridDim.x * blockDim.x) {
    const uint32_t P = p0 + slot / lp.spp;
    // scene of launch pixel P: the last entry with pix_begin <= P
    uint32_t lo = 0, hi = lp.n_scenes - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (tab[mid].pix_begin <= P)
        lo = mid;
      else
        hi = mid - 1;
    }
    const WfScene& e = tab[lo];
    uint32_t pid, smp, ent;
    slot_pixel(e, p0, slot, lp.spp, lp.stride, pid, smp, ent);
    const ViewDev& vw = find_view(e.views, e.n_views, pid);
    const uint32_t l = pid - vw.offset;
    const PathRng rng = path_rng(e, pid, smp, si);
    float3 o;
    const float3 d = camera_ray(vw, l % vw.w, l / vw.w, rng, o);
    w.ray_o[slot] = make_float4(o.x, o.y, o.z, __int_as_float(-1));
    w.ray_d[slot] = make_float4(d.x, d.y, d.z, 0.0f);
    w.beta[slot] = make_float4(1.0f, 1.0f, 1.0f, __uint_as_float(pack_state(0, lo)));
    w.rad[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    w.q0[slot] = slot;
    if (w.nv) w.nv[slot] = 0;
  }
}

// ---------------------------------------------------------------------------
// Reordering of a closest-hit queue (secondary rays): a counting sort of its
// entries by bin, bin = (direction cell, origin cell).  The direction cell is
// the cube-map face of the dominant axis and sign, split into dirs x dirs
// squares (dirs = 0: one cell for all directions); the origin cell one of
// cells^3 boxes of the scene's bounding box.  Only the order in which the
// traversal takes the rays changes: each ray's result is the same.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 1024;

// Bin of the ray from o in direction d (any length) of scene b (table entry
// e): scene major, then direction cell, then origin cell in the scene's
// bounding box; always below g.n_bins for the chunk's scenes.
__device__ __forceinline__ uint32_t ray_bin(const BinGrid& g, const WfScene& e, uint32_t b, float3 o, float3 d) {
  const int c = g.cells;
  const float fc = (float)c;
  const int cx = min(max((int)((o.x - e.bb_lo.x) * (e.bb_inv.x * fc)), 0), c - 1);
  const int cy = min(max((int)((o.y - e.bb_lo.y) * (e.bb_inv.y * fc)), 0), c - 1);
  const int cz = min(max((int)((o.z - e.bb_lo.z) * (e.bb_inv.z * fc)), 0), c - 1);
  const uint32_t cell = (uint32_t)((cz * c + cy) * c + cx);
  const uint32_t base = (b - g.scene0) * g.per_scene;
  if (g.dirs == 0) return base + cell;
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int face;
  float u, v, m;
  if (ax >= ay && ax >= az) {
    face = d.x < 0.0f ? 1 : 0;
    u = d.y;
    v = d.z;
    m = ax;
  } else if (ay >= az) {
    face = d.y < 0.0f ? 3 : 2;
    u = d.x;
    v = d.z;
    m = ay;
  } else {
    face = d.z < 0.0f ? 5 : 4;
    u = d.x;
    v = d.y;
    m = az;
  }
  // (u / m + 1) / 2 in [0, 1] on the face, in dirs squares
  const float k = 0.5f * (float)g.dirs / fmaxf(m, 1e-30f);
  const int iu = min(max((int)((u + m) * k), 0), g.dirs - 1);
  const int iv = min(max((int)((v + m) * k), 0), g.dirs - 1);
  const uint32_t dir = (uint32_t)((face * g.dirs + iu) * g.dirs + iv);
  return base + dir * (uint32_t)(c * c * c) + cell;
}

// The sort kernels take the queue in groups of 8 entries per thread (one
// 16-byte load of their bins; the key array is padded to whole groups).
// Neighbouring entries (samples of one pixel) often share a bin, so each
// thread adds a run of equal bins with one shared atomic.
__device__ __forceinline__ void load_bins8(const uint16_t* keys, uint32_t g, uint32_t k[8]) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(keys) + g);
  k[0] = v.x & 0xffffu, k[1] = v.x >> 16, k[2] = v.y & 0xffffu, k[3] = v.y >> 16;
  k[4] = v.z & 0xffffu, k[5] = v.z >> 16, k[6] = v.w & 0xffffu, k[7] = v.w >> 16;
}

// Adds the first m (1..8) of the group's 8 bins to h, one atomic per run.
__device__ __forceinline__ void count_bins8(uint32_t* h, const uint32_t k[8], uint32_t m) {
  uint32_t run = 1u, last = k[0];
#pragma unroll
  for (uint32_t j = 1; j < 8; ++j) {
    if (j >= m) break;
    if (k[j] == last) {
      ++run;
    } else {
      atomicAdd(&h[last], run);
      last = k[j];
      run = 1u;
    }
  }
  atomicAdd(&h[last], run);
}

// Counts of the bins of queue `cur`'s entries (their bins written by the
// stage that appended them), added to `bins` (cleared before).
__global__ void __launch_bounds__(kSortThreads) wf_bin_count(uint32_t n_bins, WfDev w, int cur,
                                                            const uint16_t* keys, uint32_t* bins) {
  extern __shared__ uint32_t h[];
  for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t n = w.cnt[cur];
  const uint32_t ng = (n + 7u) / 8u;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    uint32_t k[8];
    load_bins8(keys, g, k);
    count_bins8(h, k, min(8u, n - 8u * g));
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x)
    if (h[i]) atomicAdd(&bins[i], h[i]);
}

// Counts -> exclusive offsets, in place (one block of kSortThreads threads,
// at most 8 bins each).
__global__ void __launch_bounds__(kSortThreads) wf_bin_scan(uint32_t* bins, uint32_t n_bins) {
  __shared__ uint32_t ws[kSortThreads / 32];
  const uint32_t per = (n_bins + kSortThreads - 1) / kSortThreads;
  const uint32_t b0 = threadIdx.x * per;
  uint32_t v[8];
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < 8; ++k) {
    v[k] = (k < per && b0 + k < n_bins) ? bins[b0 + k] : 0u;
    sum += v[k];
  }
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= (uint32_t)off) x += y;
  }
  if (lane == 31u) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = ws[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= (uint32_t)off) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  uint32_t run = x - sum + (warp ? ws[warp - 1] : 0u);
#pragma unroll
  for (uint32_t k = 0; k < 8; ++k) {
    if (k < per && b0 + k < n_bins) bins[b0 + k] = run;
    run += v[k];
  }
}

// Each block takes a contiguous part of the queue (rays of neighbouring
// pixels stay together within a bin), reserves its share of every bin with
// one atomic and writes its slots there, a run of equal bins at a time.
__global__ void __launch_bounds__(kSortThreads) wf_bin_scatter(uint32_t n_bins, WfDev w, int cur,
                                                              const uint16_t* keys, uint32_t* bins,
                                                              uint32_t* order) {
  extern __shared__ uint32_t h[];
  for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t n = w.cnt[cur];
  const uint32_t ng = (n + 7u) / 8u;
  const uint32_t per = (ng + gridDim.x - 1u) / gridDim.x;
  const uint32_t lo = min(ng, blockIdx.x * per), hi = min(ng, lo + per);
  for (uint32_t g = lo + threadIdx.x; g < hi; g += blockDim.x) {
    uint32_t k[8];
    load_bins8(keys, g, k);
    count_bins8(h, k, min(8u, n - 8u * g));
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x) {
    const uint32_t c = h[i];
    if (c) h[i] = atomicAdd(&bins[i], c);
  }
  __syncthreads();
  const uint32_t* qin = queue(w, cur);
  for (uint32_t g = lo + threadIdx.x; g < hi; g += blockDim.x) {
    uint32_t k[8], slot[8];
    load_bins8(keys, g, k);
    const uint32_t m = min(8u, n - 8u * g);
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) slot[j] = j < m ? qin[8u * g + j] : 0u;
    uint32_t pos = 0u;
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      if (j >= m) break;
      if (j == 0 || k[j] != k[j - 1]) {  // a run starts: reserve its places
        uint32_t len = 1u;
#pragma unroll
        for (uint32_t t = j + 1; t < 8; ++t) {
          if (t >= m || k[t] != k[j]) break;
          ++len;
        }
        pos = atomicAdd(&h[k[j]], len);
      }
      order[pos++] = slot[j];
    }
  }
}

// ---------------------------------------------------------------------------
// Persistent traversal with warp refills.  kMode 0: closest hit of queue
// `cur` into w.hit; 1: shadow rays, adding the forward contribution of the
// unoccluded ones; 2: shadow rays, visibility flag only (adjoint).
// ---------------------------------------------------------------------------
// Traversal stack: the top kShortStack entries of each lane live in shared
// memory (entry e of thread t at [e * kWfThreads + t], so a warp's accesses
// fall in distinct banks whatever its lanes' depths); deeper entries spill to
// a per-lane local array.  An entry is (node link, entry distance bits).
constexpr int kShortStack = 12;

struct Trav {
  RayPre r;
  float3 oinv;
  float tmax;
  int skip_a, skip_b;
  int node, sp;
  int tri, tri_end;  // wide traversals: triangles of the current leaf still to test
  int gnode;         // 8-wide: node whose hit slots are being entered
  uint32_t gmask;    // 8-wide: its hit slots not yet entered (visiting order)
  uint32_t sgn;      // 8-wide: direction sign bits of the ray
  uint2 deep[kStackSize - kShortStack];
  int best, best_orig;
  float bt, bu, bv;
  bool occluded;
  uint32_t n_nodes, n_tests;
};

__device__ __forceinline__ void st_push(uint2* sh, Trav& T, int ref, float t) {
  const uint2 e = make_uint2((uint32_t)ref, __float_as_uint(t));
  if (T.sp < kShortStack)
    sh[T.sp * kWfThreads] = e;
  else
    T.deep[T.sp - kShortStack] = e;
  ++T.sp;
}

__device__ __forceinline__ uint2 st_pop(const uint2* sh, Trav& T) {
  --T.sp;
  return T.sp < kShortStack ? sh[T.sp * kWfThreads] : T.deep[T.sp - kShortStack];
}

__device__ __forceinline__ void trav_init(Trav& T, float3 o, float3 d, float tmax, int skip_a, int skip_b) {
  T.r = ray_pre(o, d);
  T.oinv = f3(o.x * T.r.inv.x, o.y * T.r.inv.y, o.z * T.r.inv.z);
  T.tmax = tmax;
  T.skip_a = skip_a;
  T.skip_b = skip_b;
  T.node = 0;
  T.sp = 0;
  T.tri = T.tri_end = 0;
  T.gnode = 0;
  T.gmask = 0u;
  T.sgn = ray_sgn(T.r);
  T.best = -1;
  T.best_orig = 0x7fffffff;
  T.bt = tmax;
  T.bu = T.bv = 0.0f;
  T.occluded = false;
  T.n_nodes = T.n_tests = 0;
}

template <bool kAny>
__device__ __forceinline__ bool leaf_tests(const SceneDev& s, Trav& T, int leaf) {
  int first, count;
  decode_leaf(leaf, first, count);
  T.n_tests += count;
  for (int i = first; i < first + count; ++i) {
    if (i == T.skip_a || i == T.skip_b) continue;
    const float4 q0 = __ldg(&s.tris[3 * i + 0]);
    const float4 q1 = __ldg(&s.tris[3 * i + 1]);
    const float4 q2 = __ldg(&s.tris[3 * i + 2]);
    float t, u, v;
    if (kAny) {
      if (tri_test(T.r, xyz(q0), xyz(q1), xyz(q2), T.tmax, t, u, v)) {
        T.occluded = true;
        return true;
      }
    } else if (tri_test(T.r, xyz(q0), xyz(q1), xyz(q2), T.bt * 1.0000002f, t, u, v)) {
      const int orig = __float_as_int(q0.w);
      if (t < T.bt || (t == T.bt && orig < T.best_orig)) {
        T.best = i;
        T.bt = t;
        T.bu = u;
        T.bv = v;
        T.best_orig = orig;
      }
    }
  }
  return false;
}

// Binary nodes: runs up to `steps` node visits; true when the traversal is over.
template <bool kAny>
__device__ __forceinline__ bool trav_run2(const SceneDev& s, Trav& T, uint2* sh, int steps, uint32_t* err) {
  for (int it = 0; it < steps; ++it) {
    if (T.node >= 0) {
      ++T.n_nodes;
      const float4 n0 = __ldg(&s.nodes[4 * T.node + 0]);
      const float4 n1 = __ldg(&s.nodes[4 * T.node + 1]);
      const float4 n2 = __ldg(&s.nodes[4 * T.node + 2]);
      const float4 n3 = __ldg(&s.nodes[4 * T.node + 3]);
      float t0, t1;
      box2(T.r, T.oinv, n0, n1, n2, kAny ? T.tmax : T.bt, t0, t1);
      const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      const bool h0 = t0 != __int_as_float(0x7f800000);
      const bool h1 = t1 != __int_as_float(0x7f800000);
      if (h0 && h1) {
        if (T.sp >= kStackSize) {
          atomicOr(err, kErrStack);
          T.best = -1;
          T.occluded = true;
          return true;
        }
        if (!kAny && t1 < t0) {
          st_push(sh, T, c0, 0.0f);
          T.node = c1;
        } else {
          st_push(sh, T, c1, 0.0f);
          T.node = c0;
        }
        continue;
      }
      if (h0 || h1) {
        T.node = h0 ? c0 : c1;
        continue;
      }
    } else if (leaf_tests<kAny>(s, T, T.node)) {
      return true;
    }
    if (T.sp == 0) return true;
    T.node = (int)st_pop(sh, T).x;
  }
  return false;
}

// Makes link `ref` the lane's next unit of work: an inner node to test, or
// the triangle range of a leaf.
__device__ __forceinline__ void trav_enter(Trav& T, int ref) {
  if (ref >= 0) {
    T.node = ref;
  } else {
    int first, count;
    decode_leaf(ref, first, count);
    T.node = -1;
    T.tri = first;
    T.tri_end = first + count;
    T.n_tests += count;
  }
}

// One triangle of the current leaf; true when a shadow ray is blocked.
template <bool kAny>
__device__ __forceinline__ bool tri_unit(const SceneDev& s, Trav& T) {
  const int i = T.tri++;
  if (i == T.skip_a || i == T.skip_b) return false;
  const float4 q0 = __ldg(&s.tris[3 * i + 0]);
  const float4 q1 = __ldg(&s.tris[3 * i + 1]);
  const float4 q2 = __ldg(&s.tris[3 * i + 2]);
  float t, u, v;
  if (kAny) {
    if (tri_test(T.r, xyz(q0), xyz(q1), xyz(q2), T.tmax, t, u, v)) {
      T.occluded = true;
      return true;
    }
  } else if (tri_test(T.r, xyz(q0), xyz(q1), xyz(q2), T.bt * 1.0000002f, t, u, v)) {
    const int orig = __float_as_int(q0.w);
    if (t < T.bt || (t == T.bt && orig < T.best_orig)) {
      T.best = i;
      T.bt = t;
      T.bu = u;
      T.bv = v;
      T.best_orig = orig;
    }
  }
  return false;
}

// Pops to the next stack entry still in range (closest hit: entry distance
// not beyond the current hit) and makes it the lane's unit of work; true
// when the stack is empty (the traversal is over).  4-wide nodes.
template <bool kAny>
__device__ __forceinline__ bool advance4(Trav& T, uint2* sh) {
  uint2 e;
  for (;;) {
    if (T.sp == 0) return true;
    e = st_pop(sh, T);
    if (kAny || __uint_as_float(e.y) <= T.bt * 1.0000005f) break;
  }
  trav_enter(T, (int)e.x);
  return false;
}

// 8-wide nodes: enters the next hit slot of the current group, popping
// groups (node, remaining slots) as they run out; true when none is left.
__device__ __forceinline__ bool advance8(const SceneDev& s, Trav& T, uint2* sh) {
  while (T.gmask == 0u) {
    if (T.sp == 0) return true;
    const uint2 e = st_pop(sh, T);
    T.gnode = (int)e.x;
    T.gmask = e.y;
  }
  const int k = __ffs(T.gmask) - 1;
  T.gmask &= T.gmask - 1u;
  trav_enter(T, node8_link(s, T.gnode, k ^ (int)T.sgn));
  return false;
}

// One triangle of the lane's current leaf, then (leaf done) the next unit;
// true when the traversal is over (a shadow ray blocked, or nothing left).
template <bool kAny, int kWidth>
__device__ __forceinline__ bool tri_step(const SceneDev& s, Trav& T, uint2* sh) {
  if (tri_unit<kAny>(s, T)) return true;
  if (T.tri < T.tri_end) return false;
  return kWidth == 8 ? advance8(s, T, sh) : advance4<kAny>(T, sh);
}

// One 4-wide node test: hit children nearest first (for shadow rays too: an
// occluder near the shading point is found after fewer visits, -5% shadow
// traversal time on the 61k room against slot order), the nearest entered;
// a missed node pops the next entry.
template <bool kAny>
__device__ __forceinline__ bool node_step4(const SceneDev& s, Trav& T, uint2* sh, uint32_t* err) {
  if (T.node >= 0) {
    ++T.n_nodes;
    float tn[4];
    int ref[4];
    const uint32_t mask = node4_children(s, T.node, T.r, kAny ? T.tmax : T.bt, tn, ref);
    const int k = __popc(mask);
    if (k > 0) {
      if (T.sp + k - 1 > kStackSize) {
        atomicOr(err, kErrStack);
        T.best = -1;
        T.occluded = true;
        return true;
      }
      sort4(tn, ref);
#pragma unroll
      for (int i = 3; i >= 1; --i)
        if (i < k) st_push(sh, T, ref[i], tn[i]);
      trav_enter(T, ref[0]);
      return false;
    }
  }
  return advance4<kAny>(T, sh);
}

// One 8-wide node test: a node with hits becomes the current group (the
// group it replaces, if it still has slots, goes on the stack as (node,
// remaining slots)); then the next hit slot is entered.  Entered leaves are
// not re-tested against a closer hit (their triangle tests are).
template <bool kAny>
__device__ __forceinline__ bool node_step8(const SceneDev& s, Trav& T, uint2* sh, uint32_t* err) {
  if (T.node >= 0) {
    ++T.n_nodes;
    const uint32_t m = node8_hits(s, T.node, T.r, kAny ? T.tmax : T.bt, T.sgn);
    if (m) {
      if (T.gmask) {
        if (T.sp >= kStackSize) {
          atomicOr(err, kErrStack);
          T.best = -1;
          T.occluded = true;
          return true;
        }
        st_push(sh, T, T.gnode, __uint_as_float(T.gmask));
      }
      T.gnode = T.node;
      T.gmask = m;
    }
    T.node = -1;
  }
  return advance8(s, T, sh);
}

// Stores a finished ray's result: the hit record (closest), the unoccluded
// light contribution (forward shadow rays) or the visibility flag (adjoint
// shadow rays).
template <int kMode>
__device__ __forceinline__ void trace_finish(const WfDev& w, const uint32_t* qsrc, uint32_t i, const Trav& T,
                                             const SceneDev& sd) {
  count_ray(sd, kMode != 0 ? 1 : 0, T.n_nodes, T.n_tests);
  if (kMode == 0) {
    const uint32_t slot = qsrc[i];
    w.hit[slot] = make_float4(__int_as_float(T.best), T.bt, T.bu, T.bv);
  } else if (kMode == 1) {
    if (!T.occluded) {
      const uint32_t slot = w.sh_meta[i].x;
      const float4 c = w.sh_c[i];
      float4 r = w.rad[slot];
      r.x += c.x;
      r.y += c.y;
      r.z += c.z;
      w.rad[slot] = r;
    }
  } else {
    w.sh_vis[i] = T.occluded ? 0u : 1u;
  }
}

// Persistent traversal: each warp fetches rays for its idle lanes with one
// atomic, then steps its lanes' traversals.
//  * 4- and 8-wide BVHs: every step is one unit of work per lane, a node
//    test or a single triangle test, and the warp runs one kind per step:
//    triangle tests when at least as many lanes wait at a triangle as at a
//    node, node tests otherwise (the other lanes sit the step out).  Letting
//    both kinds run in one step serialises the two code paths with most
//    lanes masked off in each.  The warp refetches once `steps` of its lanes
//    are idle (or all are); the lanes whose rays have ended store their
//    results then, together, rather than each in the step its ray ends
//    (with one or two lanes active).
//  * Binary BVH: rounds of `steps` node visits, whole leaves at a time, and a
//    refetch after each round.
// Closest hit takes queue `cur`'s slots in the order of `order` when given
// (the same slots reordered by bin), else in queue order.
template <int kMode, int kWidth>
__global__ void __launch_bounds__(kWfThreads, 8) wf_trace(const WfScene* tab, WfDev w, int cur, int steps,
                                                       int one_scene, const uint32_t* order, uint32_t* err) {
  constexpr bool kAny = kMode != 0;
  if (!kAny && blockIdx.x == 0 && threadIdx.x == 0) {
    w.cnt[cur ? 0 : 1] = 0;  // next queue, filled by the shading stage
    w.cnt[2] = 0;            // shadow queue
    w.cnt[4] = 0;            // shadow fetch counter
  }
  const uint32_t n = kAny ? w.cnt[2] : w.cnt[cur];
  const uint32_t* qsrc = order ? order : queue(w, cur);
  uint32_t* fetch = kAny ? &w.cnt[4] : &w.cnt[3];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int refill = min(max(steps, 1), 32);
  __shared__ uint2 s_stack[kShortStack * kWfThreads];
  uint2* sh = s_stack + threadIdx.x;
  Trav T;
  SceneDev sd = tab[0].s;
  int64_t item = -1;
  bool fin = false;      // wide BVHs: the lane's ray has ended, its result not yet stored
  bool drained = false;  // warp-uniform: the queue has no rays left
  for (;;) {
    if (fin) {  // results are stored at the refill, by all ended lanes together
      trace_finish<kMode>(w, qsrc, (uint32_t)item, T, sd);
      item = -1;
      fin = false;
    }
    const bool need = item < 0 && !drained;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      uint32_t base = 0;
      if ((int)lane == leader) base = atomicAdd(fetch, (uint32_t)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      drained = base + (uint32_t)__popc(m) >= n;
      const uint32_t i = base + (uint32_t)__popc(m & lt_mask);
      if (need && i < n) {
        item = i;
        // a launch over one scene skips the lookup of the ray's scene
        const uint32_t slot = kAny ? w.sh_meta[i].x : qsrc[i];
        if (!one_scene) sd = tab[state_scene(__float_as_uint(w.beta[slot].w))].s;
        if (kAny) {
          const float4 o = w.sh_o[i], d = w.sh_d[i];
          trav_init(T, xyz(o), xyz(d), d.w, __float_as_int(o.w), (int)w.sh_meta[i].y);
        } else {
          const float4 o = w.ray_o[slot], d = w.ray_d[slot];
          trav_init(T, xyz(o), xyz(d), __int_as_float(0x7f800000), __float_as_int(o.w), -1);
        }
      }
    }
    if (__all_sync(0xffffffffu, item < 0)) break;
    if constexpr (kWidth == 2) {
      if (item >= 0 && trav_run2<kAny>(sd, T, sh, steps, err)) {
        trace_finish<kMode>(w, qsrc, (uint32_t)item, T, sd);
        item = -1;
      }
    } else {
      for (;;) {
        const bool live = item >= 0 && !fin;
        const bool at_tri = live && T.tri < T.tri_end;
        const unsigned ml = __ballot_sync(0xffffffffu, live);
        const unsigned mt = __ballot_sync(0xffffffffu, at_tri);
        if (ml == 0u || (!drained && 32 - __popc(ml) >= refill)) break;
        const bool tri_phase = __popc(mt) >= __popc(ml & ~mt);
        if (live && at_tri == tri_phase)
          fin = at_tri        ? tri_step<kAny, kWidth>(sd, T, sh)
                : kWidth == 8 ? node_step8<kAny>(sd, T, sh, err)
                              : node_step4<kAny>(sd, T, sh, err);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Forward shading of queue `cur`.
// ---------------------------------------------------------------------------
// The shading and adjoint stages ask for 8 resident blocks of 128 threads per
// SM (at most 64 registers, a few bytes spilled): they wait on scattered
// path-state loads, and the extra warps hide more of that latency.
// kD: the Disney material model (sampler, BRDF and NEE pdf) in place of
// Lambert + GGX; the rest of the stage is shared.
template <bool kD>
__global__ void __launch_bounds__(kWfThreads, 8) wf_shade_fwd(const WfScene* tab, WfParams lp, uint32_t p0,
                                                           WfDev w, int cur) {
  if (blockIdx.x == 0 && threadIdx.x == 0) w.cnt[3] = 0;  // closest fetch counter of the next vertex
  const uint32_t n = w.cnt[cur];
  const uint32_t si = set_iter(lp);
  uint32_t* qin = queue(w, cur);
  uint32_t* qout = queue(w, cur ^ 1);
  uint32_t* nout = &w.cnt[cur ^ 1];
  for (uint32_t q0 = blockIdx.x * blockDim.x; q0 < n; q0 += gridDim.x * blockDim.x) {
    const uint32_t q = q0 + threadIdx.x;
    const bool act = q < n;
    const uint32_t slot = act ? qin[q] : 0u;
    const float4 hh = act ? w.hit[slot] : make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
    const int tri = __float_as_int(hh.x);
    const float4 bt = act ? w.beta[slot] : make_float4(0.f, 0.f, 0.f, __uint_as_float(kDead));
    const uint32_t st = __float_as_uint(bt.w);
    const uint32_t k = state_k(st), b = state_scene(st);
    bool cont = false, shadow = false, query = false, record = false;
    uint32_t path_id = 0;
    NeeResult ne;
    float3 shc = f3(0.f, 0.f, 0.f);
    float3 beta = xyz(bt), wo = f3(0.f, 0.f, 0.f), org = f3(0.f, 0.f, 0.f);
    float pdf = 0.0f;
    Vtx v;
    if (tri >= 0) {
      const WfScene& e = tab[lp.n_scenes == 1 ? 0u : b];
      const double W = *e.t.W;
      const bool light_on = lp.nee && W > 0.0;
      const float4 rd = w.ray_d[slot];
      Hit h;
      h.tri = tri;
      h.t = hh.y;
      h.u = hh.z;
      h.v = hh.w;
      v = make_vertex(e.s, h, xyz(rd), lp.profile);
      // a training pass gathers only what the path finds after the cache vertex
      const bool gather = !lp.cache_record || k > lp.cache_k;
      if (v.prof > 0.0f && gather) {
        const float wb = emission_weight(e.t, v, h.t, k > 0, light_on, rd.w, lp.mis);
        if (wb > 0.0f) {
          const float3 L = beta * xyz(__ldg(&e.t.emis[v.seg])) * (wb * v.prof);
          const float4 r = w.rad[slot];
          w.rad[slot] = make_float4(r.x + L.x, r.y + L.y, r.z + L.z, 0.0f);
        }
      }
      if (k < lp.max_depth && k == lp.cache_k && !lp.cache_record) {
        query = true;  // the cache supplies the reflected radiance from here
      } else if (k < lp.max_depth) {
        if (k == lp.cache_k) {
          record = true;  // training record; the target is gathered with unit throughput
          beta = f3(1.0f, 1.0f, 1.0f);
        }
        uint32_t pid, smp, ent;
        slot_pixel(e, p0, slot, lp.spp, lp.stride, pid, smp, ent);
        path_id = pid * lp.spp + smp;
        const PathRng rng = path_rng(e, pid, smp, si);
        const float4 ua = rng.draw(k, 0), ub = rng.draw(k, 1);
        if constexpr (kD) {
          float3 X, Y;
          hit_frame(e.s, tri, v.ns, X, Y);
          float m[kDisneyMat];
          load_disney(e.dis, v.seg, m);
          if (light_on) {
            ne = nee_prepare_with(e.s, e.t, v, ua, ub, W, lp.profile, lp.mis,
                                  [&](float3 wl) { return disney_pdf(e.dis, v.seg, v.ns, X, Y, v.wi, wl); });
            if (ne.valid) {
              shc = beta * disney_eval(m, v.ns, X, Y, v.wi, ne.wl) * xyz(__ldg(&e.t.emis[ne.seg])) * ne.k;
              shadow = true;
            }
          }
          if (dot(v.wi, v.ns) > 0.0f) {
            wo = disney_sample(e.dis, v.seg, v.ns, X, Y, v.wi, ua.x, ua.y, ua.z);
            pdf = disney_pdf(e.dis, v.seg, v.ns, X, Y, v.wi, wo);
            const float co = dot(wo, v.ns);
            if (dot(wo, v.ng) > 0.0f && co > 0.0f && pdf > 0.0f) {
              beta = beta * disney_eval(m, v.ns, X, Y, v.wi, wo) * (co / pdf);
              org = v.x + v.ng * e.s.eps;
              cont = true;
            }
          }
        } else {
          const float4 ma = __ldg(&e.t.mat_a[v.seg]), mb = __ldg(&e.t.mat_b[v.seg]);
          const float4 sa = __ldg(&e.t.samp[v.seg]);
          if (light_on && (!lp.cache_record || k >= lp.cache_k)) {
            ne = nee_prepare(e.s, e.t, v, ua, ub, W, lp.profile, lp.mis, sa.y, sa.x);
            if (ne.valid) {
              const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, ne.wl);
              shc = beta * bv.f * xyz(__ldg(&e.t.emis[ne.seg])) * ne.k;
              shadow = true;
            }
          }
          if (dot(v.wi, v.ns) > 0.0f) {
            wo = bsdf_sample(__ldg(&e.t.pspec[v.seg]), sa.x, v.ns, v.wi, ua.x, ua.y, ua.z);
            pdf = bsdf_pdf(sa.y, sa.x, v.ns, v.wi, wo);
            const float co = dot(wo, v.ns);
            if (dot(wo, v.ng) > 0.0f && co > 0.0f && pdf > 0.0f) {
              const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, wo);
              beta = beta * bv.f * (co / pdf);
              org = v.x + v.ng * e.s.eps;
              cont = true;
            }
          }
        }
      }
    }
    if (lp.cache_k != kNoCache) {
      const uint32_t qi = enqueue(&lp.cb.counts[0], query);
      if (query) {
        lp.cb.q.x[qi] = make_float4(v.x.x, v.x.y, v.x.z, __int_as_float(v.seg));
        lp.cb.q.d[qi] = make_float4(v.wi.x, v.wi.y, v.wi.z, __uint_as_float(slot));
        lp.cb.q.n[qi] = make_float4(v.ns.x, v.ns.y, v.ns.z, 0.0f);
        lp.cb.q.u[qi] = make_float4(beta.x, beta.y, beta.z, 0.0f);
      }
      const uint32_t ri = enqueue(&lp.cb.counts[1], record);
      if (record && ri < lp.cb.r_cap) {
        lp.cb.r.x[ri] = make_float4(v.x.x, v.x.y, v.x.z, __int_as_float(v.seg));
        lp.cb.r.d[ri] = make_float4(v.wi.x, v.wi.y, v.wi.z, __uint_as_float(slot));
        lp.cb.r.n[ri] = make_float4(v.ns.x, v.ns.y, v.ns.z, __uint_as_float(path_id));
      }
    }
    const uint32_t sq = enqueue(&w.cnt[2], shadow);
    if (shadow) {
      w.sh_o[sq] = make_float4(ne.so.x, ne.so.y, ne.so.z, __int_as_float(tri));
      w.sh_d[sq] = make_float4(ne.sd.x, ne.sd.y, ne.sd.z, ne.st);
      w.sh_meta[sq] = make_uint4(slot, (uint32_t)ne.tri, 0u, (uint32_t)ne.seg);
      w.sh_c[sq] = make_float4(shc.x, shc.y, shc.z, 0.0f);
    }
    const uint32_t ci = enqueue(nout, cont);
    if (cont) {
      qout[ci] = slot;
      if (lp.keys) lp.keys[ci] = (uint16_t)ray_bin(lp.bin, tab[lp.n_scenes == 1 ? 0u : b], b, org, wo);
      w.ray_o[slot] = make_float4(org.x, org.y, org.z, __int_as_float(tri));
      w.ray_d[slot] = make_float4(wo.x, wo.y, wo.z, pdf);
      w.beta[slot] = make_float4(beta.x, beta.y, beta.z, __uint_as_float(pack_state(k + 1, b)));
    }
  }
}

// Per-pixel reduction of a chunk: mean (and mean of squares) into the
// scene's optional outputs, or the residual of its target and the scene's
// loss, accumulated per block (rows[block * n_scenes + scene]).
__global__ void __launch_bounds__(kWfThreads) wf_reduce(const WfScene* tab, WfParams lp, uint32_t p0,
                                                        uint32_t n_pix, WfDev w, double* rows, int first_chunk) {
  extern __shared__ double sloss[];
  for (uint32_t i = threadIdx.x; i < lp.n_scenes; i += blockDim.x) sloss[i] = 0.0;
  __syncthreads();
  const float inv = 1.0f / (float)lp.spp;
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n_pix; l += gridDim.x * blockDim.x) {
    float3 a = f3(0.f, 0.f, 0.f), a2 = f3(0.f, 0.f, 0.f);
    for (uint32_t smp = 0; smp < lp.spp; ++smp) {
      const float3 L = xyz(w.rad[l * lp.spp + smp]);
      a = a + L;
      a2 = a2 + L * L;
    }
    const uint32_t b = state_scene(__float_as_uint(w.beta[l * lp.spp].w));
    const WfScene& e = tab[b];
    const uint32_t ent = p0 + l - e.pix_begin + e.pix_base;
    const uint32_t pid = e.pick ? e.pick[ent] : ent;
    const uint32_t o = ent - e.pix_base;
    const float3 mean = a * inv;
    if (e.img) {
      e.img[3 * o + 0] = mean.x;
      e.img[3 * o + 1] = mean.y;
      e.img[3 * o + 2] = mean.z;
    }
    if (e.msq) {
      e.msq[3 * o + 0] = a2.x * inv;
      e.msq[3 * o + 1] = a2.y * inv;
      e.msq[3 * o + 2] = a2.z * inv;
    }
    if (e.target) {
      const float r[3] = {mean.x - e.target[3 * pid], mean.y - e.target[3 * pid + 1],
                          mean.z - e.target[3 * pid + 2]};
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (lp.loss_kind == 0) {
          e.g_img[3 * ent + c] = 2.0f * r[c] * e.g_scale;
          acc += (double)r[c] * (double)r[c];
        } else {
          e.g_img[3 * ent + c] = (r[c] > 0.0f ? 1.0f : (r[c] < 0.0f ? -1.0f : 0.0f)) * e.g_scale;
          acc += fabs((double)r[c]);
        }
      }
      atomicAdd(&sloss[b], acc);
    }
  }
  __syncthreads();
  if (rows)
    for (uint32_t i = threadIdx.x; i < lp.n_scenes; i += blockDim.x) {
      double* r = &rows[(size_t)blockIdx.x * lp.n_scenes + i];
      *r = first_chunk ? sloss[i] : *r + sloss[i];
    }
}

// ---------------------------------------------------------------------------
// Adjoint stages.  Shared accumulators cover segments [seg_lo, seg_lo + seg_n)
// of the launch's concatenated segment space: P values per segment (10, or
// 16 for the Disney model) at a stride of P + 1 floats, an odd stride, so
// that lanes adding parameter j of different segments fall in different
// banks (at stride 10 only 16 of the 32 banks are reachable for a given j;
// at 16, two).  Global accumulators and the per-block gradient rows keep
// stride P.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr uint32_t acc_shared_floats(uint32_t P, uint32_t seg_n) { return (P + 1u) * seg_n; }

__device__ __forceinline__ void acc_zero(float* sacc, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sacc[i] = 0.0f;
  __syncthreads();
}

// Adds the block's shared accumulators (stride P + 1) to its gradient row
// (np = P * seg_n values, stride P).
template <uint32_t P>
__device__ __forceinline__ void acc_flush(const float* sacc, uint32_t np, float* blk) {
  __syncthreads();
  float* row = blk + (size_t)blockIdx.x * np;
  for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) {
    const float v = sacc[(i / P) * (P + 1u) + i % P];
    if (v != 0.0f) row[i] += v;
  }
}

// Warp-aggregated scatter: adds v[0..N) to acc[base + j] for every lane whose
// base is >= 0.  All 32 lanes of the warp call it together.  When every
// contributing lane targets the same parameters (the same segment of the
// same scene: a warp holds samples of one pixel, which mostly see the same
// surface), the values are summed by a shuffle butterfly and one lane adds
// the N sums; otherwise each lane adds its own values.  (Grouping lanes by
// target with __match_any_sync and reducing every group was measured slower:
// its shuffles cost more than the atomics they save in these latency-bound
// stages; so was reducing only the lanes that share the first lane's
// target.)
template <int N>
__device__ __forceinline__ void warp_scatter(float* acc, int base, const float (&v)[N]) {
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned want = __ballot_sync(0xffffffffu, base >= 0);
  if (!want) return;
  const int b0 = __shfl_sync(0xffffffffu, base, __ffs(want) - 1);
  if (__popc(want) > 1 && __all_sync(0xffffffffu, base < 0 || base == b0)) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float x = base >= 0 ? v[j] : 0.0f;
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if (lane == 0 && x != 0.0f) atomicAdd(&acc[b0 + j], x);
    }
  } else if (base >= 0) {
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (v[j] != 0.0f) atomicAdd(&acc[base + j], v[j]);
  }
}

__device__ __forceinline__ void warp_scatter3(float* acc, int base, float3 a) {
  const float v[3] = {a.x, a.y, a.z};
  warp_scatter<3>(acc, base, v);
}

// Accumulator index of parameter j of segment `seg` of scene entry e.
__device__ __forceinline__ int acc_ix(const WfScene& e, const WfParams& lp, int seg, int j) {
  return (lp.gacc ? 10 : 11) * ((int)e.seg_offset + seg - (int)lp.seg_lo) + j;
}

__device__ __forceinline__ float3 pixel_grad(const WfScene& e, uint32_t entry, float inv_spp) {
  return f3(e.g_img[3 * entry], e.g_img[3 * entry + 1], e.g_img[3 * entry + 2]) * inv_spp;
}

// The same for the Disney model's 16 values per segment.
__device__ __forceinline__ int acc_ix16(const WfScene& e, const WfParams& lp, int seg, int j) {
  return (lp.gacc ? kDisneyStride : kDisneyStride + 1) * ((int)e.seg_offset + seg - (int)lp.seg_lo) + j;
}


// Continuation terms of the paths that finish: (dw_l / dtheta) . (g * U_l)
// for every vertex l.  All 32 lanes call it; lanes with act = false (or with
// fewer vertices) add nothing, and the sums go through warp_scatter.  The
// Disney model rebuilds vertex l (shading normal, tangent frame) from its
// stored triangle, barycentrics and directions and contracts the BRDF
// Jacobian there with g * U_l * cos/pdf.
template <bool kD>
__device__ __forceinline__ void finish_path(const WfDev& w, const WfScene* e, const WfParams& lp, uint32_t slot,
                                            uint32_t nv_slot, float3 gp, float* sacc, bool act) {
  const uint32_t nv = act ? nv_slot : 0u;
  const uint32_t nmax = __reduce_max_sync(0xffffffffu, nv);
  for (uint32_t l = 0; l < nmax; ++l) {
    if constexpr (kD) {
      float g[kDisneyMat];
      int base = -1;
      if (l < nv) {
        const size_t ix = (size_t)l * w.cap + slot;
        const float4 T = w.aT[ix], U = w.aU[ix], Wi = w.aWi[ix], Wo = w.aWo[ix];
        const float2 R = w.aR[ix];
        const float3 q = gp * xyz(U) * T.w;
        if (q.x != 0.0f || q.y != 0.0f || q.z != 0.0f) {
          Hit h;
          h.tri = __float_as_int(Wi.w);
          h.t = 0.0f;
          h.u = R.x;
          h.v = Wo.w;
          const Vtx v = make_vertex(e->s, h, -xyz(Wi), lp.profile);
          float3 X, Y;
          hit_frame(e->s, h.tri, v.ns, X, Y);
          const int sg = __float_as_int(R.y);
          float m[kDisneyMat];
          load_disney(e->dis, sg, m);
          if (disney_vjp(m, v.ns, X, Y, xyz(Wi), xyz(Wo), q, g)) base = acc_ix16(*e, lp, sg, 0);
        }
      }
      if (base < 0)
        for (int j = 0; j < kDisneyMat; ++j) g[j] = 0.0f;
      warp_scatter<kDisneyMat>(sacc, base, g);
    } else {
      float g[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      int base = -1;
      if (l < nv) {
        const size_t ix = (size_t)l * w.cap + slot;
        const float4 T = w.aT[ix], U = w.aU[ix];
        const float2 R = w.aR[ix];
        const int sg = __float_as_int(R.y);
        const float3 q = gp * xyz(U);
        const float4 mb = __ldg(&e->t.mat_b[sg]);
        g[0] = q.x * T.w;
        g[1] = q.y * T.w;
        g[2] = q.z * T.w;
        g[3] = q.x * U.w;
        g[4] = q.y * U.w;
        g[5] = q.z * U.w;
        g[6] = dot(q, f3(mb.x, mb.y, mb.z)) * R.x;
        base = acc_ix(*e, lp, sg, 0);
      }
      warp_scatter<7>(sacc, base, g);
    }
  }
}

// U_l += T_l * C for the path's nv earlier vertices.  The carry is read in
// groups of kG vertices whose loads are all issued before the first use
// (the stages are latency-bound; nv <= kMaxAdjointDepth).  Stages short of
// registers take smaller groups.
template <uint32_t kG>
__device__ __forceinline__ void add_to_carry(const WfDev& w, uint32_t slot, uint32_t nv, float3 C) {
#pragma unroll
  for (uint32_t l0 = 0; l0 < (uint32_t)kMaxAdjointDepth; l0 += kG) {
    if (l0 >= nv) break;
    float4 T[kG], U[kG];
#pragma unroll
    for (uint32_t j = 0; j < kG; ++j)
      if (l0 + j < nv) {
        const size_t ix = (size_t)(l0 + j) * w.cap + slot;
        T[j] = w.aT[ix];
        U[j] = w.aU[ix];
      }
#pragma unroll
    for (uint32_t j = 0; j < kG; ++j)
      if (l0 + j < nv) {
        U[j].x += T[j].x * C.x;
        U[j].y += T[j].y * C.y;
        U[j].z += T[j].z * C.z;
        w.aU[(size_t)(l0 + j) * w.cap + slot] = U[j];
      }
  }
}

// T_l *= wgt for the path's nv earlier vertices (the new vertex's BSDF
// weight joins their throughputs), loads grouped as in add_to_carry.
__device__ __forceinline__ void scale_carry(const WfDev& w, uint32_t slot, uint32_t nv, float3 wgt) {
#pragma unroll
  for (uint32_t l0 = 0; l0 < (uint32_t)kMaxAdjointDepth; l0 += 4) {
    if (l0 >= nv) break;
    float4 T[4];
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j)
      if (l0 + j < nv) T[j] = w.aT[(size_t)(l0 + j) * w.cap + slot];
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j)
      if (l0 + j < nv) {
        T[j].x *= wgt.x;
        T[j].y *= wgt.y;
        T[j].z *= wgt.z;
        w.aT[(size_t)(l0 + j) * w.cap + slot] = T[j];
      }
  }
}

// Stage A: emission at the vertex, its contribution to the carry, and the
// next-event candidate (with, for the Disney model, the material derivative
// of its term, added if the shadow ray finds the light).
template <bool kD>
__global__ void __launch_bounds__(kWfThreads, 8) wf_adj_a(const WfScene* tab, WfParams lp, uint32_t p0, WfDev w,
                                                       int cur) {
  extern __shared__ float sacc_sh[];
  float* sacc = lp.gacc ? lp.gacc : sacc_sh;
  const uint32_t np = (kD ? 16u : 10u) * lp.seg_n;
  if (!lp.gacc) acc_zero(sacc, acc_shared_floats(kD ? 16u : 10u, lp.seg_n));
  const uint32_t n = w.cnt[cur];
  const uint32_t si = set_iter(lp);
  const float inv_spp = 1.0f / (float)lp.spp;
  uint32_t* qin = queue(w, cur);
  // warp-uniform trip count: every lane reaches the warp-collective scatters
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t q0 = blockIdx.x * blockDim.x + threadIdx.x - lane; q0 < n; q0 += gridDim.x * blockDim.x) {
    const uint32_t q = q0 + lane;
    const bool act = q < n;
    const uint32_t slot = act ? qin[q] : 0u;
    float4 hh = make_float4(__int_as_float(-1), 0.f, 0.f, 0.f), bt = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 rd = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t nv = 0;
    if (act) {  // the slot's state, all loads issued together
      hh = w.hit[slot];
      bt = w.beta[slot];
      rd = w.ray_d[slot];
      nv = w.nv[slot];
    }
    const int tri = __float_as_int(hh.x);
    const uint32_t st = __float_as_uint(bt.w);
    const uint32_t k = state_k(st), b = state_scene(st);
    const WfScene& e = tab[lp.n_scenes == 1 ? 0u : b];
    uint32_t pid = 0, smp = 0, ent = 0;
    float3 gp = f3(0.f, 0.f, 0.f);
    if (act) {
      slot_pixel(e, p0, slot, lp.spp, lp.stride, pid, smp, ent);
      gp = pixel_grad(e, ent, inv_spp);
    }
    bool shadow = false, query = false, finish = false;
    NeeResult ne;
    float3 ge = f3(0.f, 0.f, 0.f), gm = f3(0.f, 0.f, 0.f), cn = f3(0.f, 0.f, 0.f);
    float spec = 0.0f, dsdr = 0.0f;
    float gd[kDisneyMat];
    int vseg = 0;
    int ebase = -1;  // accumulator of the emission found here
    float3 ev = f3(0.f, 0.f, 0.f);
    float4 cq = make_float4(0.f, 0.f, 0.f, 0.f);
    Vtx cv;
    if (!act) {
    } else if (tri < 0) {
      finish = true;
      w.beta[slot] = make_float4(bt.x, bt.y, bt.z, __uint_as_float(st | kDead));
    } else {
      const double W = *e.t.W;
      const bool light_on = lp.nee && W > 0.0;
      const float3 beta = xyz(bt);
      Hit h;
      h.tri = tri;
      h.t = hh.y;
      h.u = hh.z;
      h.v = hh.w;
      const Vtx v = make_vertex(e.s, h, xyz(rd), lp.profile);
      vseg = v.seg;
      if (v.prof > 0.0f) {
        const float wb = emission_weight(e.t, v, h.t, k > 0, light_on, rd.w, lp.mis);
        if (wb > 0.0f) {
          const float f = wb * v.prof;
          add_to_carry<2>(w, slot, nv, xyz(__ldg(&e.t.emis[v.seg])) * f);
          ebase = kD ? acc_ix16(e, lp, v.seg, kDisneyMat) : acc_ix(e, lp, v.seg, 7);
          ev = gp * beta * (f * e.es);
        }
      }
      if (k == lp.max_depth) {
        finish = true;
        w.beta[slot] = make_float4(bt.x, bt.y, bt.z, __uint_as_float(st | kDead));
      } else if (k == lp.cache_k) {
        // the cache's prediction and its parameter derivative close the path
        query = true;
        const float3 u = gp * beta;
        cq = make_float4(u.x, u.y, u.z, 0.0f);
        cv = v;
      } else if (light_on) {
        const PathRng rng = path_rng(e, pid, smp, si);
        const float4 ua = rng.draw(k, 0), ub = rng.draw(k, 1);
        if constexpr (kD) {
          float3 X, Y;
          hit_frame(e.s, tri, v.ns, X, Y);
          ne = nee_prepare_with(e.s, e.t, v, ua, ub, W, lp.profile, lp.mis,
                                [&](float3 wl) { return disney_pdf(e.dis, v.seg, v.ns, X, Y, v.wi, wl); });
          if (ne.valid) {
            float m[kDisneyMat];
            load_disney(e.dis, v.seg, m);
            const float3 fv = disney_eval(m, v.ns, X, Y, v.wi, ne.wl);
            const float3 Le = xyz(__ldg(&e.t.emis[ne.seg]));
            ge = gp * beta * fv * (ne.k * e.es);
            cn = fv * Le * ne.k;
            if (!disney_vjp(m, v.ns, X, Y, v.wi, ne.wl, gp * beta * Le * ne.k, gd))
              for (int j = 0; j < kDisneyMat; ++j) gd[j] = 0.0f;
            shadow = true;
          }
        } else {
          const float4 sa = __ldg(&e.t.samp[v.seg]);
          ne = nee_prepare(e.s, e.t, v, ua, ub, W, lp.profile, lp.mis, sa.y, sa.x);
          if (ne.valid) {
            const float4 ma = __ldg(&e.t.mat_a[v.seg]), mb = __ldg(&e.t.mat_b[v.seg]);
            const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, ne.wl);
            const float3 Le = xyz(__ldg(&e.t.emis[ne.seg]));
            ge = gp * beta * bv.f * (ne.k * e.es);
            gm = gp * beta * Le * ne.k;
            cn = bv.f * Le * ne.k;
            spec = bv.sp.s;
            dsdr = bv.sp.ds_dr;
            shadow = true;
          }
        }
      }
    }
    warp_scatter3(sacc, ebase, ev);
    finish_path<kD>(w, &e, lp, slot, nv, gp, sacc, finish);
    if (lp.cache_k != kNoCache) {
      const uint32_t qi = enqueue(&lp.cb.counts[0], query);
      if (query) {
        lp.cb.q.x[qi] = make_float4(cv.x.x, cv.x.y, cv.x.z, __int_as_float(cv.seg));
        lp.cb.q.d[qi] = make_float4(cv.wi.x, cv.wi.y, cv.wi.z, __uint_as_float(slot));
        lp.cb.q.n[qi] = make_float4(cv.ns.x, cv.ns.y, cv.ns.z, 0.0f);
        lp.cb.q.u[qi] = cq;
      }
    }
    const uint32_t sq = enqueue(&w.cnt[2], shadow);
    if (shadow) {
      w.sh_o[sq] = make_float4(ne.so.x, ne.so.y, ne.so.z, __int_as_float(tri));
      w.sh_d[sq] = make_float4(ne.sd.x, ne.sd.y, ne.sd.z, ne.st);
      w.sh_meta[sq] = make_uint4(slot, (uint32_t)ne.tri, (uint32_t)vseg, (uint32_t)ne.seg);
      w.sh_ge[sq] = make_float4(ge.x, ge.y, ge.z, 0.0f);
      w.sh_gm[sq] = make_float4(gm.x, gm.y, gm.z, spec);
      w.sh_n[sq] = make_float4(cn.x, cn.y, cn.z, dsdr);
      if constexpr (kD) {
        float4* dv = w.sh_dv + 4 * (size_t)sq;
        dv[0] = make_float4(gd[0], gd[1], gd[2], gd[3]);
        dv[1] = make_float4(gd[4], gd[5], gd[6], gd[7]);
        dv[2] = make_float4(gd[8], gd[9], gd[10], gd[11]);
        dv[3] = make_float4(gd[12], 0.0f, 0.0f, 0.0f);
      }
    }
  }
  if (!lp.gacc) acc_flush<kD ? 16u : 10u>(sacc, np, w.blk);
}

// Unoccluded next-event terms: light emission (Eq. 5), the vertex material
// (Eq. 6 at this vertex) and the carry of the earlier vertices.  A launch
// over one scene skips reading the slot's state word for its scene.
template <bool kD>
__global__ void __launch_bounds__(kWfThreads) wf_adj_connect(const WfScene* tab, WfParams lp, WfDev w) {
  extern __shared__ float sacc_sh[];
  float* sacc = lp.gacc ? lp.gacc : sacc_sh;
  const uint32_t np = (kD ? 16u : 10u) * lp.seg_n;
  if (!lp.gacc) acc_zero(sacc, acc_shared_floats(kD ? 16u : 10u, lp.seg_n));
  const uint32_t n = w.cnt[2];
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x - lane; i0 < n; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + lane;
    const bool vis = i < n && w.sh_vis[i];
    int lbase = -1, mbase = -1;  // accumulators of the light's emission and the vertex material
    float3 ge3 = f3(0.f, 0.f, 0.f);
    if constexpr (kD) {
      float g[kDisneyMat];
      for (int j = 0; j < kDisneyMat; ++j) g[j] = 0.0f;
      if (vis) {
        const uint4 m = w.sh_meta[i];
        const WfScene& e = tab[lp.n_scenes == 1 ? 0u : state_scene(__float_as_uint(w.beta[m.x].w))];
        const float4 ge = w.sh_ge[i], cn = w.sh_n[i];
        lbase = acc_ix16(e, lp, (int)m.w, kDisneyMat);
        ge3 = xyz(ge);
        const float4* dv = w.sh_dv + 4 * (size_t)i;
        const float4 d0 = dv[0], d1 = dv[1], d2 = dv[2], d3 = dv[3];
        const float gg[kDisneyMat] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w, d2.x, d2.y, d2.z, d2.w, d3.x};
        for (int j = 0; j < kDisneyMat; ++j) g[j] = gg[j];
        mbase = acc_ix16(e, lp, (int)m.z, 0);
        add_to_carry<4>(w, m.x, w.nv[m.x], xyz(cn));
      }
      warp_scatter3(sacc, lbase, ge3);
      warp_scatter<kDisneyMat>(sacc, mbase, g);
      continue;
    }
    float g[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (vis) {
      const uint4 m = w.sh_meta[i];
      const WfScene& e = tab[lp.n_scenes == 1 ? 0u : state_scene(__float_as_uint(w.beta[m.x].w))];
      const float4 ge = w.sh_ge[i], gm = w.sh_gm[i], cn = w.sh_n[i];
      lbase = acc_ix(e, lp, (int)m.w, 7);
      ge3 = xyz(ge);
      const float3 q = xyz(gm);
      const float4 mb = __ldg(&e.t.mat_b[m.z]);
      g[0] = q.x * (1.0f / kPi);
      g[1] = q.y * (1.0f / kPi);
      g[2] = q.z * (1.0f / kPi);
      g[3] = q.x * gm.w;
      g[4] = q.y * gm.w;
      g[5] = q.z * gm.w;
      g[6] = dot(q, f3(mb.x, mb.y, mb.z)) * cn.w;
      mbase = acc_ix(e, lp, (int)m.z, 0);
      add_to_carry<4>(w, m.x, w.nv[m.x], xyz(cn));
    }
    warp_scatter3(sacc, lbase, ge3);
    warp_scatter<7>(sacc, mbase, g);
  }
  if (!lp.gacc) acc_flush<kD ? 16u : 10u>(sacc, np, w.blk);
}

// Stage B: BRDF sampling; the new vertex joins the carry.
template <bool kD>
__global__ void __launch_bounds__(kWfThreads, 8) wf_adj_b(const WfScene* tab, WfParams lp, uint32_t p0, WfDev w,
                                                       int cur) {
  extern __shared__ float sacc_sh[];
  float* sacc = lp.gacc ? lp.gacc : sacc_sh;
  const uint32_t np = (kD ? 16u : 10u) * lp.seg_n;
  if (!lp.gacc) acc_zero(sacc, acc_shared_floats(kD ? 16u : 10u, lp.seg_n));
  if (blockIdx.x == 0 && threadIdx.x == 0) w.cnt[3] = 0;
  const uint32_t n = w.cnt[cur];
  const uint32_t si = set_iter(lp);
  const float inv_spp = 1.0f / (float)lp.spp;
  uint32_t* qin = queue(w, cur);
  uint32_t* qout = queue(w, cur ^ 1);
  uint32_t* nout = &w.cnt[cur ^ 1];
  // warp-uniform trip count: every lane reaches the warp-collective scatters
  for (uint32_t q0 = blockIdx.x * blockDim.x; q0 < n; q0 += gridDim.x * blockDim.x) {
    const uint32_t q = q0 + threadIdx.x;
    const bool act = q < n;
    const uint32_t slot = act ? qin[q] : 0u;
    // the slot's state, all loads issued together
    float4 bt = make_float4(0.f, 0.f, 0.f, __uint_as_float(kDead)), hh = bt, rd = bt;
    uint32_t nv = 0;
    if (act) {
      bt = w.beta[slot];
      hh = w.hit[slot];
      rd = w.ray_d[slot];
      nv = w.nv[slot];
    }
    const uint32_t st = __float_as_uint(bt.w);
    bool cont = false, finish = false;
    float3 org = f3(0.f, 0.f, 0.f), wo = f3(0.f, 0.f, 0.f), beta = xyz(bt);
    float pdf = 0.0f;
    int tri = -1;
    const uint32_t k = state_k(st), b = state_scene(st);
    const WfScene& e = tab[lp.n_scenes == 1 ? 0u : b];
    float3 gfin = f3(0.f, 0.f, 0.f);
    if (!(st & kDead)) {
      tri = __float_as_int(hh.x);
      Hit h;
      h.tri = tri;
      h.t = hh.y;
      h.u = hh.z;
      h.v = hh.w;
      const Vtx v = make_vertex(e.s, h, xyz(rd), lp.profile);
      uint32_t pid, smp, ent;
      slot_pixel(e, p0, slot, lp.spp, lp.stride, pid, smp, ent);
      const PathRng rng = path_rng(e, pid, smp, si);
      const float4 ua = rng.draw(k, 0);
      if constexpr (kD) {
        if (dot(v.wi, v.ns) > 0.0f) {
          float3 X, Y;
          hit_frame(e.s, tri, v.ns, X, Y);
          wo = disney_sample(e.dis, v.seg, v.ns, X, Y, v.wi, ua.x, ua.y, ua.z);
          pdf = disney_pdf(e.dis, v.seg, v.ns, X, Y, v.wi, wo);
          const float co = dot(wo, v.ns);
          if (dot(wo, v.ng) > 0.0f && co > 0.0f && pdf > 0.0f) {
            float m[kDisneyMat];
            load_disney(e.dis, v.seg, m);
            const float kk = co / pdf;
            const float3 wgt = disney_eval(m, v.ns, X, Y, v.wi, wo) * kk;
            scale_carry(w, slot, nv, wgt);
            const size_t ix = (size_t)nv * w.cap + slot;
            w.aT[ix] = make_float4(beta.x, beta.y, beta.z, kk);
            w.aU[ix] = make_float4(0.f, 0.f, 0.f, 0.f);
            w.aR[ix] = make_float2(h.u, __int_as_float(v.seg));
            w.aWi[ix] = make_float4(v.wi.x, v.wi.y, v.wi.z, __int_as_float(tri));
            w.aWo[ix] = make_float4(wo.x, wo.y, wo.z, h.v);
            w.nv[slot] = nv + 1;
            beta = beta * wgt;
            org = v.x + v.ng * e.s.eps;
            cont = true;
          }
        }
      } else if (dot(v.wi, v.ns) > 0.0f) {
        const float4 sa = __ldg(&e.t.samp[v.seg]);
        wo = bsdf_sample(__ldg(&e.t.pspec[v.seg]), sa.x, v.ns, v.wi, ua.x, ua.y, ua.z);
        pdf = bsdf_pdf(sa.y, sa.x, v.ns, v.wi, wo);
        const float co = dot(wo, v.ns);
        if (dot(wo, v.ng) > 0.0f && co > 0.0f && pdf > 0.0f) {
          const float4 ma = __ldg(&e.t.mat_a[v.seg]), mb = __ldg(&e.t.mat_b[v.seg]);
          const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, wo);
          const float kk = co / pdf;
          const float3 wgt = bv.f * kk;
          scale_carry(w, slot, nv, wgt);
          const size_t ix = (size_t)nv * w.cap + slot;
          w.aT[ix] = make_float4(beta.x, beta.y, beta.z, kk * (1.0f / kPi));
          w.aU[ix] = make_float4(0.f, 0.f, 0.f, kk * bv.sp.s);
          w.aR[ix] = make_float2(kk * bv.sp.ds_dr, __int_as_float(v.seg));
          w.nv[slot] = nv + 1;
          beta = beta * wgt;
          org = v.x + v.ng * e.s.eps;
          cont = true;
        }
      }
      if (!cont) {
        finish = true;
        gfin = pixel_grad(e, ent, inv_spp);
        w.beta[slot] = make_float4(bt.x, bt.y, bt.z, __uint_as_float(st | kDead));
      }
    }
    finish_path<kD>(w, &e, lp, slot, nv, gfin, sacc, finish);
    const uint32_t ci = enqueue(nout, cont);
    if (cont) {
      qout[ci] = slot;
      if (lp.keys) lp.keys[ci] = (uint16_t)ray_bin(lp.bin, tab[lp.n_scenes == 1 ? 0u : b], b, org, wo);
      w.ray_o[slot] = make_float4(org.x, org.y, org.z, __int_as_float(tri));
      w.ray_d[slot] = make_float4(wo.x, wo.y, wo.z, pdf);
      w.beta[slot] = make_float4(beta.x, beta.y, beta.z, __uint_as_float(pack_state(k + 1, b)));
    }
  }
  if (!lp.gacc) acc_flush<kD ? 16u : 10u>(sacc, np, w.blk);
}

// Paths closed by the cache: its prediction joins the earlier vertices'
// carry (Eq. 6 through their BSDF factors), its parameter derivative goes to
// the terminal segment's kd, ks and roughness, and the path finishes.
__global__ void __launch_bounds__(kWfThreads) wf_adj_cache(const WfScene* tab, WfParams lp, uint32_t p0, WfDev w) {
  extern __shared__ float sacc_sh[];
  float* sacc = lp.gacc ? lp.gacc : sacc_sh;
  const uint32_t np = 10u * lp.seg_n;
  if (!lp.gacc) acc_zero(sacc, acc_shared_floats(10u, lp.seg_n));
  const uint32_t n = lp.cb.counts[0];
  const float inv_spp = 1.0f / (float)lp.spp;
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t q0 = blockIdx.x * blockDim.x + threadIdx.x - lane; q0 < n; q0 += gridDim.x * blockDim.x) {
    const uint32_t q = q0 + lane;
    const bool act = q < n;
    const uint32_t slot = act ? __float_as_uint(lp.cb.q.d[q].w) : 0u;
    const uint32_t st = act ? __float_as_uint(w.beta[slot].w) : 0u;
    const uint32_t nv = act ? w.nv[slot] : 0u;
    const WfScene& e = tab[lp.n_scenes == 1 ? 0u : state_scene(st)];
    float g[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int base = -1;
    float3 gp = f3(0.f, 0.f, 0.f);
    if (act) {
      const int seg = __float_as_int(lp.cb.q.x[q].w);
      add_to_carry<2>(w, slot, nv, xyz(lp.cb.qc[q]));
      const float* dp = lp.cb.qdp + 8 * (size_t)q;
#pragma unroll
      for (int j = 0; j < 7; ++j) g[j] = dp[j];
      base = acc_ix(e, lp, seg, 0);
      uint32_t pid, smp, ent;
      slot_pixel(e, p0, slot, lp.spp, lp.stride, pid, smp, ent);
      gp = pixel_grad(e, ent, inv_spp);
    }
    warp_scatter<7>(sacc, base, g);
    finish_path<false>(w, &e, lp, slot, nv, gp, sacc, act);
    if (act) w.beta[slot].w = __uint_as_float(st | kDead);
  }
  if (!lp.gacc) acc_flush<10u>(sacc, np, w.blk);
}

// grad_acc[i] += sum over block rows (FP64), for the chunk's parameters.
// Block b covers parameters 32b .. 32b+31: warp w sums rows w, w+32, ...
// (lane l reads parameter 32b+l, so a warp reads 128 contiguous bytes per
// row), then warp 0 adds the 32 warp sums in a fixed order: the result does
// not depend on scheduling.
constexpr int kReduceWarps = 32;
__global__ void __launch_bounds__(32 * kReduceWarps) wf_blk_reduce(const float* blk, int rows, uint32_t np,
                                                                    double* grad_acc) {
  __shared__ double part[kReduceWarps][33];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t i = blockIdx.x * 32u + lane;
  double s = 0.0;
  if (i < np)
    for (int r = (int)warp; r < rows; r += kReduceWarps) s += (double)blk[(size_t)r * np + i];
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < np) {
    double t = 0.0;
    for (int k = 0; k < kReduceWarps; ++k) t += part[k][lane];
    grad_acc[i] += t;
  }
}

// Pixel batches (Sec. 4.5): entry b of a scene with N pixels is
// floor(x * N / 2^32), x the first word of Philox4x32-10 at the scene's key
// and counter (b, 0, (4 << 24) | iteration, 0).  Launch pixels of scenes
// without a batch are skipped.
constexpr uint32_t kSetPick = 4u;
__global__ void __launch_bounds__(kWfThreads) wf_pick_k(const WfScene* tab, uint32_t n_scenes, uint32_t n_launch,
                                                        const uint32_t* iter_dev, uint32_t iter) {
  const uint32_t it = iter_dev ? *iter_dev : iter;
  for (uint32_t P = blockIdx.x * blockDim.x + threadIdx.x; P < n_launch; P += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (tab[mid].pix_begin <= P)
        lo = mid;
      else
        hi = mid - 1;
    }
    const WfScene& e = tab[lo];
    if (!e.pick) continue;
    const uint32_t b = P - e.pix_begin;
    const uint4 x = philox4x32_10(make_uint4(b, 0u, (kSetPick << 24) | (it & 0xffffffu), 0u), e.key);
    e.pick[b] = (uint32_t)(((uint64_t)x.x * (uint64_t)e.n_all) >> 32);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static WfDev wf_dev(const WfBuffers& b) {
  WfDev w;
  w.ray_o = b.ray_o;
  w.ray_d = b.ray_d;
  w.hit = b.hit;
  w.beta = b.beta;
  w.rad = b.rad;
  w.q0 = b.q0;
  w.q1 = b.q1;
  w.cnt = b.cnt;
  w.sh_o = b.sh_o;
  w.sh_d = b.sh_d;
  w.sh_meta = b.sh_meta;
  w.sh_c = b.sh_c;
  w.sh_vis = b.sh_vis;
  w.aT = b.aT;
  w.aU = b.aU;
  w.aR = b.aR;
  w.nv = b.nv;
  w.sh_ge = b.sh_ge;
  w.sh_gm = b.sh_gm;
  w.sh_n = b.sh_n;
  w.aWi = b.aWi;
  w.aWo = b.aWo;
  w.sh_dv = b.sh_dv;
  w.blk = b.blk;
  w.cap = b.cap;
  return w;
}

static int wf_grid(const Launcher& L) { return L.num_sms * L.wf_blocks_per_sm; }

// One full wave of a grid-stride kernel: every SM holds as many blocks as fit
// (or the configured count), so each SM gets the same share of the work and
// there is no partial second wave.
template <typename K>
static int one_wave(const Launcher& L, K kernel, size_t smem) {
  if (L.wf_fixed_blocks > 0) return L.num_sms * L.wf_fixed_blocks;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kWfThreads, smem) != cudaSuccess || b < 1) b = 1;
  return L.num_sms * b;
}

int wf_max_blocks(const Launcher& L) { return std::max(wf_grid(L), L.wf_max_rows); }

// Brackets a stage launch for the caller's timing hook (kernel ids of ipt.h).
struct StageMark {
  const WfHook* hook;
  StageMark(const WfHook* h, int id) : hook(h) {
    if (hook && hook->begin) hook->begin(hook->user, id);
  }
  ~StageMark() {
    if (hook && hook->end) hook->end(hook->user);
  }
};
#define IPT_STAGE(id) StageMark stage_mark_(hook, id)

static WfParams wf_params(const TraceParams& tp, int loss_kind, uint32_t n_scenes, const uint32_t* iter_dev) {
  WfParams p;
  p.set = tp.set;
  p.iter = (uint32_t)(tp.iteration & 0xffffffu);
  p.iter_dev = iter_dev;
  p.spp = tp.spp;
  p.stride = tp.sample_stride ? tp.sample_stride : tp.spp;
  p.max_depth = tp.max_depth;
  p.nee = tp.nee;
  p.mis = tp.mis;
  p.profile = tp.profile;
  p.loss_kind = loss_kind;
  p.n_scenes = n_scenes;
  p.seg_lo = 0;
  p.seg_n = 0;
  p.gacc = nullptr;
  p.cache_k = kNoCache;
  p.cache_record = 0;
  p.cb = CacheBuffers{};
  p.bin = BinGrid{};
  p.keys = nullptr;
  return p;
}

static void wf_cache_params(WfParams& p, const CachePass* cache, uint32_t max_depth) {
  if (!cache || cache->b_term >= max_depth) return;
  p.cache_k = cache->b_term;
  p.cache_record = cache->record;
  p.cb = cache->buf;
}

static uint32_t total_pixels(const std::vector<WfScene>& tab) {
  return tab.empty() ? 0u : tab.back().pix_begin + tab.back().n_pix;
}

// BVH width every scene of the table can be traversed with: 8 when all of
// them select the 8-wide BVH, 4 when all have a wide one, else 2.
static int table_width(const std::vector<WfScene>& tab) {
  bool w8 = true, w4 = true;
  for (const WfScene& e : tab) {
    w8 = w8 && e.s.wide == 2 && e.s.nodes8;
    w4 = w4 && e.s.wide >= 1 && e.s.nodes4;
  }
  return w8 ? 8 : (w4 ? 4 : 2);
}

// One launch of traversal mode kMode over the table's BVH width.
template <int kMode>
static void launch_trace(int width, int grid, const WfScene* tab_dev, int n_scenes, const WfDev& w, int cur,
                         int steps, uint32_t* err, cudaStream_t st, const uint32_t* order = nullptr) {
  const int one = n_scenes == 1 ? 1 : 0;
  if (width == 8)
    wf_trace<kMode, 8><<<grid, kWfThreads, 0, st>>>(tab_dev, w, cur, steps, one, order, err);
  else if (width == 4)
    wf_trace<kMode, 4><<<grid, kWfThreads, 0, st>>>(tab_dev, w, cur, steps, one, order, err);
  else
    wf_trace<kMode, 2><<<grid, kWfThreads, 0, st>>>(tab_dev, w, cur, steps, one, order, err);
}

// Secondary closest-hit rays are reordered when the launcher asks for it:
// sets the chunk's bin grid and key array (the shading and adjoint stages
// then write each appended ray's bin).  A chunk over several scenes keeps
// their bins apart (scene major) and coarsens the grid until all its scenes'
// bins fit the kSortMaxBins the shared histograms hold.
static void sort_setup(const Launcher& L, const std::vector<WfScene>& tab, const WfBuffers& wb, const WfChunk& c,
                       WfParams& lp) {
  lp.keys = nullptr;
  lp.bin = BinGrid{};
  if (L.sort_cells <= 0 || !wb.qs || !wb.keys || !wb.bins) return;
  uint32_t b0 = 0;
  while (b0 + 1 < tab.size() && tab[b0].pix_begin + tab[b0].n_pix <= c.p0) ++b0;
  uint32_t b1 = b0 + 1;
  while (b1 < tab.size() && tab[b1].pix_begin < c.p0 + c.n_pix) ++b1;
  const uint32_t nsc = b1 - b0;
  BinGrid g;
  g.cells = L.sort_cells;
  g.dirs = L.sort_dirs;
  for (;;) {
    g.per_scene = (g.dirs ? 6u * (uint32_t)(g.dirs * g.dirs) : 1u) * (uint32_t)(g.cells * g.cells * g.cells);
    if ((uint64_t)g.per_scene * nsc <= kSortMaxBins) break;
    if (g.cells > 1) {
      --g.cells;
    } else if (g.dirs > 0) {
      --g.dirs;
    } else {
      return;  // more scenes in the chunk than bins: queue order
    }
  }
  g.scene0 = b0;
  g.n_bins = g.per_scene * nsc;
  lp.bin = g;
  lp.keys = wb.keys;
}

// Reorders queue `cur` by the bins its entries were given; returns the order
// the closest-hit traversal takes.
static const uint32_t* sort_queue(const Launcher& L, const WfParams& lp, const WfBuffers& wb, const WfDev& w,
                                  int cur, cudaStream_t st) {
  const uint32_t nb = lp.bin.n_bins;
  const size_t sm = nb * sizeof(uint32_t);
  if (cudaMemsetAsync(wb.bins, 0, sm, st) != cudaSuccess) return nullptr;
  wf_bin_count<<<2 * L.num_sms, kSortThreads, sm, st>>>(nb, w, cur, wb.keys, wb.bins);
  wf_bin_scan<<<1, kSortThreads, 0, st>>>(wb.bins, nb);
  wf_bin_scatter<<<2 * L.num_sms, kSortThreads, sm, st>>>(nb, w, cur, wb.keys, wb.bins, wb.qs);
  return wb.qs;
}

// Chunks of at most cap / spp pixels; an adjoint chunk also ends before a
// scene whose segments would take its accumulator range past max_seg.
std::vector<WfChunk> wf_plan(const std::vector<WfScene>& tab, uint32_t cap, uint32_t spp, uint32_t max_seg) {
  std::vector<WfChunk> out;
  const uint32_t per_chunk = cap / spp;
  const uint32_t total = total_pixels(tab);
  uint32_t p = 0;
  size_t b = 0;
  while (p < total) {
    while (b + 1 < tab.size() && tab[b].pix_begin + tab[b].n_pix <= p) ++b;
    WfChunk c;
    c.p0 = p;
    c.seg_lo = tab[b].seg_offset;
    uint32_t end = std::min(total, p + per_chunk);
    size_t bb = b;
    while (bb + 1 < tab.size() && tab[bb + 1].pix_begin < end) {
      const WfScene& nx = tab[bb + 1];
      if (nx.seg_offset + nx.n_seg - c.seg_lo > max_seg) {
        end = nx.pix_begin;
        break;
      }
      ++bb;
    }
    c.n_pix = end - p;
    c.seg_n = tab[bb].seg_offset + tab[bb].n_seg - c.seg_lo;
    out.push_back(c);
    p = end;
  }
  return out;
}

cudaError_t wf_forward(const Launcher& L, const WfScene* tab_dev, const std::vector<WfScene>& tab,
                       const TraceParams& tp, int loss_kind, const uint32_t* iter_dev, const WfBuffers& wb,
                       double* loss_rows, uint32_t* err, cudaStream_t st, const WfHook* hook,
                       const CachePass* cache, bool disney) {
  const uint32_t ns = (uint32_t)tab.size();
  if (disney && cache) return cudaErrorInvalidValue;
  WfParams lp = wf_params(tp, loss_kind, ns, iter_dev);
  wf_cache_params(lp, cache, tp.max_depth);
  const bool query = lp.cache_k != kNoCache && !lp.cache_record;
  const bool record = lp.cache_k != kNoCache && lp.cache_record;
  const uint32_t last_k = query ? lp.cache_k : tp.max_depth;
  const WfDev w = wf_dev(wb);
  if (wb.cap < tp.spp || ns == 0) return cudaErrorInvalidValue;
  if (lp.cache_k != kNoCache && (ns != 1 || cache->buf.q_cap < wb.cap)) return cudaErrorInvalidValue;
  const int width = table_width(tab);
  const int grid = wf_grid(L);
  const int grid_cam = one_wave(L, wf_camera, 0);
  const int grid_sh = disney ? one_wave(L, wf_shade_fwd<true>, 0) : one_wave(L, wf_shade_fwd<false>, 0);
  const int red_grid = loss_partials_capacity(L);
  const size_t red_smem = sizeof(double) * ns;
  const std::vector<WfChunk> chunks = wf_plan(tab, wb.cap, tp.spp, 0xffffffffu);
  int first = 1;
  for (const WfChunk& c : chunks) {
    const uint32_t slots = c.n_pix * tp.spp;
    sort_setup(L, tab, wb, c, lp);
    {
      IPT_STAGE(7);
      wf_camera<<<grid_cam, kWfThreads, 0, st>>>(tab_dev, lp, c.p0, slots, w);
    }
    int cur = 0;
    for (uint32_t k = 0; k <= last_k; ++k) {
      const uint32_t* order = nullptr;
      if (k > 0 && lp.keys) {  // the camera rays (k = 0) are coherent already
        IPT_STAGE(21);
        order = sort_queue(L, lp, wb, w, cur, st);
      }
      {
        IPT_STAGE(8);
        launch_trace<0>(width, grid, tab_dev, (int)tab.size(), w, cur, L.wf_steps, err, st, order);
      }
      {
        IPT_STAGE(10);
        if (disney)
          wf_shade_fwd<true><<<grid_sh, kWfThreads, 0, st>>>(tab_dev, lp, c.p0, w, cur);
        else
          wf_shade_fwd<false><<<grid_sh, kWfThreads, 0, st>>>(tab_dev, lp, c.p0, w, cur);
      }
      if (k < last_k && k < tp.max_depth && tp.nee && !(record && k < lp.cache_k)) {
        IPT_STAGE(9);
        launch_trace<1>(width, grid, tab_dev, (int)tab.size(), w, cur, L.wf_steps, err, st);
      }
      cur ^= 1;
    }
    if (query) {
      IPT_STAGE(16);
      CacheOut o{};
      o.rad = wb.rad;
      cudaError_t e = cache_infer(cache->net, lp.cb.q, tab[0].t.mat_a, tab[0].t.mat_b, lp.cb.counts, wb.cap, o,
                                  false, L.num_sms, st);
      if (e != cudaSuccess) return e;
    }
    if (record) {
      IPT_STAGE(18);
      cudaError_t e = cache_targets(lp.cb, wb.rad, st);
      if (e != cudaSuccess) return e;
    } else {
      IPT_STAGE(14);
      wf_reduce<<<red_grid, kWfThreads, red_smem, st>>>(tab_dev, lp, c.p0, c.n_pix, w, loss_rows, first);
    }
    first = 0;
  }
  return cudaGetLastError();
}

uint32_t wf_max_segments() { return (200u * 1024u) / (10u * sizeof(float)); }

template <bool kD>
static cudaError_t wf_adjoint_model(const Launcher& L, const WfScene* tab_dev, const std::vector<WfScene>& tab,
                                    const TraceParams& tp, const uint32_t* iter_dev, const WfBuffers& wb,
                                    double* grad_acc, uint32_t* err, cudaStream_t st, const WfHook* hook,
                                    const CachePass* cache);

cudaError_t wf_adjoint(const Launcher& L, const WfScene* tab_dev, const std::vector<WfScene>& tab,
                       const TraceParams& tp, const uint32_t* iter_dev, const WfBuffers& wb, double* grad_acc,
                       uint32_t* err, cudaStream_t st, const WfHook* hook, const CachePass* cache,
                       bool disney) {
  if (disney) return wf_adjoint_model<true>(L, tab_dev, tab, tp, iter_dev, wb, grad_acc, err, st, hook, nullptr);
  return wf_adjoint_model<false>(L, tab_dev, tab, tp, iter_dev, wb, grad_acc, err, st, hook, cache);
}

// kD: the Disney model (16 values per segment, chunks of at most 10/16 of
// the Lambert + GGX segment limit so the shared accumulators keep their size).
template <bool kD>
static cudaError_t wf_adjoint_model(const Launcher& L, const WfScene* tab_dev, const std::vector<WfScene>& tab,
                                    const TraceParams& tp, const uint32_t* iter_dev, const WfBuffers& wb,
                                    double* grad_acc, uint32_t* err, cudaStream_t st, const WfHook* hook,
                                    const CachePass* cache) {
  constexpr uint32_t P = kD ? 16u : 10u;
  const uint32_t max_seg = kD ? wf_max_segments() * 10u / 16u : wf_max_segments();
  const uint32_t ns = (uint32_t)tab.size();
  WfParams lp = wf_params(tp, 0, ns, iter_dev);
  if (cache && cache->record) return cudaErrorInvalidValue;
  if (kD && (!wb.aWi || !wb.aWo || !wb.sh_dv)) return cudaErrorInvalidValue;
  wf_cache_params(lp, cache, tp.max_depth);
  const bool query = lp.cache_k != kNoCache;
  const uint32_t last_k = query ? lp.cache_k : tp.max_depth;
  const WfDev w = wf_dev(wb);
  if (wb.cap < tp.spp || !wb.aT || ns == 0 || tp.max_depth > wb.depth_cap) return cudaErrorInvalidValue;
  if (query && (ns != 1 || cache->buf.q_cap < wb.cap)) return cudaErrorInvalidValue;
  const int width = table_width(tab);
  const int grid = wf_grid(L);
  const int grid_cam = one_wave(L, wf_camera, 0);
  const std::vector<WfChunk> chunks = wf_plan(tab, wb.cap, tp.spp, max_seg);
  // chunks of more than max_seg segments (one scene with that many)
  // accumulate with atomics in global memory instead of shared memory
  uint32_t max_np = 0, max_shared = 0;
  for (const WfChunk& c : chunks) {
    max_np = std::max(max_np, P * c.seg_n);
    if (c.seg_n <= max_seg) max_shared = std::max(max_shared, acc_shared_floats(P, c.seg_n));
  }
  if (max_np > wb.blk_params) return cudaErrorInvalidValue;
  const size_t shmem = max_shared * sizeof(float);
  if (shmem > 48 * 1024) {
    cudaFuncSetAttribute(wf_adj_a<kD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    cudaFuncSetAttribute(wf_adj_connect<kD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    cudaFuncSetAttribute(wf_adj_b<kD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    cudaFuncSetAttribute(wf_adj_cache, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  }
  for (const WfChunk& c : chunks) {
    lp.seg_lo = c.seg_lo;
    lp.seg_n = c.seg_n;
    sort_setup(L, tab, wb, c, lp);
    const uint32_t np = P * c.seg_n;
    const bool global = c.seg_n > max_seg;
    lp.gacc = global ? wb.blk : nullptr;
    const size_t sm = global ? 0 : acc_shared_floats(P, c.seg_n) * sizeof(float);
    // each adjoint stage runs one wave at its own occupancy for this
    // accumulator size; block b of every stage adds into gradient row b
    // (all blocks into row 0 in global mode)
    const int g_a = one_wave(L, wf_adj_a<kD>, sm), g_c = one_wave(L, wf_adj_connect<kD>, sm);
    const int g_b = one_wave(L, wf_adj_b<kD>, sm), g_q = one_wave(L, wf_adj_cache, sm);
    const int rows = global ? 1 : std::max(std::max(g_a, g_c), std::max(g_b, g_q));
    if (rows > wf_max_blocks(L)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(wb.blk, 0, (size_t)rows * np * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const uint32_t slots = c.n_pix * tp.spp;
    {
      IPT_STAGE(7);
      wf_camera<<<grid_cam, kWfThreads, 0, st>>>(tab_dev, lp, c.p0, slots, w);
    }
    int cur = 0;
    for (uint32_t k = 0; k <= last_k; ++k) {
      const uint32_t* order = nullptr;
      if (k > 0 && lp.keys) {  // the camera rays (k = 0) are coherent already
        IPT_STAGE(21);
        order = sort_queue(L, lp, wb, w, cur, st);
      }
      {
        IPT_STAGE(8);
        launch_trace<0>(width, grid, tab_dev, (int)tab.size(), w, cur, L.wf_steps, err, st, order);
      }
      {
        IPT_STAGE(11);
        wf_adj_a<kD><<<g_a, kWfThreads, sm, st>>>(tab_dev, lp, c.p0, w, cur);
      }
      if (k < last_k) {
        if (tp.nee) {
          {
            IPT_STAGE(9);
            launch_trace<2>(width, grid, tab_dev, (int)tab.size(), w, cur, L.wf_steps, err, st);
          }
          IPT_STAGE(12);
          wf_adj_connect<kD><<<g_c, kWfThreads, sm, st>>>(tab_dev, lp, w);
        }
        IPT_STAGE(13);
        wf_adj_b<kD><<<g_b, kWfThreads, sm, st>>>(tab_dev, lp, c.p0, w, cur);
      }
      cur ^= 1;
    }
    if (query) {
      {
        IPT_STAGE(17);
        CacheOut o{};
        o.c = lp.cb.qc;
        o.dp = lp.cb.qdp;
        e = cache_infer(cache->net, lp.cb.q, tab[0].t.mat_a, tab[0].t.mat_b, lp.cb.counts, wb.cap, o, true,
                        L.num_sms, st);
        if (e != cudaSuccess) return e;
      }
      IPT_STAGE(13);
      wf_adj_cache<<<g_q, kWfThreads, sm, st>>>(tab_dev, lp, c.p0, w);
    }
    IPT_STAGE(14);
    wf_blk_reduce<<<(np + 31) / 32, 32 * kReduceWarps, 0, st>>>(wb.blk, rows, np, grad_acc + P * c.seg_lo);
  }
  return cudaGetLastError();
}

cudaError_t wf_pick(const WfScene* tab_dev, const std::vector<WfScene>& tab, const uint32_t* iter_dev,
                    uint32_t iter, cudaStream_t st) {
  if (tab.empty()) return cudaSuccess;
  const WfScene& last = tab.back();
  const uint32_t n_launch = last.pix_begin + last.n_pix;
  const uint32_t blocks = std::min<uint32_t>((n_launch + kWfThreads - 1) / kWfThreads, 4096u);
  wf_pick_k<<<std::max(blocks, 1u), kWfThreads, 0, st>>>(tab_dev, (uint32_t)tab.size(), n_launch, iter_dev, iter);
  return cudaGetLastError();
}

cudaError_t wf_init(Launcher* L) {
  // the fewest resident blocks of any traversal variant, so that every
  // width's persistent grid fits in one wave
  int b = 1 << 30;
  const void* variants[] = {(const void*)wf_trace<0, 2>, (const void*)wf_trace<0, 4>, (const void*)wf_trace<0, 8>,
                            (const void*)wf_trace<1, 2>, (const void*)wf_trace<1, 4>, (const void*)wf_trace<1, 8>,
                            (const void*)wf_trace<2, 2>, (const void*)wf_trace<2, 4>, (const void*)wf_trace<2, 8>};
  for (const void* k : variants) {
    int bk = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bk, k, kWfThreads, 0);
    if (e != cudaSuccess) return e;
    b = std::min(b, bk);
  }
  L->wf_blocks_per_sm = b < 1 ? 1 : b;
  if (L->wf_fixed_blocks > 0) L->wf_blocks_per_sm = L->wf_fixed_blocks;
  // gradient rows: the widest one-wave grid of an adjoint stage (accumulators
  // in dynamic shared memory only lower the occupancy)
  int rows = 0;
  rows = std::max(rows, one_wave(*L, wf_adj_a<false>, 0));
  rows = std::max(rows, one_wave(*L, wf_adj_connect<false>, 0));
  rows = std::max(rows, one_wave(*L, wf_adj_b<false>, 0));
  rows = std::max(rows, one_wave(*L, wf_adj_a<true>, 0));
  rows = std::max(rows, one_wave(*L, wf_adj_connect<true>, 0));
  rows = std::max(rows, one_wave(*L, wf_adj_b<true>, 0));
  rows = std::max(rows, one_wave(*L, wf_adj_cache, 0));
  L->wf_max_rows = rows;
  return cudaSuccess;
}

}  // namespace ipt
