// Kernels of one nested-SGD iteration of inverse path tracing:
//   k_prepare   per-segment tables from the parameters (light selection CDF,
//               lobe probabilities): the per-iteration form of the emission-
//               proportional light selection of Appendix E;
//   k_forward   Monte Carlo pixel estimates (Eq. 1-2) with MIS (App. A.2),
//               optionally fused with the residual of the loss (Eq. 3);
//   k_adjoint   derivative paths from an independent sample set (Sec. 3.3),
//               scattering g . dI/dTheta (Eq. 5-6) into per-block shared
//               accumulators;
//   k_finalize  loss and gradient reduction;
//   k_adam      Adam + L1 emission regulariser + clamps (Sec. 4.4-4.5), then
//               the tables for the next iteration;
//   k_trace_rays, k_philox: the ray-casting and random-number primitives.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ipt_device.cuh"
#include "ipt_internal.h"
#include "ipt_path.cuh"
#include "ipt_wavefront.h"

namespace ipt {

__global__ void k_prepare(const float* params, const float* sparams, uint32_t S, float es,
                          const double* seg_area, SegBuffers t) {
  build_tables(params, sparams, S, es, seg_area, t);
}

// Radiance estimate of one camera path.
__device__ float3 forward_path(const SceneDev& s, const SegDev& t, const ViewDev& vw, uint32_t px, uint32_t py,
                               uint32_t pid, uint32_t sample, const PathParams& pp, double W,
                               uint32_t* err) {
  PathRng rng;
  rng.base = make_uint4(pid, sample, pp.set_iter, 0);
  rng.key = pp.key;
  float3 o;
  float3 d = camera_ray(vw, px, py, rng, o);
  float3 beta = f3(1.0f, 1.0f, 1.0f), L = f3(0.0f, 0.0f, 0.0f);
  const bool light_on = pp.nee && W > 0.0;
  int skip = -1;
  float prev_pdf = 0.0f;
  for (uint32_t k = 0;; ++k) {
    const Hit h = trace_closest(s, o, d, __int_as_float(0x7f800000), skip, err);
    if (h.tri < 0) break;
    const Vtx v = make_vertex(s, h, d, pp.profile);
    if (v.prof > 0.0f) {
      const float wb = emission_weight(t, v, h.t, k > 0, light_on, prev_pdf, pp.mis);
      if (wb > 0.0f) L = L + beta * xyz(__ldg(&t.emis[v.seg])) * (wb * v.prof);
    }
    if (k == pp.max_depth) break;
    const float4 ua = rng.draw(k, 0), ub = rng.draw(k, 1);
    const float4 ma = __ldg(&t.mat_a[v.seg]), mb = __ldg(&t.mat_b[v.seg]);
    const float4 sa = __ldg(&t.samp[v.seg]);
    if (light_on) {
      const NeeResult ne = next_event(s, t, v, ua, ub, W, pp.profile, pp.mis, sa.y, sa.x, err);
      if (ne.valid) {
        const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, ne.wl);
        L = L + beta * bv.f * xyz(__ldg(&t.emis[ne.seg])) * ne.k;
      }
    }
    if (!(dot(v.wi, v.ns) > 0.0f)) break;
    const float3 wo = bsdf_sample(__ldg(&t.pspec[v.seg]), sa.x, v.ns, v.wi, ua.x, ua.y, ua.z);
    const float pdf = bsdf_pdf(sa.y, sa.x, v.ns, v.wi, wo);
    const float co = dot(wo, v.ns);
    if (!(dot(wo, v.ng) > 0.0f) || !(co > 0.0f) || !(pdf > 0.0f)) break;
    const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, wo);
    beta = beta * bv.f * (co / pdf);
    prev_pdf = pdf;
    o = v.x + v.ng * s.eps;
    d = wo;
    skip = h.tri;
  }
  return L;
}

__device__ __forceinline__ void add3(float* acc, int i, float3 v) {
  atomicAdd(&acc[i], v.x);
  atomicAdd(&acc[i + 1], v.y);
  atomicAdd(&acc[i + 2], v.z);
}

// Derivative of one camera path, contracted with the pixel's upstream
// gradient gp and scattered into acc (S x 10).  Eq. 5-6 differentiate the
// product of BSDFs along each light path; here each continuing vertex l keeps
// T_l (the throughput with its own weight w_l left out) and U_l (the sum of
// later contributions through T_l), so that d/dTheta_l of the whole path is
// (dw_l/dTheta) . U_l without dividing by w_l.  Emission and the local NEE term
// are differentiated on the spot.  Pdfs and MIS weights are held constant.
template <int MAXD>
__device__ void adjoint_path(const SceneDev& s, const SegDev& t, const ViewDev& vw, uint32_t px, uint32_t py,
                             uint32_t pid, uint32_t sample, const PathParams& pp, double W, float3 gp,
                             float* acc, uint32_t* err) {
  PathRng rng;
  rng.base = make_uint4(pid, sample, pp.set_iter, 0);
  rng.key = pp.key;
  float3 o;
  float3 d = camera_ray(vw, px, py, rng, o);
  float3 beta = f3(1.0f, 1.0f, 1.0f);
  const bool light_on = pp.nee && W > 0.0;
  const float es = pp.emission_scale;
  float3 T[MAXD], U[MAXD];
  float AD[MAXD], AS[MAXD], AR[MAXD];
  int SG[MAXD];
  int nv = 0;
  int skip = -1;
  float prev_pdf = 0.0f;
  for (uint32_t k = 0;; ++k) {
    const Hit h = trace_closest(s, o, d, __int_as_float(0x7f800000), skip, err);
    if (h.tri < 0) break;
    const Vtx v = make_vertex(s, h, d, pp.profile);
    float3 C = f3(0.0f, 0.0f, 0.0f);
    if (v.prof > 0.0f) {
      const float wb = emission_weight(t, v, h.t, k > 0, light_on, prev_pdf, pp.mis);
      if (wb > 0.0f) {
        const float f = wb * v.prof;
        C = xyz(__ldg(&t.emis[v.seg])) * f;
        add3(acc, 10 * v.seg + 7, gp * beta * (f * es));  // Eq. 5 at the hit
      }
    }
    const bool last = k == pp.max_depth;
    const float4 ma = __ldg(&t.mat_a[v.seg]), mb = __ldg(&t.mat_b[v.seg]);
    const float4 sa = __ldg(&t.samp[v.seg]);
    float4 ua = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!last) {
      ua = rng.draw(k, 0);
      const float4 ub = rng.draw(k, 1);
      if (light_on) {
        const NeeResult ne = next_event(s, t, v, ua, ub, W, pp.profile, pp.mis, sa.y, sa.x, err);
        if (ne.valid) {
          const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, ne.wl);
          const float3 Le = xyz(__ldg(&t.emis[ne.seg]));
          C = C + bv.f * Le * ne.k;
          add3(acc, 10 * ne.seg + 7, gp * beta * bv.f * (ne.k * es));        // Eq. 5, light end
          const float3 q = gp * beta * Le * ne.k;                              // Eq. 6, l = this vertex
          add3(acc, 10 * v.seg + 0, q * (1.0f / kPi));
          add3(acc, 10 * v.seg + 3, q * bv.sp.s);
          atomicAdd(&acc[10 * v.seg + 6], dot(q, f3(mb.x, mb.y, mb.z)) * bv.sp.ds_dr);
        }
      }
    }
#pragma unroll
    for (int l = 0; l < MAXD; ++l)
      if (l < nv) U[l] = U[l] + T[l] * C;
    if (last || !(dot(v.wi, v.ns) > 0.0f)) break;
    const float3 wo = bsdf_sample(__ldg(&t.pspec[v.seg]), sa.x, v.ns, v.wi, ua.x, ua.y, ua.z);
    const float pdf = bsdf_pdf(sa.y, sa.x, v.ns, v.wi, wo);
    const float co = dot(wo, v.ns);
    if (!(dot(wo, v.ng) > 0.0f) || !(co > 0.0f) || !(pdf > 0.0f)) break;
    const BrdfVal bv = brdf_eval(ma, mb, v.ns, v.wi, wo);
    const float kk = co / pdf;
    const float3 w = bv.f * kk;
#pragma unroll
    for (int l = 0; l < MAXD; ++l) {
      if (l < nv) T[l] = T[l] * w;
      if (l == nv) {
        T[l] = beta;
        U[l] = f3(0.0f, 0.0f, 0.0f);
        AD[l] = kk * (1.0f / kPi);
        AS[l] = kk * bv.sp.s;
        AR[l] = kk * bv.sp.ds_dr;
        SG[l] = v.seg;
      }
    }
    ++nv;
    beta = beta * w;
    prev_pdf = pdf;
    o = v.x + v.ng * s.eps;
    d = wo;
    skip = h.tri;
  }
#pragma unroll
  for (int l = 0; l < MAXD; ++l) {
    if (l < nv) {
      const float3 q = gp * U[l];
      const int sg = SG[l];
      add3(acc, 10 * sg + 0, q * AD[l]);
      add3(acc, 10 * sg + 3, q * AS[l]);
      const float4 mb = __ldg(&t.mat_b[sg]);
      atomicAdd(&acc[10 * sg + 6], dot(q, f3(mb.x, mb.y, mb.z)) * AR[l]);
    }
  }
}

// ---------------------------------------------------------------------------
// Forward kernel: each pixel is handled by `group` lanes of one warp, each
// lane tracing spp / group samples; the lanes' sums are combined with
// butterfly shuffles, so the pixel estimate is deterministic.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_forward(SceneDev s, SegDev t, const ViewDev* views,
                                                           uint32_t n_views, uint32_t pix_begin, uint32_t n_pix,
                                                           PathParams pp, float* img, float* msq,
                                                           const float* target, float* g_out,
                                                           double* loss_partials, float g_scale, int loss_kind,
                                                           uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t G = pp.group;
  const uint32_t ppw = 32u / G;
  const uint32_t sub = lane & (G - 1u);
  const uint32_t warps_per_block = blockDim.x >> 5;
  const uint32_t n_tasks = (n_pix + ppw - 1) / ppw;
  const uint32_t stride = gridDim.x * warps_per_block;
  const double W = *t.W;
  const float inv_spp = 1.0f / (float)pp.spp;
  double loss_acc = 0.0;
  for (uint32_t task = blockIdx.x * warps_per_block + (threadIdx.x >> 5); task < n_tasks; task += stride) {
    const uint32_t local = task * ppw + lane / G;
    const bool active = local < n_pix;
    float3 a = f3(0.f, 0.f, 0.f), a2 = f3(0.f, 0.f, 0.f);
    uint32_t pid = pix_begin + local;
    if (active) {
      uint32_t s0 = 0;
      if (pp.pick) {
        pid = pp.pick[local];
        s0 = local * pp.stride;
      }
      const ViewDev& vw = find_view(views, n_views, pid);
      const uint32_t lp = pid - vw.offset;
      const uint32_t px = lp % vw.w, py = lp / vw.w;
      for (uint32_t smp = sub; smp < pp.spp; smp += G) {
        const float3 L = forward_path(s, t, vw, px, py, pid, s0 + smp, pp, W, err);
        a = a + L;
        a2 = a2 + L * L;
      }
    }
    for (uint32_t off = G >> 1; off >= 1; off >>= 1) {
      a.x += __shfl_xor_sync(0xffffffffu, a.x, off);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, off);
      a.z += __shfl_xor_sync(0xffffffffu, a.z, off);
      a2.x += __shfl_xor_sync(0xffffffffu, a2.x, off);
      a2.y += __shfl_xor_sync(0xffffffffu, a2.y, off);
      a2.z += __shfl_xor_sync(0xffffffffu, a2.z, off);
    }
    if (active && sub == 0) {
      const float3 mean = a * inv_spp;
      if (img) {
        img[3 * local + 0] = mean.x;
        img[3 * local + 1] = mean.y;
        img[3 * local + 2] = mean.z;
      }
      if (msq) {
        msq[3 * local + 0] = a2.x * inv_spp;
        msq[3 * local + 1] = a2.y * inv_spp;
        msq[3 * local + 2] = a2.z * inv_spp;
      }
      if (target) {
        // a pixel batch reads the target of the drawn pixel (the caller passes
        // the whole target image); otherwise target is indexed like the outputs
        const uint32_t ti = pp.pick ? pid : local;
        const float r[3] = {mean.x - target[3 * ti + 0], mean.y - target[3 * ti + 1],
                            mean.z - target[3 * ti + 2]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (loss_kind == 0) {
            g_out[3 * local + c] = 2.0f * r[c] * g_scale;
            loss_acc += (double)r[c] * (double)r[c];
          } else {
            g_out[3 * local + c] = (r[c] > 0.0f ? 1.0f : (r[c] < 0.0f ? -1.0f : 0.0f)) * g_scale;
            loss_acc += fabs((double)r[c]);
          }
        }
      }
    }
  }
  if (loss_partials) {
    __shared__ double red[kBlockThreads / 32];
    for (int off = 16; off >= 1; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
    if (lane == 0) red[threadIdx.x >> 5] = loss_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (uint32_t w = 0; w < warps_per_block; ++w) sum += red[w];
      loss_partials[blockIdx.x] = sum;
    }
  }
}

// Pixels [pix_begin, pix_begin + n_pix) of the concatenated views; g_img is
// indexed relative to pix_begin.
template <int MAXD>
__global__ void __launch_bounds__(kBlockThreads) k_adjoint(SceneDev s, SegDev t, const ViewDev* views,
                                                           uint32_t n_views, uint32_t pix_begin, uint32_t n_pix,
                                                           PathParams pp, const float* g_img, double* grad_acc,
                                                           float* gacc, uint32_t* err) {
  // per-block accumulators in shared memory, or (scenes with too many
  // segments for it) one zeroed accumulator in global memory
  extern __shared__ float sgrad_sh[];
  float* sgrad = gacc ? gacc : sgrad_sh;
  const uint32_t n_par = 10u * s.n_seg;
  if (!gacc)
    for (uint32_t i = threadIdx.x; i < n_par; i += blockDim.x) sgrad[i] = 0.0f;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t G = pp.group;
  const uint32_t ppw = 32u / G;
  const uint32_t sub = lane & (G - 1u);
  const uint32_t warps_per_block = blockDim.x >> 5;
  const uint32_t n_tasks = (n_pix + ppw - 1) / ppw;
  const uint32_t stride = gridDim.x * warps_per_block;
  const double W = *t.W;
  const float inv_spp = 1.0f / (float)pp.spp;
  for (uint32_t task = blockIdx.x * warps_per_block + (threadIdx.x >> 5); task < n_tasks; task += stride) {
    const uint32_t local = task * ppw + lane / G;
    if (local >= n_pix) continue;
    const uint32_t pid = pp.pick ? pp.pick[local] : pix_begin + local;
    const uint32_t s0 = pp.pick ? local * pp.stride : 0u;
    const float3 gp = f3(g_img[3 * local], g_img[3 * local + 1], g_img[3 * local + 2]) * inv_spp;
    if (gp.x == 0.0f && gp.y == 0.0f && gp.z == 0.0f) continue;
    const ViewDev& vw = find_view(views, n_views, pid);
    const uint32_t lp = pid - vw.offset;
    const uint32_t px = lp % vw.w, py = lp / vw.w;
    for (uint32_t smp = sub; smp < pp.spp; smp += G)
      adjoint_path<MAXD>(s, t, vw, px, py, pid, s0 + smp, pp, W, gp, sgrad, err);
  }
  __syncthreads();
  if (!gacc)
    for (uint32_t i = threadIdx.x; i < n_par; i += blockDim.x) {
      const float v = sgrad[i];
      if (v != 0.0f) atomicAdd(&grad_acc[i], (double)v);
    }
}

// ---------------------------------------------------------------------------
// Batched megakernel: the paths of every scene of a batch's launch table in
// one forward and one adjoint launch (the small pixel batches of Sec. 4.5
// are latency-bound, and a stage-by-stage wavefront pays ~45 launches per
// iteration).  Launch pixel p belongs to the table entry whose pixel range
// holds it; each scene keeps its own Philox key, emission scale, pixel draw,
// target and segment range, so its paths are the ones it traces alone.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t table_scene(const WfScene* tab, uint32_t n, uint32_t p) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (tab[mid].pix_begin <= p)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ PathParams scene_params(const PathParams& base, const WfScene& e, uint32_t set_iter) {
  PathParams p = base;
  p.key = e.key;
  p.emission_scale = e.es;
  p.set_iter = set_iter;
  p.pick = e.pick;
  return p;
}

// Residual pass: the upstream gradient of every entry and, per block, each
// scene's loss sum (rows[block * n_scenes + scene], the layout of the
// wavefront's reduction).
// Four resident blocks per SM (at most 128 registers), as the single-scene
// forward: the grid is one loss row per block of a full wave.
__global__ void __launch_bounds__(kBlockThreads, 4)
    k_forward_batch(const WfScene* tab, uint32_t n_scenes, uint32_t total, PathParams pp, uint32_t set,
                    const uint32_t* iter_dev, int loss_kind, double* loss_rows, uint32_t* err) {
  extern __shared__ double sloss[];
  for (uint32_t i = threadIdx.x; i < n_scenes; i += blockDim.x) sloss[i] = 0.0;
  __syncthreads();
  const uint32_t set_iter = (set << 24) | (*iter_dev & 0xFFFFFFu);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t G = pp.group;
  const uint32_t ppw = 32u / G;
  const uint32_t sub = lane & (G - 1u);
  const uint32_t warps_per_block = blockDim.x >> 5;
  const uint32_t n_tasks = (total + ppw - 1) / ppw;
  const uint32_t stride = gridDim.x * warps_per_block;
  const float inv_spp = 1.0f / (float)pp.spp;
  for (uint32_t task = blockIdx.x * warps_per_block + (threadIdx.x >> 5); task < n_tasks; task += stride) {
    const uint32_t p = task * ppw + lane / G;
    const bool active = p < total;
    float3 a = f3(0.f, 0.f, 0.f);
    uint32_t b = 0, entry = 0, pid = 0;
    if (active) {
      b = table_scene(tab, n_scenes, p);
      const WfScene& e = tab[b];
      entry = p - e.pix_begin + e.pix_base;
      pid = e.pick ? e.pick[entry] : entry;
      const uint32_t s0 = e.pick ? entry * pp.stride : 0u;
      const PathParams q = scene_params(pp, e, set_iter);
      const double W = *e.t.W;
      const ViewDev& vw = find_view(e.views, e.n_views, pid);
      const uint32_t lp = pid - vw.offset;
      const uint32_t px = lp % vw.w, py = lp / vw.w;
      for (uint32_t smp = sub; smp < pp.spp; smp += G) a = a + forward_path(e.s, e.t, vw, px, py, pid, s0 + smp, q, W, err);
    }
    for (uint32_t off = G >> 1; off >= 1; off >>= 1) {
      a.x += __shfl_xor_sync(0xffffffffu, a.x, off);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, off);
      a.z += __shfl_xor_sync(0xffffffffu, a.z, off);
    }
    if (active && sub == 0) {
      const WfScene& e = tab[b];
      const float3 mean = a * inv_spp;
      const uint32_t ti = e.pick ? pid : entry;
      const float r[3] = {mean.x - e.target[3 * ti + 0], mean.y - e.target[3 * ti + 1], mean.z - e.target[3 * ti + 2]};
      double l = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (loss_kind == 0) {
          e.g_img[3 * entry + c] = 2.0f * r[c] * e.g_scale;
          l += (double)r[c] * (double)r[c];
        } else {
          e.g_img[3 * entry + c] = (r[c] > 0.0f ? 1.0f : (r[c] < 0.0f ? -1.0f : 0.0f)) * e.g_scale;
          l += fabs((double)r[c]);
        }
      }
      atomicAdd(&sloss[b], l);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n_scenes; i += blockDim.x) loss_rows[(size_t)blockIdx.x * n_scenes + i] = sloss[i];
}

// Derivative pass: every entry's paths into the batch's packed segment
// accumulators (shared per block, or global when they do not fit).
template <int MAXD>
__global__ void __launch_bounds__(kBlockThreads)
    k_adjoint_batch(const WfScene* tab, uint32_t n_scenes, uint32_t total, uint32_t n_par, PathParams pp,
                    uint32_t set, const uint32_t* iter_dev, double* grad_acc, float* gacc, uint32_t* err) {
  extern __shared__ float bgrad_sh[];
  float* acc = gacc ? gacc : bgrad_sh;
  if (!gacc)
    for (uint32_t i = threadIdx.x; i < n_par; i += blockDim.x) acc[i] = 0.0f;
  __syncthreads();
  const uint32_t set_iter = (set << 24) | (*iter_dev & 0xFFFFFFu);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t G = pp.group;
  const uint32_t ppw = 32u / G;
  const uint32_t sub = lane & (G - 1u);
  const uint32_t warps_per_block = blockDim.x >> 5;
  const uint32_t n_tasks = (total + ppw - 1) / ppw;
  const uint32_t stride = gridDim.x * warps_per_block;
  const float inv_spp = 1.0f / (float)pp.spp;
  for (uint32_t task = blockIdx.x * warps_per_block + (threadIdx.x >> 5); task < n_tasks; task += stride) {
    const uint32_t p = task * ppw + lane / G;
    if (p >= total) continue;
    const WfScene& e = tab[table_scene(tab, n_scenes, p)];
    const uint32_t entry = p - e.pix_begin + e.pix_base;
    const uint32_t pid = e.pick ? e.pick[entry] : entry;
    const uint32_t s0 = e.pick ? entry * pp.stride : 0u;
    const float3 gp = f3(e.g_img[3 * entry], e.g_img[3 * entry + 1], e.g_img[3 * entry + 2]) * inv_spp;
    if (gp.x == 0.0f && gp.y == 0.0f && gp.z == 0.0f) continue;
    const PathParams q = scene_params(pp, e, set_iter);
    const double W = *e.t.W;
    const ViewDev& vw = find_view(e.views, e.n_views, pid);
    const uint32_t lp = pid - vw.offset;
    const uint32_t px = lp % vw.w, py = lp / vw.w;
    float* sacc = acc + 10u * e.seg_offset;
    for (uint32_t smp = sub; smp < pp.spp; smp += G)
      adjoint_path<MAXD>(e.s, e.t, vw, px, py, pid, s0 + smp, q, W, gp, sacc, err);
  }
  __syncthreads();
  if (!gacc)
    for (uint32_t i = threadIdx.x; i < n_par; i += blockDim.x) {
      const float v = acc[i];
      if (v != 0.0f) atomicAdd(&grad_acc[i], (double)v);
    }
}

__global__ void k_add_to_double(const float* src, uint32_t n, double* dst) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] += (double)src[i];
}

// One block: fixed-order sums (deterministic for a fixed grid).
__global__ void k_finalize(const double* loss_partials, int n_partials, double* loss_dev,
                           const double* grad_acc, float* grad_out, uint32_t n_params) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n_partials; i += blockDim.x) s += loss_partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss_dev) *loss_dev = red[0];
  if (grad_out)
    for (uint32_t i = threadIdx.x; i < n_params; i += blockDim.x) grad_out[i] = (float)grad_acc[i];
}

// Adam on the concatenated parameters of a batch, one block per member,
// followed by that member's tables for the next iteration.
__device__ __forceinline__ void adam_range(float* params, float* m, float* v, const uint8_t* free_mask,
                                           const double* grad_acc, const float* grad_f, uint32_t begin,
                                           uint32_t end, uint32_t g_begin, const AdamHost& a, int step,
                                           uint32_t lane0, uint32_t lanes) {
  const float bc1 = 1.0f - powf(a.beta1, (float)step);
  const float bc2 = 1.0f - powf(a.beta2, (float)step);
  for (uint32_t i = begin + lane0; i < end; i += lanes) {
    if (free_mask && !free_mask[i]) continue;
    const uint32_t j = i % 10u;
    float g = grad_f ? grad_f[i] : (float)grad_acc[g_begin + (i - begin)];
    const float th = params[i];
    if (j >= 7) g += a.l1 * (th > 0.0f ? 1.0f : (th < 0.0f ? -1.0f : 0.0f));
    const float mi = a.beta1 * m[i] + (1.0f - a.beta1) * g;
    const float vi = a.beta2 * v[i] + (1.0f - a.beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float nt = th - a.lr * (mi / bc1) / (sqrtf(vi / bc2) + a.eps);
    if (j < 6)
      nt = fminf(fmaxf(nt, 0.0f), 1.0f);
    else if (j == 6)
      nt = fminf(fmaxf(nt, 0.02f), 1.0f);
    else
      nt = fmaxf(nt, 0.0f);
    params[i] = nt;
  }
}

// True on every thread of the block when the loss (nullable) or any of the n
// gradient values (FP64 accumulators, or FP32 when grad_f is given) is NaN or
// infinite.
__device__ __forceinline__ bool block_nonfinite(const double* loss, const double* grad_acc, const float* grad_f,
                                                uint32_t n) {
  bool bad = loss && !isfinite(*loss);
  for (uint32_t i = threadIdx.x; i < n && !bad; i += blockDim.x)
    bad = grad_f ? !isfinite(grad_f[i]) : !isfinite(grad_acc[i]);
  return __syncthreads_or(bad) != 0;
}

// A member whose loss or gradient is not finite keeps its parameters and
// Adam moments (the step is skipped for it alone) and sets the error word.
__global__ void k_adam_batch(const BatchMember* members, float* params, float* m, float* v,
                             const uint8_t* free_mask, const double* grad_acc, const uint32_t* iter_dev,
                             AdamHost a, const double* losses, uint32_t* err) {
  const BatchMember mb = members[blockIdx.x];
  if (!mb.active) return;
  const int step = (int)*iter_dev + 1;
  if (block_nonfinite(losses + blockIdx.x, grad_acc + 10u * mb.grad_offset, nullptr, 10u * mb.n_seg)) {
    if (threadIdx.x == 0) atomicOr(err, kErrNonFinite);
  } else {
    adam_range(params, m, v, free_mask, grad_acc, nullptr, 10u * mb.seg_offset, 10u * (mb.seg_offset + mb.n_seg),
               10u * mb.grad_offset, a, step, threadIdx.x, blockDim.x);
  }
  __syncthreads();
  const float* p = params + 10u * mb.seg_offset;
  build_tables(p, p, mb.n_seg, mb.es, mb.seg_area, mb.tab);
}

__global__ void k_prepare_batch(const BatchMember* members, const float* params) {
  const BatchMember mb = members[blockIdx.x];
  const float* p = params + 10u * mb.seg_offset;
  build_tables(p, p, mb.n_seg, mb.es, mb.seg_area, mb.tab);
}

// Loss of each member from the per-block rows of the launch table (n_tab
// entries: the active members).
__global__ void k_batch_losses(const double* rows, int n_rows, const BatchMember* members, uint32_t n_tab,
                               double* loss) {
  __shared__ double red[256];
  const uint32_t b = blockIdx.x;
  if (!members[b].active) {  // traced nothing this step
    if (threadIdx.x == 0) loss[b] = 0.0;
    return;
  }
  const uint32_t slot = members[b].slot;
  double s = 0.0;
  for (int r = threadIdx.x; r < n_rows; r += blockDim.x) s += rows[(size_t)r * n_tab + slot];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[b] = red[0] * (double)members[b].inv_n;
}

__global__ void k_tick(uint32_t* counter) { *counter += 1u; }

// With a non-finite loss or gradient the update is skipped: parameters, Adam
// moments and the step count stay those of the last good step, and the
// error word reports it.  The tables are rebuilt either way.
__global__ void k_adam(float* params, float* m, float* v, const uint8_t* free_mask,
                       const double* grad_acc, const float* grad_f, int* step_dev, AdamHost a, uint32_t S,
                       float es, const double* seg_area, SegBuffers t, const double* loss, uint32_t* err) {
  const int step = *step_dev + 1;
  const bool bad = block_nonfinite(loss, grad_acc, grad_f, 10u * S);
  if (!bad) adam_range(params, m, v, free_mask, grad_acc, grad_f, 0, 10u * S, 0u, a, step, threadIdx.x, blockDim.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bad)
      atomicOr(err, kErrNonFinite);
    else
      *step_dev = step;
  }
  build_tables(params, params, S, es, seg_area, t);
}

// The same check for launches over a grid: one block decides, *flag = 1
// when the step must be skipped.
__global__ void __launch_bounds__(1024) k_finite_guard(const double* loss, const double* grad_acc,
                                                       const float* grad_f, uint32_t n, uint32_t* flag,
                                                       uint32_t* err) {
  const bool bad = block_nonfinite(loss, grad_acc, grad_f, n);
  if (threadIdx.x == 0) {
    *flag = bad ? 1u : 0u;
    if (bad) atomicOr(err, kErrNonFinite);
  }
}

// Scenes with many segments (per-triangle parameters): Adam over a grid, the
// per-segment tables over a grid, and the light CDF by one block that keeps
// the sequential FP64 summation order of build_tables.  The terms of
// non-emitting segments are exact zeros, so the running sum changes only at
// emitters: those are added in order by one thread, and every other entry
// takes the running value of the last emitter before it.
constexpr uint32_t kWideSegments = 4096;

__global__ void k_adam_wide(float* params, float* m, float* v, const uint8_t* free_mask, const double* grad_acc,
                            const float* grad_f, const int* step_dev, AdamHost a, uint32_t S, const uint32_t* skip) {
  if (*skip) return;
  const int step = *step_dev + 1;
  adam_range(params, m, v, free_mask, grad_acc, grad_f, 0, 10u * S, 0u, a, step,
             blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void k_tables_seg(const float* params, const float* sparams, uint32_t S, float es, SegBuffers t) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const float* p = params + 10 * s;
    const float* q = sparams + 10 * s;
    const float r = p[6];
    t.mat_a[s] = make_float4(p[0], p[1], p[2], r);
    t.mat_b[s] = make_float4(p[3], p[4], p[5], fmaxf(r * r, 1e-4f));
    t.emis[s] = make_float4(es * p[7], es * p[8], es * p[9], 0.0f);
    const double ld = lum_d(q[0], q[1], q[2]);
    const double ls = lum_d(q[3], q[4], q[5]);
    const double sum = __dadd_rn(ld, ls);
    t.pspec[s] = sum > 0.0 ? __ddiv_rn(ls, sum) : 0.0;
    double le = lum_d(q[7], q[8], q[9]);
    if (!(le > 0.0)) le = 0.0;
    t.lum[s] = le;
  }
}

// One block of 1024 threads; bumps *step_dev when given (after Adam) unless
// *skip says the Adam step was skipped.
__global__ void __launch_bounds__(1024) k_tables_cdf(uint32_t S, const double* seg_area, SegBuffers t,
                                                     int* step_dev, const uint32_t* skip) {
  __shared__ double term[1024];
  __shared__ unsigned nz[32];
  __shared__ double warp_end[32];
  __shared__ double carry, start;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
  if (tid == 0) carry = 0.0;
  for (uint32_t base = 0; base < S; base += 1024u) {
    const uint32_t i = base + tid;
    if (tid == 0) start = carry;
    const double a = i < S ? __dmul_rn(t.lum[i], seg_area[i]) : 0.0;
    term[tid] = a;
    const unsigned m = __ballot_sync(0xffffffffu, a != 0.0);
    if (lane == 0) nz[wid] = m;
    __syncthreads();
    if (tid == 0) {
      double acc = carry;
      for (int w = 0; w < 32; ++w) {
        for (unsigned b = nz[w]; b; b &= b - 1u) {
          const int j = w * 32 + __ffs(b) - 1;
          acc = __dadd_rn(acc, term[j]);
          term[j] = acc;
        }
        warp_end[w] = acc;
      }
      carry = acc;
    }
    __syncthreads();
    // running value after the last emitter at or before this entry
    const unsigned upto = nz[wid] & (0xffffffffu >> (31u - lane));
    double c;
    if (upto)
      c = term[wid * 32 + 31 - __clz(upto)];
    else
      c = wid > 0 ? warp_end[wid - 1] : start;
    if (i < S) t.cdf[i] = c;
    __syncthreads();
  }
  if (tid == 0) {
    *t.W = carry;
    if (step_dev && !(skip && *skip)) *step_dev += 1;
  }
}

__global__ void k_tables_samp(const float* sparams, uint32_t S, SegBuffers t) {
  const double W = *t.W;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const float rs = sparams[10 * s + 6];
    const double le = t.lum[s];
    t.samp[s] = make_float4(fmaxf(rs * rs, 1e-4f), (float)t.pspec[s],
                            (W > 0.0 && le > 0.0) ? (float)(le / W) : 0.0f, 0.0f);
  }
}

static cudaError_t launch_tables_wide(const SceneBuffers& s, const SegBuffers& t, const float* params,
                                      const float* sparams, int* step_dev, const uint32_t* skip, cudaStream_t st) {
  const int grid = (int)std::min<uint32_t>((s.n_seg + 255u) / 256u, 1024u);
  k_tables_seg<<<grid, 256, 0, st>>>(params, sparams, s.n_seg, s.emission_scale, t);
  k_tables_cdf<<<1, 1024, 0, st>>>(s.n_seg, s.seg_area, t, step_dev, skip);
  k_tables_samp<<<grid, 256, 0, st>>>(sparams, s.n_seg, t);
  return cudaGetLastError();
}


__global__ void k_trace_rays(SceneDev s, const uint32_t* orig_to_internal, uint32_t n, const float* orig,
                             const float* dir, const int32_t* skip, int32_t* tri_out, float* t_out,
                             float* u_out, float* v_out, uint32_t* err) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float3 o = f3(orig[3 * i], orig[3 * i + 1], orig[3 * i + 2]);
  const float3 d = f3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
  int sk = -1;
  if (skip && skip[i] >= 0 && (uint32_t)skip[i] < s.n_tri) sk = (int)orig_to_internal[skip[i]];
  const Hit h = trace_closest(s, o, d, __int_as_float(0x7f800000), sk, err);
  tri_out[i] = h.tri >= 0 ? __float_as_int(__ldg(&s.tris[3 * h.tri]).w) : -1;
  if (t_out) t_out[i] = h.t;
  if (u_out) u_out[i] = h.u;
  if (v_out) v_out[i] = h.v;
}

__global__ void k_philox(uint32_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 o = philox4x32_10(c, make_uint2(key[2 * i], key[2 * i + 1]));
  out[4 * i] = o.x;
  out[4 * i + 1] = o.y;
  out[4 * i + 2] = o.z;
  out[4 * i + 3] = o.w;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <int MAXD>
static void adjoint_occupancy(int* out) {
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_adjoint<MAXD>, kBlockThreads, 16384);
}

cudaError_t init_launcher(Launcher* L, int device) {
  cudaError_t e = cudaDeviceGetAttribute(&L->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->fwd_blocks_per_sm, k_forward, kBlockThreads, 0);
  if (e != cudaSuccess) return e;
  adjoint_occupancy<2>(&L->adj_blocks_per_sm[0]);
  adjoint_occupancy<4>(&L->adj_blocks_per_sm[1]);
  adjoint_occupancy<6>(&L->adj_blocks_per_sm[2]);
  adjoint_occupancy<8>(&L->adj_blocks_per_sm[3]);
  for (int i = 0; i < 4; ++i)
    if (L->adj_blocks_per_sm[i] < 1) L->adj_blocks_per_sm[i] = 1;
  if (L->fwd_blocks_per_sm < 1) L->fwd_blocks_per_sm = 1;
  e = wf_init(L);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int loss_partials_capacity(const Launcher& L) { return L.num_sms * L.fwd_blocks_per_sm; }

static int grid_for(uint64_t n_tasks_warps, int blocks_cap) {
  const uint64_t per_block = kBlockThreads / 32;
  uint64_t g = (n_tasks_warps + per_block - 1) / per_block;
  if (g > (uint64_t)blocks_cap) g = blocks_cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_prepare(const SceneBuffers& s, const SegBuffers& t, const float* params,
                           const float* sparams, cudaStream_t st) {
  if (s.n_seg > kWideSegments) return launch_tables_wide(s, t, params, sparams ? sparams : params, nullptr, nullptr, st);
  k_prepare<<<1, 256, 0, st>>>(params, sparams ? sparams : params, s.n_seg, s.emission_scale, s.seg_area, t);
  return cudaGetLastError();
}

cudaError_t launch_forward(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                           const ViewHost* views_dev, uint32_t n_views, uint32_t pix_begin,
                           uint32_t n_pix, const TraceParams& tp, float* img, float* msq,
                           const float* target, float* g_out, double* loss_partials,
                           float g_scale, int loss_kind, uint32_t* err, cudaStream_t st) {
  const PathParams pp = make_path_params(tp, s);
  const uint64_t tasks = (n_pix + (32 / pp.group) - 1) / (32 / pp.group);
  const int cap = L.num_sms * L.fwd_blocks_per_sm;
  // with a loss the grid is fixed, so the partial sums reduce in a fixed order
  const int grid = loss_partials ? cap : grid_for(tasks, cap);
  k_forward<<<grid, kBlockThreads, 0, st>>>(scene_dev(s), seg_dev(t), reinterpret_cast<const ViewDev*>(views_dev),
                                             n_views, pix_begin, n_pix, pp, img, msq, target, g_out,
                                             loss_partials, g_scale, loss_kind, err);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                           const ViewHost* views_dev, uint32_t n_views, uint32_t pix_begin, uint32_t n_pix,
                           const TraceParams& tp, const float* g_img, double* grad_acc,
                           float* gacc_scratch, uint32_t* err, cudaStream_t st) {
  const PathParams pp = make_path_params(tp, s);
  const uint64_t tasks = (n_pix + (32 / pp.group) - 1) / (32 / pp.group);
  // above wf_max_segments() segments the accumulators move to global memory
  const bool global = s.n_seg > wf_max_segments();
  if (global && !gacc_scratch) return cudaErrorInvalidValue;
  float* gacc = global ? gacc_scratch : nullptr;
  const size_t shmem = global ? 0 : sizeof(float) * 10u * s.n_seg;
  if (global) {
    cudaError_t e = cudaMemsetAsync(gacc, 0, sizeof(float) * 10u * s.n_seg, st);
    if (e != cudaSuccess) return e;
  }
  const ViewDev* vd = reinterpret_cast<const ViewDev*>(views_dev);
  const int md = tp.max_depth < 1 ? 1 : (int)tp.max_depth;
#define IPT_LAUNCH_ADJ(D, I)                                                                         \
  {                                                                                                  \
    if (shmem > 48 * 1024)                                                                           \
      cudaFuncSetAttribute(k_adjoint<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);  \
    const int grid = grid_for(tasks, L.num_sms * L.adj_blocks_per_sm[I]);                            \
    k_adjoint<D><<<grid, kBlockThreads, shmem, st>>>(scene_dev(s), seg_dev(t), vd, n_views, pix_begin, n_pix, pp, \
                                                     g_img, grad_acc, gacc, err);                    \
  }
  if (md <= 2)
    IPT_LAUNCH_ADJ(2, 0)
  else if (md <= 4)
    IPT_LAUNCH_ADJ(4, 1)
  else if (md <= 6)
    IPT_LAUNCH_ADJ(6, 2)
  else
    IPT_LAUNCH_ADJ(8, 3)
#undef IPT_LAUNCH_ADJ
  if (global) k_add_to_double<<<(10u * s.n_seg + 255) / 256, 256, 0, st>>>(gacc, 10u * s.n_seg, grad_acc);
  return cudaGetLastError();
}

static PathParams batch_path_params(const TraceParams& tp) {
  PathParams p{};
  p.spp = tp.spp;
  p.group = lanes_per_pixel(tp.spp);
  p.max_depth = tp.max_depth;
  p.nee = tp.nee;
  p.mis = tp.mis;
  p.profile = tp.profile;
  p.stride = tp.sample_stride ? tp.sample_stride : tp.spp;
  return p;
}

cudaError_t launch_forward_batch(const Launcher& L, const WfScene* tab_dev, uint32_t n_scenes, uint32_t total,
                                 const TraceParams& tp, const uint32_t* iter_dev, int loss_kind, double* loss_rows,
                                 uint32_t* err, cudaStream_t st) {
  // one block per loss row: every row of the batch's loss reduction is written
  k_forward_batch<<<loss_partials_capacity(L), kBlockThreads, sizeof(double) * n_scenes, st>>>(
      tab_dev, n_scenes, total, batch_path_params(tp), tp.set, iter_dev, loss_kind, loss_rows, err);
  return cudaGetLastError();
}

uint32_t batch_shared_params() { return (96u * 1024u) / (uint32_t)sizeof(float); }

cudaError_t launch_adjoint_batch(const Launcher& L, const WfScene* tab_dev, uint32_t n_scenes, uint32_t total,
                                 uint32_t n_seg, const TraceParams& tp, const uint32_t* iter_dev, double* grad_acc,
                                 float* gacc_scratch, uint32_t* err, cudaStream_t st) {
  const PathParams pp = batch_path_params(tp);
  const uint32_t n_par = 10u * n_seg;
  const bool global = n_par > batch_shared_params();
  if (global && !gacc_scratch) return cudaErrorInvalidValue;
  float* gacc = global ? gacc_scratch : nullptr;
  const size_t shmem = global ? 0 : sizeof(float) * n_par;
  if (global) {
    cudaError_t e = cudaMemsetAsync(gacc, 0, sizeof(float) * n_par, st);
    if (e != cudaSuccess) return e;
  }
  const uint64_t tasks = ((uint64_t)total + (32 / pp.group) - 1) / (32 / pp.group);
  const int md = tp.max_depth < 1 ? 1 : (int)tp.max_depth;
#define IPT_LAUNCH_ADJB(D, I)                                                                              \
  {                                                                                                        \
    if (shmem > 48 * 1024)                                                                                 \
      cudaFuncSetAttribute(k_adjoint_batch<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);  \
    const int grid = grid_for(tasks, L.num_sms * L.adj_blocks_per_sm[I]);                                  \
    k_adjoint_batch<D><<<grid, kBlockThreads, shmem, st>>>(tab_dev, n_scenes, total, n_par, pp, tp.set,    \
                                                           iter_dev, grad_acc, gacc, err);                 \
  }
  if (md <= 2)
    IPT_LAUNCH_ADJB(2, 0)
  else if (md <= 4)
    IPT_LAUNCH_ADJB(4, 1)
  else if (md <= 6)
    IPT_LAUNCH_ADJB(6, 2)
  else
    IPT_LAUNCH_ADJB(8, 3)
#undef IPT_LAUNCH_ADJB
  if (global) k_add_to_double<<<(n_par + 255) / 256, 256, 0, st>>>(gacc, n_par, grad_acc);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* loss_partials, int n_partials, double* loss_dev,
                            const double* grad_acc, float* grad_out, uint32_t n_params,
                            cudaStream_t st) {
  k_finalize<<<1, 256, 0, st>>>(loss_partials, n_partials, loss_dev, grad_acc, grad_out, n_params);
  return cudaGetLastError();
}

cudaError_t launch_adam(const SceneBuffers& s, const SegBuffers& t, float* params, float* m,
                        float* v, const uint8_t* free_mask, const double* grad_acc,
                        const float* grad_f, int* step_dev, const AdamHost& a, const double* loss,
                        uint32_t* guard, uint32_t* err, cudaStream_t st) {
  if (s.n_seg > kWideSegments) {
    k_finite_guard<<<1, 1024, 0, st>>>(loss, grad_acc, grad_f, 10u * s.n_seg, guard, err);
    const int grid = (int)std::min<uint32_t>((10u * s.n_seg + 255u) / 256u, 2048u);
    k_adam_wide<<<grid, 256, 0, st>>>(params, m, v, free_mask, grad_acc, grad_f, step_dev, a, s.n_seg, guard);
    return launch_tables_wide(s, t, params, params, step_dev, guard, st);
  }
  k_adam<<<1, 256, 0, st>>>(params, m, v, free_mask, grad_acc, grad_f, step_dev, a, s.n_seg,
                            s.emission_scale, s.seg_area, t, loss, err);
  return cudaGetLastError();
}

cudaError_t launch_adam_batch(const BatchMember* members, uint32_t n_members, float* params, float* m, float* v,
                              const uint8_t* free_mask, const double* grad_acc, const uint32_t* iter_dev,
                              const AdamHost& a, const double* losses, uint32_t* err, cudaStream_t st) {
  k_adam_batch<<<n_members, 256, 0, st>>>(members, params, m, v, free_mask, grad_acc, iter_dev, a, losses, err);
  return cudaGetLastError();
}

cudaError_t launch_prepare_batch(const BatchMember* members, uint32_t n_members, const float* params,
                                 cudaStream_t st) {
  k_prepare_batch<<<n_members, 256, 0, st>>>(members, params);
  return cudaGetLastError();
}

cudaError_t launch_batch_losses(const double* rows, int n_rows, const BatchMember* members, uint32_t n,
                                uint32_t n_tab, double* loss, cudaStream_t st) {
  k_batch_losses<<<n, 256, 0, st>>>(rows, n_rows, members, n_tab, loss);
  return cudaGetLastError();
}

cudaError_t launch_tick(uint32_t* counter, cudaStream_t st) {
  k_tick<<<1, 1, 0, st>>>(counter);
  return cudaGetLastError();
}

cudaError_t launch_trace_rays(const SceneBuffers& s, uint32_t n, const float* orig,
                              const float* dir, const int32_t* skip, int32_t* tri_out,
                              float* t_out, float* u_out, float* v_out, uint32_t* err,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int block = 128;
  k_trace_rays<<<(n + block - 1) / block, block, 0, st>>>(scene_dev(s), s.orig_to_internal, n, orig, dir, skip,
                                                           tri_out, t_out, u_out, v_out, err);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_philox<<<(n + 255) / 256, 256, 0, st>>>(n, ctr, key, out);
  return cudaGetLastError();
}

}  // namespace ipt
