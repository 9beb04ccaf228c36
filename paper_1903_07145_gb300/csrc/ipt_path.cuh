// Path construction shared by the megakernel and the wavefront integrator:
// per-segment tables, vertex set-up, MIS weights, camera rays, next-event
// estimation and BRDF evaluation.  Both integrators draw the same random
// numbers at the same (vertex, call) slots, so they build identical paths.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ipt_device.cuh"
#include "ipt_internal.h"

namespace ipt {

constexpr double kLumR = 0.2126, kLumG = 0.7152, kLumB = 0.0722;  // Rec. 709 luminance

struct PathParams {
  uint2 key;
  uint32_t set_iter;  // (set << 24) | (iteration & 0xFFFFFF)
  uint32_t spp;
  uint32_t group;     // lanes per pixel (power of two dividing spp, <= 32)
  uint32_t max_depth;
  int nee, mis, profile;
  float emission_scale;
  // pixel batch: launch pixel i is entry i, tracing scene pixel pick[i] with
  // sample counters i * stride + s (nullptr: launch pixel i is pixel
  // pix_begin + i with counters s)
  const uint32_t* pick;
  uint32_t stride;
};

__host__ __device__ inline uint32_t lanes_per_pixel(uint32_t spp) {
  uint32_t g = 1;
  while (g < 32 && (spp % (2 * g)) == 0) g *= 2;
  return g;
}

inline PathParams make_path_params(const TraceParams& tp, const SceneBuffers& s) {
  PathParams p;
  p.key = make_uint2((uint32_t)(tp.seed & 0xFFFFFFFFu), (uint32_t)(tp.seed >> 32) ^ tp.scene_id);
  p.set_iter = (tp.set << 24) | (uint32_t)(tp.iteration & 0xFFFFFFu);
  p.spp = tp.spp;
  p.group = lanes_per_pixel(tp.spp);
  p.max_depth = tp.max_depth;
  p.nee = tp.nee;
  p.mis = tp.mis;
  p.profile = tp.profile;
  p.emission_scale = s.emission_scale;
  p.pick = tp.pick;
  p.stride = tp.sample_stride ? tp.sample_stride : tp.spp;
  return p;
}

inline SceneDev scene_dev(const SceneBuffers& s) {
  SceneDev d;
  d.nodes = s.nodes;
  d.nodes4 = s.nodes4;
  d.nodes8 = s.nodes8;
  d.tris = s.tris;
  d.vnrm = s.vnrm;
  d.seg_tris = s.seg_tris;
  d.seg_begin = s.seg_begin;
  d.tri_cdf = s.tri_cdf;
  d.seg_area = s.seg_area;
  d.n_seg = s.n_seg;
  d.n_tri = s.n_tri;
  d.eps = s.eps;
  d.counters = s.counters;
  d.wide = s.wide;
  return d;
}

inline SegDev seg_dev(const SegBuffers& t) {
  SegDev d;
  d.mat_a = t.mat_a;
  d.mat_b = t.mat_b;
  d.emis = t.emis;
  d.samp = t.samp;
  d.pspec = t.pspec;
  d.cdf = t.cdf;
  d.W = t.W;
  return d;
}

// ---------------------------------------------------------------------------
// Parameter tables.  Decisions that pick an integer (light segment, lobe) are
// taken in FP64 from FP64 tables evaluated without contraction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lum_d(double r, double g, double b) {
  return __dadd_rn(__dadd_rn(__dmul_rn(kLumR, r), __dmul_rn(kLumG, g)), __dmul_rn(kLumB, b));
}

inline __device__ void build_tables(const float* params, const float* sparams, uint32_t S, float es,
                             const double* seg_area, SegBuffers t) {
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
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
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (uint32_t s = 0; s < S; ++s) {
      acc = __dadd_rn(acc, __dmul_rn(t.lum[s], seg_area[s]));
      t.cdf[s] = acc;
    }
    *t.W = acc;
  }
  __syncthreads();
  const double W = *t.W;
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
    const float rs = sparams[10 * s + 6];
    const double le = t.lum[s];
    t.samp[s] = make_float4(fmaxf(rs * rs, 1e-4f), (float)t.pspec[s],
                            (W > 0.0 && le > 0.0) ? (float)(le / W) : 0.0f, 0.0f);
  }
}


// ---------------------------------------------------------------------------
// Path construction shared by the forward and adjoint kernels.
// ---------------------------------------------------------------------------
struct Vtx {
  int tri, seg;
  float3 x, ng, ns, wi;  // normals oriented to the incoming side
  float cos_e;           // wi . n_g (unflipped): > 0 on the emitting face
  float prof;            // emission profile toward wi
};

__device__ __forceinline__ Vtx make_vertex(const SceneDev& s, const Hit& h, float3 d, int profile) {
  Vtx v;
  v.tri = h.tri;
  const float4 q0 = __ldg(&s.tris[3 * h.tri + 0]);
  const float4 q1 = __ldg(&s.tris[3 * h.tri + 1]);
  const float4 q2 = __ldg(&s.tris[3 * h.tri + 2]);
  v.seg = __float_as_int(q1.w);
  const float w0 = 1.0f - h.u - h.v;
  const float3 p0 = xyz(q0), p1 = xyz(q1), p2 = xyz(q2);
  v.x = p0 * w0 + p1 * h.u + p2 * h.v;
  const float3 ng0 = normalize(cross(p1 - p0, p2 - p0));
  float3 ns = ng0;
  if (s.vnrm) {
    const float3 a = xyz(__ldg(&s.vnrm[3 * h.tri + 0]));
    const float3 b = xyz(__ldg(&s.vnrm[3 * h.tri + 1]));
    const float3 c = xyz(__ldg(&s.vnrm[3 * h.tri + 2]));
    ns = normalize(a * w0 + b * h.u + c * h.v);
  }
  v.wi = -d;
  v.cos_e = dot(v.wi, ng0);
  v.prof = profile == 0 ? fmaxf(0.0f, v.cos_e) : (v.cos_e > 0.0f ? 1.0f : 0.0f);
  const float sg = v.cos_e < 0.0f ? -1.0f : 1.0f;
  v.ng = ng0 * sg;
  v.ns = ns * sg;
  return v;
}

// MIS weight of emission found by BRDF sampling (power heuristic, beta = 2).
__device__ __forceinline__ float emission_weight(const SegDev& t, const Vtx& v, float dist, bool after_scatter,
                                                 bool prev_light, float prev_pdf, int mis) {
  if (!after_scatter || !prev_light) return 1.0f;
  const float pa = __ldg(&t.samp[v.seg]).z;
  if (!(pa > 0.0f) || !(v.cos_e > 0.0f)) return 1.0f;
  if (!mis) return 0.0f;
  const float pl = pa * dist * dist / v.cos_e;
  return prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl);
}

__device__ __forceinline__ float3 camera_ray(const ViewDev& vw, uint32_t px, uint32_t py, const PathRng& rng,
                                             float3& org) {
  const float4 u = rng.draw(0, 2);
  const float ndc_x = 2.0f * ((float)px + u.x) / (float)vw.w - 1.0f;
  const float ndc_y = 1.0f - 2.0f * ((float)py + u.y) / (float)vw.h;
  const float3 dc = f3(ndc_x * vw.tx, ndc_y * vw.ty, -1.0f);
  const float* M = vw.m;
  org = f3(M[3], M[7], M[11]);
  return normalize(f3(M[0] * dc.x + M[1] * dc.y + M[2] * dc.z, M[4] * dc.x + M[5] * dc.y + M[6] * dc.z,
                      M[8] * dc.x + M[9] * dc.y + M[10] * dc.z));
}

struct NeeResult {
  bool valid;
  int seg;       // emitting segment
  int tri;       // light triangle (internal id)
  float3 wl;
  float k;       // cos_x * profile * (cos_l / r^2) / p_A * w_light
  float3 so;     // shadow ray: origin, unit direction, extent
  float3 sd;
  float st;
};

// Light selection proportional to lum(e_s) A_s, then area within the segment,
// then a uniform point (sqrt parameterisation).  Returns the candidate with
// its shadow ray (from the offset point, skipping both end triangles); the
// candidate counts only if that ray is unoccluded.  bsdf_pdf_to(wl) is the
// material sampler's solid-angle pdf towards wl (for the MIS weight).
template <class PdfTo>
__device__ __forceinline__ NeeResult nee_prepare_with(const SceneDev& s, const SegDev& t, const Vtx& v, float4 ua,
                                                      float4 ub, double W, int profile, int mis,
                                                      const PdfTo& bsdf_pdf_to) {
  NeeResult r;
  r.valid = false;
  const int sl = upper_bound_d(t.cdf, 0, (int)s.n_seg, (double)ua.w * W);
  const int b = (int)__ldg(&s.seg_begin[sl]), e = (int)__ldg(&s.seg_begin[sl + 1]);
  if (e <= b) return r;  // a segment without triangles is never selectable; guard anyway
  const int j = upper_bound_d(s.tri_cdf, b, e, (double)ub.x * __ldg(&s.seg_area[sl]));
  const int lt = (int)__ldg(&s.seg_tris[j]);
  const float3 p0 = xyz(__ldg(&s.tris[3 * lt + 0]));
  const float3 p1 = xyz(__ldg(&s.tris[3 * lt + 1]));
  const float3 p2 = xyz(__ldg(&s.tris[3 * lt + 2]));
  const float su = sqrtf(ub.y);
  const float b0 = 1.0f - su, b1 = ub.z * su, b2 = 1.0f - b0 - b1;
  const float3 y = p0 * b0 + p1 * b1 + p2 * b2;
  const float3 dl = y - v.x;
  const float r2 = dot(dl, dl);
  const float3 wl = dl * rsqrtf(r2);
  const float3 nl = normalize(cross(p1 - p0, p2 - p0));
  const float cos_l = -dot(wl, nl);
  const float lprof = profile == 0 ? fmaxf(0.0f, cos_l) : (cos_l > 0.0f ? 1.0f : 0.0f);
  const float cxg = dot(wl, v.ng), cxs = dot(wl, v.ns);
  if (!(lprof > 0.0f) || !(cxg > 0.0f) || !(cxs > 0.0f) || !(dot(v.wi, v.ns) > 0.0f)) return r;
  r.so = v.x + v.ng * s.eps;
  const float3 ds = y - r.so;
  const float rs = sqrtf(dot(ds, ds));
  r.sd = ds * (1.0f / rs);
  r.st = rs * 0.99999f;
  const float pA = __ldg(&t.samp[sl]).z;
  float wlight = 1.0f;
  if (mis) {
    const float pl = pA * r2 / cos_l;
    const float pb = bsdf_pdf_to(wl);
    wlight = pl * pl / (pl * pl + pb * pb);
  }
  r.valid = true;
  r.seg = sl;
  r.tri = lt;
  r.wl = wl;
  r.k = cxs * lprof * (cos_l / r2) / pA * wlight;
  return r;
}

// Lambert + GGX: the mixture sampler of bsdf_sample.
__device__ __forceinline__ NeeResult nee_prepare(const SceneDev& s, const SegDev& t, const Vtx& v, float4 ua,
                                                 float4 ub, double W, int profile, int mis, float P, float a_s) {
  return nee_prepare_with(s, t, v, ua, ub, W, profile, mis,
                          [&](float3 wl) { return bsdf_pdf(P, a_s, v.ns, v.wi, wl); });
}

// Next-event estimation with the visibility test done in place.
__device__ __forceinline__ NeeResult next_event(const SceneDev& s, const SegDev& t, const Vtx& v, float4 ua,
                                                float4 ub, double W, int profile, int mis, float P,
                                                float a_s, uint32_t* err) {
  NeeResult r = nee_prepare(s, t, v, ua, ub, W, profile, mis, P, a_s);
  if (r.valid && trace_any(s, r.so, r.sd, r.st, v.tri, r.tri, err)) r.valid = false;
  return r;
}

struct BrdfVal {
  float3 f;
  Spec sp;
};

__device__ __forceinline__ BrdfVal brdf_eval(float4 ma, float4 mb, float3 n, float3 wi, float3 wo) {
  const float ci = dot(n, wi), co = dot(n, wo);
  const float3 h = normalize(wi + wo);
  BrdfVal b;
  b.sp = spec_term(ci, co, dot(n, h), ma.w, mb.w);
  b.f = f3(ma.x, ma.y, ma.z) * (1.0f / kPi) + f3(mb.x, mb.y, mb.z) * b.sp.s;
  return b;
}

__device__ __forceinline__ const ViewDev& find_view(const ViewDev* views, uint32_t n_views, uint32_t p) {
  uint32_t v = n_views - 1;
  while (v > 0 && p < views[v].offset) --v;
  return views[v];
}


}  // namespace ipt
