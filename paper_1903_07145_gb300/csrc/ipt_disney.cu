// Disney material model on the megakernel integrator: per-segment tables
// from the 16-value parameter blocks, the forward pixel estimate (Eq. 1-2
// with NEE and MIS) and its adjoint (Eq. 5-6), and Adam with the model's
// clamps.  Path construction, light selection, random-number slots and the
// residual follow the Lambert + GGX kernels; only the material differs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipt_disney.cuh"
#include "ipt_internal.h"

namespace ipt {
namespace {

constexpr int kDisneyThreads = 128;

// Per-segment tables of one scene (one block): material values, emission,
// the FP64 lobe probabilities and sampling widths from the sampling
// parameters, and the emission-proportional light-selection CDF.
__device__ void disney_tables_body(const float* params, const float* sparams, uint32_t S, float es,
                                   const double* seg_area, const SegBuffers& t, const DisneyBuffers& d) {
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
    const float* p = params + kDisneyStride * s;
    const float* q = sparams + kDisneyStride * s;
    d.mat[4 * s + 0] = make_float4(p[0], p[1], p[2], p[3]);
    d.mat[4 * s + 1] = make_float4(p[4], p[5], p[6], p[7]);
    d.mat[4 * s + 2] = make_float4(p[8], p[9], p[10], p[11]);
    d.mat[4 * s + 3] = make_float4(p[12], 0.0f, 0.0f, 0.0f);
    t.emis[s] = make_float4(es * p[13], es * p[14], es * p[15], 0.0f);
    // lobe weights (1 - mu) lum(base), (1 - mu) 0.08 specular + mu lum(base),
    // clearcoat / 4, in FP64 without contraction
    const double lb = lum_d(q[0], q[1], q[2]);
    const double om = __dsub_rn(1.0, (double)q[4]);
    const double wd = __dmul_rn(om, lb);
    const double ws = __dadd_rn(__dmul_rn(__dmul_rn(om, 0.08), (double)q[5]), __dmul_rn((double)q[4], lb));
    const double wc = __dmul_rn(0.25, (double)q[11]);
    const double sum = __dadd_rn(__dadd_rn(wd, ws), wc);
    double p0 = 1.0, p1 = 0.0, p2 = 0.0;
    if (sum > 0.0) {
      p0 = __ddiv_rn(wd, sum);
      p1 = __ddiv_rn(ws, sum);
      p2 = __ddiv_rn(wc, sum);
    }
    d.lobe[s] = make_double2(p0, __dadd_rn(p0, p1));
    const float k = sqrtf(1.0f - 0.9f * q[8]);
    const float r2 = q[7] * q[7];
    d.samp[2 * s] = make_float4(fmaxf(r2 / k, 1e-3f), fmaxf(r2 * k, 1e-3f), 0.1f - 0.099f * q[12], 0.0f);
    d.samp[2 * s + 1] = make_float4((float)p0, (float)p1, (float)p2, 0.0f);
    double le = lum_d(q[13], q[14], q[15]);
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
    const double le = t.lum[s];
    t.samp[s] = make_float4(0.0f, 0.0f, (W > 0.0 && le > 0.0) ? (float)(le / W) : 0.0f, 0.0f);
  }
}

__global__ void k_disney_tables(const float* params, const float* sparams, uint32_t S, float es,
                                const double* seg_area, SegBuffers t, DisneyBuffers d) {
  disney_tables_body(params, sparams, S, es, seg_area, t, d);
}

// A non-finite loss or gradient skips the update (parameters, moments and
// step count unchanged) and sets the error word; the tables are rebuilt
// either way.
__global__ void k_disney_adam(float* params, float* m, float* v, const uint8_t* free_mask, const double* grad_acc,
                              const float* grad_f, int* step_dev, AdamHost a, uint32_t S, float es,
                              const double* seg_area, SegBuffers t, DisneyBuffers d, const double* loss,
                              uint32_t* err) {
  const int step = *step_dev + 1;
  const float bc1 = 1.0f - powf(a.beta1, (float)step);
  const float bc2 = 1.0f - powf(a.beta2, (float)step);
  bool bad = loss && !isfinite(*loss);
  for (uint32_t i = threadIdx.x; i < kDisneyStride * S && !bad; i += blockDim.x)
    bad = grad_f ? !isfinite(grad_f[i]) : !isfinite(grad_acc[i]);
  bad = __syncthreads_or(bad) != 0;
  for (uint32_t i = threadIdx.x; !bad && i < kDisneyStride * S; i += blockDim.x) {
    if (free_mask && !free_mask[i]) continue;
    const uint32_t j = i % kDisneyStride;
    float g = grad_f ? grad_f[i] : (float)grad_acc[i];
    const float th = params[i];
    if (j >= (uint32_t)kDisneyMat) g += a.l1 * (th > 0.0f ? 1.0f : (th < 0.0f ? -1.0f : 0.0f));
    const float mi = a.beta1 * m[i] + (1.0f - a.beta1) * g;
    const float vi = a.beta2 * v[i] + (1.0f - a.beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float nt = th - a.lr * (mi / bc1) / (sqrtf(vi / bc2) + a.eps);
    if (j < (uint32_t)kDisneyMat)
      nt = fminf(fmaxf(nt, j == 7 ? 0.02f : 0.0f), 1.0f);
    else
      nt = fmaxf(nt, 0.0f);
    params[i] = nt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bad)
      atomicOr(err, kErrNonFinite);
    else
      *step_dev = step;
  }
  disney_tables_body(params, params, S, es, seg_area, t, d);
}

// acc[j] += sum_c q_c d f_c(wi, wo) / d m_j for the 13 material values.
__device__ __forceinline__ void disney_grad(const float (&m)[kDisneyMat], float3 n, float3 X, float3 Y, float3 wi,
                                            float3 wo, float3 q, float* acc) {
  float g[kDisneyMat];
  if (!disney_vjp(m, n, X, Y, wi, wo, q, g)) return;
#pragma unroll
  for (int j = 0; j < kDisneyMat; ++j)
    if (g[j] != 0.0f) atomicAdd(&acc[j], g[j]);
}

__device__ __forceinline__ void add3d(float* acc, int i, float3 v) {
  atomicAdd(&acc[i], v.x);
  atomicAdd(&acc[i + 1], v.y);
  atomicAdd(&acc[i + 2], v.z);
}

// Radiance estimate of one camera path (the Lambert + GGX forward path with
// the Disney material and sampler).
__device__ float3 disney_forward_path(const SceneDev& s, const SegDev& t, const DisneyDev& D, const ViewDev& vw,
                                      uint32_t px, uint32_t py, uint32_t pid, uint32_t sample, const PathParams& pp,
                                      double W, uint32_t* err) {
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
    float3 X, Y;
    hit_frame(s, h.tri, v.ns, X, Y);
    float m[kDisneyMat];
    load_disney(D, v.seg, m);
    if (light_on) {
      NeeResult ne = nee_prepare_with(s, t, v, ua, ub, W, pp.profile, pp.mis,
                                      [&](float3 wl) { return disney_pdf(D, v.seg, v.ns, X, Y, v.wi, wl); });
      if (ne.valid && trace_any(s, ne.so, ne.sd, ne.st, v.tri, ne.tri, err)) ne.valid = false;
      if (ne.valid) L = L + beta * disney_eval(m, v.ns, X, Y, v.wi, ne.wl) * xyz(__ldg(&t.emis[ne.seg])) * ne.k;
    }
    if (!(dot(v.wi, v.ns) > 0.0f)) break;
    const float3 wo = disney_sample(D, v.seg, v.ns, X, Y, v.wi, ua.x, ua.y, ua.z);
    const float pdf = disney_pdf(D, v.seg, v.ns, X, Y, v.wi, wo);
    const float co = dot(wo, v.ns);
    if (!(dot(wo, v.ng) > 0.0f) || !(co > 0.0f) || !(pdf > 0.0f)) break;
    beta = beta * disney_eval(m, v.ns, X, Y, v.wi, wo) * (co / pdf);
    prev_pdf = pdf;
    o = v.x + v.ng * s.eps;
    d = wo;
    skip = h.tri;
  }
  return L;
}

// Derivative of one camera path contracted with the pixel's upstream
// gradient gp, scattered into acc (16 per segment).  As in the Lambert + GGX
// adjoint, vertex l keeps T_l (throughput without its own weight) and U_l
// (later contributions through T_l); its weight w_l = f_r(wi, wo) cos / pdf
// is differentiated at the end, when U_l is known, from the stored
// directions.  Emission (Eq. 5) and the local NEE term are differentiated on
// the spot; pdfs and MIS weights are held constant.
template <int MAXD>
__device__ void disney_adjoint_path(const SceneDev& s, const SegDev& t, const DisneyDev& D, const ViewDev& vw,
                                    uint32_t px, uint32_t py, uint32_t pid, uint32_t sample, const PathParams& pp,
                                    double W, float3 gp, float* acc, uint32_t* err) {
  PathRng rng;
  rng.base = make_uint4(pid, sample, pp.set_iter, 0);
  rng.key = pp.key;
  float3 o;
  float3 d = camera_ray(vw, px, py, rng, o);
  float3 beta = f3(1.0f, 1.0f, 1.0f);
  const bool light_on = pp.nee && W > 0.0;
  const float es = pp.emission_scale;
  float3 T[MAXD], U[MAXD], WI[MAXD], WO[MAXD], NS[MAXD], TX[MAXD];
  float KK[MAXD];
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
        add3d(acc, kDisneyStride * v.seg + kDisneyMat, gp * beta * (f * es));  // Eq. 5 at the hit
      }
    }
    const bool last = k == pp.max_depth;
    float3 X = f3(1.0f, 0.0f, 0.0f), Y = f3(0.0f, 1.0f, 0.0f);
    float m[kDisneyMat];
    float4 ua = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!last) {
      hit_frame(s, h.tri, v.ns, X, Y);
      load_disney(D, v.seg, m);
      ua = rng.draw(k, 0);
      const float4 ub = rng.draw(k, 1);
      if (light_on) {
        NeeResult ne = nee_prepare_with(s, t, v, ua, ub, W, pp.profile, pp.mis,
                                        [&](float3 wl) { return disney_pdf(D, v.seg, v.ns, X, Y, v.wi, wl); });
        if (ne.valid && trace_any(s, ne.so, ne.sd, ne.st, v.tri, ne.tri, err)) ne.valid = false;
        if (ne.valid) {
          const float3 fv = disney_eval(m, v.ns, X, Y, v.wi, ne.wl);
          const float3 Le = xyz(__ldg(&t.emis[ne.seg]));
          C = C + fv * Le * ne.k;
          add3d(acc, kDisneyStride * ne.seg + kDisneyMat, gp * beta * fv * (ne.k * es));  // Eq. 5, light end
          disney_grad(m, v.ns, X, Y, v.wi, ne.wl, gp * beta * Le * ne.k, acc + kDisneyStride * v.seg);  // Eq. 6
        }
      }
    }
#pragma unroll
    for (int l = 0; l < MAXD; ++l)
      if (l < nv) U[l] = U[l] + T[l] * C;
    if (last || !(dot(v.wi, v.ns) > 0.0f)) break;
    const float3 wo = disney_sample(D, v.seg, v.ns, X, Y, v.wi, ua.x, ua.y, ua.z);
    const float pdf = disney_pdf(D, v.seg, v.ns, X, Y, v.wi, wo);
    const float co = dot(wo, v.ns);
    if (!(dot(wo, v.ng) > 0.0f) || !(co > 0.0f) || !(pdf > 0.0f)) break;
    const float kk = co / pdf;
    const float3 w = disney_eval(m, v.ns, X, Y, v.wi, wo) * kk;
#pragma unroll
    for (int l = 0; l < MAXD; ++l) {
      if (l < nv) T[l] = T[l] * w;
      if (l == nv) {
        T[l] = beta;
        U[l] = f3(0.0f, 0.0f, 0.0f);
        WI[l] = v.wi;
        WO[l] = wo;
        NS[l] = v.ns;
        TX[l] = X;
        KK[l] = kk;
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
#pragma unroll 1
  for (int l = 0; l < MAXD; ++l) {
    if (l >= nv) break;
    float3 wi, wo, n, X, Uq;
    float kk;
    int sg;
    // select vertex l's record (register arrays indexed by a constant)
#pragma unroll
    for (int i = 0; i < MAXD; ++i)
      if (i == l) {
        wi = WI[i];
        wo = WO[i];
        n = NS[i];
        X = TX[i];
        Uq = U[i];
        kk = KK[i];
        sg = SG[i];
      }
    const float3 q = gp * Uq * kk;
    if (q.x == 0.0f && q.y == 0.0f && q.z == 0.0f) continue;
    float m[kDisneyMat];
    load_disney(D, sg, m);
    disney_grad(m, n, X, cross(n, X), wi, wo, q, acc + kDisneyStride * sg);
  }
}

__global__ void __launch_bounds__(kDisneyThreads)
    k_disney_forward(SceneDev s, SegDev t, DisneyDev D, const ViewDev* views, uint32_t n_views, uint32_t pix_begin,
                     uint32_t n_pix, PathParams pp, float* img, float* msq, const float* target, float* g_out,
                     double* loss_partials, float g_scale, int loss_kind, uint32_t* err) {
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
        const float3 L = disney_forward_path(s, t, D, vw, px, py, pid, s0 + smp, pp, W, err);
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
        const uint32_t ti = pp.pick ? pid : local;
        const float r[3] = {mean.x - target[3 * ti + 0], mean.y - target[3 * ti + 1], mean.z - target[3 * ti + 2]};
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
    __shared__ double red[kDisneyThreads / 32];
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

template <int MAXD>
__global__ void __launch_bounds__(kDisneyThreads)
    k_disney_adjoint(SceneDev s, SegDev t, DisneyDev D, const ViewDev* views, uint32_t n_views, uint32_t pix_begin,
                     uint32_t n_pix, PathParams pp, const float* g_img, double* grad_acc, float* gacc,
                     uint32_t* err) {
  extern __shared__ float dsgrad_sh[];
  float* sgrad = gacc ? gacc : dsgrad_sh;
  const uint32_t n_par = (uint32_t)kDisneyStride * s.n_seg;
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
      disney_adjoint_path<MAXD>(s, t, D, vw, px, py, pid, s0 + smp, pp, W, gp, sgrad, err);
  }
  __syncthreads();
  if (!gacc)
    for (uint32_t i = threadIdx.x; i < n_par; i += blockDim.x) {
      const float v = sgrad[i];
      if (v != 0.0f) atomicAdd(&grad_acc[i], (double)v);
    }
}

__global__ void k_disney_add_to_double(const float* src, uint32_t n, double* dst) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] += (double)src[i];
}

}  // namespace

// Shared-memory accumulators of one adjoint block: 16 floats per segment.
uint32_t disney_max_shared_segments() { return (96u * 1024u) / (4u * (uint32_t)kDisneyStride); }

cudaError_t launch_disney_tables(const SceneBuffers& s, const SegBuffers& t, const DisneyBuffers& d,
                                 const float* params, const float* sparams, cudaStream_t st) {
  k_disney_tables<<<1, 256, 0, st>>>(params, sparams ? sparams : params, s.n_seg, s.emission_scale, s.seg_area, t,
                                     d);
  return cudaGetLastError();
}

static int disney_grid(uint64_t n_pix, uint32_t group, int cap) {
  const uint64_t tasks = (n_pix + (32 / group) - 1) / (32 / group);
  const uint64_t per_block = kDisneyThreads / 32;
  uint64_t g = (tasks + per_block - 1) / per_block;
  if (g > (uint64_t)cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_disney_forward(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                                  const DisneyBuffers& d, const ViewHost* views_dev, uint32_t n_views,
                                  uint32_t pix_begin, uint32_t n_pix, const TraceParams& tp, float* img, float* msq,
                                  const float* target, float* g_out, double* loss_partials, float g_scale,
                                  int loss_kind, uint32_t* err, cudaStream_t st) {
  const PathParams pp = make_path_params(tp, s);
  // the loss partials hold one row per block of the fixed loss grid
  const int cap = loss_partials_capacity(L);
  const int grid = loss_partials ? cap : disney_grid(n_pix, pp.group, cap);
  k_disney_forward<<<grid, kDisneyThreads, 0, st>>>(scene_dev(s), seg_dev(t), DisneyDev{d.mat, d.lobe, d.samp},
                                                    reinterpret_cast<const ViewDev*>(views_dev), n_views, pix_begin,
                                                    n_pix, pp, img, msq, target, g_out, loss_partials, g_scale,
                                                    loss_kind, err);
  return cudaGetLastError();
}

cudaError_t launch_disney_adjoint(const Launcher& L, const SceneBuffers& s, const SegBuffers& t,
                                  const DisneyBuffers& d, const ViewHost* views_dev, uint32_t n_views,
                                  uint32_t pix_begin, uint32_t n_pix, const TraceParams& tp, const float* g_img,
                                  double* grad_acc, float* gacc_scratch, uint32_t* err, cudaStream_t st) {
  const PathParams pp = make_path_params(tp, s);
  const uint32_t n_par = (uint32_t)kDisneyStride * s.n_seg;
  const bool global = s.n_seg > disney_max_shared_segments();
  if (global && !gacc_scratch) return cudaErrorInvalidValue;
  float* gacc = global ? gacc_scratch : nullptr;
  const size_t shmem = global ? 0 : sizeof(float) * n_par;
  if (global) {
    cudaError_t e = cudaMemsetAsync(gacc, 0, sizeof(float) * n_par, st);
    if (e != cudaSuccess) return e;
  }
  const DisneyDev D{d.mat, d.lobe, d.samp};
  const ViewDev* vd = reinterpret_cast<const ViewDev*>(views_dev);
  const int md = tp.max_depth < 1 ? 1 : (int)tp.max_depth;
  const int cap = L.num_sms * 4;
#define IPT_LAUNCH_DADJ(DEPTH)                                                                                     \
  {                                                                                                                \
    if (shmem > 48 * 1024)                                                                                         \
      cudaFuncSetAttribute(k_disney_adjoint<DEPTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);     \
    k_disney_adjoint<DEPTH><<<disney_grid(n_pix, pp.group, cap), kDisneyThreads, shmem, st>>>(                     \
        scene_dev(s), seg_dev(t), D, vd, n_views, pix_begin, n_pix, pp, g_img, grad_acc, gacc, err);              \
  }
  if (md <= 2)
    IPT_LAUNCH_DADJ(2)
  else if (md <= 4)
    IPT_LAUNCH_DADJ(4)
  else if (md <= 6)
    IPT_LAUNCH_DADJ(6)
  else
    IPT_LAUNCH_DADJ(8)
#undef IPT_LAUNCH_DADJ
  if (global) k_disney_add_to_double<<<(n_par + 255) / 256, 256, 0, st>>>(gacc, n_par, grad_acc);
  return cudaGetLastError();
}

cudaError_t launch_disney_adam(const SceneBuffers& s, const SegBuffers& t, const DisneyBuffers& d, float* params,
                               float* m, float* v, const uint8_t* free_mask, const double* grad_acc,
                               const float* grad_f, int* step_dev, const AdamHost& a, const double* loss,
                               uint32_t* err, cudaStream_t st) {
  k_disney_adam<<<1, 256, 0, st>>>(params, m, v, free_mask, grad_acc, grad_f, step_dev, a, s.n_seg,
                                   s.emission_scale, s.seg_area, t, d, loss, err);
  return cudaGetLastError();
}

}  // namespace ipt
