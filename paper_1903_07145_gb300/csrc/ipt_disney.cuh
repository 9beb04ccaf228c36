// Disney material model on the device (Sec. 4.1: a base colour and ten more
// scalars in [0, 1]; Burley, "Physically-Based Shading at Disney", SIGGRAPH
// 2012 course notes), with the base colour taken as linear RGB.
//
// Parameter block per segment (16 floats): base colour 0-2, subsurface 3,
// metallic 4, specular 5, specular tint 6, roughness 7, anisotropic 8,
// sheen 9, sheen tint 10, clearcoat 11, clearcoat gloss 12, emission 13-15.
//
// f_r = diffuse + sheen + specular + clearcoat, with l = wo, v = wi, h the
// half vector, S(c) = (1 - c)^5, C_t = base / lum(base) (white when black):
//   diffuse   (1 - metallic) base / pi [(1 - subsurface) fD + subsurface fSS]
//             (Burley's retro-reflective diffuse and its Hanrahan-Krueger-like
//             subsurface approximation);
//   sheen     (1 - metallic) sheen S(l.h) (1 + sheen_tint (C_t - 1));
//   specular  anisotropic GGX D with a_x = max(1e-3, r^2 / k), a_y =
//             max(1e-3, r^2 k), k = sqrt(1 - 0.9 anisotropic); Schlick
//             Fresnel from C0 = (1 - metallic) 0.08 specular (1 + spec_tint
//             (C_t - 1)) + metallic base; separable Smith masking g(l) g(v)
//             with g(w) = 1 / (n.w + |(a_x w.X, a_y w.Y, n.w)|);
//   clearcoat clearcoat / 4 * GTR1(a_c = 0.1 - 0.099 gloss) * (0.04 + 0.96
//             S(l.h)) * Smith masking of width 0.25.
// The tangent X is the hit triangle's first edge made orthogonal to the
// shading normal; Y = n x X.
//
// The derivatives the adjoint needs (the 3 x 13 Jacobian of f_r with respect
// to the material values, contracted with an RGB weight) come from
// forward-mode dual numbers: the same templated evaluation run on Dual13.
#pragma once

#include "ipt_device.cuh"
#include "ipt_path.cuh"

namespace ipt {

constexpr int kDisneyMat = 13;     // material values per segment
constexpr int kDisneyStride = 16;  // material + emission
constexpr float kLumRf = (float)kLumR, kLumGf = (float)kLumG, kLumBf = (float)kLumB;

struct Dual13 {
  float v;
  float d[kDisneyMat];
};
__device__ __forceinline__ Dual13 dc(float x) {
  Dual13 r;
  r.v = x;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = 0.0f;
  return r;
}
__device__ __forceinline__ Dual13 operator+(const Dual13& a, const Dual13& b) {
  Dual13 r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
__device__ __forceinline__ Dual13 operator-(const Dual13& a, const Dual13& b) {
  Dual13 r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
__device__ __forceinline__ Dual13 operator*(const Dual13& a, const Dual13& b) {
  Dual13 r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
__device__ __forceinline__ Dual13 operator*(const Dual13& a, float b) {
  Dual13 r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] * b;
  return r;
}
__device__ __forceinline__ Dual13 operator*(float b, const Dual13& a) { return a * b; }
__device__ __forceinline__ Dual13 operator+(const Dual13& a, float b) {
  Dual13 r = a;
  r.v += b;
  return r;
}
__device__ __forceinline__ Dual13 operator+(float b, const Dual13& a) { return a + b; }
__device__ __forceinline__ Dual13 operator-(const Dual13& a, float b) {
  Dual13 r = a;
  r.v -= b;
  return r;
}
__device__ __forceinline__ Dual13 operator-(float b, const Dual13& a) {
  Dual13 r;
  r.v = b - a.v;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = -a.d[i];
  return r;
}
// 1 / a
__device__ __forceinline__ Dual13 rcp(const Dual13& a) {
  Dual13 r;
  r.v = 1.0f / a.v;
  const float k = -r.v * r.v;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] * k;
  return r;
}
__device__ __forceinline__ Dual13 operator/(const Dual13& a, const Dual13& b) { return a * rcp(b); }
__device__ __forceinline__ Dual13 operator/(float a, const Dual13& b) { return rcp(b) * a; }
__device__ __forceinline__ Dual13 operator/(const Dual13& a, float b) { return a * (1.0f / b); }
__device__ __forceinline__ Dual13 dsqrt(const Dual13& a) {
  Dual13 r;
  r.v = sqrtf(a.v);
  const float k = 0.5f / r.v;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] * k;
  return r;
}
__device__ __forceinline__ Dual13 dlog(const Dual13& a) {
  Dual13 r;
  r.v = logf(a.v);
  const float k = 1.0f / a.v;
#pragma unroll
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] * k;
  return r;
}
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ float dlog(float a) { return logf(a); }
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ float val(const Dual13& a) { return a.v; }
// max(a, c) with a constant c (zero derivative where c wins)
__device__ __forceinline__ float floor_at(float a, float c) { return a > c ? a : c; }
__device__ __forceinline__ Dual13 floor_at(const Dual13& a, float c) { return a.v > c ? a : dc(c); }
template <class T>
__device__ __forceinline__ T zero_like();
template <>
__device__ __forceinline__ float zero_like<float>() {
  return 0.0f;
}
template <>
__device__ __forceinline__ Dual13 zero_like<Dual13>() {
  return dc(0.0f);
}

__device__ __forceinline__ float schlick_w(float c) {
  const float m = fminf(1.0f, fmaxf(0.0f, 1.0f - c));
  const float m2 = m * m;
  return m2 * m2 * m;
}

// Tangent frame at shading normal n from the triangle edge e1.
__device__ __forceinline__ void tangent_frame(float3 e1, float3 n, float3& X, float3& Y) {
  float3 t = e1 - n * dot(n, e1);
  const float l2 = dot(t, t);
  if (!(l2 > 1e-24f * dot(e1, e1))) {
    float3 b2;
    onb(n, t, b2);
  } else {
    t = t * rsqrtf(l2);
  }
  X = t;
  Y = cross(n, X);
}

template <class T>
__device__ __forceinline__ void disney_widths(const T& r, const T& aniso, T& ax, T& ay) {
  const T k = dsqrt(1.0f - 0.9f * aniso);
  ax = floor_at(r * r / k, 1e-3f);
  ay = floor_at(r * r * k, 1e-3f);
}

// GTR with gamma = 1 at n.h = ch.
template <class T>
__device__ __forceinline__ T gtr1(float ch, const T& a) {
  const T a2 = a * a;
  return (a2 - 1.0f) / (kPi * dlog(a2) * (1.0f + (a2 - 1.0f) * (ch * ch)));
}

// f_r per channel for the 13 material values m (float, or Dual13 for the
// derivatives); zero unless both directions lie above the shading hemisphere.
template <class T>
__device__ __forceinline__ void disney_f(const T (&m)[kDisneyMat], float3 n, float3 X, float3 Y, float3 wi,
                                         float3 wo, T (&f)[3]) {
  const float cl = dot(n, wo), cv = dot(n, wi);
  if (!(cl > 0.0f) || !(cv > 0.0f)) {
    f[0] = f[1] = f[2] = zero_like<T>();
    return;
  }
  const float3 h = normalize(wi + wo);
  const float ch = dot(n, h), cd = dot(wo, h);
  const float Sl = schlick_w(cl), Sv = schlick_w(cv), Sd = schlick_w(cd);
  const T lb = m[0] * kLumRf + m[1] * kLumGf + m[2] * kLumBf;
  T tint[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) tint[c] = val(lb) > 0.0f ? m[c] / lb : zero_like<T>() + 1.0f;
  // diffuse with the subsurface blend
  const T fd90 = 0.5f + (2.0f * cd * cd) * m[7];
  const T fd = (1.0f + (fd90 - 1.0f) * Sl) * (1.0f + (fd90 - 1.0f) * Sv);
  const T f90 = (cd * cd) * m[7];
  const T fss0 = (1.0f + (f90 - 1.0f) * Sl) * (1.0f + (f90 - 1.0f) * Sv);
  const T fss = 1.25f * (fss0 * (1.0f / (cl + cv) - 0.5f) + 0.5f);
  const T diff = (1.0f - m[4]) * ((1.0f - m[3]) * fd + m[3] * fss) * (1.0f / kPi);
  // anisotropic GGX with separable masking
  T ax, ay;
  disney_widths(m[7], m[8], ax, ay);
  const float hx = dot(h, X), hy = dot(h, Y);
  const T q = (hx * hx) / (ax * ax) + (hy * hy) / (ay * ay) + ch * ch;
  const T Ds = 1.0f / (kPi * ax * ay * q * q);
  const float lx = dot(wo, X), ly = dot(wo, Y), vx = dot(wi, X), vy = dot(wi, Y);
  const T gl = 1.0f / (cl + dsqrt((lx * lx) * (ax * ax) + (ly * ly) * (ay * ay) + cl * cl));
  const T gv = 1.0f / (cv + dsqrt((vx * vx) * (ax * ax) + (vy * vy) * (ay * ay) + cv * cv));
  const T spec_geo = Ds * gl * gv;
  // clearcoat
  const T ac = 0.1f - 0.099f * m[12];
  const float gcl = 1.0f / (cl + sqrtf(0.0625f + 0.9375f * cl * cl));
  const float gcv = 1.0f / (cv + sqrtf(0.0625f + 0.9375f * cv * cv));
  const T coat = 0.25f * m[11] * gtr1(ch, ac) * ((0.04f + 0.96f * Sd) * gcl * gcv);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T C0 = (1.0f - m[4]) * 0.08f * m[5] * (1.0f + m[6] * (tint[c] - 1.0f)) + m[4] * m[c];
    const T Fs = C0 + (1.0f - C0) * Sd;
    const T sheen = (1.0f - m[4]) * m[9] * Sd * (1.0f + m[10] * (tint[c] - 1.0f));
    f[c] = m[c] * diff + sheen + Fs * spec_geo + coat;
  }
}

// Per-segment sampling data (built from the sampling parameters):
//   lobe: FP64 cumulative lobe probabilities (P_d, P_d + P_s) for the lobe
//         decision; samp: (a_x, a_y, a_c, -) and (P_d, P_s, P_c, -) in FP32.
struct DisneyDev {
  const float4* mat;    // 4 per segment: material values 0-12, then 0
  const double2* lobe;
  const float4* samp;   // 2 per segment
};

__device__ __forceinline__ void load_disney(const DisneyDev& D, int seg, float (&m)[kDisneyMat]) {
  const float4 a = __ldg(&D.mat[4 * seg]), b = __ldg(&D.mat[4 * seg + 1]);
  const float4 c = __ldg(&D.mat[4 * seg + 2]), d = __ldg(&D.mat[4 * seg + 3]);
  m[0] = a.x, m[1] = a.y, m[2] = a.z, m[3] = a.w;
  m[4] = b.x, m[5] = b.y, m[6] = b.z, m[7] = b.w;
  m[8] = c.x, m[9] = c.y, m[10] = c.z, m[11] = c.w;
  m[12] = d.x;
}

// Solid-angle pdf of the sampler (cosine diffuse, visible anisotropic GGX
// normals, GTR1 clearcoat normals) mixed by the lobe probabilities.
__device__ __forceinline__ float disney_pdf(const DisneyDev& D, int seg, float3 n, float3 X, float3 Y, float3 wi,
                                            float3 wo) {
  const float cv = dot(n, wi), cl = dot(n, wo);
  if (!(cv > 0.0f) || !(cl > 0.0f)) return 0.0f;
  const float4 w = __ldg(&D.samp[2 * seg]), p = __ldg(&D.samp[2 * seg + 1]);
  const float3 h = normalize(wi + wo);
  const float ch = dot(n, h);
  float pdf = p.x * cl * (1.0f / kPi);
  if (p.y > 0.0f) {
    const float hx = dot(h, X), hy = dot(h, Y);
    const float q = (hx * hx) / (w.x * w.x) + (hy * hy) / (w.y * w.y) + ch * ch;
    const float Dn = 1.0f / (kPi * w.x * w.y * q * q);
    const float vx = dot(wi, X), vy = dot(wi, Y);
    const float lam = 0.5f * (sqrtf(1.0f + (vx * vx * w.x * w.x + vy * vy * w.y * w.y) / (cv * cv)) - 1.0f);
    pdf += p.y * Dn / (1.0f + lam) / (4.0f * cv);
  }
  if (p.z > 0.0f) {
    const float wh = dot(wo, h);
    if (wh > 0.0f) pdf += p.z * gtr1(ch, w.z) * ch / (4.0f * wh);
  }
  return pdf;
}

// Direction from the lobe chosen by u_lobe (FP64 comparison with the
// cumulative probabilities) and (u1, u2).
__device__ __forceinline__ float3 disney_sample(const DisneyDev& D, int seg, float3 n, float3 X, float3 Y,
                                                float3 wi, float u_lobe, float u1, float u2) {
  const double2 cum = __ldg(&D.lobe[seg]);
  const float4 w = __ldg(&D.samp[2 * seg]);
  float sphi, cphi;
  sincospif(2.0f * u2, &sphi, &cphi);
  const float rr = sqrtf(u1);
  if ((double)u_lobe < cum.x) {
    float3 b1, b2;
    onb(n, b1, b2);
    return b1 * (rr * cphi) + b2 * (rr * sphi) + n * sqrtf(fmaxf(0.0f, 1.0f - u1));
  }
  float3 hw;
  if ((double)u_lobe < cum.y) {
    const float3 vl = f3(dot(wi, X), dot(wi, Y), dot(wi, n));
    const float3 vh = normalize(f3(w.x * vl.x, w.y * vl.y, vl.z));
    const float lensq = vh.x * vh.x + vh.y * vh.y;
    const float3 t1 = lensq > 0.0f ? f3(-vh.y, vh.x, 0.0f) * rsqrtf(lensq) : f3(1.0f, 0.0f, 0.0f);
    const float3 t2 = cross(vh, t1);
    const float q1 = rr * cphi;
    float q2 = rr * sphi;
    const float s = 0.5f * (1.0f + vh.z);
    q2 = (1.0f - s) * sqrtf(fmaxf(0.0f, 1.0f - q1 * q1)) + s * q2;
    const float3 nh = t1 * q1 + t2 * q2 + vh * sqrtf(fmaxf(0.0f, 1.0f - q1 * q1 - q2 * q2));
    const float3 ne = normalize(f3(w.x * nh.x, w.y * nh.y, fmaxf(0.0f, nh.z)));
    hw = X * ne.x + Y * ne.y + n * ne.z;
  } else {
    const float a2 = w.z * w.z;
    const float c2 = (1.0f - powf(a2, 1.0f - u1)) / (1.0f - a2);
    const float ct = sqrtf(fmaxf(0.0f, c2)), st = sqrtf(fmaxf(0.0f, 1.0f - c2));
    float3 b1, b2;
    onb(n, b1, b2);
    hw = b1 * (st * cphi) + b2 * (st * sphi) + n * ct;
  }
  return hw * (2.0f * dot(wi, hw)) - wi;
}

}  // namespace ipt
