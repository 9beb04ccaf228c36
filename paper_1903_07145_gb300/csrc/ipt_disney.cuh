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
// forward-mode dual numbers (DualN: a value and N tangents) where the
// chain rule is long, and hand-derived partials where it is short.
#pragma once

#include "ipt_device.cuh"
#include "ipt_path.cuh"

namespace ipt {

constexpr int kDisneyMat = 13;     // material values per segment
constexpr int kDisneyStride = 16;  // material + emission
constexpr float kLumRf = (float)kLumR, kLumGf = (float)kLumG, kLumBf = (float)kLumB;

// Forward-mode dual number: a value and N tangents.
template <int N>
struct DualN {
  float v;
  float d[N];
};
template <int N>
__device__ __forceinline__ DualN<N> dconst(float x) {
  DualN<N> r;
  r.v = x;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = 0.0f;
  return r;
}
// the value x with tangent e_i
template <int N>
__device__ __forceinline__ DualN<N> dvar(float x, int i) {
  DualN<N> r = dconst<N>(x);
  r.d[i] = 1.0f;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator+(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator-(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator*(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator*(const DualN<N>& a, float b) {
  DualN<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator*(float b, const DualN<N>& a) {
  return a * b;
}
template <int N>
__device__ __forceinline__ DualN<N> operator+(const DualN<N>& a, float b) {
  DualN<N> r = a;
  r.v += b;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator+(float b, const DualN<N>& a) {
  return a + b;
}
template <int N>
__device__ __forceinline__ DualN<N> operator-(const DualN<N>& a, float b) {
  DualN<N> r = a;
  r.v -= b;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator-(float b, const DualN<N>& a) {
  DualN<N> r;
  r.v = b - a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> rcp(const DualN<N>& a) {
  DualN<N> r;
  r.v = 1.0f / a.v;
  const float k = -r.v * r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * k;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator/(const DualN<N>& a, const DualN<N>& b) {
  return a * rcp(b);
}
template <int N>
__device__ __forceinline__ DualN<N> operator/(float a, const DualN<N>& b) {
  return rcp(b) * a;
}
template <int N>
__device__ __forceinline__ DualN<N> operator/(const DualN<N>& a, float b) {
  return a * (1.0f / b);
}
template <int N>
__device__ __forceinline__ DualN<N> dsqrt(const DualN<N>& a) {
  DualN<N> r;
  r.v = sqrtf(a.v);
  const float k = 0.5f / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * k;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> dlog(const DualN<N>& a) {
  DualN<N> r;
  r.v = logf(a.v);
  const float k = 1.0f / a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * k;
  return r;
}
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ float dlog(float a) { return logf(a); }
__device__ __forceinline__ float val(float a) { return a; }
template <int N>
__device__ __forceinline__ float val(const DualN<N>& a) {
  return a.v;
}
// max(a, c) with a constant c (zero derivative where c wins)
__device__ __forceinline__ float floor_at(float a, float c) { return a > c ? a : c; }
template <int N>
__device__ __forceinline__ DualN<N> floor_at(const DualN<N>& a, float c) {
  return a.v > c ? a : dconst<N>(c);
}
template <class T>
struct Zero {
  __device__ static T get();
};
template <>
struct Zero<float> {
  __device__ static float get() { return 0.0f; }
};
template <int N>
struct Zero<DualN<N>> {
  __device__ static DualN<N> get() { return dconst<N>(0.0f); }
};
template <class T>
__device__ __forceinline__ T zero_like() {
  return Zero<T>::get();
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

// Geometry of one evaluation: cosines with the shading normal, tangent-frame
// components and Schlick weights.
struct DisneyGeo {
  float cl, cv, ch, cd;  // n.wo, n.wi, n.h, wo.h
  float hx, hy, lx, ly, vx, vy;
  float Sl, Sv, Sd;
};

__device__ __forceinline__ bool disney_geo(float3 n, float3 X, float3 Y, float3 wi, float3 wo, DisneyGeo& g) {
  g.cl = dot(n, wo);
  g.cv = dot(n, wi);
  if (!(g.cl > 0.0f) || !(g.cv > 0.0f)) return false;
  const float3 h = normalize(wi + wo);
  g.ch = dot(n, h);
  g.cd = dot(wo, h);
  g.hx = dot(h, X), g.hy = dot(h, Y);
  g.lx = dot(wo, X), g.ly = dot(wo, Y), g.vx = dot(wi, X), g.vy = dot(wi, Y);
  g.Sl = schlick_w(g.cl), g.Sv = schlick_w(g.cv), g.Sd = schlick_w(g.cd);
  return true;
}

// D_s g(l) g(v) of the anisotropic GGX lobe at widths (ax, ay).
template <class T>
__device__ __forceinline__ T ggx_geo(const T& ax, const T& ay, const DisneyGeo& g) {
  const T q = (g.hx * g.hx) / (ax * ax) + (g.hy * g.hy) / (ay * ay) + g.ch * g.ch;
  const T Ds = 1.0f / (kPi * ax * ay * q * q);
  const T gl = 1.0f / (g.cl + dsqrt((g.lx * g.lx) * (ax * ax) + (g.ly * g.ly) * (ay * ay) + g.cl * g.cl));
  const T gv = 1.0f / (g.cv + dsqrt((g.vx * g.vx) * (ax * ax) + (g.vy * g.vy) * (ay * ay) + g.cv * g.cv));
  return Ds * gl * gv;
}

// Separable Smith masking of the clearcoat (width 0.25), both directions.
__device__ __forceinline__ float coat_masking(const DisneyGeo& g) {
  return 1.0f / ((g.cl + sqrtf(0.0625f + 0.9375f * g.cl * g.cl)) * (g.cv + sqrtf(0.0625f + 0.9375f * g.cv * g.cv)));
}

// f_r per channel for the 13 material values m (float, or DualN for the
// derivatives); zero unless both directions lie above the shading hemisphere.
template <class T>
__device__ __forceinline__ void disney_f(const T (&m)[kDisneyMat], float3 n, float3 X, float3 Y, float3 wi,
                                         float3 wo, T (&f)[3]) {
  DisneyGeo G;
  if (!disney_geo(n, X, Y, wi, wo, G)) {
    f[0] = f[1] = f[2] = zero_like<T>();
    return;
  }
  const float cl = G.cl, cv = G.cv, ch = G.ch, cd = G.cd, Sl = G.Sl, Sv = G.Sv, Sd = G.Sd;
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
  const T spec_geo = ggx_geo(ax, ay, G);
  // clearcoat
  const T ac = 0.1f - 0.099f * m[12];
  const T coat = 0.25f * m[11] * gtr1(ch, ac) * ((0.04f + 0.96f * Sd) * coat_masking(G));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T C0 = (1.0f - m[4]) * 0.08f * m[5] * (1.0f + m[6] * (tint[c] - 1.0f)) + m[4] * m[c];
    const T Fs = C0 + (1.0f - C0) * Sd;
    const T sheen = (1.0f - m[4]) * m[9] * Sd * (1.0f + m[10] * (tint[c] - 1.0f));
    f[c] = m[c] * diff + sheen + Fs * spec_geo + coat;
  }
}

// Contracted derivative g_j = sum_c q_c d f_c / d m_j of the 13 material
// values, by the chain rule written out per parameter; the GGX term's two
// widths and the clearcoat's GTR1 width go through 2- and 1-tangent dual
// numbers.  With lum(base) = 0 the tint is the constant white (no base-colour
// derivative through it), as in the evaluation.  Returns false (g untouched)
// unless both directions lie above the shading hemisphere.
__device__ __forceinline__ bool disney_vjp(const float (&m)[kDisneyMat], float3 n, float3 X, float3 Y, float3 wi,
                                          float3 wo, float3 q3, float (&g)[kDisneyMat]) {
  DisneyGeo G;
  if (!disney_geo(n, X, Y, wi, wo, G)) return false;
  const float q[3] = {q3.x, q3.y, q3.z};
  const float lw[3] = {kLumRf, kLumGf, kLumBf};
  const float sub = m[3], met = m[4], spc = m[5], spt = m[6], rho = m[7], shn = m[9], sht = m[10], cc = m[11];
  const float lb = m[0] * kLumRf + m[1] * kLumGf + m[2] * kLumBf;
  const bool tinted = lb > 0.0f;
  float tint[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) tint[c] = tinted ? m[c] / lb : 1.0f;
  // diffuse and subsurface, with their roughness derivatives
  const float cd2 = G.cd * G.cd;
  const float A = 0.5f + 2.0f * cd2 * rho - 1.0f, B = cd2 * rho - 1.0f;
  const float fd = (1.0f + A * G.Sl) * (1.0f + A * G.Sv);
  const float dfd = 2.0f * cd2 * (G.Sl * (1.0f + A * G.Sv) + G.Sv * (1.0f + A * G.Sl));
  const float fss0 = (1.0f + B * G.Sl) * (1.0f + B * G.Sv);
  const float k_ss = 1.25f * (1.0f / (G.cl + G.cv) - 0.5f);
  const float fss = k_ss * fss0 + 0.625f;
  const float dfss = k_ss * cd2 * (G.Sl * (1.0f + B * G.Sv) + G.Sv * (1.0f + B * G.Sl));
  const float mixd = (1.0f - sub) * fd + sub * fss;
  const float diff = (1.0f - met) * mixd * (1.0f / kPi);
  // specular geometry and its derivatives in (roughness, anisotropic)
  DualN<2> ax, ay;
  disney_widths(dvar<2>(rho, 0), dvar<2>(m[8], 1), ax, ay);
  const DualN<2> S = ggx_geo(ax, ay, G);
  // clearcoat and its derivative in the gloss
  const DualN<1> Dc = gtr1(G.ch, 0.1f - 0.099f * dvar<1>(m[12], 0));
  const float cF = (0.04f + 0.96f * G.Sd) * coat_masking(G);
  const float oSd = 1.0f - G.Sd;
  float Qb = 0.0f, Qs = 0.0f, QF = 0.0f, Qt = 0.0f, Qsh = 0.0f, Qspt = 0.0f, Qmet = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float tc = 1.0f + spt * (tint[c] - 1.0f);
    const float sc = 1.0f + sht * (tint[c] - 1.0f);
    const float C0 = (1.0f - met) * 0.08f * spc * tc + met * m[c];
    const float Fs = C0 * oSd + G.Sd;
    Qb += q[c] * m[c];
    Qs += q[c];
    QF += q[c] * Fs;
    Qt += q[c] * tint[c];
    Qsh += q[c] * sc;
    Qspt += q[c] * tc;
    Qmet += q[c] * (-m[c] * mixd * (1.0f / kPi) - shn * G.Sd * sc + oSd * S.v * (m[c] - 0.08f * spc * tc));
  }
  // base colour: its own diffuse and metallic Fresnel terms, and the tint of
  // sheen and specular through d tint_c / d base_k = (delta_ck - tint_c w_k) / lb
  const float K = (1.0f - met) * (shn * G.Sd * sht + oSd * S.v * 0.08f * spc * spt);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    g[k] = q[k] * (diff + oSd * S.v * met) + (tinted ? K * (q[k] - lw[k] * Qt) / lb : 0.0f);
  g[3] = Qb * (1.0f - met) * (fss - fd) * (1.0f / kPi);
  g[4] = Qmet;
  g[5] = oSd * S.v * (1.0f - met) * 0.08f * Qspt;
  g[6] = oSd * S.v * (1.0f - met) * 0.08f * spc * (Qt - Qs);
  g[7] = Qb * (1.0f - met) * ((1.0f - sub) * dfd + sub * dfss) * (1.0f / kPi) + QF * S.d[0];
  g[8] = QF * S.d[1];
  g[9] = (1.0f - met) * G.Sd * Qsh;
  g[10] = (1.0f - met) * shn * G.Sd * (Qt - Qs);
  g[11] = Qs * 0.25f * Dc.v * cF;
  g[12] = Qs * 0.25f * cc * cF * Dc.d[0];
  return true;
}

// Per-segment sampling data (built from the sampling parameters):
//   lobe: FP64 cumulative lobe probabilities (P_d, P_d + P_s) for the lobe
//         decision; samp: (a_x, a_y, a_c, -) and (P_d, P_s, P_c, -) in FP32.

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

// Tangent frame of the hit triangle at the oriented shading normal.
__device__ __forceinline__ void hit_frame(const SceneDev& s, int tri, float3 ns, float3& X, float3& Y) {
  const float3 p0 = xyz(__ldg(&s.tris[3 * tri + 0]));
  const float3 p1 = xyz(__ldg(&s.tris[3 * tri + 1]));
  tangent_frame(p1 - p0, ns, X, Y);
}

__device__ __forceinline__ float3 disney_eval(const float (&m)[kDisneyMat], float3 n, float3 X, float3 Y, float3 wi,
                                              float3 wo) {
  float f[3];
  disney_f(m, n, X, Y, wi, wo, f);
  return f3(f[0], f[1], f[2]);
}

}  // namespace ipt
