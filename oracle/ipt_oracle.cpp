// FP64 CPU oracle for Inverse Path Tracing (Azinovic, Li, Kaplanyan, Niessner,
// CVPR 2019).
//
// TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg may load this library.  It shares no code, header or table
// with the CUDA path: it is a plain, slow, double-precision restatement of the
// method, used to check the GPU results.
//
// What it computes, and where the paper defines it:
//   * path-integral pixel estimate, Eq. 1, with the measurement contribution of
//     Eq. 2: emitted radiance at the light end times the product of BRDFs
//     (cosines and sampling pdfs folded into the estimator);
//   * emission profile L_e(x, w) = e (w . n)_+  (Sec. 4.3);
//   * MIS of BRDF sampling with light sampling (Appendix A.2, Appendix E),
//     light selection proportional to the current emission (Appendix E);
//   * gradients by the product rule, Eq. 5 (emission) and Eq. 6 (materials),
//     evaluated literally per sampled light path with explicit products over
//     i != l, never by division;
//   * per-object (segment) constant parameters (Sec. 4.2).
// Readings where the paper is silent (BRDF = Lambert + GGX without Fresnel,
// power-heuristic MIS, box pixel filter, frozen sampling parameters, the
// random-number dimension map) are the same conventions the CUDA path follows
// and are listed in the design notes.
//
// Parity status: pinned (Philox known-answer vectors, BVH vs brute force,
// furnace closed form, polygon-light irradiance, GGX normalisation and weak
// white furnace, linearity in emission, finite differences of the gradient).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kLumR = 0.2126, kLumG = 0.7152, kLumB = 0.0722;  // Rec. 709

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double length(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 normalize(V3 a) { return a * (1.0 / length(a)); }
inline double comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As
// Easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 Philox S-box; the key is
// bumped by the Weyl constants before every round after the first.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = (uint64_t)M0 * c0;
    const uint64_t p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// 32-bit word -> uniform in [0,1) with 24 significant bits (exact in FP32).
inline double to_unit(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

struct Rng {
  uint32_t key[2];
  uint32_t base[3];  // pixel id, sample id, (set << 24) | iteration
  // Four uniforms for one (vertex, call) slot of the dimension map.
  void draw(uint32_t vertex, uint32_t call, double u[4]) const {
    uint32_t c[4] = {base[0], base[1], base[2], vertex * 4u + call};
    uint32_t o[4];
    philox4x32_10(c, key, o);
    for (int i = 0; i < 4; ++i) u[i] = to_unit(o[i]);
  }
};

// ---------------------------------------------------------------------------
// Scene: triangle mesh with per-triangle segment ids (Sec. 4.2), plus a simple
// binary BVH (median split) used only to answer the same closest-hit query
// as the brute-force loop faster.
// ---------------------------------------------------------------------------
struct Node {
  V3 lo, hi;
  int left, right;  // children, or -1 for a leaf
  int first, count; // leaf triangle range in bvh_tris
};

struct Scene {
  uint32_t nt = 0, ns = 0;
  std::vector<V3> p0, p1, p2;  // triangle corners
  std::vector<V3> n0, n1, n2;  // vertex normals (copies of the geometric one if none)
  bool has_normals = false;
  std::vector<V3> ng;          // unit geometric normal (winding order)
  std::vector<double> area;
  std::vector<uint32_t> seg;
  double diameter = 1.0;
  // Light sampling support: triangles grouped by segment, in increasing id.
  std::vector<uint32_t> seg_begin;  // ns + 1
  std::vector<uint32_t> seg_tris;
  std::vector<double> tri_cdf;      // inclusive area prefix inside the segment
  std::vector<double> seg_area;
  std::vector<Node> nodes;
  std::vector<uint32_t> bvh_tris;
};

V3 load3(const float* a, size_t i) { return {(double)a[3 * i], (double)a[3 * i + 1], (double)a[3 * i + 2]}; }

int build_bvh(Scene& s, std::vector<uint32_t>& ids, int first, int count,
              const std::vector<V3>& cen) {
  Node nd;
  nd.lo = {1e300, 1e300, 1e300};
  nd.hi = {-1e300, -1e300, -1e300};
  V3 clo = nd.lo, chi = nd.hi;
  for (int i = first; i < first + count; ++i) {
    const uint32_t t = ids[i];
    for (const V3& q : {s.p0[t], s.p1[t], s.p2[t]}) {
      nd.lo = {std::min(nd.lo.x, q.x), std::min(nd.lo.y, q.y), std::min(nd.lo.z, q.z)};
      nd.hi = {std::max(nd.hi.x, q.x), std::max(nd.hi.y, q.y), std::max(nd.hi.z, q.z)};
    }
    const V3 c = cen[t];
    clo = {std::min(clo.x, c.x), std::min(clo.y, c.y), std::min(clo.z, c.z)};
    chi = {std::max(chi.x, c.x), std::max(chi.y, c.y), std::max(chi.z, c.z)};
  }
  const double pad = 1e-9 * s.diameter;  // cover rounding of the hit test
  nd.lo = nd.lo - V3{pad, pad, pad};
  nd.hi = nd.hi + V3{pad, pad, pad};
  const int me = (int)s.nodes.size();
  s.nodes.push_back(nd);
  if (count <= 4) {
    s.nodes[me].left = s.nodes[me].right = -1;
    s.nodes[me].first = first;
    s.nodes[me].count = count;
    return me;
  }
  const V3 ext = chi - clo;
  const int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
  const int mid = first + count / 2;
  std::nth_element(ids.begin() + first, ids.begin() + mid, ids.begin() + first + count,
                   [&](uint32_t a, uint32_t b) {
                     const double ca = comp(cen[a], axis), cb = comp(cen[b], axis);
                     return ca < cb || (ca == cb && a < b);
                   });
  const int l = build_bvh(s, ids, first, mid - first, cen);
  const int r = build_bvh(s, ids, mid, first + count - mid, cen);
  s.nodes[me].left = l;
  s.nodes[me].right = r;
  s.nodes[me].first = 0;
  s.nodes[me].count = 0;
  return me;
}

// Moller-Trumbore in FP64, two-sided.  Hit point = (1-u-v) p0 + u p1 + v p2.
inline bool tri_hit(const Scene& s, uint32_t t, V3 o, V3 d, double& th, double& uh, double& vh) {
  const V3 e1 = s.p1[t] - s.p0[t];
  const V3 e2 = s.p2[t] - s.p0[t];
  const V3 pv = cross(d, e2);
  const double det = dot(e1, pv);
  if (det == 0.0) return false;
  const double inv = 1.0 / det;
  const V3 tv = o - s.p0[t];
  const double u = dot(tv, pv) * inv;
  if (u < 0.0 || u > 1.0) return false;
  const V3 qv = cross(tv, e1);
  const double v = dot(d, qv) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  th = dot(e2, qv) * inv;
  uh = u;
  vh = v;
  return true;
}

inline bool box_hit(const Node& n, V3 o, V3 d, double tmin, double tmax) {
  double t0 = tmin, t1 = tmax;
  for (int k = 0; k < 3; ++k) {
    const double ok = comp(o, k), dk = comp(d, k);
    const double lo = comp(n.lo, k), hi = comp(n.hi, k);
    if (dk == 0.0) {
      if (ok < lo || ok > hi) return false;
      continue;
    }
    double a = (lo - ok) / dk, b = (hi - ok) / dk;
    if (a > b) std::swap(a, b);
    t0 = std::max(t0, a);
    t1 = std::min(t1, b);
    if (t0 > t1) return false;
  }
  return true;
}

struct Hit {
  int tri = -1;
  double t = 0, u = 0, v = 0;
};

// Closest hit with t in (tmin, tmax), skipping one triangle; equal t keeps the
// smaller triangle id.
Hit closest(const Scene& s, V3 o, V3 d, double tmin, double tmax, int skip, bool brute) {
  Hit h;
  double best = tmax;
  auto consider = [&](uint32_t t) {
    if ((int)t == skip) return;
    double th, uh, vh;
    if (!tri_hit(s, t, o, d, th, uh, vh)) return;
    if (!(th > tmin)) return;
    const bool better = h.tri < 0 ? th < tmax : (th < best || (th == best && (int)t < h.tri));
    if (better) {
      best = th;
      h.tri = (int)t;
      h.t = th;
      h.u = uh;
      h.v = vh;
    }
  };
  if (brute || s.nodes.empty()) {
    for (uint32_t t = 0; t < s.nt; ++t) consider(t);
    return h;
  }
  int stack[128];
  int sp = 0;
  stack[sp++] = 0;
  while (sp) {
    const Node& n = s.nodes[stack[--sp]];
    if (!box_hit(n, o, d, tmin, best)) continue;
    if (n.left < 0) {
      for (int i = n.first; i < n.first + n.count; ++i) consider(s.bvh_tris[i]);
    } else {
      stack[sp++] = n.left;
      stack[sp++] = n.right;
    }
  }
  return h;
}

// Any hit with t in (tmin, tmax), skipping two triangles.
bool occluded(const Scene& s, V3 o, V3 d, double tmin, double tmax, int skip_a, int skip_b) {
  int stack[128];
  int sp = 0;
  stack[sp++] = 0;
  while (sp) {
    const Node& n = s.nodes[stack[--sp]];
    if (!box_hit(n, o, d, tmin, tmax)) continue;
    if (n.left < 0) {
      for (int i = n.first; i < n.first + n.count; ++i) {
        const uint32_t t = s.bvh_tris[i];
        if ((int)t == skip_a || (int)t == skip_b) continue;
        double th, uh, vh;
        if (tri_hit(s, t, o, d, th, uh, vh) && th > tmin && th < tmax) return true;
      }
    } else {
      stack[sp++] = n.left;
      stack[sp++] = n.right;
    }
  }
  return false;
}

// ---------------------------------------------------------------------------
// Material model.  The paper uses a Disney-style model with perceptual [0,1]
// parameters (Sec. 4.1); this path narrows it to Lambert + GGX:
//   f_r = kd / pi + ks * D(h) G2(wi, wo) / (4 |n.wi| |n.wo|),  alpha = max(r^2, 1e-4)
// GGX normal distribution, height-correlated Smith masking-shadowing, no
// Fresnel (ks is the specular reflectance scale, keeping f_r linear in kd, ks).
// ---------------------------------------------------------------------------
struct Mat {
  double kd[3], ks[3], r, e[3];
};

inline Mat mat_of(const double* p) {
  Mat m;
  for (int c = 0; c < 3; ++c) {
    m.kd[c] = p[c];
    m.ks[c] = p[3 + c];
    m.e[c] = p[7 + c];
  }
  m.r = p[6];
  return m;
}

inline double alpha_of(double r) { return std::max(r * r, 1e-4); }
inline double dalpha_dr(double r) { return (r * r > 1e-4) ? 2.0 * r : 0.0; }

inline double ggx_D(double nh, double a) {
  if (nh <= 0) return 0.0;
  const double a2 = a * a;
  const double q = nh * nh * (a2 - 1.0) + 1.0;
  return a2 / (kPi * q * q);
}
inline double ggx_dD_da(double nh, double a) {
  if (nh <= 0) return 0.0;
  const double a2 = a * a;
  const double q = nh * nh * (a2 - 1.0) + 1.0;
  // D = a^2 / (pi q^2), dq/da = 2 a nh^2
  return 2.0 * a / (kPi * q * q) - a2 * 2.0 * (2.0 * a * nh * nh) / (kPi * q * q * q);
}
inline double smith_lambda(double c, double a) {
  const double c2 = c * c;
  const double t2 = (1.0 - c2) / c2;
  return 0.5 * (-1.0 + std::sqrt(1.0 + a * a * t2));
}
inline double smith_dlambda_da(double c, double a) {
  const double c2 = c * c;
  const double t2 = (1.0 - c2) / c2;
  return 0.5 * a * t2 / std::sqrt(1.0 + a * a * t2);
}
inline double smith_G1(double c, double a) { return 1.0 / (1.0 + smith_lambda(c, a)); }

// Specular factor s = D G2 / (4 ci co) and ds/dr, for ci, co > 0.
inline void spec_term(double ci, double co, double nh, double r, double& s, double& ds_dr) {
  const double a = alpha_of(r);
  const double D = ggx_D(nh, a);
  const double li = smith_lambda(ci, a), lo = smith_lambda(co, a);
  const double G2 = 1.0 / (1.0 + li + lo);
  const double den = 4.0 * ci * co;
  s = D * G2 / den;
  const double dG2 = -G2 * G2 * (smith_dlambda_da(ci, a) + smith_dlambda_da(co, a));
  const double ds_da = (ggx_dD_da(nh, a) * G2 + D * dG2) / den;
  ds_dr = ds_da * dalpha_dr(r);
}

struct BrdfEval {
  double f[3];     // f_r per channel
  double spec;     // D G2 / (4 ci co)
  double dspec_dr;
  bool valid;      // both directions above the shading hemisphere
};

inline BrdfEval brdf_eval(const Mat& m, V3 n, V3 wi, V3 wo) {
  BrdfEval b{};
  const double ci = dot(n, wi), co = dot(n, wo);
  if (!(ci > 0.0) || !(co > 0.0)) {
    b.valid = false;
    return b;
  }
  b.valid = true;
  const V3 h = normalize(wi + wo);
  spec_term(ci, co, dot(n, h), m.r, b.spec, b.dspec_dr);
  for (int c = 0; c < 3; ++c) b.f[c] = m.kd[c] / kPi + m.ks[c] * b.spec;
  return b;
}

inline double lum3(const double* c) { return kLumR * c[0] + kLumG * c[1] + kLumB * c[2]; }

// Probability of choosing the specular lobe (from the sampling parameters).
inline double spec_prob(const Mat& ms) {
  const double ld = lum3(ms.kd), ls = lum3(ms.ks);
  const double sum = ld + ls;
  return sum > 0.0 ? ls / sum : 0.0;
}

// Orthonormal basis around unit n: Duff, Burgess, Christensen, Hery, Kensler,
// Liani, Villemin, "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017.
inline void onb(V3 n, V3& b1, V3& b2) {
  const double sign = std::copysign(1.0, n.z);
  const double a = -1.0 / (sign + n.z);
  const double b = n.x * n.y * a;
  b1 = {1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x};
  b2 = {b, sign + n.y * n.y * a, -n.y};
}

// Mixture pdf (solid angle) of sampling wo from wi, with sampling params ms.
inline double bsdf_pdf(const Mat& ms, V3 n, V3 wi, V3 wo) {
  const double ci = dot(n, wi), co = dot(n, wo);
  if (!(ci > 0.0) || !(co > 0.0)) return 0.0;
  const double P = spec_prob(ms);
  const double pd = co / kPi;
  double ps = 0.0;
  if (P > 0.0) {
    const double a = alpha_of(ms.r);
    const V3 h = normalize(wi + wo);
    ps = smith_G1(ci, a) * ggx_D(dot(n, h), a) / (4.0 * ci);
  }
  return (1.0 - P) * pd + P * ps;
}

// Sample wo: lobe by u_lobe < P_spec; diffuse = cosine-weighted hemisphere
// (r = sqrt(u1), phi = 2 pi u2); specular = GGX visible normals (Heitz,
// "Sampling the GGX Distribution of Visible Normals", JCGT 7(4), 2018), then
// mirror wi about the sampled normal.
inline V3 bsdf_sample(const Mat& ms, V3 n, V3 wi, double u_lobe, double u1, double u2) {
  V3 b1, b2;
  onb(n, b1, b2);
  const double P = spec_prob(ms);
  if (u_lobe < P) {
    const double a = alpha_of(ms.r);
    const V3 vl = {dot(wi, b1), dot(wi, b2), dot(wi, n)};
    const V3 vh = normalize(V3{a * vl.x, a * vl.y, vl.z});
    const double lensq = vh.x * vh.x + vh.y * vh.y;
    const V3 t1 = lensq > 0.0 ? V3{-vh.y, vh.x, 0.0} * (1.0 / std::sqrt(lensq)) : V3{1.0, 0.0, 0.0};
    const V3 t2 = cross(vh, t1);
    const double rr = std::sqrt(u1);
    const double phi = 2.0 * kPi * u2;
    const double q1 = rr * std::cos(phi);
    double q2 = rr * std::sin(phi);
    const double s = 0.5 * (1.0 + vh.z);
    q2 = (1.0 - s) * std::sqrt(1.0 - q1 * q1) + s * q2;
    const V3 nh = t1 * q1 + t2 * q2 + vh * std::sqrt(std::max(0.0, 1.0 - q1 * q1 - q2 * q2));
    const V3 ne = normalize(V3{a * nh.x, a * nh.y, std::max(0.0, nh.z)});
    const V3 hw = b1 * ne.x + b2 * ne.y + n * ne.z;
    return hw * (2.0 * dot(wi, hw)) - wi;
  }
  const double rr = std::sqrt(u1);
  const double phi = 2.0 * kPi * u2;
  const V3 l = {rr * std::cos(phi), rr * std::sin(phi), std::sqrt(std::max(0.0, 1.0 - u1))};
  return b1 * l.x + b2 * l.y + n * l.z;
}

// ---------------------------------------------------------------------------
// Disney material model (Sec. 4.1: a base colour and ten further scalars, all
// in [0, 1]).  Restated from Burley, "Physically-Based Shading at Disney",
// SIGGRAPH 2012 course notes, with the base colour taken as linear RGB.
// Per segment 16 values: base colour (0-2), subsurface (3), metallic (4),
// specular (5), specular tint (6), roughness (7), anisotropic (8), sheen (9),
// sheen tint (10), clearcoat (11), clearcoat gloss (12), emission (13-15).
//
// With l = wo, v = wi, h their half vector, S(c) = (1 - c)^5, rho the
// roughness, mu metallic, sigma subsurface, C_t = base / lum(base) (white
// for a black base):
//   diffuse   (1 - mu) base / pi [(1 - sigma) fD + sigma fSS],
//             fD  = (1 + (FD90 - 1) S(n.l)) (1 + (FD90 - 1) S(n.v)), FD90 = 1/2 + 2 rho (l.h)^2,
//             fSS = 5/4 [FSS (1 / (n.l + n.v) - 1/2) + 1/2],
//             FSS = (1 + (F90 - 1) S(n.l)) (1 + (F90 - 1) S(n.v)), F90 = rho (l.h)^2;
//   sheen     (1 - mu) sheen S(l.h) (1 + sheen_tint (C_t - 1));
//   specular  D_s F_s G_s: anisotropic GGX (GTR, gamma = 2),
//             a_x = max(1e-3, rho^2 / k), a_y = max(1e-3, rho^2 k), k = sqrt(1 - 0.9 aniso),
//             F_s = C0 + (1 - C0) S(l.h),
//             C0 = (1 - mu) 0.08 specular (1 + spec_tint (C_t - 1)) + mu base,
//             G_s = g(l) g(v), g(w) = 1 / (n.w + sqrt((w.X a_x)^2 + (w.Y a_y)^2 + (n.w)^2))
//             (separable Smith masking with the 1 / (4 n.l n.v) folded in);
//   clearcoat clearcoat / 4 D_c F_c G_c: GTR with gamma = 1 and a_c = 0.1 - 0.099 gloss,
//             D_c = (a_c^2 - 1) / (pi ln(a_c^2) (1 + (a_c^2 - 1) (n.h)^2)),
//             F_c = 0.04 + 0.96 S(l.h), G_c = g_c(l) g_c(v) with width 0.25.
// X, Y: tangent frame (the hit triangle's first edge made orthogonal to the
// shading normal, then n x X).  Derivatives with respect to the 13 material
// values are exact first derivatives by forward-mode dual numbers.
// ---------------------------------------------------------------------------
constexpr int kDisneyMat = 13;
constexpr int kDisneyStride = 16;

struct Dual {
  double v;
  double d[kDisneyMat];
};
inline Dual dconst(double x) {
  Dual r;
  r.v = x;
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = 0.0;
  return r;
}
inline Dual dvar(double x, int i) {
  Dual r = dconst(x);
  r.d[i] = 1.0;
  return r;
}
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v + b.v;
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v - b.v;
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v * b.v;
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v / b.v;
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
inline Dual operator+(const Dual& a, double b) { return a + dconst(b); }
inline Dual operator+(double a, const Dual& b) { return dconst(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - dconst(b); }
inline Dual operator-(double a, const Dual& b) { return dconst(a) - b; }
inline Dual operator*(const Dual& a, double b) { return a * dconst(b); }
inline Dual operator*(double a, const Dual& b) { return dconst(a) * b; }
inline Dual operator/(const Dual& a, double b) { return a / dconst(b); }
inline Dual operator/(double a, const Dual& b) { return dconst(a) / b; }
inline Dual sqrt(const Dual& a) {
  Dual r;
  r.v = std::sqrt(a.v);
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
inline Dual log(const Dual& a) {
  Dual r;
  r.v = std::log(a.v);
  for (int i = 0; i < kDisneyMat; ++i) r.d[i] = a.d[i] / a.v;
  return r;
}
inline double sqrt(double a) { return std::sqrt(a); }
inline double log(double a) { return std::log(a); }
inline double value(double x) { return x; }
inline double value(const Dual& x) { return x.v; }
// max(a, c) for a constant c (zero derivative where the constant wins)
inline double floor_at(double a, double c) { return a > c ? a : c; }
inline Dual floor_at(const Dual& a, double c) { return a.v > c ? a : dconst(c); }

inline double schlick_w(double c) {
  const double m = std::min(1.0, std::max(0.0, 1.0 - c));
  return m * m * m * m * m;
}

// Tangent frame at shading normal n from a triangle edge e1.
inline void tangent_frame(V3 e1, V3 n, V3& X, V3& Y) {
  V3 t = e1 - n * dot(n, e1);
  double len = length(t);
  if (!(len > 1e-12 * length(e1))) {
    V3 b2;
    onb(n, t, b2);
    len = 1.0;
  }
  X = t * (1.0 / len);
  Y = cross(n, X);
}

// Anisotropic widths (a_x, a_y) from roughness and anisotropy.
template <class T>
inline void disney_widths(const T& rho, const T& ani, T& ax, T& ay) {
  const T k = sqrt(1.0 - 0.9 * ani);
  ax = floor_at(rho * rho / k, 1e-3);
  ay = floor_at(rho * rho * k, 1e-3);
}

inline double clearcoat_width(double gloss) { return 0.1 - 0.099 * gloss; }

// GTR, gamma = 1 (the clearcoat lobe's normal distribution).
template <class T>
inline T gtr1(double ch, const T& a) {
  const T a2 = a * a;
  return (a2 - 1.0) / (kPi * log(a2) * (1.0 + (a2 - 1.0) * (ch * ch)));
}

// f_r per channel for the 13 material values m (double, or Dual for the
// derivatives); zero unless both directions are above the shading hemisphere.
template <class T>
void disney_f(const T* m, V3 n, V3 X, V3 Y, V3 wi, V3 wo, T f[3]) {
  const double cl = dot(n, wo), cv = dot(n, wi);
  if (!(cl > 0.0) || !(cv > 0.0)) {
    for (int c = 0; c < 3; ++c) f[c] = m[0] * 0.0;
    return;
  }
  const V3 h = normalize(wi + wo);
  const double ch = dot(n, h), cd = dot(wo, h);
  const double Sl = schlick_w(cl), Sv = schlick_w(cv), Sd = schlick_w(cd);
  const T& sub = m[3];
  const T& met = m[4];
  const T& spc = m[5];
  const T& spt = m[6];
  const T& rho = m[7];
  const T& shn = m[9];
  const T& sht = m[10];
  const T& cc = m[11];
  const T lb = m[0] * kLumR + m[1] * kLumG + m[2] * kLumB;
  T tint[3];
  for (int c = 0; c < 3; ++c) tint[c] = value(lb) > 0.0 ? m[c] / lb : m[c] * 0.0 + 1.0;
  // diffuse with the subsurface blend
  const T fd90 = 0.5 + (2.0 * cd * cd) * rho;
  const T fd = (1.0 + (fd90 - 1.0) * Sl) * (1.0 + (fd90 - 1.0) * Sv);
  const T f90 = (cd * cd) * rho;
  const T fss0 = (1.0 + (f90 - 1.0) * Sl) * (1.0 + (f90 - 1.0) * Sv);
  const T fss = 1.25 * (fss0 * (1.0 / (cl + cv) - 0.5) + 0.5);
  const T diff = (1.0 - met) * ((1.0 - sub) * fd + sub * fss) * (1.0 / kPi);
  // anisotropic GGX
  T ax, ay;
  disney_widths(rho, m[8], ax, ay);
  const double hx = dot(h, X), hy = dot(h, Y);
  const T q = (hx * hx) / (ax * ax) + (hy * hy) / (ay * ay) + ch * ch;
  const T Ds = 1.0 / (kPi * ax * ay * q * q);
  const double lx = dot(wo, X), ly = dot(wo, Y), vx = dot(wi, X), vy = dot(wi, Y);
  const T gl = 1.0 / (cl + sqrt((lx * lx) * (ax * ax) + (ly * ly) * (ay * ay) + cl * cl));
  const T gv = 1.0 / (cv + sqrt((vx * vx) * (ax * ax) + (vy * vy) * (ay * ay) + cv * cv));
  const T spec_geo = Ds * gl * gv;
  // clearcoat
  const T ac = 0.1 - 0.099 * m[12];
  const double gcl = 1.0 / (cl + std::sqrt(0.0625 + cl * cl - 0.0625 * cl * cl));
  const double gcv = 1.0 / (cv + std::sqrt(0.0625 + cv * cv - 0.0625 * cv * cv));
  const T coat = 0.25 * cc * gtr1(ch, ac) * ((0.04 + 0.96 * Sd) * gcl * gcv);
  for (int c = 0; c < 3; ++c) {
    const T C0 = (1.0 - met) * 0.08 * spc * (1.0 + spt * (tint[c] - 1.0)) + met * m[c];
    const T Fs = C0 + (1.0 - C0) * Sd;
    const T sheen = (1.0 - met) * shn * Sd * (1.0 + sht * (tint[c] - 1.0));
    f[c] = m[c] * diff + sheen + Fs * spec_geo + coat;
  }
}

// Lobe probabilities (diffuse, specular, clearcoat) from the sampling
// parameters: weights (1 - mu) lum(base), (1 - mu) 0.08 specular + mu lum(base)
// and clearcoat / 4, normalised (all diffuse when they sum to zero).
inline void disney_lobes(const double* m, double p[3]) {
  const double lb = kLumR * m[0] + kLumG * m[1] + kLumB * m[2];
  const double wd = (1.0 - m[4]) * lb;
  const double ws = (1.0 - m[4]) * 0.08 * m[5] + m[4] * lb;
  const double wc = 0.25 * m[11];
  const double sum = wd + ws + wc;
  if (!(sum > 0.0)) {
    p[0] = 1.0;
    p[1] = p[2] = 0.0;
    return;
  }
  p[0] = wd / sum;
  p[1] = ws / sum;
  p[2] = wc / sum;
}

// Solid-angle pdf of the Disney sampler: cosine-weighted diffuse, visible
// anisotropic GGX normals (Heitz 2018, stretched by a_x, a_y in the tangent
// frame) and GTR1 normals for the clearcoat, mixed by the lobe probabilities.
inline double disney_pdf(const double* ms, V3 n, V3 X, V3 Y, V3 wi, V3 wo) {
  const double cv = dot(n, wi), cl = dot(n, wo);
  if (!(cv > 0.0) || !(cl > 0.0)) return 0.0;
  double p[3];
  disney_lobes(ms, p);
  const V3 h = normalize(wi + wo);
  const double ch = dot(n, h);
  double pdf = p[0] * cl / kPi;
  if (p[1] > 0.0) {
    double ax, ay;
    disney_widths(ms[7], ms[8], ax, ay);
    const double hx = dot(h, X), hy = dot(h, Y);
    const double q = (hx * hx) / (ax * ax) + (hy * hy) / (ay * ay) + ch * ch;
    const double D = 1.0 / (kPi * ax * ay * q * q);
    const double vx = dot(wi, X), vy = dot(wi, Y);
    const double lam = 0.5 * (std::sqrt(1.0 + (vx * vx * ax * ax + vy * vy * ay * ay) / (cv * cv)) - 1.0);
    pdf += p[1] * D / (1.0 + lam) / (4.0 * cv);
  }
  if (p[2] > 0.0) {
    const double wh = dot(wo, h);
    if (wh > 0.0) pdf += p[2] * gtr1(ch, clearcoat_width(ms[12])) * ch / (4.0 * wh);
  }
  return pdf;
}

// Sample wo from wi: lobe by u_lobe against the cumulative lobe
// probabilities, then (u1, u2) as in the lobe's sampler.
inline V3 disney_sample(const double* ms, V3 n, V3 X, V3 Y, V3 wi, double u_lobe, double u1, double u2) {
  double p[3];
  disney_lobes(ms, p);
  const double rr = std::sqrt(u1);
  const double phi = 2.0 * kPi * u2;
  if (u_lobe < p[0]) {
    V3 b1, b2;
    onb(n, b1, b2);
    return b1 * (rr * std::cos(phi)) + b2 * (rr * std::sin(phi)) + n * std::sqrt(std::max(0.0, 1.0 - u1));
  }
  V3 hw;
  if (u_lobe < p[0] + p[1]) {
    double ax, ay;
    disney_widths(ms[7], ms[8], ax, ay);
    const V3 vl = {dot(wi, X), dot(wi, Y), dot(wi, n)};
    const V3 vh = normalize(V3{ax * vl.x, ay * vl.y, vl.z});
    const double lensq = vh.x * vh.x + vh.y * vh.y;
    const V3 t1 = lensq > 0.0 ? V3{-vh.y, vh.x, 0.0} * (1.0 / std::sqrt(lensq)) : V3{1.0, 0.0, 0.0};
    const V3 t2 = cross(vh, t1);
    const double q1 = rr * std::cos(phi);
    double q2 = rr * std::sin(phi);
    const double s = 0.5 * (1.0 + vh.z);
    q2 = (1.0 - s) * std::sqrt(1.0 - q1 * q1) + s * q2;
    const V3 nh = t1 * q1 + t2 * q2 + vh * std::sqrt(std::max(0.0, 1.0 - q1 * q1 - q2 * q2));
    const V3 ne = normalize(V3{ax * nh.x, ay * nh.y, std::max(0.0, nh.z)});
    hw = X * ne.x + Y * ne.y + n * ne.z;
  } else {
    // GTR1: cos^2 theta_h = (1 - a^(2 (1 - u1))) / (1 - a^2)
    const double a2 = clearcoat_width(ms[12]) * clearcoat_width(ms[12]);
    const double c2 = (1.0 - std::pow(a2, 1.0 - u1)) / (1.0 - a2);
    const double ct = std::sqrt(std::max(0.0, c2)), st = std::sqrt(std::max(0.0, 1.0 - c2));
    V3 b1, b2;
    onb(n, b1, b2);
    hw = b1 * (st * std::cos(phi)) + b2 * (st * std::sin(phi)) + n * ct;
  }
  return hw * (2.0 * dot(wi, hw)) - wi;
}

// ---------------------------------------------------------------------------
// Light selection proportional to current emission (Appendix E keeps these
// probabilities per object in a Fenwick tree; here the object distribution is
// rebuilt per call).  Object s is chosen with probability
// lum(e_s) A_s / W, then triangle t of s with probability A_t / A_s, then a
// uniform point on t, so the area density is p_A = lum(e_s) / W.
// ---------------------------------------------------------------------------
struct LightDist {
  std::vector<double> cdf;  // inclusive, per segment
  std::vector<double> lum;  // lum(e_s), clamped at 0
  double W = 0.0;
};

// Emission of segment k sits at offset stride - 3 of its parameter block
// (10 values per segment for Lambert + GGX, 16 for the Disney model).
LightDist light_dist(const Scene& s, const double* sparams, int stride = 10) {
  LightDist L;
  L.cdf.resize(s.ns);
  L.lum.resize(s.ns);
  double acc = 0.0;
  for (uint32_t k = 0; k < s.ns; ++k) {
    const double* e = sparams + (size_t)stride * k + (stride - 3);
    double l = kLumR * e[0] + kLumG * e[1] + kLumB * e[2];
    if (!(l > 0.0)) l = 0.0;
    L.lum[k] = l;
    acc = acc + l * s.seg_area[k];
    L.cdf[k] = acc;
  }
  L.W = acc;
  return L;
}

struct LightSample {
  int tri;
  int seg;
  V3 y;
  double pA;
};

LightSample light_sample(const Scene& s, const LightDist& L, double u_seg, double u_tri,
                         double ua, double ub) {
  LightSample ls;
  const double target = u_seg * L.W;
  uint32_t k = 0;
  while (k + 1 < s.ns && !(target < L.cdf[k])) ++k;
  ls.seg = (int)k;
  const uint32_t b = s.seg_begin[k], e = s.seg_begin[k + 1];
  const double t2 = u_tri * s.seg_area[k];
  uint32_t j = b;
  while (j + 1 < e && !(t2 < s.tri_cdf[j])) ++j;
  const uint32_t t = s.seg_tris[j];
  ls.tri = (int)t;
  const double su = std::sqrt(ua);
  const double b0 = 1.0 - su, b1 = ub * su, b2 = 1.0 - b0 - b1;
  ls.y = s.p0[t] * b0 + s.p1[t] * b1 + s.p2[t] * b2;
  ls.pA = L.lum[k] / L.W;
  return ls;
}

// ---------------------------------------------------------------------------
// Options and camera (the oracle's own definitions).
// ---------------------------------------------------------------------------
}  // namespace

extern "C" {

typedef struct {
  double cam_to_world[12];  // row-major 3x4: right, up, backward, position columns
  double fov_y_deg;
  uint32_t width, height;
} ora_camera;

typedef struct {
  uint32_t spp;
  uint32_t max_depth;
  int32_t nee;
  int32_t mis;
  int32_t profile;  // 0 cosine (Sec. 4.3), 1 uniform (front face)
  uint32_t set;     // 0 residual, 1 derivative, 2 target, 3 cache
  uint32_t iteration;
  uint32_t scene_id;
  uint64_t seed;
  double emission_scale;
  uint32_t pixel_offset;  // global id of pixel 0 of this view (= sum of earlier views' W*H)
  uint32_t model;         // 0: Lambert + GGX (10 values per segment), 1: Disney (16)
} ora_opts;

}  // extern "C"

namespace {

struct PathVertex {
  int tri, seg;
  V3 x, ns, ng;    // normals oriented to the incoming side
  V3 tx, ty;       // tangent frame (Disney model)
  V3 wi;           // towards the previous vertex
  double prof;     // emission profile toward wi (0 on the back face)
  double w_bsdf;   // MIS weight of emission found at this vertex
  // next-event estimation
  bool nee;
  int l_seg;
  V3 wl;
  double nee_k;    // cos_x * profile(light) * (cos_l / r^2) / p_A * w_light
  // continuation
  bool cont;
  V3 wo;
  double cont_k;   // cos_o / pdf
};

struct Ctx {
  const Scene* s;
  const double* params;
  const double* sparams;
  const ora_opts* o;
  LightDist L;
  double eps;  // spawn offset along the oriented geometric normal
  int disney;  // material model: Disney (16 values per segment) or Lambert + GGX (10)
  int stride;
};

// Sampling pdf and direction at a path vertex, for the context's model.
inline double vertex_pdf(const Ctx& C, const PathVertex& v, V3 wo) {
  if (C.disney) return disney_pdf(C.sparams + kDisneyStride * v.seg, v.ns, v.tx, v.ty, v.wi, wo);
  return bsdf_pdf(mat_of(C.sparams + 10 * v.seg), v.ns, v.wi, wo);
}
inline V3 vertex_sample(const Ctx& C, const PathVertex& v, double ul, double u1, double u2) {
  if (C.disney) return disney_sample(C.sparams + kDisneyStride * v.seg, v.ns, v.tx, v.ty, v.wi, ul, u1, u2);
  return bsdf_sample(mat_of(C.sparams + 10 * v.seg), v.ns, v.wi, ul, u1, u2);
}

// One camera path for pixel (px, py), sample index `sample`, following the
// dimension map: vertex k, call 0 -> (u_lobe, u_dir1, u_dir2, u_light_seg),
// call 1 -> (u_light_tri, u_light_a, u_light_b, unused), vertex 0 call 2 ->
// (u_jitter_x, u_jitter_y, unused, unused).
std::vector<PathVertex> trace_path(const Ctx& C, const ora_camera& cam, uint32_t px, uint32_t py,
                                   uint32_t sample) {
  const Scene& s = *C.s;
  const ora_opts& o = *C.o;
  Rng rng;
  rng.key[0] = (uint32_t)(o.seed & 0xFFFFFFFFu);
  rng.key[1] = (uint32_t)(o.seed >> 32) ^ o.scene_id;
  rng.base[0] = o.pixel_offset + py * cam.width + px;
  rng.base[1] = sample;
  rng.base[2] = (o.set << 24) | (o.iteration & 0xFFFFFFu);

  double u[4];
  rng.draw(0, 2, u);
  const double ndc_x = 2.0 * ((double)px + u[0]) / cam.width - 1.0;
  const double ndc_y = 1.0 - 2.0 * ((double)py + u[1]) / cam.height;
  const double th = std::tan(0.5 * cam.fov_y_deg * kPi / 180.0);
  const double aspect = (double)cam.width / (double)cam.height;
  const V3 dc = {ndc_x * th * aspect, ndc_y * th, -1.0};
  const double* M = cam.cam_to_world;
  V3 d = normalize(V3{M[0] * dc.x + M[1] * dc.y + M[2] * dc.z, M[4] * dc.x + M[5] * dc.y + M[6] * dc.z,
                      M[8] * dc.x + M[9] * dc.y + M[10] * dc.z});
  V3 org = {M[3], M[7], M[11]};
  int skip = -1;
  double prev_pdf = 0.0;  // solid-angle pdf of the direction that led here
  bool prev_nee = false;  // light sampling was possible at the previous vertex
  std::vector<PathVertex> path;
  const bool light_on = o.nee && C.L.W > 0.0;
  for (uint32_t k = 0; k <= o.max_depth; ++k) {
    const Hit h = closest(s, org, d, 0.0, 1e300, skip, false);
    if (h.tri < 0) break;
    PathVertex v{};
    v.tri = h.tri;
    v.seg = (int)s.seg[h.tri];
    const uint32_t t = (uint32_t)h.tri;
    const double w0 = 1.0 - h.u - h.v;
    v.x = s.p0[t] * w0 + s.p1[t] * h.u + s.p2[t] * h.v;
    v.wi = -d;
    const V3 ng0 = s.ng[t];
    V3 ns = s.has_normals ? normalize(s.n0[t] * w0 + s.n1[t] * h.u + s.n2[t] * h.v) : ng0;
    // emission leaves the front face only (profile is the clamped cosine)
    const double cos_e = dot(v.wi, ng0);
    v.prof = o.profile == 0 ? std::max(0.0, cos_e) : (cos_e > 0.0 ? 1.0 : 0.0);
    // MIS weight of BRDF-sampled emission
    v.w_bsdf = 1.0;
    if (k > 0 && prev_nee) {
      const double pa = C.L.lum[v.seg] > 0.0 ? C.L.lum[v.seg] / C.L.W : 0.0;
      if (pa > 0.0 && cos_e > 0.0) {
        const double pl = pa * h.t * h.t / cos_e;
        v.w_bsdf = o.mis ? prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl) : 0.0;
      }
    }
    // two-sided shading: orient both normals to the incoming side
    const double sg = cos_e < 0.0 ? -1.0 : 1.0;
    v.ng = ng0 * sg;
    v.ns = ns * sg;
    if (C.disney) tangent_frame(s.p1[t] - s.p0[t], v.ns, v.tx, v.ty);
    v.nee = false;
    v.cont = false;
    if (k == o.max_depth) {
      path.push_back(v);
      break;
    }
    double ua[4], ub[4];
    rng.draw(k, 0, ua);
    rng.draw(k, 1, ub);
    if (light_on) {
      const LightSample ls = light_sample(s, C.L, ua[3], ub[0], ub[1], ub[2]);
      const V3 dl = ls.y - v.x;
      const double r2 = dot(dl, dl);
      const double r = std::sqrt(r2);
      const V3 wl = dl * (1.0 / r);
      const V3 so = v.x + v.ng * C.eps;  // shadow ray leaves from the offset point
      const V3 ds = ls.y - so;
      const double rs = length(ds);
      const double cos_l = -dot(wl, s.ng[ls.tri]);
      const double lprof = o.profile == 0 ? std::max(0.0, cos_l) : (cos_l > 0.0 ? 1.0 : 0.0);
      const double cxg = dot(wl, v.ng), cxs = dot(wl, v.ns);
      if (lprof > 0.0 && cxg > 0.0 && cxs > 0.0 && dot(v.wi, v.ns) > 0.0 &&
          !occluded(s, so, ds * (1.0 / rs), 0.0, rs * (1.0 - 1e-5), h.tri, ls.tri)) {
        double wlight = 1.0;
        if (o.mis) {
          const double pl = ls.pA * r2 / cos_l;
          const double pb = vertex_pdf(C, v, wl);
          wlight = pl * pl / (pl * pl + pb * pb);
        }
        v.nee = true;
        v.l_seg = ls.seg;
        v.wl = wl;
        v.nee_k = cxs * lprof * (cos_l / r2) / ls.pA * wlight;
      }
    }
    prev_nee = light_on;
    if (!(dot(v.wi, v.ns) > 0.0)) {
      path.push_back(v);
      break;
    }
    const V3 wo = vertex_sample(C, v, ua[0], ua[1], ua[2]);
    const double pdf = vertex_pdf(C, v, wo);
    if (!(dot(wo, v.ng) > 0.0) || !(dot(wo, v.ns) > 0.0) || !(pdf > 0.0)) {
      path.push_back(v);
      break;
    }
    v.cont = true;
    v.wo = wo;
    v.cont_k = dot(wo, v.ns) / pdf;
    path.push_back(v);
    prev_pdf = pdf;
    org = v.x + v.ng * C.eps;
    d = wo;
    skip = h.tri;
  }
  return path;
}

// One light path ending at a path vertex: emission factor times BSDF factors.
struct BsdfFactor {
  int vtx;      // path vertex
  V3 wo;        // outgoing direction used at that vertex
  double k;     // constant factor (cos / pdf, or the NEE geometry term)
};

// Radiance and (optionally) g-weighted parameter gradient of one path, by
// enumerating its light paths (one per emission event) and applying Eq. 2,
// Eq. 5 and Eq. 6 to each.
void disney_value_and_grad(const Ctx& C, const std::vector<PathVertex>& path, const double* g,
                           double L[3], double* grad);

void path_value_and_grad(const Ctx& C, const std::vector<PathVertex>& path, const double* g,
                         double L[3], double* grad) {
  if (C.disney) {
    disney_value_and_grad(C, path, g, L, grad);
    return;
  }
  const double es = C.o->emission_scale;
  L[0] = L[1] = L[2] = 0.0;
  std::vector<BsdfFactor> fs;
  auto light_path = [&](const std::vector<BsdfFactor>& f, int e_seg, double ek) {
    // value_c = es * e_{seg,c} * ek * prod_i f_r,c(i) k_i
    const size_t n = f.size();
    std::vector<BrdfEval> be(n);
    std::vector<Mat> mats(n);
    for (size_t i = 0; i < n; ++i) {
      const PathVertex& pv = path[f[i].vtx];
      mats[i] = mat_of(C.params + 10 * pv.seg);
      be[i] = brdf_eval(mats[i], pv.ns, pv.wi, f[i].wo);
    }
    const Mat me = mat_of(C.params + 10 * e_seg);
    for (int c = 0; c < 3; ++c) {
      double prod = 1.0;
      for (size_t i = 0; i < n; ++i) prod *= be[i].f[c] * f[i].k;
      const double Le = es * me.e[c] * ek;
      L[c] += Le * prod;
      if (!grad) continue;
      // Eq. 5: d/d e_c of the emission, times the product of BSDF factors
      grad[10 * e_seg + 7 + c] += g[c] * es * ek * prod;
      // Eq. 6: sum over l of d f_r(l) times the product over i != l
      for (size_t l = 0; l < n; ++l) {
        double others = 1.0;
        for (size_t i = 0; i < n; ++i)
          if (i != l) others *= be[i].f[c] * f[i].k;
        const double base = g[c] * Le * others * f[l].k;
        const int sl = path[f[l].vtx].seg;
        grad[10 * sl + c] += base / kPi;                         // d f / d kd_c
        grad[10 * sl + 3 + c] += base * be[l].spec;              // d f / d ks_c
        grad[10 * sl + 6] += base * mats[l].ks[c] * be[l].dspec_dr;  // d f / d r
      }
    }
  };
  for (size_t m = 0; m < path.size(); ++m) {
    const PathVertex& v = path[m];
    // emission found at vertex m (BRDF-sampled, or seen by the camera)
    if (v.prof > 0.0 && v.w_bsdf > 0.0) light_path(fs, v.seg, v.prof * v.w_bsdf);
    // next-event estimation at vertex m
    if (v.nee) {
      fs.push_back({(int)m, v.wl, v.nee_k});
      light_path(fs, v.l_seg, 1.0);
      fs.pop_back();
    }
    if (!v.cont) break;
    fs.push_back({(int)m, v.wo, v.cont_k});
  }
}

// Throughput beta_b (per channel) of the first b vertices' BSDF factors,
// f_r * cos / pdf, evaluated at the parameters.
void path_beta(const Ctx& C, const std::vector<PathVertex>& path, size_t b, double beta[3]) {
  beta[0] = beta[1] = beta[2] = 1.0;
  for (size_t i = 0; i < b; ++i) {
    const PathVertex& pv = path[i];
    const BrdfEval be = brdf_eval(mat_of(C.params + 10 * pv.seg), pv.ns, pv.wi, pv.wo);
    for (int c = 0; c < 3; ++c) beta[c] *= be.f[c] * pv.cont_k;
  }
}

// The cached estimator ends a path at vertex b: it keeps the emission found
// at b, drops next-event estimation and continuation there, and adds
// beta_b * Lc, where Lc is the cache's reflected radiance at b.  This is the
// path with its tail cut (the prefix).
std::vector<PathVertex> cut_at(const std::vector<PathVertex>& path, size_t b) {
  std::vector<PathVertex> head(path.begin(), path.begin() + (long)(b + 1));
  head[b].nee = false;
  head[b].cont = false;
  return head;
}

// Value and g-weighted gradient of the cache term beta_b * Lc of one path.
// Lc depends on the material parameters (kd, ks, r) of the terminal segment
// through the 3 x 7 Jacobian J; beta_b on the earlier vertices by Eq. 6.
void cache_term(const Ctx& C, const std::vector<PathVertex>& path, size_t b, const double Lc[3],
                const double J[21], const double* g, double L[3], double* grad) {
  std::vector<BrdfEval> be(b);
  std::vector<Mat> mats(b);
  for (size_t i = 0; i < b; ++i) {
    mats[i] = mat_of(C.params + 10 * path[i].seg);
    be[i] = brdf_eval(mats[i], path[i].ns, path[i].wi, path[i].wo);
  }
  const int sb = path[b].seg;
  for (int c = 0; c < 3; ++c) {
    double prod = 1.0;
    for (size_t i = 0; i < b; ++i) prod *= be[i].f[c] * path[i].cont_k;
    L[c] += Lc[c] * prod;
    if (!grad) continue;
    for (int j = 0; j < 7; ++j) grad[10 * sb + j] += g[c] * prod * J[7 * c + j];
    for (size_t l = 0; l < b; ++l) {
      double others = 1.0;
      for (size_t i = 0; i < b; ++i)
        if (i != l) others *= be[i].f[c] * path[i].cont_k;
      const double base = g[c] * Lc[c] * others * path[l].cont_k;
      const int sl = path[l].seg;
      grad[10 * sl + c] += base / kPi;
      grad[10 * sl + 3 + c] += base * be[l].spec;
      grad[10 * sl + 6] += base * mats[l].ks[c] * be[l].dspec_dr;
    }
  }
}

// The same enumeration of light paths for the Disney model: each BSDF factor
// is f_r * k with f_r from disney_f, and Eq. 6 takes its 3 x 13 Jacobian
// times the product of the other factors.
void disney_value_and_grad(const Ctx& C, const std::vector<PathVertex>& path, const double* g,
                           double L[3], double* grad) {
  const double es = C.o->emission_scale;
  const int S = kDisneyStride;
  L[0] = L[1] = L[2] = 0.0;
  std::vector<BsdfFactor> fs;
  auto light_path = [&](const std::vector<BsdfFactor>& f, int e_seg, double ek) {
    const size_t n = f.size();
    std::vector<double> fv(3 * n);
    std::vector<Dual> fd(grad ? 3 * n : 0);
    for (size_t i = 0; i < n; ++i) {
      const PathVertex& pv = path[f[i].vtx];
      const double* p = C.params + (size_t)S * pv.seg;
      disney_f(p, pv.ns, pv.tx, pv.ty, pv.wi, f[i].wo, &fv[3 * i]);
      if (grad) {
        Dual md[kDisneyMat];
        for (int j = 0; j < kDisneyMat; ++j) md[j] = dvar(p[j], j);
        disney_f(md, pv.ns, pv.tx, pv.ty, pv.wi, f[i].wo, &fd[3 * i]);
      }
    }
    const double* e = C.params + (size_t)S * e_seg + kDisneyMat;
    for (int c = 0; c < 3; ++c) {
      double prod = 1.0;
      for (size_t i = 0; i < n; ++i) prod *= fv[3 * i + c] * f[i].k;
      const double Le = es * e[c] * ek;
      L[c] += Le * prod;
      if (!grad) continue;
      grad[(size_t)S * e_seg + kDisneyMat + c] += g[c] * es * ek * prod;  // Eq. 5
      for (size_t l = 0; l < n; ++l) {                                       // Eq. 6
        double others = 1.0;
        for (size_t i = 0; i < n; ++i)
          if (i != l) others *= fv[3 * i + c] * f[i].k;
        const double base = g[c] * Le * others * f[l].k;
        double* gs = grad + (size_t)S * path[f[l].vtx].seg;
        for (int j = 0; j < kDisneyMat; ++j) gs[j] += base * fd[3 * l + c].d[j];
      }
    }
  };
  for (size_t m = 0; m < path.size(); ++m) {
    const PathVertex& v = path[m];
    if (v.prof > 0.0 && v.w_bsdf > 0.0) light_path(fs, v.seg, v.prof * v.w_bsdf);
    if (v.nee) {
      fs.push_back({(int)m, v.wl, v.nee_k});
      light_path(fs, v.l_seg, 1.0);
      fs.pop_back();
    }
    if (!v.cont) break;
    fs.push_back({(int)m, v.wo, v.cont_k});
  }
}

Ctx make_ctx(const Scene* s, const double* params, const double* sparams, const ora_opts* o) {
  Ctx C;
  C.s = s;
  C.params = params;
  C.sparams = sparams ? sparams : params;
  C.o = o;
  C.disney = o->model == 1 ? 1 : 0;
  C.stride = C.disney ? kDisneyStride : 10;
  C.L = light_dist(*s, C.sparams, C.stride);
  C.eps = 1e-5 * s->diameter;
  return C;
}

template <class F>
void parallel_for(uint32_t n, int nthreads, F f) {
  if (nthreads <= 1 || n < 2) {
    for (uint32_t i = 0; i < n; ++i) f(0, i);
    return;
  }
  std::atomic<uint32_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      for (;;) {
        const uint32_t i = next.fetch_add(1);
        if (i >= n) break;
        f(t, i);
      }
    });
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

int ora_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
  return 0;
}

void* ora_scene_create(const float* pos, uint32_t nv, const float* nrm, const uint32_t* idx,
                       uint32_t nt, const uint32_t* tri_seg, uint32_t ns) {
  Scene* s = new Scene();
  s->nt = nt;
  s->ns = ns;
  s->has_normals = nrm != nullptr;
  s->p0.resize(nt);
  s->p1.resize(nt);
  s->p2.resize(nt);
  s->n0.resize(nt);
  s->n1.resize(nt);
  s->n2.resize(nt);
  s->ng.resize(nt);
  s->area.resize(nt);
  s->seg.assign(tri_seg, tri_seg + nt);
  V3 lo = {1e300, 1e300, 1e300}, hi = {-1e300, -1e300, -1e300};
  for (uint32_t i = 0; i < nv; ++i) {
    const V3 q = load3(pos, i);
    lo = {std::min(lo.x, q.x), std::min(lo.y, q.y), std::min(lo.z, q.z)};
    hi = {std::max(hi.x, q.x), std::max(hi.y, q.y), std::max(hi.z, q.z)};
  }
  s->diameter = length(hi - lo);
  for (uint32_t t = 0; t < nt; ++t) {
    s->p0[t] = load3(pos, idx[3 * t]);
    s->p1[t] = load3(pos, idx[3 * t + 1]);
    s->p2[t] = load3(pos, idx[3 * t + 2]);
    const V3 e1 = s->p1[t] - s->p0[t], e2 = s->p2[t] - s->p0[t];
    const V3 c = cross(e1, e2);
    const double len = std::sqrt(c.x * c.x + c.y * c.y + c.z * c.z);
    s->area[t] = 0.5 * len;
    s->ng[t] = c * (1.0 / len);
    if (nrm) {
      s->n0[t] = load3(nrm, idx[3 * t]);
      s->n1[t] = load3(nrm, idx[3 * t + 1]);
      s->n2[t] = load3(nrm, idx[3 * t + 2]);
    } else {
      s->n0[t] = s->n1[t] = s->n2[t] = s->ng[t];
    }
  }
  // triangles grouped by segment (stable: increasing id), area CDFs
  s->seg_begin.assign(ns + 1, 0);
  for (uint32_t t = 0; t < nt; ++t) s->seg_begin[tri_seg[t] + 1]++;
  for (uint32_t k = 0; k < ns; ++k) s->seg_begin[k + 1] += s->seg_begin[k];
  s->seg_tris.resize(nt);
  std::vector<uint32_t> fill(s->seg_begin.begin(), s->seg_begin.end() - 1);
  for (uint32_t t = 0; t < nt; ++t) s->seg_tris[fill[tri_seg[t]]++] = t;
  s->tri_cdf.resize(nt);
  s->seg_area.assign(ns, 0.0);
  for (uint32_t k = 0; k < ns; ++k) {
    double acc = 0.0;
    for (uint32_t j = s->seg_begin[k]; j < s->seg_begin[k + 1]; ++j) {
      acc = acc + s->area[s->seg_tris[j]];
      s->tri_cdf[j] = acc;
    }
    s->seg_area[k] = acc;
  }
  // BVH
  std::vector<V3> cen(nt);
  for (uint32_t t = 0; t < nt; ++t) cen[t] = (s->p0[t] + s->p1[t] + s->p2[t]) * (1.0 / 3.0);
  s->bvh_tris.resize(nt);
  for (uint32_t t = 0; t < nt; ++t) s->bvh_tris[t] = t;
  if (nt) build_bvh(*s, s->bvh_tris, 0, (int)nt, cen);
  return s;
}

void ora_scene_destroy(void* s) { delete static_cast<Scene*>(s); }

double ora_scene_diameter(void* s) { return static_cast<Scene*>(s)->diameter; }

void ora_scene_areas(void* sp, double* tri_area, double* seg_area) {
  const Scene* s = static_cast<Scene*>(sp);
  if (tri_area) std::copy(s->area.begin(), s->area.end(), tri_area);
  if (seg_area) std::copy(s->seg_area.begin(), s->seg_area.end(), seg_area);
}

// Closest hit for n rays (origins and directions as FP64 triples); t in
// (tmin, inf), skipping skip_tri[i] (or none if skip_tri is NULL / -1).
int ora_intersect(void* sp, uint32_t n, const double* orig, const double* dir, const int32_t* skip_tri,
                  double tmin, int32_t brute, int32_t* tri_out, double* t_out, double* u_out,
                  double* v_out, int32_t nthreads) {
  const Scene* s = static_cast<Scene*>(sp);
  parallel_for(n, nthreads, [&](int, uint32_t i) {
    const V3 o = {orig[3 * i], orig[3 * i + 1], orig[3 * i + 2]};
    const V3 d = {dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]};
    const Hit h = closest(*s, o, d, tmin, 1e300, skip_tri ? skip_tri[i] : -1, brute != 0);
    tri_out[i] = h.tri;
    t_out[i] = h.t;
    if (u_out) u_out[i] = h.u;
    if (v_out) v_out[i] = h.v;
  });
  return 0;
}

// BRDF value, specular factor and its roughness derivative for one direction
// pair (params: 10 floats of one segment).  Returns 0 when below the horizon.
int ora_brdf(const double* p, const double* n, const double* wi, const double* wo, double* f3,
             double* spec, double* dspec_dr) {
  const Mat m = mat_of(p);
  const BrdfEval b = brdf_eval(m, {n[0], n[1], n[2]}, {wi[0], wi[1], wi[2]}, {wo[0], wo[1], wo[2]});
  for (int c = 0; c < 3; ++c) f3[c] = b.valid ? b.f[c] : 0.0;
  *spec = b.valid ? b.spec : 0.0;
  *dspec_dr = b.valid ? b.dspec_dr : 0.0;
  return b.valid ? 1 : 0;
}

double ora_ggx_D(double nh, double alpha) { return ggx_D(nh, alpha); }
double ora_smith_lambda(double c, double alpha) { return smith_lambda(c, alpha); }

int ora_bsdf_sample(const double* p, const double* n, const double* wi, double u_lobe, double u1,
                    double u2, double* wo, double* pdf) {
  const Mat m = mat_of(p);
  const V3 nn = {n[0], n[1], n[2]}, w = {wi[0], wi[1], wi[2]};
  const V3 o = bsdf_sample(m, nn, w, u_lobe, u1, u2);
  wo[0] = o.x;
  wo[1] = o.y;
  wo[2] = o.z;
  *pdf = bsdf_pdf(m, nn, w, o);
  return 0;
}

double ora_bsdf_pdf(const double* p, const double* n, const double* wi, const double* wo) {
  return bsdf_pdf(mat_of(p), {n[0], n[1], n[2]}, {wi[0], wi[1], wi[2]}, {wo[0], wo[1], wo[2]});
}

// Disney model at one configuration: f_r per channel and (J nullable) its
// Jacobian J[13 c + j] = d f_c / d m_j.  X: a vector in the tangent plane
// direction (made orthogonal to n here).
int ora_disney_brdf(const double* m, const double* n, const double* x, const double* wi, const double* wo,
                    double* f3, double* J) {
  const V3 nn = {n[0], n[1], n[2]};
  V3 X, Y;
  tangent_frame({x[0], x[1], x[2]}, nn, X, Y);
  const V3 vi = {wi[0], wi[1], wi[2]}, vo = {wo[0], wo[1], wo[2]};
  disney_f(m, nn, X, Y, vi, vo, f3);
  if (J) {
    Dual md[kDisneyMat], fd[3];
    for (int j = 0; j < kDisneyMat; ++j) md[j] = dvar(m[j], j);
    disney_f(md, nn, X, Y, vi, vo, fd);
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < kDisneyMat; ++j) J[kDisneyMat * c + j] = fd[c].d[j];
  }
  return (dot(nn, vi) > 0.0 && dot(nn, vo) > 0.0) ? 1 : 0;
}

double ora_disney_pdf(const double* m, const double* n, const double* x, const double* wi, const double* wo) {
  const V3 nn = {n[0], n[1], n[2]};
  V3 X, Y;
  tangent_frame({x[0], x[1], x[2]}, nn, X, Y);
  return disney_pdf(m, nn, X, Y, {wi[0], wi[1], wi[2]}, {wo[0], wo[1], wo[2]});
}

int ora_disney_sample(const double* m, const double* n, const double* x, const double* wi, double u_lobe,
                      double u1, double u2, double* wo, double* pdf) {
  const V3 nn = {n[0], n[1], n[2]}, w = {wi[0], wi[1], wi[2]};
  V3 X, Y;
  tangent_frame({x[0], x[1], x[2]}, nn, X, Y);
  const V3 o = disney_sample(m, nn, X, Y, w, u_lobe, u1, u2);
  wo[0] = o.x;
  wo[1] = o.y;
  wo[2] = o.z;
  *pdf = disney_pdf(m, nn, X, Y, w, o);
  return 0;
}

void ora_disney_lobes(const double* m, double* p3) { disney_lobes(m, p3); }

// Light selection for an array of uniforms (4 per sample): triangle, point, p_A.
int ora_light_sample(void* sp, const double* sparams, uint32_t n, const double* u, int32_t* tri,
                     double* y, double* pA) {
  const Scene* s = static_cast<Scene*>(sp);
  const LightDist L = light_dist(*s, sparams);
  if (!(L.W > 0.0)) return -1;
  for (uint32_t i = 0; i < n; ++i) {
    const LightSample ls = light_sample(*s, L, u[4 * i], u[4 * i + 1], u[4 * i + 2], u[4 * i + 3]);
    tri[i] = ls.tri;
    y[3 * i] = ls.y.x;
    y[3 * i + 1] = ls.y.y;
    y[3 * i + 2] = ls.y.z;
    pA[i] = ls.pA;
  }
  return 0;
}

// Render pixels of one view: mean and mean of squares per channel over the
// opts->spp samples.  pixels: linear ids py*W+px (NULL = all, in order).
// sample_base: per listed pixel, the sample counter of its first sample
// (NULL = 0); a pixel drawn into a stochastic pixel batch (Sec. 4.5) uses
// samples b*spp .. b*spp+spp-1 for batch entry b.
int ora_render(void* sp, const ora_camera* cam, const double* params, const double* sparams,
               const ora_opts* o, const uint32_t* pixels, const uint32_t* sample_base, uint32_t npix,
               double* mean, double* msq, int32_t nthreads) {
  const Scene* s = static_cast<Scene*>(sp);
  const Ctx C = make_ctx(s, params, sparams, o);
  parallel_for(npix, nthreads, [&](int, uint32_t i) {
    const uint32_t pid = pixels ? pixels[i] : i;
    const uint32_t px = pid % cam->width, py = pid / cam->width;
    const uint32_t s0 = sample_base ? sample_base[i] : 0u;
    double acc[3] = {0, 0, 0}, acc2[3] = {0, 0, 0};
    for (uint32_t smp = 0; smp < o->spp; ++smp) {
      const std::vector<PathVertex> path = trace_path(C, *cam, px, py, s0 + smp);
      double L[3];
      path_value_and_grad(C, path, nullptr, L, nullptr);
      for (int c = 0; c < 3; ++c) {
        acc[c] += L[c];
        acc2[c] += L[c] * L[c];
      }
    }
    for (int c = 0; c < 3; ++c) {
      mean[3 * i + c] = acc[c] / o->spp;
      if (msq) msq[3 * i + c] = acc2[c] / o->spp;
    }
  });
  return 0;
}

// Vector-Jacobian product: grad[S * stride] += sum_pixels sum_c g[pixel,c] *
// d(mean over opts->spp samples of I_c)/d(params), with pdfs, MIS weights and
// light selection held at sparams.  sample_base as in ora_render.
int ora_gradient(void* sp, const ora_camera* cam, const double* params, const double* sparams,
                 const ora_opts* o, const uint32_t* pixels, const uint32_t* sample_base, uint32_t npix,
                 const double* g, double* grad, int32_t nthreads) {
  const Scene* s = static_cast<Scene*>(sp);
  const Ctx C = make_ctx(s, params, sparams, o);
  const int nt = std::max(1, nthreads);
  std::vector<std::vector<double>> part(nt, std::vector<double>((size_t)C.stride * s->ns, 0.0));
  parallel_for(npix, nt, [&](int tid, uint32_t i) {
    const uint32_t pid = pixels ? pixels[i] : i;
    const uint32_t px = pid % cam->width, py = pid / cam->width;
    const double gs[3] = {g[3 * i] / o->spp, g[3 * i + 1] / o->spp, g[3 * i + 2] / o->spp};
    const uint32_t s0 = sample_base ? sample_base[i] : 0u;
    for (uint32_t smp = 0; smp < o->spp; ++smp) {
      const std::vector<PathVertex> path = trace_path(C, *cam, px, py, s0 + smp);
      double L[3];
      path_value_and_grad(C, path, gs, L, part[tid].data());
    }
  });
  for (int t = 0; t < nt; ++t)
    for (size_t k = 0; k < part[t].size(); ++k) grad[k] += part[t][k];
  return 0;
}

// Path vertex count statistics (tests and sizing): number of closest-hit and
// shadow rays traced for the given pixels.
int ora_count_rays(void* sp, const ora_camera* cam, const double* params, const double* sparams,
                   const ora_opts* o, const uint32_t* pixels, uint32_t npix, uint64_t* n_vertices,
                   uint64_t* n_nee) {
  const Scene* s = static_cast<Scene*>(sp);
  const Ctx C = make_ctx(s, params, sparams, o);
  uint64_t nv = 0, nn = 0;
  for (uint32_t i = 0; i < npix; ++i) {
    const uint32_t pid = pixels ? pixels[i] : i;
    for (uint32_t smp = 0; smp < o->spp; ++smp) {
      const auto path = trace_path(C, *cam, pid % cam->width, pid / cam->width, smp);
      nv += path.size();
      for (const auto& v : path) nn += v.nee ? 1 : 0;
    }
  }
  *n_vertices = nv;
  *n_nee = nn;
  return 0;
}


// Cached estimator, per path (pixel i, sample k -> row i * spp + k): the
// prefix value (the path cut at vertex b_term, keeping the emission found
// there), and, where the path reaches vertex b_term < max_depth, the
// throughput beta_b, position, direction towards the previous vertex,
// oriented shading normal and segment of that vertex (seg = -1 otherwise:
// the prefix is then the whole path).
int ora_cache_terminals(void* sp, const ora_camera* cam, const double* params, const double* sparams,
                        const ora_opts* o, uint32_t b_term, const uint32_t* pixels, uint32_t npix,
                        double* prefix, double* beta, double* x, double* wi, double* ns, int32_t* seg,
                        int32_t nthreads) {
  const Scene* s = static_cast<Scene*>(sp);
  const Ctx C = make_ctx(s, params, sparams, o);
  parallel_for(npix, nthreads, [&](int, uint32_t i) {
    const uint32_t pid = pixels ? pixels[i] : i;
    for (uint32_t smp = 0; smp < o->spp; ++smp) {
      const size_t r = (size_t)i * o->spp + smp;
      const std::vector<PathVertex> path = trace_path(C, *cam, pid % cam->width, pid / cam->width, smp);
      const bool term = b_term < o->max_depth && path.size() > b_term;
      double L[3];
      path_value_and_grad(C, term ? cut_at(path, b_term) : path, nullptr, L, nullptr);
      double bb[3] = {0.0, 0.0, 0.0};
      if (term) path_beta(C, path, b_term, bb);
      const PathVertex* v = term ? &path[b_term] : nullptr;
      for (int c = 0; c < 3; ++c) {
        prefix[3 * r + c] = L[c];
        beta[3 * r + c] = bb[c];
        x[3 * r + c] = v ? comp(v->x, c) : 0.0;
        wi[3 * r + c] = v ? comp(v->wi, c) : 0.0;
        ns[3 * r + c] = v ? comp(v->ns, c) : 0.0;
      }
      seg[r] = v ? v->seg : -1;
    }
  });
  return 0;
}

// Vector-Jacobian product of the cached estimator: as ora_gradient, with
// every path cut at b_term and its cache term beta_b * Lc added.  cval
// (rows x 3) and cjac (rows x 3 x 7, d Lc_c / d (kd, ks, r)) are given per
// path row (i * spp + k); rows without a terminal vertex are ignored.
int ora_cache_gradient(void* sp, const ora_camera* cam, const double* params, const double* sparams,
                       const ora_opts* o, uint32_t b_term, const uint32_t* pixels, uint32_t npix, const double* g,
                       const double* cval, const double* cjac, double* grad, int32_t nthreads) {
  const Scene* s = static_cast<Scene*>(sp);
  const Ctx C = make_ctx(s, params, sparams, o);
  const int nt = std::max(1, nthreads);
  std::vector<std::vector<double>> part(nt, std::vector<double>(10 * (size_t)s->ns, 0.0));
  parallel_for(npix, nt, [&](int tid, uint32_t i) {
    const uint32_t pid = pixels ? pixels[i] : i;
    const double gs[3] = {g[3 * i] / o->spp, g[3 * i + 1] / o->spp, g[3 * i + 2] / o->spp};
    for (uint32_t smp = 0; smp < o->spp; ++smp) {
      const size_t r = (size_t)i * o->spp + smp;
      const std::vector<PathVertex> path = trace_path(C, *cam, pid % cam->width, pid / cam->width, smp);
      const bool term = b_term < o->max_depth && path.size() > b_term;
      double L[3];
      path_value_and_grad(C, term ? cut_at(path, b_term) : path, gs, L, part[tid].data());
      if (term) cache_term(C, path, b_term, cval + 3 * r, cjac + 21 * r, gs, L, part[tid].data());
    }
  });
  for (int t = 0; t < nt; ++t)
    for (size_t k = 0; k < part[t].size(); ++k) grad[k] += part[t][k];
  return 0;
}

// Training records of the cache: full-length paths (normally set 3); where a
// path reaches vertex b_term < max_depth, its position, direction, oriented
// shading normal, segment and the target: the reflected radiance the path
// estimates there, i.e. everything it gathers from vertex b_term on except
// the emission found at b_term, divided by beta_b (the sub-path from b_term
// with unit throughput).  seg = -1 where the path ends earlier.
int ora_cache_records(void* sp, const ora_camera* cam, const double* params, const double* sparams,
                      const ora_opts* o, uint32_t b_term, const uint32_t* pixels, uint32_t npix, double* x,
                      double* wi, double* ns, int32_t* seg, double* target, int32_t nthreads) {
  const Scene* s = static_cast<Scene*>(sp);
  const Ctx C = make_ctx(s, params, sparams, o);
  parallel_for(npix, nthreads, [&](int, uint32_t i) {
    const uint32_t pid = pixels ? pixels[i] : i;
    for (uint32_t smp = 0; smp < o->spp; ++smp) {
      const size_t r = (size_t)i * o->spp + smp;
      const std::vector<PathVertex> path = trace_path(C, *cam, pid % cam->width, pid / cam->width, smp);
      const bool term = b_term < o->max_depth && path.size() > b_term;
      double L[3] = {0.0, 0.0, 0.0};
      if (term) {
        std::vector<PathVertex> tail(path.begin() + (long)b_term, path.end());
        tail[0].prof = 0.0;
        path_value_and_grad(C, tail, nullptr, L, nullptr);
      }
      const PathVertex* v = term ? &path[b_term] : nullptr;
      for (int c = 0; c < 3; ++c) {
        x[3 * r + c] = v ? comp(v->x, c) : 0.0;
        wi[3 * r + c] = v ? comp(v->wi, c) : 0.0;
        ns[3 * r + c] = v ? comp(v->ns, c) : 0.0;
        target[3 * r + c] = L[c];
      }
      seg[r] = v ? v->seg : -1;
    }
  });
  return 0;
}

}  // extern "C"
