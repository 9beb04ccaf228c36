// Device building blocks of the GB300 inverse path tracer: float3 algebra,
// Philox4x32-10, the scene layout in HBM, watertight ray casting over a
// binary BVH, the Lambert + GGX material model and its sampling routines.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ipt {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kStackSize = 64;
constexpr uint32_t kErrStack = 1u;      // traversal stack would overflow
constexpr uint32_t kErrNonFinite = 2u;  // a loss or gradient was NaN or infinite: the Adam step was skipped

// ---------------------------------------------------------------------------
// float3 algebra
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return a * rsqrtf(dot(a, a)); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
__device__ __forceinline__ float comp(float3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Bumping the key after
// each round is the same as bumping it before every round but the first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// top 24 bits -> [0,1), exactly representable in FP32 and FP64
__device__ __forceinline__ float to_unit(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// Counter layout of one path: (pixel id, sample id, (set << 24) | iteration,
// 4 * vertex + call).  Calls: 0 -> (u_lobe, u_dir1, u_dir2, u_light_segment),
// 1 -> (u_light_triangle, u_light_a, u_light_b, -), vertex 0 call 2 ->
// (u_jitter_x, u_jitter_y, -, -).
struct PathRng {
  uint4 base;  // w holds nothing; set per draw
  uint2 key;
  __device__ __forceinline__ float4 draw(uint32_t vertex, uint32_t call) const {
    const uint4 o = philox4x32_10(make_uint4(base.x, base.y, base.z, vertex * 4u + call), key);
    return make_float4(to_unit(o.x), to_unit(o.y), to_unit(o.z), to_unit(o.w));
  }
};

// ---------------------------------------------------------------------------
// Scene layout in device memory.
//   nodes: 4 float4 per inner node of a binary BVH, both children's boxes in
//     the parent: (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y), (c1 same),
//     (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z), (child0, child1 as int bits).
//     child >= 0: inner node index; child < 0: leaf, v = -child - 1,
//     first triangle = v >> 3, count = (v & 7) + 1.
//   tris: 3 float4 per triangle in leaf order; p0.w = original triangle id,
//     p1.w = segment id (both as int bits).
//   vnrm: 3 float4 per triangle (vertex normals) or nullptr.
//   Light selection (static): seg_tris lists the triangles of each segment
//     (internal ids, by increasing original id), seg_begin[s]..seg_begin[s+1];
//     tri_cdf is the inclusive FP64 area prefix inside each segment.
// ---------------------------------------------------------------------------
struct SceneDev {
  const float4* nodes;
  const uint4* nodes4;  // 4-wide quantized nodes (4 x uint4 each), or nullptr
  const uint4* nodes8;  // 8-wide quantized nodes (6 x uint4 each), or nullptr
  const float4* tris;
  const float4* vnrm;
  const uint32_t* seg_tris;
  const uint32_t* seg_begin;
  const double* tri_cdf;
  const double* seg_area;
  uint32_t n_seg;
  uint32_t n_tri;
  float eps;  // spawn offset along the oriented geometric normal
  unsigned long long* counters;  // optional: closest rays, shadow rays, node visits, triangle tests
  int wide;   // 0: binary BVH, 1: 4-wide, 2: 8-wide quantized BVH
};

// kind 0: closest-hit ray, 1: shadow ray
__device__ __forceinline__ void count_ray(const SceneDev& s, int kind, uint32_t nodes, uint32_t tests) {
  if (s.counters) {
    atomicAdd(&s.counters[kind], 1ull);
    atomicAdd(&s.counters[2 + 2 * kind], (unsigned long long)nodes);
    atomicAdd(&s.counters[3 + 2 * kind], (unsigned long long)tests);
  }
}

// Per-segment tables derived from the parameters (rebuilt whenever the
// parameters change).  Evaluation uses params; sampling uses sampling params.
struct SegDev {
  const float4* mat_a;   // kd.rgb, roughness            (params)
  const float4* mat_b;   // ks.rgb, alpha = max(r^2,1e-4) (params)
  const float4* emis;    // emission_scale * e.rgb, -    (params)
  const float4* samp;    // alpha_s, P_spec (float), p_A = lum_s / W (float), -   (sampling)
  const double* pspec;   // P_spec in FP64 (lobe decision)
  const double* cdf;     // inclusive FP64 prefix of lum(e_s) A_s
  const double* W;       // total; 0 disables light sampling
};

// Disney material model tables (see ipt_disney.cuh); null pointers when a
// scene traces with Lambert + GGX.
struct DisneyDev {
  const float4* mat;    // 4 per segment: the 13 material values, then zeros
  const double2* lobe;  // cumulative lobe probabilities (P_d, P_d + P_s), FP64
  const float4* samp;   // 2 per segment: (a_x, a_y, a_c, 0), (P_d, P_s, P_c, 0)
};

struct ViewDev {
  float m[12];      // cam_to_world, row-major 3x4
  float tx, ty;     // tan(fov/2) * aspect, tan(fov/2)
  uint32_t w, h;
  uint32_t offset;  // global id of this view's first pixel
  uint32_t pad[3];
};

struct Hit {
  int tri;      // internal (leaf-order) id, -1 = miss
  float t, u, v;
};

// ---------------------------------------------------------------------------
// Watertight ray/triangle test: Woop, Benthin, Wald, "Watertight Ray/Triangle
// Intersection", JCGT 2(1), 2013.  The edge functions are evaluated without
// FMA contraction so that a shared edge gives the same value (up to sign) in
// both triangles; exact zeros are re-evaluated in FP64.
// ---------------------------------------------------------------------------
struct RayPre {
  float3 o, d, inv;
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ RayPre ray_pre(float3 o, float3 d) {
  RayPre r;
  r.o = o;
  r.d = d;
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  r.kx = r.kz + 1 == 3 ? 0 : r.kz + 1;
  r.ky = r.kx + 1 == 3 ? 0 : r.kx + 1;
  if (comp(d, r.kz) < 0.0f) {
    const int t = r.kx;
    r.kx = r.ky;
    r.ky = t;
  }
  const float dz = comp(d, r.kz);
  r.Sx = comp(d, r.kx) / dz;
  r.Sy = comp(d, r.ky) / dz;
  r.Sz = 1.0f / dz;
  const float tiny = 1e-30f;
  r.inv = f3(1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
             1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
             1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
  return r;
}

// Returns true and (t, u, v) on a hit with 0 < t < tmax.
__device__ __forceinline__ bool tri_test(const RayPre& r, float3 p0, float3 p1, float3 p2, float tmax,
                                         float& t_out, float& u_out, float& v_out) {
  const float3 A = p0 - r.o, B = p1 - r.o, C = p2 - r.o;
  const float Az0 = comp(A, r.kz), Bz0 = comp(B, r.kz), Cz0 = comp(C, r.kz);
  const float Ax = __fsub_rn(comp(A, r.kx), __fmul_rn(r.Sx, Az0));
  const float Ay = __fsub_rn(comp(A, r.ky), __fmul_rn(r.Sy, Az0));
  const float Bx = __fsub_rn(comp(B, r.kx), __fmul_rn(r.Sx, Bz0));
  const float By = __fsub_rn(comp(B, r.ky), __fmul_rn(r.Sy, Bz0));
  const float Cx = __fsub_rn(comp(C, r.kx), __fmul_rn(r.Sx, Cz0));
  const float Cy = __fsub_rn(comp(C, r.ky), __fmul_rn(r.Sy, Cz0));
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
  const float det = U + V + W;
  if (det == 0.0f) return false;
  const float T = U * (r.Sz * Az0) + V * (r.Sz * Bz0) + W * (r.Sz * Cz0);
  const float inv = 1.0f / det;
  const float t = T * inv;
  if (!(t > 0.0f) || !(t < tmax)) return false;
  t_out = t;
  u_out = V * inv;
  v_out = W * inv;
  return true;
}

__device__ __forceinline__ void decode_leaf(int child, int& first, int& count) {
  const int v = -child - 1;
  first = v >> 3;
  count = (v & 7) + 1;
}

// Slab test of both children; returns entry distances (or +inf on a miss).
__device__ __forceinline__ void box2(const RayPre& r, float3 oinv, float4 n0, float4 n1, float4 n2,
                                     float tmax, float& t0, float& t1) {
  const float far_scale = 1.0000005f;  // conservative far bound (a few ulps)
  const float a_lx = n0.x * r.inv.x - oinv.x, a_hx = n0.y * r.inv.x - oinv.x;
  const float a_ly = n0.z * r.inv.y - oinv.y, a_hy = n0.w * r.inv.y - oinv.y;
  const float a_lz = n2.x * r.inv.z - oinv.z, a_hz = n2.y * r.inv.z - oinv.z;
  const float b_lx = n1.x * r.inv.x - oinv.x, b_hx = n1.y * r.inv.x - oinv.x;
  const float b_ly = n1.z * r.inv.y - oinv.y, b_hy = n1.w * r.inv.y - oinv.y;
  const float b_lz = n2.z * r.inv.z - oinv.z, b_hz = n2.w * r.inv.z - oinv.z;
  const float an = fmaxf(fmaxf(fminf(a_lx, a_hx), fminf(a_ly, a_hy)), fmaxf(fminf(a_lz, a_hz), 0.0f));
  const float af = fminf(fminf(fmaxf(a_lx, a_hx), fmaxf(a_ly, a_hy)), fminf(fmaxf(a_lz, a_hz), tmax)) * far_scale;
  const float bn = fmaxf(fmaxf(fminf(b_lx, b_hx), fminf(b_ly, b_hy)), fmaxf(fminf(b_lz, b_hz), 0.0f));
  const float bf = fminf(fminf(fmaxf(b_lx, b_hx), fmaxf(b_ly, b_hy)), fminf(fmaxf(b_lz, b_hz), tmax)) * far_scale;
  t0 = an <= af ? an : __int_as_float(0x7f800000);
  t1 = bn <= bf ? bn : __int_as_float(0x7f800000);
}

// ---------------------------------------------------------------------------
// 4-wide node with 8-bit child boxes (see the scene builder): entry distances
// of its children (or +inf), and their links.
// ---------------------------------------------------------------------------

// Three-input minimum / maximum (one instruction on sm_100 and later; NaN
// operands are ignored as by fminf / fmaxf).
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// One 64-byte node as two 256-bit read-only loads (the node array is 64-byte
// aligned: cudaMalloc base, 64-byte records).
__device__ __forceinline__ void load_node4(const uint4* p, uint4& a, uint4& c, uint4& qa, uint4& qb) {
  asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(c.x), "=r"(c.y), "=r"(c.z), "=r"(c.w)
      : "l"(p));
  asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(qa.x), "=r"(qa.y), "=r"(qa.z), "=r"(qa.w), "=r"(qb.x), "=r"(qb.y), "=r"(qb.z), "=r"(qb.w)
      : "l"(p + 2));
}

// Byte i of w as the float 1 + byte * 2^-15 (the byte placed in mantissa
// bits 8-15 of 1.0; exact).
__device__ __forceinline__ float q_unit(uint32_t w, int i) {
  return __uint_as_float(__byte_perm(w, 0x3F800000u, 0x7604u | ((uint32_t)i << 4)));
}

// Slab test of the (up to) four children.
//  * Near / far planes: the plane distance t(q) = (origin + q * scale - o) / d
//    is monotonic in the byte q, so for each axis the near plane is the lower
//    byte when d >= 0 and the upper byte when d < 0: one select per axis and
//    node instead of a min/max per child and axis.
//  * One instruction per plane after the byte extraction: with
//    u = 1 + q * 2^-15 (q_unit), t(q) = u * A + B where A = 2^15 * scale / d and
//    B = (origin - o) / d - A, evaluated as one fma.  Rounding B, and the
//    margins below, add absolute errors of at most 2^-24 |A| each to a plane
//    distance of that axis (beyond the relative rounding the far-plane factor
//    1.0000005 covers).  A itself is a rounded product (the node stores
//    2^15 * scale as a float), but B carries the same A, so its rounding
//    enters t only through (u - 1) * A, u - 1 < 2^-7: below 2^-31 |A|.  Each axis's near planes therefore use B - 2^-22 |A|
//    and its far planes B + 2^-22 |A| (a widening of 2^-7 of a code on each
//    side, a few times the error bound): a child box is never missed because
//    of it.
__device__ __forceinline__ uint32_t node4_children(const SceneDev& s, int node, const RayPre& r, float tmax,
                                                   float tn[4], int ref[4]) {
  uint4 a, c, qa, qb;
  load_node4(&s.nodes4[4 * node], a, c, qa, qb);
  // 2^15 * scale of each axis, stored in words 3, 14 and 15
  const float sx = __uint_as_float(a.w), sy = __uint_as_float(qb.z), sz = __uint_as_float(qb.w);
  const float Ax = sx * r.inv.x, Bx = fmaf(__uint_as_float(a.x) - r.o.x, r.inv.x, -Ax);
  const float Ay = sy * r.inv.y, By = fmaf(__uint_as_float(a.y) - r.o.y, r.inv.y, -Ay);
  const float Az = sz * r.inv.z, Bz = fmaf(__uint_as_float(a.z) - r.o.z, r.inv.z, -Az);
  const float Bnx = fmaf(fabsf(Ax), -0x1p-22f, Bx), Bfx = fmaf(fabsf(Ax), 0x1p-22f, Bx);
  const float Bny = fmaf(fabsf(Ay), -0x1p-22f, By), Bfy = fmaf(fabsf(Ay), 0x1p-22f, By);
  const float Bnz = fmaf(fabsf(Az), -0x1p-22f, Bz), Bfz = fmaf(fabsf(Az), 0x1p-22f, Bz);
  const bool nx = r.inv.x < 0.0f, ny = r.inv.y < 0.0f, nz = r.inv.z < 0.0f;
  const uint32_t nwx = nx ? qa.y : qa.x, fwx = nx ? qa.x : qa.y;
  const uint32_t nwy = ny ? qa.w : qa.z, fwy = ny ? qa.z : qa.w;
  const uint32_t nwz = nz ? qb.y : qb.x, fwz = nz ? qb.x : qb.y;
  ref[0] = (int)c.x;
  ref[1] = (int)c.y;
  ref[2] = (int)c.z;
  ref[3] = (int)c.w;
  uint32_t mask = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float tnx = fmaf(q_unit(nwx, i), Ax, Bnx), tfx = fmaf(q_unit(fwx, i), Ax, Bfx);
    const float tny = fmaf(q_unit(nwy, i), Ay, Bny), tfy = fmaf(q_unit(fwy, i), Ay, Bfy);
    const float tnz = fmaf(q_unit(nwz, i), Az, Bnz), tfz = fmaf(q_unit(fwz, i), Az, Bfz);
    const float tnear = max3f(tnx, tny, fmaxf(tnz, 0.0f));
    const float tfar = min3f(tfx, tfy, fminf(tfz, tmax)) * 1.0000005f;
    const bool hit = tnear <= tfar;  // empty slots hold inverted boxes
    tn[i] = hit ? tnear : __int_as_float(0x7f800000);
    mask |= hit ? (1u << i) : 0u;
  }
  return mask;
}

// ---------------------------------------------------------------------------
// 8-wide node with 8-bit child boxes (96 bytes; the node test reads the first
// 64 with two 256-bit loads, the slots' links are read one at a time as the
// slots are entered).  Children sit in slots by octant (see the scene
// builder), so a ray visits the slots in the order of (slot ^ sgn), sgn the
// sign bits of its direction: no sort, and one stack entry per node (its
// remaining hit slots) instead of one per child.  Returns the mask of hit
// slots in visiting order (bit k: slot k ^ sgn); the plane arithmetic and
// its conservative margins are those of node4_children.
__device__ __forceinline__ uint32_t node8_hits(const SceneDev& s, int node, const RayPre& r, float tmax,
                                               uint32_t sgn) {
  uint4 a, b, c, d;
  load_node4(&s.nodes8[6 * node], a, b, c, d);  // words 0-7 (a, b) and 8-15 (c, d)
  const float sx = __uint_as_float(((a.w & 0xffu) + 15u) << 23);
  const float sy = __uint_as_float((((a.w >> 8) & 0xffu) + 15u) << 23);
  const float sz = __uint_as_float((((a.w >> 16) & 0xffu) + 15u) << 23);
  const uint32_t valid = a.w >> 24;
  const float Ax = sx * r.inv.x, Bx = fmaf(__uint_as_float(a.x) - r.o.x, r.inv.x, -Ax);
  const float Ay = sy * r.inv.y, By = fmaf(__uint_as_float(a.y) - r.o.y, r.inv.y, -Ay);
  const float Az = sz * r.inv.z, Bz = fmaf(__uint_as_float(a.z) - r.o.z, r.inv.z, -Az);
  const float Bnx = fmaf(fabsf(Ax), -0x1p-22f, Bx), Bfx = fmaf(fabsf(Ax), 0x1p-22f, Bx);
  const float Bny = fmaf(fabsf(Ay), -0x1p-22f, By), Bfy = fmaf(fabsf(Ay), 0x1p-22f, By);
  const float Bnz = fmaf(fabsf(Az), -0x1p-22f, Bz), Bfz = fmaf(fabsf(Az), 0x1p-22f, Bz);
  const bool nx = sgn & 1u, ny = sgn & 2u, nz = sgn & 4u;
  // near / far plane words of slots 0-3 (index 0) and 4-7 (index 1)
  const uint32_t nwx[2] = {nx ? b.z : b.x, nx ? b.w : b.y}, fwx[2] = {nx ? b.x : b.z, nx ? b.y : b.w};
  const uint32_t nwy[2] = {ny ? c.z : c.x, ny ? c.w : c.y}, fwy[2] = {ny ? c.x : c.z, ny ? c.y : c.w};
  const uint32_t nwz[2] = {nz ? d.z : d.x, nz ? d.w : d.y}, fwz[2] = {nz ? d.x : d.z, nz ? d.y : d.w};
  uint32_t mask = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int h = i >> 2, q = i & 3;
    const float tnx = fmaf(q_unit(nwx[h], q), Ax, Bnx), tfx = fmaf(q_unit(fwx[h], q), Ax, Bfx);
    const float tny = fmaf(q_unit(nwy[h], q), Ay, Bny), tfy = fmaf(q_unit(fwy[h], q), Ay, Bfy);
    const float tnz = fmaf(q_unit(nwz[h], q), Az, Bnz), tfz = fmaf(q_unit(fwz[h], q), Az, Bfz);
    const float tnear = max3f(tnx, tny, fmaxf(tnz, 0.0f));
    const float tfar = min3f(tfx, tfy, fminf(tfz, tmax)) * 1.0000005f;
    mask |= (tnear <= tfar ? 1u : 0u) << (i ^ (int)sgn);
  }
  // empty slots: their bit moves with the same permutation
  uint32_t vp = valid;
  if (sgn & 1u) vp = ((vp & 0x55u) << 1) | ((vp >> 1) & 0x55u);
  if (sgn & 2u) vp = ((vp & 0x33u) << 2) | ((vp >> 2) & 0x33u);
  if (sgn & 4u) vp = ((vp & 0x0fu) << 4) | ((vp >> 4) & 0x0fu);
  return mask & vp;
}

// Link of slot `slot` of 8-wide node `node`.
__device__ __forceinline__ int node8_link(const SceneDev& s, int node, int slot) {
  return (int)__ldg(reinterpret_cast<const uint32_t*>(&s.nodes8[6 * node]) + 16 + slot);
}

// Direction sign bits of a ray (bit k set: component k negative).
__device__ __forceinline__ uint32_t ray_sgn(const RayPre& r) {
  return (r.inv.x < 0.0f ? 1u : 0u) | (r.inv.y < 0.0f ? 2u : 0u) | (r.inv.z < 0.0f ? 4u : 0u);
}

// Sorts four (distance, link) pairs by distance (misses carry +inf).
__device__ __forceinline__ void sort4(float t[4], int r[4]) {
#define IPT_CSWAP(i, j)                 \
  if (t[j] < t[i]) {                    \
    const float tt = t[i];              \
    t[i] = t[j];                        \
    t[j] = tt;                          \
    const int rr = r[i];                \
    r[i] = r[j];                        \
    r[j] = rr;                          \
  }
  IPT_CSWAP(0, 1)
  IPT_CSWAP(2, 3)
  IPT_CSWAP(0, 2)
  IPT_CSWAP(1, 3)
  IPT_CSWAP(1, 2)
#undef IPT_CSWAP
}

// Closest hit in (0, tmax), skipping one internal triangle id; equal t keeps
// the smaller original id.  On stack overflow the ray reports a miss and the
// error word is set.
__device__ __forceinline__ Hit trace_closest2(const SceneDev& s, float3 o, float3 d, float tmax, int skip,
                                              uint32_t* err) {
  const RayPre r = ray_pre(o, d);
  const float3 oinv = f3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
  Hit h;
  h.tri = -1;
  h.t = tmax;
  h.u = h.v = 0.0f;
  int best_orig = 0x7fffffff;
  int stack[kStackSize];
  int sp = 0;
  int node = 0;
  uint32_t n_nodes = 0, n_tests = 0;
  for (;;) {
    if (node >= 0) {
      ++n_nodes;
      const float4 n0 = __ldg(&s.nodes[4 * node + 0]);
      const float4 n1 = __ldg(&s.nodes[4 * node + 1]);
      const float4 n2 = __ldg(&s.nodes[4 * node + 2]);
      const float4 n3 = __ldg(&s.nodes[4 * node + 3]);
      float t0, t1;
      box2(r, oinv, n0, n1, n2, h.t, t0, t1);
      const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      const bool h0 = t0 != __int_as_float(0x7f800000);
      const bool h1 = t1 != __int_as_float(0x7f800000);
      if (h0 && h1) {
        if (sp >= kStackSize) {
          atomicOr(err, kErrStack);
          h.tri = -1;
          return h;
        }
        if (t1 < t0) {
          stack[sp++] = c0;
          node = c1;
        } else {
          stack[sp++] = c1;
          node = c0;
        }
        continue;
      }
      if (h0 || h1) {
        node = h0 ? c0 : c1;
        continue;
      }
    } else {
      int first, count;
      decode_leaf(node, first, count);
      n_tests += count;
      for (int i = first; i < first + count; ++i) {
        if (i == skip) continue;
        const float4 q0 = __ldg(&s.tris[3 * i + 0]);
        const float4 q1 = __ldg(&s.tris[3 * i + 1]);
        const float4 q2 = __ldg(&s.tris[3 * i + 2]);
        float t, u, v;
        if (tri_test(r, xyz(q0), xyz(q1), xyz(q2), h.t * 1.0000002f, t, u, v)) {
          const int orig = __float_as_int(q0.w);
          if (t < h.t || (t == h.t && orig < best_orig)) {
            h.tri = i;
            h.t = t;
            h.u = u;
            h.v = v;
            best_orig = orig;
          }
        }
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  count_ray(s, 0, n_nodes, n_tests);
  return h;
}

// Any hit in (0, tmax), skipping two internal triangle ids.
__device__ __forceinline__ bool trace_any2(const SceneDev& s, float3 o, float3 d, float tmax, int skip_a,
                                           int skip_b, uint32_t* err) {
  const RayPre r = ray_pre(o, d);
  const float3 oinv = f3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
  int stack[kStackSize];
  int sp = 0;
  int node = 0;
  uint32_t n_nodes = 0, n_tests = 0;
  for (;;) {
    if (node >= 0) {
      ++n_nodes;
      const float4 n0 = __ldg(&s.nodes[4 * node + 0]);
      const float4 n1 = __ldg(&s.nodes[4 * node + 1]);
      const float4 n2 = __ldg(&s.nodes[4 * node + 2]);
      const float4 n3 = __ldg(&s.nodes[4 * node + 3]);
      float t0, t1;
      box2(r, oinv, n0, n1, n2, tmax, t0, t1);
      const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      const bool h0 = t0 != __int_as_float(0x7f800000);
      const bool h1 = t1 != __int_as_float(0x7f800000);
      if (h0 && h1) {
        if (sp >= kStackSize) {
          atomicOr(err, kErrStack);
          return true;
        }
        stack[sp++] = c1;
        node = c0;
        continue;
      }
      if (h0 || h1) {
        node = h0 ? c0 : c1;
        continue;
      }
    } else {
      int first, count;
      decode_leaf(node, first, count);
      n_tests += count;
      for (int i = first; i < first + count; ++i) {
        if (i == skip_a || i == skip_b) continue;
        const float4 q0 = __ldg(&s.tris[3 * i + 0]);
        const float4 q1 = __ldg(&s.tris[3 * i + 1]);
        const float4 q2 = __ldg(&s.tris[3 * i + 2]);
        float t, u, v;
        if (tri_test(r, xyz(q0), xyz(q1), xyz(q2), tmax, t, u, v)) {
          count_ray(s, 1, n_nodes, n_tests);
          return true;
        }
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  count_ray(s, 1, n_nodes, n_tests);
  return false;
}

// The same two queries over the 4-wide quantized BVH.
__device__ __forceinline__ Hit trace_closest4(const SceneDev& s, float3 o, float3 d, float tmax, int skip,
                                              uint32_t* err) {
  const RayPre r = ray_pre(o, d);
  Hit h;
  h.tri = -1;
  h.t = tmax;
  h.u = h.v = 0.0f;
  int best_orig = 0x7fffffff;
  int stack[kStackSize];
  float stack_t[kStackSize];
  int sp = 0;
  int node = 0;
  uint32_t n_nodes = 0, n_tests = 0;
  for (;;) {
    if (node >= 0) {
      ++n_nodes;
      float tn[4];
      int ref[4];
      const uint32_t mask = node4_children(s, node, r, h.t, tn, ref);
      const int k = __popc(mask);
      if (k > 0) {
        if (sp + k - 1 > kStackSize) {
          atomicOr(err, kErrStack);
          h.tri = -1;
          return h;
        }
        sort4(tn, ref);
#pragma unroll
        for (int i = 3; i >= 1; --i)
          if (i < k) {
            stack[sp] = ref[i];
            stack_t[sp] = tn[i];
            ++sp;
          }
        node = ref[0];
        continue;
      }
    } else {
      int first, count;
      decode_leaf(node, first, count);
      n_tests += count;
      for (int i = first; i < first + count; ++i) {
        if (i == skip) continue;
        const float4 q0 = __ldg(&s.tris[3 * i + 0]);
        const float4 q1 = __ldg(&s.tris[3 * i + 1]);
        const float4 q2 = __ldg(&s.tris[3 * i + 2]);
        float t, u, v;
        if (tri_test(r, xyz(q0), xyz(q1), xyz(q2), h.t * 1.0000002f, t, u, v)) {
          const int orig = __float_as_int(q0.w);
          if (t < h.t || (t == h.t && orig < best_orig)) {
            h.tri = i;
            h.t = t;
            h.u = u;
            h.v = v;
            best_orig = orig;
          }
        }
      }
    }
    bool done = false;
    for (;;) {
      if (sp == 0) {
        done = true;
        break;
      }
      --sp;
      if (stack_t[sp] <= h.t * 1.0000005f) break;
    }
    if (done) break;
    node = stack[sp];
  }
  count_ray(s, 0, n_nodes, n_tests);
  return h;
}

__device__ __forceinline__ bool trace_any4(const SceneDev& s, float3 o, float3 d, float tmax, int skip_a,
                                           int skip_b, uint32_t* err) {
  const RayPre r = ray_pre(o, d);
  int stack[kStackSize];
  int sp = 0;
  int node = 0;
  uint32_t n_nodes = 0, n_tests = 0;
  for (;;) {
    if (node >= 0) {
      ++n_nodes;
      float tn[4];
      int ref[4];
      const uint32_t mask = node4_children(s, node, r, tmax, tn, ref);
      const int k = __popc(mask);
      if (k > 0) {
        if (sp + k - 1 > kStackSize) {
          atomicOr(err, kErrStack);
          return true;
        }
        // nearest first: an occluder near the shading point ends the search sooner
        sort4(tn, ref);
#pragma unroll
        for (int i = 3; i >= 1; --i)
          if (i < k) stack[sp++] = ref[i];
        node = ref[0];
        continue;
      }
    } else {
      int first, count;
      decode_leaf(node, first, count);
      n_tests += count;
      for (int i = first; i < first + count; ++i) {
        if (i == skip_a || i == skip_b) continue;
        const float4 q0 = __ldg(&s.tris[3 * i + 0]);
        const float4 q1 = __ldg(&s.tris[3 * i + 1]);
        const float4 q2 = __ldg(&s.tris[3 * i + 2]);
        float t, u, v;
        if (tri_test(r, xyz(q0), xyz(q1), xyz(q2), tmax, t, u, v)) {
          count_ray(s, 1, n_nodes, n_tests);
          return true;
        }
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  count_ray(s, 1, n_nodes, n_tests);
  return false;
}

// The same two queries over the 8-wide quantized BVH: a stack entry is a
// node and the mask of its hit slots not yet entered (visiting order).
template <bool kAny>
__device__ __forceinline__ void trace8(const SceneDev& s, const RayPre& r, float tmax, int skip_a, int skip_b,
                                       Hit& h, bool& occluded, uint32_t* err) {
  const uint32_t sgn = ray_sgn(r);
  uint2 stack[kStackSize];
  int sp = 0;
  int best_orig = 0x7fffffff;
  int gnode = 0;
  uint32_t gmask = node8_hits(s, 0, r, tmax, sgn);
  uint32_t n_nodes = 1, n_tests = 0;
  for (;;) {
    while (gmask == 0) {
      if (sp == 0) {
        count_ray(s, kAny ? 1 : 0, n_nodes, n_tests);
        return;
      }
      --sp;
      gnode = (int)stack[sp].x;
      gmask = stack[sp].y;
    }
    const int k = __ffs(gmask) - 1;
    gmask &= gmask - 1u;
    const int ref = node8_link(s, gnode, k ^ (int)sgn);
    if (ref >= 0) {
      ++n_nodes;
      const uint32_t m = node8_hits(s, ref, r, kAny ? tmax : h.t, sgn);
      if (m) {
        if (gmask) {
          if (sp >= kStackSize) {
            atomicOr(err, kErrStack);
            h.tri = -1;
            occluded = true;
            return;
          }
          stack[sp++] = make_uint2((uint32_t)gnode, gmask);
        }
        gnode = ref;
        gmask = m;
      }
      continue;
    }
    int first, count;
    decode_leaf(ref, first, count);
    n_tests += count;
    for (int i = first; i < first + count; ++i) {
      if (i == skip_a || i == skip_b) continue;
      const float4 q0 = __ldg(&s.tris[3 * i + 0]);
      const float4 q1 = __ldg(&s.tris[3 * i + 1]);
      const float4 q2 = __ldg(&s.tris[3 * i + 2]);
      float t, u, v;
      if (kAny) {
        if (tri_test(r, xyz(q0), xyz(q1), xyz(q2), tmax, t, u, v)) {
          occluded = true;
          count_ray(s, 1, n_nodes, n_tests);
          return;
        }
      } else if (tri_test(r, xyz(q0), xyz(q1), xyz(q2), h.t * 1.0000002f, t, u, v)) {
        const int orig = __float_as_int(q0.w);
        if (t < h.t || (t == h.t && orig < best_orig)) {
          h.tri = i;
          h.t = t;
          h.u = u;
          h.v = v;
          best_orig = orig;
        }
      }
    }
  }
}

__device__ __forceinline__ Hit trace_closest8(const SceneDev& s, float3 o, float3 d, float tmax, int skip,
                                              uint32_t* err) {
  const RayPre r = ray_pre(o, d);
  Hit h;
  h.tri = -1;
  h.t = tmax;
  h.u = h.v = 0.0f;
  bool occ = false;
  trace8<false>(s, r, tmax, skip, -1, h, occ, err);
  return h;
}

__device__ __forceinline__ bool trace_any8(const SceneDev& s, float3 o, float3 d, float tmax, int skip_a,
                                           int skip_b, uint32_t* err) {
  const RayPre r = ray_pre(o, d);
  Hit h;
  h.tri = -1;
  h.t = tmax;
  h.u = h.v = 0.0f;
  bool occ = false;
  trace8<true>(s, r, tmax, skip_a, skip_b, h, occ, err);
  return occ;
}

__device__ __forceinline__ Hit trace_closest(const SceneDev& s, float3 o, float3 d, float tmax, int skip,
                                             uint32_t* err) {
  if (s.wide == 2) return trace_closest8(s, o, d, tmax, skip, err);
  return s.wide ? trace_closest4(s, o, d, tmax, skip, err) : trace_closest2(s, o, d, tmax, skip, err);
}

__device__ __forceinline__ bool trace_any(const SceneDev& s, float3 o, float3 d, float tmax, int skip_a,
                                          int skip_b, uint32_t* err) {
  if (s.wide == 2) return trace_any8(s, o, d, tmax, skip_a, skip_b, err);
  return s.wide ? trace_any4(s, o, d, tmax, skip_a, skip_b, err) : trace_any2(s, o, d, tmax, skip_a, skip_b, err);
}

// ---------------------------------------------------------------------------
// Material model: f_r = kd/pi + ks * D(h) G2 / (4 ci co), GGX D, height-
// correlated Smith G2, alpha = max(r^2, 1e-4), no Fresnel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ggx_D(float nh, float a) {
  if (!(nh > 0.0f)) return 0.0f;
  const float a2 = a * a;
  const float q = nh * nh * (a2 - 1.0f) + 1.0f;
  return a2 / (kPi * q * q);
}
__device__ __forceinline__ float ggx_dD_da(float nh, float a) {
  if (!(nh > 0.0f)) return 0.0f;
  const float a2 = a * a;
  const float q = nh * nh * (a2 - 1.0f) + 1.0f;
  return 2.0f * a / (kPi * q * q) * (1.0f - 2.0f * a2 * nh * nh / q);
}
__device__ __forceinline__ float smith_lambda(float c, float a) {
  const float c2 = c * c;
  const float t2 = (1.0f - c2) / c2;
  return 0.5f * (sqrtf(1.0f + a * a * t2) - 1.0f);
}
__device__ __forceinline__ float smith_dlambda_da(float c, float a) {
  const float c2 = c * c;
  const float t2 = (1.0f - c2) / c2;
  return 0.5f * a * t2 * rsqrtf(1.0f + a * a * t2);
}

struct Spec {
  float s;      // D G2 / (4 ci co)
  float ds_dr;  // d s / d roughness
};

// r: roughness (for d alpha / d r), a = max(r^2, 1e-4)
__device__ __forceinline__ Spec spec_term(float ci, float co, float nh, float r, float a) {
  const float D = ggx_D(nh, a);
  const float G2 = 1.0f / (1.0f + smith_lambda(ci, a) + smith_lambda(co, a));
  const float inv_den = 1.0f / (4.0f * ci * co);
  Spec sp;
  sp.s = D * G2 * inv_den;
  const float dG2 = -G2 * G2 * (smith_dlambda_da(ci, a) + smith_dlambda_da(co, a));
  const float dsda = (ggx_dD_da(nh, a) * G2 + D * dG2) * inv_den;
  sp.ds_dr = r * r > 1e-4f ? dsda * 2.0f * r : 0.0f;
  return sp;
}

// Orthonormal basis around unit n (Duff et al., JCGT 6(1), 2017).
__device__ __forceinline__ void onb(float3 n, float3& b1, float3& b2) {
  const float sign = copysignf(1.0f, n.z);
  const float a = -1.0f / (sign + n.z);
  const float b = n.x * n.y * a;
  b1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  b2 = f3(b, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float smith_G1(float c, float a) { return 1.0f / (1.0f + smith_lambda(c, a)); }

// Mixture pdf (solid angle) for sampling wo given wi; P = specular probability.
__device__ __forceinline__ float bsdf_pdf(float P, float a_s, float3 n, float3 wi, float3 wo) {
  const float ci = dot(n, wi), co = dot(n, wo);
  if (!(ci > 0.0f) || !(co > 0.0f)) return 0.0f;
  float ps = 0.0f;
  if (P > 0.0f) {
    const float3 h = normalize(wi + wo);
    ps = smith_G1(ci, a_s) * ggx_D(dot(n, h), a_s) / (4.0f * ci);
  }
  return (1.0f - P) * (co * (1.0f / kPi)) + P * ps;
}

// Lobe by u_lobe < P_spec (FP64 decision); diffuse: cosine-weighted
// (r = sqrt(u1), phi = 2 pi u2); specular: GGX visible normals (Heitz, JCGT
// 7(4), 2018) and a mirror reflection of wi.
__device__ __forceinline__ float3 bsdf_sample(double P, float a_s, float3 n, float3 wi, float u_lobe,
                                              float u1, float u2) {
  float3 b1, b2;
  onb(n, b1, b2);
  float sphi, cphi;
  sincospif(2.0f * u2, &sphi, &cphi);
  const float rr = sqrtf(u1);
  if ((double)u_lobe < P) {
    const float3 vl = f3(dot(wi, b1), dot(wi, b2), dot(wi, n));
    const float3 vh = normalize(f3(a_s * vl.x, a_s * vl.y, vl.z));
    const float lensq = vh.x * vh.x + vh.y * vh.y;
    const float3 t1 = lensq > 0.0f ? f3(-vh.y, vh.x, 0.0f) * rsqrtf(lensq) : f3(1.0f, 0.0f, 0.0f);
    const float3 t2 = cross(vh, t1);
    const float q1 = rr * cphi;
    float q2 = rr * sphi;
    const float s = 0.5f * (1.0f + vh.z);
    q2 = (1.0f - s) * sqrtf(fmaxf(0.0f, 1.0f - q1 * q1)) + s * q2;
    const float3 nh = t1 * q1 + t2 * q2 + vh * sqrtf(fmaxf(0.0f, 1.0f - q1 * q1 - q2 * q2));
    const float3 ne = normalize(f3(a_s * nh.x, a_s * nh.y, fmaxf(0.0f, nh.z)));
    const float3 hw = b1 * ne.x + b2 * ne.y + n * ne.z;
    return hw * (2.0f * dot(wi, hw)) - wi;
  }
  const float z = sqrtf(fmaxf(0.0f, 1.0f - u1));
  return b1 * (rr * cphi) + b2 * (rr * sphi) + n * z;
}

// First index i in [b, e) with x < a[i] (e - 1 if none); a non-decreasing.
__device__ __forceinline__ int upper_bound_d(const double* a, int b, int e, double x) {
  int lo = b, hi = e - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (x < __ldg(&a[mid]))
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

}  // namespace ipt
