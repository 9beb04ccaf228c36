// Learned radiance cache on BF16 tensor cores.
//
// Input of a row (80 values): the multiresolution hash-grid encoding of the
// position (Mueller et al. 2022: 16 levels x 2 features, 2^19 entries per
// level, resolutions 16..2048 spaced geometrically, trilinear interpolation
// of the 8 cell corners, dense indexing where a level's vertices fit the
// table, else the xor-of-primes spatial hash), real spherical harmonics of
// degrees 0..3 of the direction and of the normal (16 + 16), the terminal
// segment's kd, ks and roughness (7), zeros (9).  Network: 80 -> 64 -> 64 ->
// 64 -> 64 -> 16, ReLU on hidden layers, no biases; the first 3 outputs are
// the predicted reflected radiance.
//
// Each warp runs 16 rows through the network with mma.sync m16n8k16 (BF16
// operands, FP32 accumulation).  The encoded input tile is staged in shared
// memory; a layer's FP32 accumulator fragments are exactly the next layer's
// A fragments once packed to BF16, so hidden activations stay in registers,
// and the inference VJP needs only their ReLU masks (one register per layer).
// Inference blocks of 16 warps share one weight image (two blocks per SM).
// The backward pass loads the transposed weights with ldmatrix.trans from the
// same out-major image.  Training keeps the block's 64 rows of activations
// and pre-activation gradients in shared memory, so each warp then forms
// whole weight-gradient tiles over all 64 rows (K = rows) and accumulates
// them in a block-private FP32 copy, flushed once per launch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "ipt_cache.h"

namespace ipt {
namespace {

constexpr int kThreads = 128;   // 4 warps
constexpr int kTileRows = 64;   // rows of one block tile (16 per warp)
constexpr int kXs = 88;         // BF16 row stride of the input tile and W1t
constexpr int kHs = 72;         // hidden tiles, W2t..W5t
constexpr int kYs = 24;         // output-gradient tile
constexpr int kXw = kXs / 2, kHw = kHs / 2, kYw = kYs / 2;  // strides in 32-bit words

// BF16 weight image offsets (elements).
constexpr int kWt1 = 0, kWt2 = 64 * kXs, kWt3 = kWt2 + 64 * kHs, kWt4 = kWt3 + 64 * kHs, kWt5 = kWt4 + 64 * kHs;
// FP32 master weight offsets: W1 80 x 64, W2..W4 64 x 64, W5 64 x 16, in-major.
constexpr int kW1 = 0, kW2 = 80 * 64, kW3 = kW2 + 4096, kW4 = kW3 + 4096, kW5 = kW4 + 4096;

// Shared-memory layout (bytes, 16-byte aligned regions).
constexpr int kSmWt = 0;
constexpr int kSmX = kSmWt + (int)kCacheWtElems * 2;
constexpr int kSmMeta = kSmX + kTileRows * kXs * 2;
constexpr int kSmH = kSmMeta + kTileRows * 16;
constexpr int kSmDz = kSmH + 4 * kTileRows * kHs * 2;
constexpr int kSmDy = kSmDz + 4 * kTileRows * kHs * 2;
constexpr int kSmDw = kSmDy + kTileRows * kYs * 2;
constexpr int kSmEnd = kSmDw + (int)kCacheWeights * 4;
constexpr int kSmemTrain = kSmEnd;  // weights, tiles, activations, pre-activation gradients, dY, dW
static_assert(kSmX % 16 == 0 && kSmMeta % 16 == 0 && kSmH % 16 == 0 && kSmDz % 16 == 0 && kSmDy % 16 == 0 &&
                  kSmDw % 16 == 0,
              "shared regions must be 16-byte aligned");
static_assert(kSmemTrain <= 227 * 1024, "training tile exceeds shared memory");

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float2 unpack2(uint32_t w) {
  const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&w);
  return __bfloat1622float2(v);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four transposed 8x8 BF16 matrices; lane l gives the row address of matrix
// l / 8, row l % 8.
__device__ __forceinline__ void ldsm4t(uint32_t r[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Real spherical harmonics of degrees 0..3 of a unit vector.
__device__ __forceinline__ void sh16(float3 d, float o[16]) {
  const float x = d.x, y = d.y, z = d.z;
  const float xx = x * x, yy = y * y, zz = z * z;
  o[0] = 0.28209479177387814f;
  o[1] = -0.4886025119029199f * y;
  o[2] = 0.4886025119029199f * z;
  o[3] = -0.4886025119029199f * x;
  o[4] = 1.0925484305920792f * x * y;
  o[5] = -1.0925484305920792f * y * z;
  o[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
  o[7] = -1.0925484305920792f * x * z;
  o[8] = 0.5462742152960396f * (xx - yy);
  o[9] = -0.5900435899266435f * y * (3.0f * xx - yy);
  o[10] = 2.890611442640554f * x * y * z;
  o[11] = -0.4570457994644658f * y * (5.0f * zz - 1.0f);
  o[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
  o[13] = -0.4570457994644658f * x * (5.0f * zz - 1.0f);
  o[14] = 1.445305721320277f * z * (xx - yy);
  o[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
}

// Table indices and trilinear weights of the 8 corners of level l's cell.
// res: the levels' resolutions, staged in shared memory (dynamic index).
__device__ __forceinline__ void level_corners(const int* res, uint32_t dense_mask, int l, float3 x, uint32_t idx[8],
                                              float w[8]) {
  const int n = res[l];
  const float px = x.x * (float)n, py = x.y * (float)n, pz = x.z * (float)n;
  const float gx = floorf(px), gy = floorf(py), gz = floorf(pz);
  const int ix = (int)gx, iy = (int)gy, iz = (int)gz;
  const float fx = px - gx, fy = py - gy, fz = pz - gz;
  const bool dense = (dense_mask >> l) & 1u;
  const uint32_t s1 = (uint32_t)n + 1u;
  const uint32_t base = (uint32_t)l * kCacheT;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t cx = (uint32_t)min(ix + (c & 1), n);
    const uint32_t cy = (uint32_t)min(iy + ((c >> 1) & 1), n);
    const uint32_t cz = (uint32_t)min(iz + ((c >> 2) & 1), n);
    w[c] = ((c & 1) ? fx : 1.0f - fx) * ((c & 2) ? fy : 1.0f - fy) * ((c & 4) ? fz : 1.0f - fz);
    const uint32_t h = dense ? cx + cy * s1 + cz * s1 * s1 : (cx ^ (cy * 2654435761u) ^ (cz * 805459861u));
    idx[c] = base + (h & (kCacheT - 1u));
  }
}

__device__ __forceinline__ float3 unit_pos(const CacheNet& net, float4 x) {
  return make_float3(fminf(fmaxf((x.x - net.lo.x) * net.inv_ext.x, 0.0f), 1.0f),
                     fminf(fmaxf((x.y - net.lo.y) * net.inv_ext.y, 0.0f), 1.0f),
                     fminf(fmaxf((x.z - net.lo.z) * net.inv_ext.z, 0.0f), 1.0f));
}

// Encodes rows [r0, r0 + 16) (valid below `end`) into the warp's input tile
// X (16 x kXs BF16) and its row metadata (unit position, valid flag).
__device__ __forceinline__ void encode_rows(const CacheNet& net, const int* res, const CacheRows& rows, const float4* mat_a,
                            const float4* mat_b, uint32_t r0, uint32_t end, uint32_t* X, float4* meta, int lane) {
  const int row = lane & 15;
  const uint32_t r = r0 + (uint32_t)row;
  const bool valid = r < end;
  uint32_t* xr = X + row * kXw;
  if (lane < 16) {
    const float4 xq = valid ? rows.x[r] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float3 p = unit_pos(net, xq);
    meta[row] = make_float4(p.x, p.y, p.z, valid ? 1.0f : 0.0f);
    float4 ma = make_float4(0.f, 0.f, 0.f, 0.f), mb = ma;
    if (valid) {
      const int seg = __float_as_int(xq.w);
      ma = __ldg(&mat_a[seg]);
      mb = __ldg(&mat_b[seg]);
    }
    xr[32] = pack2(ma.x, ma.y);  // kd r, g
    xr[33] = pack2(ma.z, mb.x);  // kd b, ks r
    xr[34] = pack2(mb.y, mb.z);  // ks g, b
    xr[35] = pack2(ma.w, 0.0f);  // roughness
#pragma unroll
    for (int i = 36; i < 40; ++i) xr[i] = 0u;
  }
  {
    float3 dir = make_float3(0.f, 0.f, 1.f);
    if (valid) {
      const float4 v = lane < 16 ? rows.d[r] : rows.n[r];
      dir = make_float3(v.x, v.y, v.z);
    }
    float sh[16];
    sh16(dir, sh);
    const int w0 = lane < 16 ? 16 : 24;  // columns 32.. and 48..
#pragma unroll
    for (int i = 0; i < 8; ++i) xr[w0 + i] = valid ? pack2(sh[2 * i], sh[2 * i + 1]) : 0u;
  }
  __syncwarp();
#pragma unroll 1
  for (int i = 0; i < 8; ++i) {
    const int item = lane + 32 * i;
    const int rr = item & 15, l = item >> 4;
    const float4 m = meta[rr];
    uint32_t word = 0u;
    if (m.w != 0.0f) {
      uint32_t idx[8];
      float w[8];
      level_corners(res, net.dense, l, make_float3(m.x, m.y, m.z), idx, w);
      float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float2 v = __ldg(&net.table[idx[c]]);
        f0 += w[c] * v.x;
        f1 += w[c] * v.y;
      }
      word = pack2(f0, f1);
    }
    X[rr * kXw + l] = word;
  }
  __syncwarp();
}

// One forward layer: c[NT] = a[KT] x W (W out-major with row stride S words*2).
template <int KT, int NT, int SW>
__device__ __forceinline__ void layer_fwd(const uint32_t* Wt, const uint32_t (&a)[KT][4], float (&c)[NT][4],
                                          int g, int t) {
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      const uint32_t* p = Wt + (8 * j + g) * SW + 8 * kk + t;
      mma16816(c[j], a[kk], p[0], p[4]);
    }
  }
}

// ReLU, BF16 A fragments of the next layer, and (optionally) the activation
// tile H (warp rows, row stride kHw words).
template <bool kStore>
__device__ __forceinline__ void relu_pack(const float (&c)[8][4], uint32_t (&a)[4][4], uint32_t* H, int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t lo = pack2(fmaxf(c[j][0], 0.0f), fmaxf(c[j][1], 0.0f));
    const uint32_t hi = pack2(fmaxf(c[j][2], 0.0f), fmaxf(c[j][3], 0.0f));
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    if (kStore) {
      H[g * kHw + 4 * j + t] = lo;
      H[(g + 8) * kHw + 4 * j + t] = hi;
    }
  }
}

// Forward pass of the warp's 16 rows from its input tile; hidden
// activations of layer i go to H + i * hstride when kStore.
template <bool kStore>
__device__ __forceinline__ void net_forward(const uint32_t* Wt, const uint32_t* X, uint32_t* H, int hstride,
                                            float (&y)[2][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  float c[8][4];
  uint32_t h[4][4];
  {
    uint32_t a[5][4];
#pragma unroll
    for (int kk = 0; kk < 5; ++kk) {
      a[kk][0] = X[g * kXw + 8 * kk + t];
      a[kk][1] = X[(g + 8) * kXw + 8 * kk + t];
      a[kk][2] = X[g * kXw + 8 * kk + 4 + t];
      a[kk][3] = X[(g + 8) * kXw + 8 * kk + 4 + t];
    }
    layer_fwd<5, 8, kXw>(Wt + kWt1 / 2, a, c, g, t);
  }
  relu_pack<kStore>(c, h, H, g, t);
  layer_fwd<4, 8, kHw>(Wt + kWt2 / 2, h, c, g, t);
  relu_pack<kStore>(c, h, H + hstride, g, t);
  layer_fwd<4, 8, kHw>(Wt + kWt3 / 2, h, c, g, t);
  relu_pack<kStore>(c, h, H + 2 * hstride, g, t);
  layer_fwd<4, 8, kHw>(Wt + kWt4 / 2, h, c, g, t);
  relu_pack<kStore>(c, h, H + 3 * hstride, g, t);
  layer_fwd<4, 2, kHw>(Wt + kWt5 / 2, h, y, g, t);
}

// One backward layer: c (n-tile pairs [JP0, JP1) over the layer's inputs) =
// a (gradient at the layer's outputs, KT k-tiles) x W^T, with W^T loaded by
// ldmatrix.trans from the out-major BF16 image (row stride S elements).
template <int KT, int JP0, int JP1, int S>
__device__ __forceinline__ void layer_bwd(const __nv_bfloat16* Wt, const uint32_t (&a)[KT][4],
                                          float (&c)[2 * (JP1 - JP0)][4], int lane) {
  const int m = lane >> 3, r = lane & 7;
#pragma unroll
  for (int jp = JP0; jp < JP1; ++jp) {
    float* c0 = c[2 * (jp - JP0)];
    float* c1 = c[2 * (jp - JP0) + 1];
    c0[0] = c0[1] = c0[2] = c0[3] = 0.0f;
    c1[0] = c1[1] = c1[2] = c1[3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      uint32_t b[4];
      ldsm4t(b, Wt + (16 * kk + r + 8 * (m & 1)) * S + 16 * jp + 8 * (m >> 1));
      mma16816(c0, a[kk], b[0], b[1]);
      mma16816(c1, a[kk], b[2], b[3]);
    }
  }
}

// dZ = dH * (H > 0) at the fragment positions, packed to A fragments and
// (optionally) stored as a BF16 tile.
template <bool kStore>
__device__ __forceinline__ void relu_grad(const float (&dh)[8][4], const uint32_t* H, uint32_t (&a)[4][4],
                                          uint32_t* Dz, int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float2 h0 = unpack2(H[g * kHw + 4 * j + t]);
    const float2 h1 = unpack2(H[(g + 8) * kHw + 4 * j + t]);
    const uint32_t lo = pack2(h0.x > 0.0f ? dh[j][0] : 0.0f, h0.y > 0.0f ? dh[j][1] : 0.0f);
    const uint32_t hi = pack2(h1.x > 0.0f ? dh[j][2] : 0.0f, h1.y > 0.0f ? dh[j][3] : 0.0f);
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    if (kStore) {
      Dz[g * kHw + 4 * j + t] = lo;
      Dz[(g + 8) * kHw + 4 * j + t] = hi;
    }
  }
}

// ReLU masks of a hidden layer in one register per lane: bit 4j + k is the
// fragment element k of n-tile j (k = 0, 1: row g; k = 2, 3: row g + 8) and
// is set where the BF16 activation is positive.  The input VJP needs only
// these masks, so inference keeps no activation tile in shared memory.
__device__ __forceinline__ uint32_t relu_pack_mask(const float (&c)[8][4], uint32_t (&a)[4][4]) {
  uint32_t mask = 0u;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t lo = pack2(fmaxf(c[j][0], 0.0f), fmaxf(c[j][1], 0.0f));
    const uint32_t hi = pack2(fmaxf(c[j][2], 0.0f), fmaxf(c[j][3], 0.0f));
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    mask |= ((lo & 0x7FFFu) ? 1u : 0u) << (4 * j);
    mask |= ((lo & 0x7FFF0000u) ? 1u : 0u) << (4 * j + 1);
    mask |= ((hi & 0x7FFFu) ? 1u : 0u) << (4 * j + 2);
    mask |= ((hi & 0x7FFF0000u) ? 1u : 0u) << (4 * j + 3);
  }
  return mask;
}

__device__ __forceinline__ void relu_grad_mask(const float (&dh)[8][4], uint32_t mask, uint32_t (&a)[4][4]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t m = mask >> (4 * j);
    a[j >> 1][(j & 1) * 2 + 0] = pack2((m & 1u) ? dh[j][0] : 0.0f, (m & 2u) ? dh[j][1] : 0.0f);
    a[j >> 1][(j & 1) * 2 + 1] = pack2((m & 4u) ? dh[j][2] : 0.0f, (m & 8u) ? dh[j][3] : 0.0f);
  }
}

// Forward pass keeping the hidden layers' ReLU masks (mask[i]: layer i + 1).
__device__ __forceinline__ void net_forward_mask(const uint32_t* Wt, const uint32_t* X, float (&y)[2][4],
                                                 uint32_t (&mask)[4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  float c[8][4];
  uint32_t h[4][4];
  {
    uint32_t a[5][4];
#pragma unroll
    for (int kk = 0; kk < 5; ++kk) {
      a[kk][0] = X[g * kXw + 8 * kk + t];
      a[kk][1] = X[(g + 8) * kXw + 8 * kk + t];
      a[kk][2] = X[g * kXw + 8 * kk + 4 + t];
      a[kk][3] = X[(g + 8) * kXw + 8 * kk + 4 + t];
    }
    layer_fwd<5, 8, kXw>(Wt + kWt1 / 2, a, c, g, t);
  }
  mask[0] = relu_pack_mask(c, h);
  layer_fwd<4, 8, kHw>(Wt + kWt2 / 2, h, c, g, t);
  mask[1] = relu_pack_mask(c, h);
  layer_fwd<4, 8, kHw>(Wt + kWt3 / 2, h, c, g, t);
  mask[2] = relu_pack_mask(c, h);
  layer_fwd<4, 8, kHw>(Wt + kWt4 / 2, h, c, g, t);
  mask[3] = relu_pack_mask(c, h);
  layer_fwd<4, 2, kHw>(Wt + kWt5 / 2, h, y, g, t);
}

// Input VJP from the masks: gradient fragments of n-tile pairs [JP0, JP1)
// of the 80 inputs.
template <int JP0, int JP1>
__device__ __forceinline__ void net_backward_mask(const __nv_bfloat16* Wtb, const uint32_t (&mask)[4],
                                                  const float (&dy)[2][4], float (&dx)[2 * (JP1 - JP0)][4],
                                                  int lane) {
  uint32_t ay[1][4];
  ay[0][0] = pack2(dy[0][0], dy[0][1]);
  ay[0][1] = pack2(dy[0][2], dy[0][3]);
  ay[0][2] = pack2(dy[1][0], dy[1][1]);
  ay[0][3] = pack2(dy[1][2], dy[1][3]);
  float dh[8][4];
  uint32_t a[4][4];
  layer_bwd<1, 0, 4, kHs>(Wtb + kWt5, ay, dh, lane);
  relu_grad_mask(dh, mask[3], a);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt4, a, dh, lane);
  relu_grad_mask(dh, mask[2], a);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt3, a, dh, lane);
  relu_grad_mask(dh, mask[1], a);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt2, a, dh, lane);
  relu_grad_mask(dh, mask[0], a);
  layer_bwd<4, JP0, JP1, kXs>(Wtb + kWt1, a, dx, lane);
}

// Backward pass of the warp's rows from dL/dy down to the inputs: returns the
// input-gradient fragments of n-tile pairs [JP0, JP1) of the 80 inputs.
// Pre-activation gradients (and dY) are stored when kStore.
template <bool kStore, int JP0, int JP1>
__device__ __forceinline__ void net_backward(const __nv_bfloat16* Wtb, const uint32_t* H, int hstride,
                                             uint32_t* Dz, uint32_t* Dy, const float (&dy)[2][4],
                                             float (&dx)[2 * (JP1 - JP0)][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  uint32_t ay[1][4];
  ay[0][0] = pack2(dy[0][0], dy[0][1]);
  ay[0][1] = pack2(dy[0][2], dy[0][3]);
  ay[0][2] = pack2(dy[1][0], dy[1][1]);
  ay[0][3] = pack2(dy[1][2], dy[1][3]);
  if (kStore) {
    Dy[g * kYw + t] = ay[0][0];
    Dy[(g + 8) * kYw + t] = ay[0][1];
    Dy[g * kYw + 4 + t] = ay[0][2];
    Dy[(g + 8) * kYw + 4 + t] = ay[0][3];
  }
  float dh[8][4];
  uint32_t a[4][4];
  layer_bwd<1, 0, 4, kHs>(Wtb + kWt5, ay, dh, lane);
  relu_grad<kStore>(dh, H + 3 * hstride, a, Dz + 3 * hstride, g, t);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt4, a, dh, lane);
  relu_grad<kStore>(dh, H + 2 * hstride, a, Dz + 2 * hstride, g, t);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt3, a, dh, lane);
  relu_grad<kStore>(dh, H + hstride, a, Dz + hstride, g, t);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt2, a, dh, lane);
  relu_grad<kStore>(dh, H, a, Dz, g, t);
  layer_bwd<4, JP0, JP1, kXs>(Wtb + kWt1, a, dx, lane);
}

__device__ __forceinline__ void load_weights(const CacheNet& net, unsigned char* sm, int* res) {
  uint4* dst = reinterpret_cast<uint4*>(sm + kSmWt);
  for (uint32_t i = threadIdx.x; i < kCacheWtElems / 8; i += blockDim.x) dst[i] = __ldg(&net.wt[i]);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int l = 0; l < kCacheLevels; ++l) res[l] = net.res[l];
  }
}

// Inference (and input VJP) over warp tiles of 16 rows; W warps share one
// shared-memory weight image.  The VJP keeps the hidden layers' ReLU masks in
// registers, so a block holds only the weights and its warps' input tiles.
constexpr int kInferWarps = 16;
template <int W>
constexpr int infer_smem() {
  return kSmX + W * 16 * kXs * 2 + W * 16 * 16;
}
static_assert(kSmX % 16 == 0 && (kSmX + kInferWarps * 16 * kXs * 2) % 16 == 0, "infer tiles must be aligned");

template <bool kVjp, int W>
__global__ void __launch_bounds__(W * 32, 2) cache_infer_k(CacheNet net, CacheRows rows, const float4* mat_a,
                                                           const float4* mat_b, const uint32_t* count_dev,
                                                           uint32_t n_max, CacheOut o) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int res[kCacheLevels];
  load_weights(net, sm, res);
  __syncthreads();
  const uint32_t n = count_dev ? min(*count_dev, n_max) : n_max;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const uint32_t* Wt = reinterpret_cast<const uint32_t*>(sm + kSmWt);
  const __nv_bfloat16* Wtb = reinterpret_cast<const __nv_bfloat16*>(sm + kSmWt);
  uint32_t* X = reinterpret_cast<uint32_t*>(sm + kSmX) + warp * 16 * kXw;
  float4* meta = reinterpret_cast<float4*>(sm + kSmX + W * 16 * kXs * 2) + warp * 16;
  const uint32_t n_tiles = (n + 15u) / 16u;
  for (uint32_t tile = blockIdx.x * (uint32_t)W + (uint32_t)warp; tile < n_tiles; tile += gridDim.x * (uint32_t)W) {
    const uint32_t r0 = tile * 16u;
    __syncwarp();
    encode_rows(net, res, rows, mat_a, mat_b, r0, n, X, meta, lane);
    float y[2][4];
    uint32_t mask[4];
    net_forward_mask(Wt, X, y, mask, lane);
    // rows g and g + 8: lane t = 0 holds outputs 0, 1 and takes 2 from lane t = 1
    const float y2a = __shfl_down_sync(0xffffffffu, y[0][0], 1);
    const float y2b = __shfl_down_sync(0xffffffffu, y[0][2], 1);
    const uint32_t ra = r0 + (uint32_t)g, rb = ra + 8u;
    if (t == 0) {
      if (ra < n) {
        const float3 C = make_float3(y[0][0], y[0][1], y2a);
        if (o.c) o.c[ra] = make_float4(C.x, C.y, C.z, 0.0f);
        if (o.rad) {
          const float4 b = rows.u[ra];
          float4* dst = &o.rad[__float_as_uint(rows.d[ra].w)];
          const float4 v = *dst;
          *dst = make_float4(v.x + b.x * C.x, v.y + b.y * C.y, v.z + b.z * C.z, v.w);
        }
      }
      if (rb < n) {
        const float3 C = make_float3(y[0][2], y[0][3], y2b);
        if (o.c) o.c[rb] = make_float4(C.x, C.y, C.z, 0.0f);
        if (o.rad) {
          const float4 b = rows.u[rb];
          float4* dst = &o.rad[__float_as_uint(rows.d[rb].w)];
          const float4 v = *dst;
          *dst = make_float4(v.x + b.x * C.x, v.y + b.y * C.y, v.z + b.z * C.z, v.w);
        }
      }
    }
    if (kVjp) {
      // upstream u on outputs 0..2: lane t = 0 takes (u.x, u.y), t = 1 (u.z, 0)
      float dy[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      if (t < 2) {
        if (ra < n) {
          const float4 u = rows.u[ra];
          dy[0][0] = t == 0 ? u.x : u.z;
          dy[0][1] = t == 0 ? u.y : 0.0f;
        }
        if (rb < n) {
          const float4 u = rows.u[rb];
          dy[0][2] = t == 0 ? u.x : u.z;
          dy[0][3] = t == 0 ? u.y : 0.0f;
        }
      }
      float dx[2][4];
      net_backward_mask<4, 5>(Wtb, mask, dy, dx, lane);
      // n-tile 8 = inputs 64..71: kd rgb, ks rgb, roughness, pad
      if (o.dp) {
        if (ra < n) *reinterpret_cast<float2*>(&o.dp[8 * (size_t)ra + 2 * t]) = make_float2(dx[0][0], dx[0][1]);
        if (rb < n) *reinterpret_cast<float2*>(&o.dp[8 * (size_t)rb + 2 * t]) = make_float2(dx[0][2], dx[0][3]);
      }
    }
  }
}

// Training gradients over block tiles of 64 rows of one minibatch.
__global__ void __launch_bounds__(kThreads) cache_grad_k(CacheNet net, CacheRows rows, const float4* mat_a,
                                                         const float4* mat_b, const uint32_t* count_dev,
                                                         uint32_t n_max, uint32_t batch, uint32_t n_batches,
                                                         CacheOut o) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int res[kCacheLevels];
  load_weights(net, sm, res);
  float* dW = reinterpret_cast<float*>(sm + kSmDw);
  for (uint32_t i = threadIdx.x; i < kCacheWeights; i += blockDim.x) dW[i] = 0.0f;
  __syncthreads();
  const uint32_t n = count_dev ? min(*count_dev, n_max) : n_max;
  const uint32_t per = (n + n_batches - 1u) / n_batches;
  const uint32_t begin = min(batch * per, n), end = min(begin + per, n);
  const uint32_t rows_n = end - begin;
  const float scale = rows_n ? 1.0f / (3.0f * (float)rows_n) : 0.0f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const uint32_t* Wt = reinterpret_cast<const uint32_t*>(sm + kSmWt);
  const __nv_bfloat16* Wtb = reinterpret_cast<const __nv_bfloat16*>(sm + kSmWt);
  uint32_t* X = reinterpret_cast<uint32_t*>(sm + kSmX) + warp * 16 * kXw;
  float4* meta = reinterpret_cast<float4*>(sm + kSmMeta) + warp * 16;
  uint32_t* H = reinterpret_cast<uint32_t*>(sm + kSmH) + warp * 16 * kHw;
  uint32_t* Dz = reinterpret_cast<uint32_t*>(sm + kSmDz) + warp * 16 * kHw;
  uint32_t* Dy = reinterpret_cast<uint32_t*>(sm + kSmDy) + warp * 16 * kYw;
  const int hstride = kTileRows * kHw;
  double loss = 0.0;
  const uint32_t n_tiles = (rows_n + kTileRows - 1u) / kTileRows;
  for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint32_t r0 = begin + tile * kTileRows + 16u * (uint32_t)warp;
    encode_rows(net, res, rows, mat_a, mat_b, r0, end, X, meta, lane);
    float y[2][4];
    net_forward<true>(Wt, X, H, hstride, y, lane);
    // relative L2: d/dy_c of (y_c - t_c)^2 / (sg(y_c)^2 + 0.01), mean over rows and channels
    const float y2a = __shfl_down_sync(0xffffffffu, y[0][0], 1);
    const float y2b = __shfl_down_sync(0xffffffffu, y[0][2], 1);
    const uint32_t ra = r0 + (uint32_t)g, rb = ra + 8u;
    float da[3] = {0.f, 0.f, 0.f}, db[3] = {0.f, 0.f, 0.f};
    if (t == 0) {
      if (ra < end) {
        const float4 tg = rows.u[ra];
        const float yy[3] = {y[0][0], y[0][1], y2a}, tt[3] = {tg.x, tg.y, tg.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float den = yy[c] * yy[c] + 0.01f, r = yy[c] - tt[c];
          loss += (double)(r * r / den);
          da[c] = 2.0f * r / den * scale;
        }
      }
      if (rb < end) {
        const float4 tg = rows.u[rb];
        const float yy[3] = {y[0][2], y[0][3], y2b}, tt[3] = {tg.x, tg.y, tg.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float den = yy[c] * yy[c] + 0.01f, r = yy[c] - tt[c];
          loss += (double)(r * r / den);
          db[c] = 2.0f * r / den * scale;
        }
      }
    }
    const float d2a = __shfl_up_sync(0xffffffffu, da[2], 1);
    const float d2b = __shfl_up_sync(0xffffffffu, db[2], 1);
    float dy[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    if (t == 0) {
      dy[0][0] = da[0];
      dy[0][1] = da[1];
      dy[0][2] = db[0];
      dy[0][3] = db[1];
    } else if (t == 1) {
      dy[0][0] = d2a;
      dy[0][2] = d2b;
    }
    float dx[4][4];
    net_backward<true, 0, 2>(Wtb, H, hstride, Dz, Dy, dy, dx, lane);
    // hash-table gradient: n-tile j holds level 4j + t (features 0, 1)
    if (o.gt) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int l = 4 * j + t;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float4 m = meta[g + 8 * h];
          if (m.w == 0.0f) continue;
          uint32_t idx[8];
          float w[8];
          level_corners(res, net.dense, l, make_float3(m.x, m.y, m.z), idx, w);
          const float d0 = dx[j][2 * h], d1 = dx[j][2 * h + 1];
#pragma unroll
          for (int c = 0; c < 8; ++c) atomicAdd(&o.gt[idx[c]], make_float2(w[c] * d0, w[c] * d1));
        }
      }
    }
    __syncthreads();
    // weight gradients over the block's 64 rows: 72 units of (layer, 16 inputs, 16 outputs)
    for (int u = warp; u < 72; u += 4) {
      const __nv_bfloat16 *A, *B;
      int sa, sb, mt, np, ostride, off;
      if (u < 20) {
        A = reinterpret_cast<const __nv_bfloat16*>(sm + kSmX);
        sa = kXs;
        B = reinterpret_cast<const __nv_bfloat16*>(sm + kSmDz);
        sb = kHs;
        mt = u >> 2;
        np = u & 3;
        ostride = 64;
        off = kW1;
      } else if (u < 68) {
        const int L = (u - 20) >> 4;  // 0..2: dW2..dW4
        A = reinterpret_cast<const __nv_bfloat16*>(sm + kSmH) + L * kTileRows * kHs;
        sa = kHs;
        B = reinterpret_cast<const __nv_bfloat16*>(sm + kSmDz) + (L + 1) * kTileRows * kHs;
        sb = kHs;
        mt = ((u - 20) & 15) >> 2;
        np = (u - 20) & 3;
        ostride = 64;
        off = kW2 + L * 4096;
      } else {
        A = reinterpret_cast<const __nv_bfloat16*>(sm + kSmH) + 3 * kTileRows * kHs;
        sa = kHs;
        B = reinterpret_cast<const __nv_bfloat16*>(sm + kSmDy);
        sb = kYs;
        mt = u - 68;
        np = 0;
        ostride = 16;
        off = kW5;
      }
      const int m = lane >> 3, r = lane & 7;
      float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        uint32_t a[4], b[4];
        ldsm4t(a, A + (16 * ks + r + 8 * (m >> 1)) * sa + 16 * mt + 8 * (m & 1));
        ldsm4t(b, B + (16 * ks + r + 8 * (m & 1)) * sb + 16 * np + 8 * (m >> 1));
        mma16816(acc[0], a, b[0], b[1]);
        mma16816(acc[1], a, b[2], b[3]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = 16 * np + 8 * h + 2 * t;
        float2* p0 = reinterpret_cast<float2*>(&dW[off + (16 * mt + g) * ostride + col]);
        float2* p1 = reinterpret_cast<float2*>(&dW[off + (16 * mt + g + 8) * ostride + col]);
        const float2 v0 = *p0, v1 = *p1;
        *p0 = make_float2(v0.x + acc[h][0], v0.y + acc[h][1]);
        *p1 = make_float2(v1.x + acc[h][2], v1.y + acc[h][3]);
      }
    }
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < kCacheWeights; i += blockDim.x) {
    const float v = dW[i];
    if (v != 0.0f) atomicAdd(&o.gw[i], v);
  }
  if (o.loss) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, s);
    if (lane == 0 && loss != 0.0) atomicAdd(o.loss, loss);
  }
}

// Position of FP32 master weight i in the BF16 image (out-major rows).
__device__ __forceinline__ int image_index(int i) {
  if (i < kW2) return kWt1 + (i % 64) * kXs + i / 64;
  if (i < kW5) {
    const int L = (i - kW2) / 4096, k = (i - kW2) % 4096;
    return kWt2 + L * 64 * kHs + (k % 64) * kHs + k / 64;
  }
  const int k = i - kW5;
  return kWt5 + (k % 16) * kHs + k / 16;
}

__global__ void cache_adam_k(float* w, float* mw, float* vw, float* gw, float* table, float* mt, float* vt,
                             float* gt, __nv_bfloat16* wt, float lr, float b1, float b2, float eps, float bc1,
                             float bc2) {
  const size_t nw = kCacheWeights, n = nw + kCacheTableFloats;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float *p, *m, *v, *gp;
    size_t k;
    if (i < nw) {
      p = w, m = mw, v = vw, gp = gw, k = i;
    } else {
      p = table, m = mt, v = vt, gp = gt, k = i - nw;
    }
    const float g = gp[k];
    const float m1 = b1 * m[k] + (1.0f - b1) * g;
    const float v1 = b2 * v[k] + (1.0f - b2) * g * g;
    m[k] = m1;
    v[k] = v1;
    gp[k] = 0.0f;
    const float np = p[k] - lr * (m1 / bc1) / (sqrtf(v1 / bc2) + eps);
    p[k] = np;
    if (i < nw) wt[image_index((int)i)] = __float2bfloat16_rn(np);
  }
}

__global__ void cache_pack_k(const float* w, __nv_bfloat16* wt) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < kCacheWeights; i += gridDim.x * blockDim.x)
    wt[image_index((int)i)] = __float2bfloat16_rn(w[i]);
}

__global__ void cache_pack_rows_k(uint32_t n, const float* x01, const float* dir, const float* nrm,
                                  const float* p7, const float* u, CacheRows rows, float4* mat_a, float4* mat_b) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    rows.x[i] = make_float4(x01[3 * i], x01[3 * i + 1], x01[3 * i + 2], __int_as_float((int)i));
    rows.d[i] = make_float4(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2], __uint_as_float(i));
    rows.n[i] = make_float4(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2], 0.0f);
    rows.u[i] = u ? make_float4(u[3 * i], u[3 * i + 1], u[3 * i + 2], 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float* q = p7 + 7 * (size_t)i;
    mat_a[i] = make_float4(q[0], q[1], q[2], q[6]);
    mat_b[i] = make_float4(q[3], q[4], q[5], 0.0f);
  }
}

__global__ void cache_unpack_k(uint32_t n, const float4* c, const float* dp, float* rgb, float* dparams) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (rgb) {
      const float4 v = c[i];
      rgb[3 * i] = v.x;
      rgb[3 * i + 1] = v.y;
      rgb[3 * i + 2] = v.z;
    }
    if (dparams)
      for (int k = 0; k < 7; ++k) dparams[7 * (size_t)i + k] = dp[8 * (size_t)i + k];
  }
}

__global__ void cache_targets_k(CacheBuffers b, const float4* rad) {
  const uint32_t lo = b.counts[2], hi = min(b.counts[1], b.r_cap);
  for (uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) {
    const float4 v = rad[__float_as_uint(b.r.d[i].w)];
    b.r.u[i] = make_float4(v.x, v.y, v.z, 0.0f);
  }
}

int grid_of(uint32_t n, int threads) {
  const uint32_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

void cache_grid(int res[kCacheLevels], uint32_t* dense) {
  const double b = std::exp((std::log((double)kCacheNMax) - std::log((double)kCacheNMin)) / (kCacheLevels - 1));
  *dense = 0u;
  for (int l = 0; l < kCacheLevels; ++l) {
    res[l] = (int)std::floor((double)kCacheNMin * std::pow(b, (double)l));
    const double v = (double)(res[l] + 1);
    if (v * v * v <= (double)kCacheT) *dense |= 1u << l;
  }
}

template <bool kVjp>
static cudaError_t launch_infer(const CacheNet& net, const CacheRows& rows, const float4* mat_a, const float4* mat_b,
                                const uint32_t* count_dev, uint32_t n, const CacheOut& out, int num_sms,
                                cudaStream_t st) {
  // the VJP needs more than 64 registers: 12 warps per block keep two blocks
  // per SM without spills
  constexpr int W = kVjp ? 12 : kInferWarps, smem = infer_smem<W>();
  cudaError_t e = cudaFuncSetAttribute(cache_infer_k<kVjp, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  static int per_sm = 0;  // resident blocks per SM at this shared-memory size (the same on every GB300)
  if (per_sm == 0) {
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cache_infer_k<kVjp, W>, W * 32, smem);
    if (e != cudaSuccess) return e;
    per_sm = b < 1 ? 1 : b;
  }
  const uint32_t tiles = (n + 16u * W - 1u) / (16u * W);
  const int grid = (int)std::max<uint32_t>(1u, std::min<uint32_t>(tiles, (uint32_t)(num_sms * per_sm)));
  cache_infer_k<kVjp, W><<<grid, W * 32, smem, st>>>(net, rows, mat_a, mat_b, count_dev, n, out);
  return cudaGetLastError();
}

cudaError_t cache_infer(const CacheNet& net, const CacheRows& rows, const float4* mat_a, const float4* mat_b,
                        const uint32_t* count_dev, uint32_t n, const CacheOut& out, bool vjp, int num_sms,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return vjp ? launch_infer<true>(net, rows, mat_a, mat_b, count_dev, n, out, num_sms, st)
             : launch_infer<false>(net, rows, mat_a, mat_b, count_dev, n, out, num_sms, st);
}

cudaError_t cache_grad(const CacheNet& net, const CacheRows& rows, const float4* mat_a, const float4* mat_b,
                       const uint32_t* count_dev, uint32_t n, uint32_t batch, uint32_t n_batches,
                       const CacheOut& out, int num_sms, cudaStream_t st) {
  if (n == 0 || n_batches == 0) return cudaSuccess;
  const uint32_t tiles = ((n + n_batches - 1u) / n_batches + kTileRows - 1u) / kTileRows;
  const int grid = (int)std::max<uint32_t>(1u, std::min<uint32_t>(tiles, (uint32_t)num_sms));
  cudaFuncSetAttribute(cache_grad_k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTrain);
  cache_grad_k<<<grid, kThreads, kSmemTrain, st>>>(net, rows, mat_a, mat_b, count_dev, n, batch, n_batches, out);
  return cudaGetLastError();
}

cudaError_t cache_adam(float* w, float* mw, float* vw, float* gw, float* table, float* mt, float* vt, float* gt,
                       uint4* wt, float lr, float beta1, float beta2, float eps, float bc1, float bc2,
                       int num_sms, cudaStream_t st) {
  cache_adam_k<<<num_sms * 8, 256, 0, st>>>(w, mw, vw, gw, table, mt, vt, gt,
                                            reinterpret_cast<__nv_bfloat16*>(wt), lr, beta1, beta2, eps, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t cache_pack_weights(const float* w, uint4* wt, cudaStream_t st) {
  cache_pack_k<<<grid_of(kCacheWeights, 256), 256, 0, st>>>(w, reinterpret_cast<__nv_bfloat16*>(wt));
  return cudaGetLastError();
}

cudaError_t cache_pack_rows(uint32_t n, const float* x01, const float* dir, const float* nrm, const float* params7,
                            const float* u, const CacheRows& rows, float4* mat_a, float4* mat_b, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cache_pack_rows_k<<<grid_of(n, 256), 256, 0, st>>>(n, x01, dir, nrm, params7, u, rows, mat_a, mat_b);
  return cudaGetLastError();
}

cudaError_t cache_unpack_out(uint32_t n, const float4* c, const float* dp, float* rgb, float* dparams,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cache_unpack_k<<<grid_of(n, 256), 256, 0, st>>>(n, c, dp, rgb, dparams);
  return cudaGetLastError();
}

cudaError_t cache_targets(const CacheBuffers& b, const float4* rad, cudaStream_t st) {
  cache_targets_k<<<grid_of(b.r_cap, 256), 256, 0, st>>>(b, rad);
  return cudaGetLastError();
}

}  // namespace ipt
