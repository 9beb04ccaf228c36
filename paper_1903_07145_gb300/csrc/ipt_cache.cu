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
// Queries run on the fifth-generation tensor cores: a block of 128 threads
// encodes 128 rows (one per thread) into a BF16 tile in shared memory, one
// thread issues each layer as tcgen05.mma (M = 128 rows) into FP32
// accumulators in tensor memory (TMEM), and every thread reads its row back
// with tcgen05.ld, applies the ReLU and writes the next layer's tile.  The
// input VJP and training run each warp's 16 rows forward and backward with
// mma.sync m16n8k16: a layer's FP32 accumulator fragments are the next
// layer's A fragments once packed to BF16, so the VJP needs only the hidden
// layers' ReLU masks (one register per layer), and the backward pass loads
// the transposed weights with ldmatrix.trans from the out-major image.  (A
// tcgen05 VJP, ten dependent MMA round trips per 128-row tile, measured 28%
// slower than these independent per-warp chains.)  Training keeps the
// block's 64 rows of inputs, activations and pre-activation gradients in
// shared memory in the core-matrix-blocked layout that the tensor cores
// read: the weight gradients dW = A^T dZ over those rows (K = rows) are one
// tcgen05.mma batch per tile, accumulated in TMEM across every tile the
// block processes, then read back and added to the global gradient once per
// launch.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
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
constexpr int kXw = kXs / 2, kHw = kHs / 2;  // strides in 32-bit words

// BF16 weight image offsets (elements).
constexpr int kWt1 = 0, kWt2 = 64 * kXs, kWt3 = kWt2 + 64 * kHs, kWt4 = kWt3 + 64 * kHs, kWt5 = kWt4 + 64 * kHs;
// FP32 master weight offsets: W1 80 x 64, W2..W4 64 x 64, W5 64 x 16, in-major.
constexpr int kW1 = 0, kW2 = 80 * 64, kW3 = kW2 + 4096, kW4 = kW3 + 4096, kW5 = kW4 + 4096;

// Shared-memory layout (bytes, 16-byte aligned regions).  Input VJP: the
// BF16 weight image, then each warp's input tile (row stride kXs) and row
// metadata (kSmemVjp).  Training: the weight image, then the block's
// 64-row tiles in the core-matrix-blocked layout of BlockTile -- X (80
// features), H1..H4 and dZ1..dZ4 (64 each), dY (16) -- the rows' metadata,
// and the weight-gradient MMAs' mbarrier and TMEM address.
constexpr int kSmWt = 0;
constexpr int kSmX = kSmWt + (int)kCacheWtElems * 2;
// bytes between consecutive 8-row groups of a blocked tile (features / 8 chunks of 128 B)
constexpr int kLboX = 10 * 128, kLboH = 8 * 128, kLboY = 2 * 128;
constexpr int kTX = kSmX;
constexpr int kTH = kTX + 8 * kLboX;       // H1..H4: 8 row groups of kLboH each
constexpr int kTDz = kTH + 4 * 8 * kLboH;  // dZ1..dZ4
constexpr int kTDy = kTDz + 4 * 8 * kLboH;
constexpr int kTMeta = kTDy + 8 * kLboY;
constexpr int kTBar = kTMeta + kTileRows * 16;  // mbarrier (8 B), TMEM address (4 B)
constexpr int kSmemTrain = kTBar + 16;
static_assert(kSmX % 16 == 0 && kTH % 16 == 0 && kTDz % 16 == 0 && kTDy % 16 == 0 && kTMeta % 16 == 0 &&
                  kTBar % 16 == 0,
              "shared regions must be 16-byte aligned");
static_assert(kSmemTrain <= 227 * 1024, "training tile exceeds shared memory");
// An M = 128 operand reads 16 feature chunks of every row group; the X and
// H tiles have fewer, so the reads of the last group run past the tile into
// the next region (never past dZ1).  The rows of D they feed are not used.
static_assert(kTX + 7 * kLboX + 16 * 128 <= kTDz && kTH + 3 * 8 * kLboH + 7 * kLboH + 16 * 128 <= kTDy,
              "M = 128 operand reads must stay inside the tiles");

// A tile of 16-bit pairs addressed by (row, word); word w of a row holds
// features 2w and 2w + 1.
struct RowTile {  // row-major, `stride` words per row
  uint32_t* p;
  int stride;
  __device__ __forceinline__ uint32_t& operator()(int r, int w) const { return p[r * stride + w]; }
};

// Core-matrix-blocked tile: 8-row groups `lbo` words apart; inside a group,
// chunks of 8 features (4 words) 32 words apart, each chunk holding its 8
// rows at 4-word steps (16 bytes).  Stored this way a [rows x features] tile
// is the no-swizzle MN-major operand of tcgen05.mma (features along M or N,
// rows along K), and the mma.sync fragment accesses (8 rows x 4 words per
// instruction) touch 32 consecutive words.
struct BlockTile {
  uint32_t* p;
  int lbo;
  __device__ __forceinline__ uint32_t& operator()(int r, int w) const {
    return p[(r >> 3) * lbo + (w >> 2) * 32 + (r & 7) * 4 + (w & 3)];
  }
  __device__ __forceinline__ BlockTile rows_from(int r0) const { return BlockTile{p + (r0 >> 3) * lbo, lbo}; }
};

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
// X (16 rows of 80 BF16 features) and its row metadata (unit position, valid
// flag).
// Encodes 16 rows into X.  kHalf: the hash-grid features come from the
// table's FP16 copy (queries) instead of the FP32 master (training and the
// input VJP, whose result depends on the table only through the ReLU
// decisions, which the FP16 rounding would move near their kinks).
template <bool kHalf, class Tile>
__device__ __forceinline__ void encode_rows(const CacheNet& net, const int* res, const CacheRows& rows, const float4* mat_a,
                            const float4* mat_b, uint32_t r0, uint32_t end, Tile X, float4* meta, int lane) {
  const int row = lane & 15;
  const uint32_t r = r0 + (uint32_t)row;
  const bool valid = r < end;
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
    X(row, 32) = pack2(ma.x, ma.y);  // kd r, g
    X(row, 33) = pack2(ma.z, mb.x);  // kd b, ks r
    X(row, 34) = pack2(mb.y, mb.z);  // ks g, b
    X(row, 35) = pack2(ma.w, 0.0f);  // roughness
#pragma unroll
    for (int i = 36; i < 40; ++i) X(row, i) = 0u;
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
    for (int i = 0; i < 8; ++i) X(row, w0 + i) = valid ? pack2(sh[2 * i], sh[2 * i + 1]) : 0u;
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
        float2 v;
        if (kHalf) {
          const uint32_t hv = __ldg(&net.table_h[idx[c]]);
          v = __half22float2(*reinterpret_cast<const __half2*>(&hv));
        } else {
          v = __ldg(&net.table[idx[c]]);
        }
        f0 += w[c] * v.x;
        f1 += w[c] * v.y;
      }
      word = pack2(f0, f1);
    }
    X(rr, l) = word;
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
// tile H (the warp's 16 rows).
template <bool kStore>
__device__ __forceinline__ void relu_pack(const float (&c)[8][4], uint32_t (&a)[4][4], BlockTile H, int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t lo = pack2(fmaxf(c[j][0], 0.0f), fmaxf(c[j][1], 0.0f));
    const uint32_t hi = pack2(fmaxf(c[j][2], 0.0f), fmaxf(c[j][3], 0.0f));
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    if (kStore) {
      H(g, 4 * j + t) = lo;
      H(g + 8, 4 * j + t) = hi;
    }
  }
}

// First-layer A fragments of the warp's 16 rows from its input tile.
template <class Tile>
__device__ __forceinline__ void input_frags(Tile X, uint32_t (&a)[5][4], int g, int t) {
#pragma unroll
  for (int kk = 0; kk < 5; ++kk) {
    a[kk][0] = X(g, 8 * kk + t);
    a[kk][1] = X(g + 8, 8 * kk + t);
    a[kk][2] = X(g, 8 * kk + 4 + t);
    a[kk][3] = X(g + 8, 8 * kk + 4 + t);
  }
}

// Forward pass of the warp's 16 rows from its input tile; hidden
// activations of layer i go to H advanced by i * hstride words when kStore.
template <bool kStore>
__device__ __forceinline__ void net_forward(const uint32_t* Wt, BlockTile X, BlockTile H, int hstride,
                                            float (&y)[2][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  float c[8][4];
  uint32_t h[4][4];
  {
    uint32_t a[5][4];
    input_frags(X, a, g, t);
    layer_fwd<5, 8, kXw>(Wt + kWt1 / 2, a, c, g, t);
  }
  relu_pack<kStore>(c, h, H, g, t);
  layer_fwd<4, 8, kHw>(Wt + kWt2 / 2, h, c, g, t);
  relu_pack<kStore>(c, h, BlockTile{H.p + hstride, H.lbo}, g, t);
  layer_fwd<4, 8, kHw>(Wt + kWt3 / 2, h, c, g, t);
  relu_pack<kStore>(c, h, BlockTile{H.p + 2 * hstride, H.lbo}, g, t);
  layer_fwd<4, 8, kHw>(Wt + kWt4 / 2, h, c, g, t);
  relu_pack<kStore>(c, h, BlockTile{H.p + 3 * hstride, H.lbo}, g, t);
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
__device__ __forceinline__ void relu_grad(const float (&dh)[8][4], BlockTile H, uint32_t (&a)[4][4],
                                          BlockTile Dz, int g, int t) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float2 h0 = unpack2(H(g, 4 * j + t));
    const float2 h1 = unpack2(H(g + 8, 4 * j + t));
    const uint32_t lo = pack2(h0.x > 0.0f ? dh[j][0] : 0.0f, h0.y > 0.0f ? dh[j][1] : 0.0f);
    const uint32_t hi = pack2(h1.x > 0.0f ? dh[j][2] : 0.0f, h1.y > 0.0f ? dh[j][3] : 0.0f);
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    if (kStore) {
      Dz(g, 4 * j + t) = lo;
      Dz(g + 8, 4 * j + t) = hi;
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
__device__ __forceinline__ void net_forward_mask(const uint32_t* Wt, RowTile X, float (&y)[2][4],
                                                 uint32_t (&mask)[4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  float c[8][4];
  uint32_t h[4][4];
  {
    uint32_t a[5][4];
    input_frags(X, a, g, t);
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
// Pre-activation gradients (and dY) are stored when kStore; layer i of H and
// Dz is hstride words after layer i - 1.
template <bool kStore, int JP0, int JP1>
__device__ __forceinline__ void net_backward(const __nv_bfloat16* Wtb, BlockTile H, int hstride, BlockTile Dz,
                                             BlockTile Dy, const float (&dy)[2][4],
                                             float (&dx)[2 * (JP1 - JP0)][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  uint32_t ay[1][4];
  ay[0][0] = pack2(dy[0][0], dy[0][1]);
  ay[0][1] = pack2(dy[0][2], dy[0][3]);
  ay[0][2] = pack2(dy[1][0], dy[1][1]);
  ay[0][3] = pack2(dy[1][2], dy[1][3]);
  if (kStore) {
    Dy(g, t) = ay[0][0];
    Dy(g + 8, t) = ay[0][1];
    Dy(g, 4 + t) = ay[0][2];
    Dy(g + 8, 4 + t) = ay[0][3];
  }
  float dh[8][4];
  uint32_t a[4][4];
  layer_bwd<1, 0, 4, kHs>(Wtb + kWt5, ay, dh, lane);
  auto at = [](BlockTile b, int i, int stride) { return BlockTile{b.p + i * stride, b.lbo}; };
  relu_grad<kStore>(dh, at(H, 3, hstride), a, at(Dz, 3, hstride), g, t);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt4, a, dh, lane);
  relu_grad<kStore>(dh, at(H, 2, hstride), a, at(Dz, 2, hstride), g, t);
  layer_bwd<4, 0, 4, kHs>(Wtb + kWt3, a, dh, lane);
  relu_grad<kStore>(dh, at(H, 1, hstride), a, at(Dz, 1, hstride), g, t);
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

// Input VJP (with the query's outputs) over warp tiles of 16 rows; the warps
// share one shared-memory weight image.  The hidden layers' ReLU masks stay
// in registers, so a block holds only the weights and its warps' input
// tiles.  The VJP needs more than 64 registers: 12 warps per block keep two
// blocks per SM without spills.
constexpr int kVjpWarps = 12;
constexpr int kSmemVjp = kSmX + kVjpWarps * 16 * kXs * 2 + kVjpWarps * 16 * 16;
static_assert(kSmX % 16 == 0 && (kSmX + kVjpWarps * 16 * kXs * 2) % 16 == 0, "VJP tiles must be aligned");

__global__ void __launch_bounds__(kVjpWarps * 32, 2) cache_vjp_k(CacheNet net, CacheRows rows, const float4* mat_a,
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
  const RowTile X{reinterpret_cast<uint32_t*>(sm + kSmX) + warp * 16 * kXw, kXw};
  float4* meta = reinterpret_cast<float4*>(sm + kSmX + kVjpWarps * 16 * kXs * 2) + warp * 16;
  const uint32_t n_tiles = (n + 15u) / 16u;
  for (uint32_t tile = blockIdx.x * (uint32_t)kVjpWarps + (uint32_t)warp; tile < n_tiles;
       tile += gridDim.x * (uint32_t)kVjpWarps) {
    const uint32_t r0 = tile * 16u;
    __syncwarp();
    encode_rows<false>(net, res, rows, mat_a, mat_b, r0, n, X, meta, lane);
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
    {
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

// ---------------------------------------------------------------------------
// Fifth-generation tensor cores (tcgen05): the training pass's weight
// gradients.  Operands come from shared memory through matrix descriptors,
// the FP32 accumulators live in tensor memory (TMEM), one thread issues the
// MMAs, and an mbarrier tracks their completion.
// ---------------------------------------------------------------------------
constexpr uint32_t kDwCols = 512;       // TMEM columns held by a training block (272 used)
constexpr uint32_t kWaitLimit = 1u << 24;  // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Descriptor of a no-swizzle operand in shared memory: start address, the
// byte offset between 8-row groups along K (lbo) and between 8-element
// chunks along M or N (sbo), descriptor version 1.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of a dense kind::f16 MMA: BF16 A and B, FP32 D,
// shape M x N, both operands MN-major (mn = true) or both K-major.
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n, bool mn = true) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (mn ? (1u << 15) | (1u << 16) : 0u) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Polls the mbarrier's phase with the given parity at most `limit` times.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// One tile's weight gradients added to the TMEM accumulators (sums over the
// tile's 64 rows, K, in four steps of 16): dW1 = X^T dZ1, dW2..dW4 =
// H1..H3^T dZ2..dZ4, dW5 = H4^T dY.  D rows (TMEM lanes) are the layer's
// inputs (M = 128; rows past 80 or 64 inputs take values that are never
// read), columns its outputs: dW1 at columns 0-63, dW2..dW4 at 64-255, dW5
// at 256-271.  accumulate = 0 overwrites (the block's first tile).
__device__ __forceinline__ void issue_weight_grads(const unsigned char* sm, uint32_t tmem, bool accumulate) {
  const uint32_t base = smem_addr(sm);
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    const uint32_t a = base + (uint32_t)(l == 0 ? kTX : kTH + (l - 1) * 8 * kLboH);
    const uint32_t alb = l == 0 ? kLboX : kLboH;
    const uint32_t b = base + (uint32_t)(l < 4 ? kTDz + l * 8 * kLboH : kTDy);
    const uint32_t blb = l < 4 ? kLboH : kLboY;
    const uint32_t idesc = umma_idesc(128, l < 4 ? 64 : 16);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      umma_bf16(tmem + 64u * (uint32_t)l, umma_sdesc(a + 2u * k * alb, alb, 128), umma_sdesc(b + 2u * k * blb, blb, 128),
                idesc, (accumulate || k > 0) ? 1u : 0u);
  }
}

// Adds the block's accumulated weight gradients to gw (FP32 master layout,
// input index first).  Warp w reads TMEM lanes 32w..32w + 31, i.e. input m =
// 32w + lane of every layer.
__device__ __forceinline__ void flush_weight_grads(uint32_t tmem, float* gw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = 32 * warp + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < 272; c0 += 16) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int l = c0 >> 6, n0 = c0 & 63;
    if (m < (l == 0 ? 80 : 64)) {
      float* dst = gw + (l == 0 ? kW1 + m * 64 : (l < 4 ? kW2 + (l - 1) * 4096 + m * 64 : kW5 + m * 16)) + n0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float v = __uint_as_float(r[j]);
        if (v != 0.0f) atomicAdd(dst + j, v);
      }
    }
  }
}

// Training gradients over block tiles of 64 rows of one minibatch.  The
// forward and backward passes run on mma.sync per warp (16 rows each); the
// weight gradients of each tile go to the tensor cores as one batch of 20
// tcgen05.mma (issued after the tile's tiles are written, waited for before
// the next tile overwrites them), accumulated in TMEM for the whole launch.
__global__ void __launch_bounds__(kThreads) cache_grad_k(CacheNet net, CacheRows rows, const float4* mat_a,
                                                         const float4* mat_b, const uint32_t* count_dev,
                                                         uint32_t n_max, uint32_t batch, uint32_t n_batches,
                                                         CacheOut o) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int res[kCacheLevels];
  load_weights(net, sm, res);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kTBar + 8);
  const uint32_t mbar = smem_addr(sm + kTBar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kDwCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t n = count_dev ? min(*count_dev, n_max) : n_max;
  const uint32_t per = (n + n_batches - 1u) / n_batches;
  const uint32_t begin = min(batch * per, n), end = min(begin + per, n);
  const uint32_t rows_n = end - begin;
  const float scale = rows_n ? 1.0f / (3.0f * (float)rows_n) : 0.0f;
  const int g = lane >> 2, t = lane & 3;
  const uint32_t* Wt = reinterpret_cast<const uint32_t*>(sm + kSmWt);
  const __nv_bfloat16* Wtb = reinterpret_cast<const __nv_bfloat16*>(sm + kSmWt);
  // the warp's 16 rows of each block tile
  const BlockTile X = BlockTile{reinterpret_cast<uint32_t*>(sm + kTX), kLboX / 4}.rows_from(16 * warp);
  const BlockTile H = BlockTile{reinterpret_cast<uint32_t*>(sm + kTH), kLboH / 4}.rows_from(16 * warp);
  const BlockTile Dz = BlockTile{reinterpret_cast<uint32_t*>(sm + kTDz), kLboH / 4}.rows_from(16 * warp);
  const BlockTile Dy = BlockTile{reinterpret_cast<uint32_t*>(sm + kTDy), kLboY / 4}.rows_from(16 * warp);
  const int hstride = 8 * kLboH / 4;  // words between layers
  float4* meta = reinterpret_cast<float4*>(sm + kTMeta) + warp * 16;
  double loss = 0.0;
  uint32_t issued = 0;  // MMA batches committed to the mbarrier
  bool failed = false;
  const uint32_t n_tiles = (rows_n + kTileRows - 1u) / kTileRows;
  for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (issued) {
      // the previous tile's MMAs read these tiles: wait before overwriting
      const bool ok = mbar_wait(mbar, (issued - 1u) & 1u, kWaitLimit);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    const uint32_t r0 = begin + tile * kTileRows + 16u * (uint32_t)warp;
    encode_rows<false>(net, res, rows, mat_a, mat_b, r0, end, X, meta, lane);
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
    // the tiles' generic-proxy writes become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      issue_weight_grads(sm, tmem, issued > 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                   : "memory");
    }
    ++issued;
  }
  // wait for the last batch (also after a failed wait: its MMAs may still run)
  bool drained = true;
  if (issued) drained = __syncthreads_or(!mbar_wait(mbar, (issued - 1u) & 1u, kWaitLimit)) == 0;
  if ((failed || !drained) && threadIdx.x == 0 && o.err) atomicOr(o.err, kErrTimeout);
  tc_fence_after();
  if (issued && drained && !failed) flush_weight_grads(tmem, o.gw);
  tc_fence_before();
  __syncthreads();
  // the TMEM is freed unless MMAs may still write it
  if (warp == 0 && drained)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kDwCols) : "memory");
  if (o.loss) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, s);
    if (lane == 0 && loss != 0.0) atomicAdd(o.loss, loss);
  }
}

// ---------------------------------------------------------------------------
// Inference on the fifth-generation tensor cores: 128-row tiles per block of
// four warps, one row per thread.  Each warp encodes its 32 rows into the
// block's input tile; per layer one thread issues the MMAs (A = the tile,
// K-major: the rows' features in 128-byte chunks; B = the layer's weights in
// the same blocked layout, K-major: each output's inputs in chunks) into a
// 128 x 64 FP32 accumulator in TMEM; every thread then reads its row back
// with tcgen05.ld, applies the ReLU and writes the next layer's BF16 tile
// (over the layer's own input tile, whose MMAs have completed).  Two blocks
// per SM: one block's gathers overlap the other's MMA round trips, and the
// 74 KB of shared memory a block takes leave most of the SM's L1 to the
// hash-table gathers (three blocks per SM, with 28 KB of L1 left, were 36%
// slower).
// ---------------------------------------------------------------------------
constexpr int kQRows = 128;
constexpr int kQLboX = 10 * 128, kQLboH = 8 * 128;  // bytes between 8-row groups (activation tiles, weights)
constexpr int kQW1 = 0;                               // 64 outputs x 80 inputs
constexpr int kQW2 = kQW1 + 8 * kQLboX;               // W2..W4: 64 x 64 each
constexpr int kQW5 = kQW2 + 3 * 8 * kQLboH;           // 16 outputs x 64 inputs
constexpr int kQX = kQW5 + 2 * kQLboH;
constexpr int kQH = kQX + (kQRows / 8) * kQLboX;      // one 128 x 64 tile
constexpr int kQMeta = kQH + (kQRows / 8) * kQLboH;
constexpr int kQBar = kQMeta + kQRows * 16;
constexpr int kSmemInferTc = kQBar + 16;
constexpr uint32_t kQCols = 128;                      // TMEM columns of a block
static_assert(kQX % 128 == 0 && kQH % 128 == 0 && kQMeta % 16 == 0 && kQBar % 16 == 0, "tile alignment");
static_assert(2 * kSmemInferTc <= 227 * 1024, "two inference blocks per SM");
static_assert(2 * kQCols <= 512, "two inference blocks' TMEM per SM");

// The out-major BF16 weight image (mma.sync layout, padded rows) re-laid in
// the blocked K-major layout: output n, input chunk c (8 inputs, 16 bytes)
// at (n / 8) * lbo + c * 128 + (n % 8) * 16.
__device__ __forceinline__ void load_weights_blocked(const CacheNet& net, unsigned char* sm, int* res) {
  const uint4* img = net.wt;  // BF16 elements, 8 per uint4
  constexpr int chunks1 = 64 * 10, chunks24 = 64 * 8, chunks5 = 16 * 8;
  constexpr int total = chunks1 + 3 * chunks24 + chunks5;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int n, c, src, dst;
    if (t < chunks1) {
      n = t / 10;
      c = t % 10;
      src = (kWt1 + n * kXs + 8 * c) / 8;
      dst = kQW1 + (n >> 3) * kQLboX + c * 128 + (n & 7) * 16;
    } else if (t < chunks1 + 3 * chunks24) {
      const int u = t - chunks1, L = u / chunks24, v = u % chunks24;
      n = v / 8;
      c = v % 8;
      src = (kWt2 + L * 64 * kHs + n * kHs + 8 * c) / 8;
      dst = kQW2 + L * 8 * kQLboH + (n >> 3) * kQLboH + c * 128 + (n & 7) * 16;
    } else {
      const int v = t - chunks1 - 3 * chunks24;
      n = v / 8;
      c = v % 8;
      src = (kWt5 + n * kHs + 8 * c) / 8;
      dst = kQW5 + (n >> 3) * kQLboH + c * 128 + (n & 7) * 16;
    }
    *reinterpret_cast<uint4*>(sm + dst) = __ldg(&img[src]);
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int l = 0; l < kCacheLevels; ++l) res[l] = net.res[l];
  }
}

// Reads 16 FP32 accumulator columns of this thread's row (TMEM lane) into r.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) r[j] = __uint_as_float(u[j]);
}

// One layer's MMAs: D[128 x n_out] = A[128 x k_in] x W^T, both K-major
// blocked (A rows grouped at a_lbo bytes, W outputs at w_lbo), K in steps of 16.
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t a, uint32_t a_lbo, uint32_t w, uint32_t w_lbo,
                                            int k_in, int n_out) {
  const uint32_t idesc = umma_idesc(128, n_out, false);
  for (int k = 0; k < k_in / 16; ++k)
    umma_bf16(tmem, umma_sdesc(a + 256u * k, 128, a_lbo), umma_sdesc(w + 256u * k, 128, w_lbo), idesc, k > 0 ? 1u : 0u);
}

__global__ void __launch_bounds__(128, 2) cache_infer_tc_k(CacheNet net, CacheRows rows, const float4* mat_a,
                                                           const float4* mat_b, const uint32_t* count_dev,
                                                           uint32_t n_max, CacheOut o) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int res[kCacheLevels];
  load_weights_blocked(net, sm, res);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kQBar + 8);
  const uint32_t mbar = smem_addr(sm + kQBar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kQCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's 32 TMEM lanes
  const uint32_t n = count_dev ? min(*count_dev, n_max) : n_max;
  const uint32_t base = smem_addr(sm);
  const BlockTile X{reinterpret_cast<uint32_t*>(sm + kQX), kQLboX / 4};
  float4* meta = reinterpret_cast<float4*>(sm + kQMeta);
  const int row = 32 * warp + lane;  // this thread's row of the tile
  uint32_t phase = 0;
  bool ok = true;
  const uint32_t n_tiles = (n + kQRows - 1u) / kQRows;
  for (uint32_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const uint32_t r0 = tile * kQRows;
    encode_rows<true>(net, res, rows, mat_a, mat_b, r0 + 32u * warp, n, X.rows_from(32 * warp), meta + 32 * warp, lane);
    encode_rows<true>(net, res, rows, mat_a, mat_b, r0 + 32u * warp + 16u, n, X.rows_from(32 * warp + 16),
                meta + 32 * warp + 16, lane);
    float y[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int l = 0; l < 5 && ok; ++l) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_fence_after();
        const uint32_t a = base + (uint32_t)(l == 0 ? kQX : kQH);
        const uint32_t a_lbo = l == 0 ? kQLboX : kQLboH;
        const uint32_t w = base + (uint32_t)(l == 0 ? kQW1 : (l < 4 ? kQW2 + (l - 1) * 8 * kQLboH : kQW5));
        const uint32_t w_lbo = l == 0 ? kQLboX : kQLboH;
        issue_layer(tmem, a, a_lbo, w, w_lbo, l == 0 ? 80 : 64, l < 4 ? 64 : 16);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                     : "memory");
      }
      ok = __syncthreads_and(mbar_wait(mbar, phase, kWaitLimit)) != 0;
      phase ^= 1u;
      tc_fence_after();
      if (!ok) break;
      if (l < 4) {
        // ReLU, BF16, this row of the next tile
        const BlockTile H{reinterpret_cast<uint32_t*>(sm + kQH), kQLboH / 4};
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
          float v[16];
          tmem_ld16(tlane + (uint32_t)c0, v);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            uint4 pk;
            pk.x = pack2(fmaxf(v[8 * q + 0], 0.f), fmaxf(v[8 * q + 1], 0.f));
            pk.y = pack2(fmaxf(v[8 * q + 2], 0.f), fmaxf(v[8 * q + 3], 0.f));
            pk.z = pack2(fmaxf(v[8 * q + 4], 0.f), fmaxf(v[8 * q + 5], 0.f));
            pk.w = pack2(fmaxf(v[8 * q + 6], 0.f), fmaxf(v[8 * q + 7], 0.f));
            *reinterpret_cast<uint4*>(&H(row, (c0 + 8 * q) / 2)) = pk;
          }
        }
      } else {
        float v[16];
        tmem_ld16(tlane, v);
        y[0] = v[0];
        y[1] = v[1];
        y[2] = v[2];
      }
    }
    if (!ok) break;
    const uint32_t r = r0 + (uint32_t)row;
    if (r < n) {
      if (o.c) o.c[r] = make_float4(y[0], y[1], y[2], 0.0f);
      if (o.rad) {
        const float4 b = rows.u[r];
        float4* dst = &o.rad[__float_as_uint(rows.d[r].w)];
        const float4 v = *dst;
        *dst = make_float4(v.x + b.x * y[0], v.y + b.y * y[1], v.z + b.z * y[2], v.w);
      }
    }
    // the next tile's encoding overwrites X (read by layer 1, done) and meta
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // MMAs in flight after a failed wait must finish before the TMEM goes back
  bool drained = ok;
  if (!ok) {
    drained = __syncthreads_and(mbar_wait(mbar, phase ^ 1u, kWaitLimit)) != 0;
    if (threadIdx.x == 0 && o.err) atomicOr(o.err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0 && drained)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kQCols) : "memory");
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
                             float* gt, __nv_bfloat16* wt, __half* table_h, float lr, float b1, float b2, float eps,
                             float bc1, float bc2) {
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
    if (i < nw)
      wt[image_index((int)i)] = __float2bfloat16_rn(np);
    else
      table_h[k] = __float2half_rn(np);
  }
}

__global__ void cache_pack_table_k(const float* table, __half* table_h) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < kCacheTableFloats;
       i += (size_t)gridDim.x * blockDim.x)
    table_h[i] = __float2half_rn(table[i]);
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

static cudaError_t launch_vjp(const CacheNet& net, const CacheRows& rows, const float4* mat_a, const float4* mat_b,
                              const uint32_t* count_dev, uint32_t n, const CacheOut& out, int num_sms,
                              cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(cache_vjp_k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemVjp);
  if (e != cudaSuccess) return e;
  static int per_sm = 0;  // resident blocks per SM at this shared-memory size (the same on every GB300)
  if (per_sm == 0) {
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cache_vjp_k, kVjpWarps * 32, kSmemVjp);
    if (e != cudaSuccess) return e;
    per_sm = b < 1 ? 1 : b;
  }
  const uint32_t tiles = (n + 16u * kVjpWarps - 1u) / (16u * kVjpWarps);
  const int grid = (int)std::max<uint32_t>(1u, std::min<uint32_t>(tiles, (uint32_t)(num_sms * per_sm)));
  cache_vjp_k<<<grid, kVjpWarps * 32, kSmemVjp, st>>>(net, rows, mat_a, mat_b, count_dev, n, out);
  return cudaGetLastError();
}

static cudaError_t launch_infer_tc(const CacheNet& net, const CacheRows& rows, const float4* mat_a,
                                   const float4* mat_b, const uint32_t* count_dev, uint32_t n, const CacheOut& out,
                                   int num_sms, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(cache_infer_tc_k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemInferTc);
  if (e != cudaSuccess) return e;
  // the smallest shared-memory carveout that holds two blocks (with the 1 KB
  // the system reserves per block): the rest of the 256 KB stays L1
  const int carveout = (2 * (kSmemInferTc + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024);
  e = cudaFuncSetAttribute(cache_infer_tc_k, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (n + kQRows - 1u) / kQRows;
  const int grid = (int)std::max<uint32_t>(1u, std::min<uint32_t>(tiles, (uint32_t)(2 * num_sms)));
  cache_infer_tc_k<<<grid, 128, kSmemInferTc, st>>>(net, rows, mat_a, mat_b, count_dev, n, out);
  return cudaGetLastError();
}

cudaError_t cache_infer(const CacheNet& net, const CacheRows& rows, const float4* mat_a, const float4* mat_b,
                        const uint32_t* count_dev, uint32_t n, const CacheOut& out, bool vjp, int num_sms,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (vjp) return launch_vjp(net, rows, mat_a, mat_b, count_dev, n, out, num_sms, st);
  return launch_infer_tc(net, rows, mat_a, mat_b, count_dev, n, out, num_sms, st);
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
                       uint4* wt, uint32_t* table_h, float lr, float beta1, float beta2, float eps, float bc1,
                       float bc2, int num_sms, cudaStream_t st) {
  cache_adam_k<<<num_sms * 8, 256, 0, st>>>(w, mw, vw, gw, table, mt, vt, gt, reinterpret_cast<__nv_bfloat16*>(wt),
                                            reinterpret_cast<__half*>(table_h), lr, beta1, beta2, eps, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t cache_pack_table(const float* table, uint32_t* table_h, cudaStream_t st) {
  cache_pack_table_k<<<grid_of((uint32_t)(kCacheTableFloats / 4), 256), 256, 0, st>>>(
      table, reinterpret_cast<__half*>(table_h));
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
