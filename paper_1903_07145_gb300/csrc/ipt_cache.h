// Learned radiance cache: sizes, device views and launchers shared by the
// wavefront integrator and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ipt {

constexpr int kCacheLevels = 16;                  // hash-grid levels
constexpr int kCacheFeatures = 2;                 // features per level
constexpr uint32_t kCacheLog2T = 19;              // entries per level = 2^19
constexpr uint32_t kCacheT = 1u << kCacheLog2T;
constexpr int kCacheNMin = 16, kCacheNMax = 2048; // coarsest and finest grid resolution
constexpr int kCacheIn = 80;                      // hash 32 | SH(dir) 16 | SH(normal) 16 | kd ks r 7 | 0 x 9
constexpr int kCacheHidden = 64;
constexpr int kCacheOut = 16;                     // first 3 are RGB
constexpr uint32_t kCacheWeights = 80 * 64 + 3 * 64 * 64 + 64 * 16;  // 18432 FP32 master weights
constexpr size_t kCacheTableFloats = (size_t)kCacheLevels * kCacheT * kCacheFeatures;
// BF16 weight image in shared memory: each layer out-major with padded rows
// (W1t 64 x 88, W2t..W4t 64 x 72, W5t 16 x 72).
constexpr uint32_t kCacheWtElems = 64 * 88 + 3 * 64 * 72 + 16 * 72;

// Device view of the network used by a pass.
struct CacheNet {
  const uint4* wt;        // BF16 weight image (kCacheWtElems / 8 uint4)
  const float2* table;    // [level][kCacheT] features (FP32 master, read by training and the VJP)
  const uint32_t* table_h;  // the same as FP16 pairs, read by queries
  float3 lo, inv_ext;     // world -> unit cube (the scene's bounding box)
  int res[kCacheLevels];  // grid resolution of each level
  uint32_t dense;         // bit l: level l indexes its (res+1)^3 vertices directly
};

// Rows of queries or training records (structure of arrays).
//   x: position (world), w = segment (int bits)
//   d: direction towards the previous vertex, w = path slot (uint bits)
//   n: oriented shading normal
//   u: forward: throughput beta; adjoint: upstream g * beta; training: target
struct CacheRows {
  float4* x;
  float4* d;
  float4* n;
  float4* u;
};

// Device error word bit: a bounded wait for the tensor cores gave up (the
// pass's results are incomplete).
constexpr uint32_t kErrTimeout = 4u;

// What a kernel writes for its rows.
struct CacheOut {
  float4* c;      // prediction per row (nullable)
  float4* rad;    // nullable: rad[slot] += u * prediction
  float* dp;      // nullable: 8 floats per row, d(u . prediction) / d(kd, ks, r), 8th = 0
  float* gw;      // training: weight gradients (accumulated)
  float2* gt;     // training: hash-table gradients (accumulated)
  double* loss;   // training: sum over rows and channels of the relative L2 terms
  uint32_t* err;  // training: error word (kErrTimeout), nullable
};

// Query and record buffers of the wavefront integrator.
struct CacheBuffers {
  CacheRows q;        // queries of the current chunk
  float4* qc;         // prediction per query
  float* qdp;         // 8 floats per query (see CacheOut::dp)
  CacheRows r;        // training records (u = target)
  uint32_t* counts;   // [0] queries in the chunk, [1] records, [2] records before the chunk
  uint32_t q_cap, r_cap;
};

// Resolutions and dense-level mask of the grid (host).
void cache_grid(int res[kCacheLevels], uint32_t* dense);

// Prediction (and, with vjp, the input vector-Jacobian product) of rows
// [0, min(*count_dev, n)) (count_dev nullable: n rows).  mat_a / mat_b hold
// (kd, r) and (ks, -) per segment id of x.w.
cudaError_t cache_infer(const CacheNet& net, const CacheRows& rows, const float4* mat_a, const float4* mat_b,
                        const uint32_t* count_dev, uint32_t n, const CacheOut& out, bool vjp, int num_sms,
                        cudaStream_t st);

// Relative-L2 loss and gradients of minibatch `batch` of `n_batches` equal
// parts of rows [0, min(*count_dev, n)); the gradient is that of the mean
// over the minibatch's rows and 3 channels (the loss sum is not scaled).
cudaError_t cache_grad(const CacheNet& net, const CacheRows& rows, const float4* mat_a, const float4* mat_b,
                       const uint32_t* count_dev, uint32_t n, uint32_t batch, uint32_t n_batches,
                       const CacheOut& out, int num_sms, cudaStream_t st);

// Adam on weights and table with the accumulated gradients (which it
// clears); rewrites the BF16 weight image and the table's FP16 copy.
// bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
cudaError_t cache_adam(float* w, float* mw, float* vw, float* gw, float* table, float* mt, float* vt, float* gt,
                       uint4* wt, uint32_t* table_h, float lr, float beta1, float beta2, float eps, float bc1,
                       float bc2, int num_sms, cudaStream_t st);

// BF16 weight image from the FP32 master weights.
cudaError_t cache_pack_weights(const float* w, uint4* wt, cudaStream_t st);
// FP16 copy of the hash table (kCacheTableFloats halves), from the FP32 master.
cudaError_t cache_pack_table(const float* table, uint32_t* table_h, cudaStream_t st);

// Rows of the evaluation entry points: row i gets x = x01[i], segment i,
// and per-row parameter tables (kd, r) / (ks, 0) from params7[i].
cudaError_t cache_pack_rows(uint32_t n, const float* x01, const float* dir, const float* nrm, const float* params7,
                            const float* u, const CacheRows& rows, float4* mat_a, float4* mat_b, cudaStream_t st);

// Per-row outputs of the evaluation entry points back to n x 3 / n x 7.
cudaError_t cache_unpack_out(uint32_t n, const float4* c, const float* dp, float* rgb, float* dparams,
                             cudaStream_t st);

// Targets of the records appended since the chunk began: u = rad[slot].
cudaError_t cache_targets(const CacheBuffers& b, const float4* rad, cudaStream_t st);

}  // namespace ipt
