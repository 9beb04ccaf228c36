// Measurement support, not part of the method: the achievable bandwidth of
// random 64-byte line gathers over a device buffer of a given size, the
// access pattern of BVH traversal (a 64-byte node or a 48-byte triangle per
// fetch, incoherent across lanes), each line fetched with the two 256-bit
// read-only loads the traversal issues for a node.  It is the denominator of
// the traversal kernels' roofline: with the scene's node and triangle arrays
// (a few MB) the gathers stay in L2.  Also the build check: which binary
// version the device runs the library's kernels from.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ipt.h"

namespace {

constexpr int kThreads = 256;
constexpr int kStreams = 4;  // independent gathers in flight per thread

__device__ __forceinline__ uint32_t mix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__global__ void __launch_bounds__(kThreads) probe_gather_k(const uint4* buf, uint32_t n_lines, uint32_t iters,
                                                           uint32_t seed, uint4* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s[kStreams];
#pragma unroll
  for (int k = 0; k < kStreams; ++k) s[k] = mix(seed ^ mix(tid * kStreams + k + 1)) | 1u;
  uint4 acc = make_uint4(0, 0, 0, 0);
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kStreams; ++k) {
      // xorshift32 (Marsaglia 2003), mapped to [0, n_lines) by a 32x32 high product
      s[k] ^= s[k] << 13;
      s[k] ^= s[k] >> 17;
      s[k] ^= s[k] << 5;
      const uint32_t line = __umulhi(s[k], n_lines);
      const uint4* p = buf + 4 * (size_t)line;
      uint4 a, b, c, d;
      asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                   : "l"(p));
      asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(c.x), "=r"(c.y), "=r"(c.z), "=r"(c.w), "=r"(d.x), "=r"(d.y), "=r"(d.z), "=r"(d.w)
                   : "l"(p + 2));
      acc.x ^= a.x ^ b.y ^ c.z ^ d.w;
      acc.y ^= a.y ^ b.z ^ c.w ^ d.x;
      acc.z ^= a.z ^ b.w ^ c.x ^ d.y;
      acc.w ^= a.w ^ b.x ^ c.y ^ d.z;
    }
  }
  // keeps the loads live; the buffer is filled so that this never holds
  if (acc.x == 0xFFFFFFFFu && acc.y == 0xFFFFFFFFu && acc.z == 0xFFFFFFFFu && acc.w == 0xFFFFFFFFu) *sink = acc;
}

__global__ void probe_fill_k(uint32_t* buf, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    buf[i] = (uint32_t)i & 0x7FFFFFFFu;
}

}  // namespace

extern "C" ipt_status ipt_probe_gather(int32_t device, uint64_t bytes, double* gbs_out) {
  if (!gbs_out || bytes < 64 * 1024 || bytes / 64 > 0xFFFFFFFFull) return IPT_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return IPT_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return IPT_ERR_CUDA;
  const uint32_t n_lines = (uint32_t)(bytes / 64);
  uint4* buf = nullptr;
  uint4* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ipt_status status = IPT_OK;
  if (cudaMalloc(&buf, (size_t)n_lines * 64) != cudaSuccess || cudaMalloc(&sink, sizeof(uint4)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    status = IPT_ERR_OUT_OF_MEMORY;
  } else {
    probe_fill_k<<<sms * 8, kThreads, 0, st>>>(reinterpret_cast<uint32_t*>(buf), (size_t)n_lines * 16);
    const int grid = sms * 8;
    // about 12 ms of gathers per timed run at 6 TB/s
    const uint32_t iters = 896;
    const double bytes_moved = (double)grid * kThreads * iters * kStreams * 64.0;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, st);
      probe_gather_k<<<grid, kThreads, 0, st>>>(buf, n_lines, iters, 0x9E3779B9u * (rep + 1), sink);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        status = IPT_ERR_CUDA;
        break;
      }
      if (rep > 0 && ms < best) best = ms;  // the first run warms the caches
    }
    if (status == IPT_OK) *gbs_out = bytes_moved / (best * 1e-3) / 1e9;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  return status;
}

extern "C" ipt_status ipt_build_info(int32_t device, int32_t* binary_version, int32_t* ptx_version) {
  if (!binary_version && !ptx_version) return IPT_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return IPT_ERR_CUDA;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, probe_gather_k) != cudaSuccess) return IPT_ERR_CUDA;
  if (binary_version) *binary_version = fa.binaryVersion;
  if (ptx_version) *ptx_version = fa.ptxVersion;
  return IPT_OK;
}
