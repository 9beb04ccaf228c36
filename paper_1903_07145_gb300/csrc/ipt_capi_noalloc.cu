// C ABI: ipt_backward_noalloc, the vector-Jacobian product without a device
// allocation at the call (include/ipt.h).
#include "ipt_capi_internal.h"

using namespace ipt_capi;

// ---------------------------------------------------------------------------
// ipt_backward_noalloc: ipt_backward for callers that may not allocate device
// memory.  Its only scratch, the FP64 gradient accumulator, is this file-scope
// array: 10 * kNoAllocMaxSegments doubles (80 KiB) that every device which
// loads the library keeps until the process exits.  Host code only sees a
// stand-in for the array; the device address is looked up by the first call
// with each context, with the context's device current, kept in the context
// (a device reset ends every context, so no address outlives one) and
// handed to the kernels.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kNoAllocMaxSegments = 1024;

static __device__ __align__(256) double g_noalloc_grad[10 * kNoAllocMaxSegments];

// Device address of g_noalloc_grad on the context's device (current).
cudaError_t noalloc_scratch(ipt_ctx* ctx, double** out) {
  if (!ctx->noalloc_acc) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_grad);
    if (e != cudaSuccess) return e;
    ctx->noalloc_acc = static_cast<double*>(p);
  }
  *out = ctx->noalloc_acc;
  return cudaSuccess;
}

}  // namespace

extern "C" ipt_status ipt_backward_noalloc(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts,
                                           uint32_t set, uint64_t iteration, const float* params,
                                           const float* sampling_params, const float* grad_image,
                                           float* grad_out) {
  DeviceScene* s;
  ipt_status st = get_scene(ctx, scene, &s);
  if (st != IPT_OK) return st;
  if ((st = check_opts(ctx, opts, true)) != IPT_OK) return st;
  if (s->views.empty()) return fail(ctx, IPT_ERR_INVALID_ARG, "no views set");
  if (!grad_image || !grad_out) return fail(ctx, IPT_ERR_INVALID_ARG, "null grad_image or grad_out");
  if (opts->spp_d == 0) return fail(ctx, IPT_ERR_INVALID_ARG, "spp_d must be positive");
  if (s->n_seg > kNoAllocMaxSegments)
    return fail(ctx, IPT_ERR_INVALID_ARG, "ipt_backward_noalloc supports at most " +
                                              std::to_string(kNoAllocMaxSegments) + " segments, scene has " +
                                              std::to_string(s->n_seg));
  IPT_CK(cudaSetDevice(ctx->device));
  double* acc = nullptr;
  IPT_CK(noalloc_scratch(ctx, &acc));
  const float* p = params ? params : s->params;
  const bool is_ctx = (p == s->params) && (sampling_params == nullptr || sampling_params == s->params);
  if (!(is_ctx && s->tab_is_ctx)) {
    Timed tm(ctx, IPT_KERNEL_PREPARE);
    IPT_CK(ipt::launch_prepare(buffers(ctx, s), s->tab, p, sampling_params ? sampling_params : p, ctx->stream));
    s->tab_is_ctx = is_ctx;
    s->tab_batch = -1;
  }
  const uint32_t np = 10u * s->n_seg;
  IPT_CK(cudaMemsetAsync(acc, 0, np * sizeof(double), ctx->stream));
  {
    Timed tm(ctx, IPT_KERNEL_ADJOINT);
    IPT_CK(ipt::launch_adjoint(ctx->L, buffers(ctx, s), s->tab, s->views_dev, (uint32_t)s->views.size(), 0,
                               (uint32_t)s->n_pix, trace_params(ctx, scene, opts, set, opts->spp_d, iteration),
                               grad_image, acc, nullptr, ctx->err_dev, ctx->stream));
  }
  Timed tm(ctx, IPT_KERNEL_FINALIZE);
  IPT_CK(ipt::launch_finalize(nullptr, 0, nullptr, acc, grad_out, np, ctx->stream));
  return IPT_OK;
}
