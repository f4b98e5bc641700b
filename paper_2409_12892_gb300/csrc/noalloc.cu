// gslm_apply_JT_noalloc: J^T u without any device allocation.
//
// The paper has no counterpart; this entry point exists for callers that must
// not allocate device memory once they are running, e.g. a service whose
// device memory is reserved up front by another allocator, or a host thread
// that may not call cudaMalloc (which can synchronise the device). The normal
// gslm_apply_JT keeps its per-segment partial sums in a context-owned buffer
// that grows with cudaMallocAsync; this variant keeps them in the fixed array
// below instead and calls no allocating routine.
//
// Set-up happens in gslm_create, not here: with the context's device current,
// it looks up the array's device address (the array's name is only a host-side
// stand-in for it), which loads this file's module and so places the array on
// that device. Every device on which a context was created holds the array
// until the process exits; the call itself only reads the stored address.
#include "internal.cuh"

// Largest cache (in non-empty tile/splat segments) the variant accepts.
static constexpr long long kNoAllocMaxSegments = 1ll << 19;

// 2^19 segments x 12 floats = 24 MiB of per-segment J^T u partials.
static __device__ __align__(256) float g_noalloc_seg_ybar[kNoAllocMaxSegments * 12];

namespace gslm {
cudaError_t noalloc_scratch_address(void** out) {
  *out = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(out, g_noalloc_seg_ybar);
  if (e != cudaSuccess) *out = nullptr;
  return e;
}
}  // namespace gslm

extern "C" gslm_status gslm_apply_JT_noalloc(gslm_ctx* ctx, const gslm_cache* cache, const float* u, float* g) {
  gslm::CacheParts cp;
  gslm::ContextParts xp;
  if (ctx == nullptr || cache == nullptr || u == nullptr || g == nullptr || !gslm::cache_parts(cache, &cp) ||
      !gslm::context_parts(ctx, cp.view.fmt, &xp)) {
    gslm::set_context_error(ctx, "apply_JT_noalloc: null argument");
    return GSLM_E_INVALID;
  }
  if (cp.view.n_seg > kNoAllocMaxSegments) {
    gslm::set_context_error(ctx, "apply_JT_noalloc: the cache has more than 524288 (tile, splat) segments, "
                                 "the most this allocation-free variant holds; use gslm_apply_JT");
    return GSLM_E_INVALID;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != xp.device) {
    cudaGetLastError();
    gslm::set_context_error(ctx, "apply_JT_noalloc: the current CUDA device is not the context's device");
    return GSLM_E_INVALID;
  }
  if (xp.noalloc_scratch == nullptr) {
    gslm::set_context_error(ctx, "apply_JT_noalloc: the fixed array could not be set up when the context was created");
    return GSLM_E_CUDA;
  }
  // Every segment slot read below is written first in this call, so nothing in
  // the shared array needs clearing.
  float* seg_ybar = static_cast<float*>(xp.noalloc_scratch);
  cudaError_t e = cp.view.fmt == GSLM_CACHE_THIN ? gslm::launch_thin_apply_JT(cp.view, u, seg_ybar, xp.st)
                                                 : gslm::launch_apply_JT(cp.view, u, seg_ybar, xp.variant_JT, xp.st);
  if (e == cudaSuccess)
    e = gslm::launch_vjp(cp.params, cp.N, cp.ld, cp.cams, cp.V, cp.smooth, cp.view.slot_seg_start,
                         cp.view.slot_seg_end, cp.view.vmask, cp.view.act_off, seg_ybar, nullptr, 1.f, g, nullptr,
                         nullptr, 0.f, nullptr, nullptr, xp.st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    gslm::set_context_error(ctx, "apply_JT_noalloc: kernel launch failed");
    return GSLM_E_CUDA;
  }
  return GSLM_OK;
}
