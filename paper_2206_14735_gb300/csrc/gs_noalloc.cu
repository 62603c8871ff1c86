// Allocation-free variant of gs_forward_backward.  The paper has no counterpart: this
// entry point exists for callers that may not allocate device memory -- for example code
// running inside a host framework that owns every device allocation (a plugin or custom
// operator whose memory must come from the framework's own pool), or a latency-critical
// loop that cannot afford the implicit device synchronisation of cudaMalloc.
//
// The fused render kernel needs per-CTA partial rows (loss sums and decoder-gradient sums)
// that gs_create would otherwise allocate.  Here they live in one file-scope device array
// of fixed size, which every GPU that loads this library holds until the process exits.
#include <cmath>

#include "gs_internal.h"

namespace {

// partial rows for up to 448 CTAs: the render kernel uses kRenderCtasPerSm (1) CTA per SM
// and the smoothness kernel kSmoothCtas (128), so devices with up to 320 SMs fit
constexpr int kNoAllocRows = 448;
constexpr size_t kNoAllocFloats = (size_t)kNoAllocRows * (kLossPad + kMlpPad) + 16;  // + default dloss, status

__device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];  // 3.04 MB

// Stream-ordered start of a call: the default upstream derivative (0,0,0,0,0,1) and a
// cleared status word, so neither depends on what an earlier call left in the array.
__global__ void noalloc_begin_kernel(float* default_dloss, int* status) {
  if (threadIdx.x < 8) default_dloss[threadIdx.x] = threadIdx.x == 5 ? 1.0f : 0.0f;
  if (threadIdx.x == 0) *status = 0;
}

// Stream-ordered end of a call: a device-side failure of this call (a bounded wait of the
// render kernel that ran out) turns every loss entry into NaN, because no context exists
// whose status gs_sync_status could report.
__global__ void noalloc_end_kernel(const int* status, float* loss) {
  if (threadIdx.x < 6 && *status != 0) loss[threadIdx.x] = nanf("");
}

}  // namespace

static gs_status noalloc_fail(gs_status s, const char* msg) {
  gs_set_thread_error(msg);
  return s;
}

extern "C" gs_status gs_forward_backward_noalloc(const gs_config* cfg, const float* theta, const gs_batch* batch,
                                                 const float* dloss, float* loss, float* grad, void* stream) {
  if (!cfg) return noalloc_fail(GS_ERR_INVALID_ARG, "gs_forward_backward_noalloc: cfg is NULL");
  const char* why = nullptr;
  const gs_status cs = gs_check_config(cfg, &why);
  if (cs != GS_OK) {
    gs_set_thread_error((std::string("gs_forward_backward_noalloc: ") + why).c_str());
    return cs;
  }
  if (cfg->precision != GS_PREC_FP32)
    return noalloc_fail(GS_ERR_UNSUPPORTED, "gs_forward_backward_noalloc: FP32 form only");
  if (cfg->arch != GS_ARCH_COMPACT)
    return noalloc_fail(GS_ERR_UNSUPPORTED, "gs_forward_backward_noalloc: GS_ARCH_COMPACT only");
  const int N = cfg->n_strat + cfg->n_guided;
  if (!theta || !loss || !grad || !batch) return noalloc_fail(GS_ERR_INVALID_ARG, "gs_forward_backward_noalloc: NULL argument");
  if ((reinterpret_cast<uintptr_t>(theta) & 15u) || (reinterpret_cast<uintptr_t>(grad) & 15u))
    return noalloc_fail(GS_ERR_ALIGN, "gs_forward_backward_noalloc: theta and grad must be 16-byte aligned");
  if (batch->R < 0 || batch->R > cfg->max_rays || batch->N != N || batch->P < 0 || batch->P > cfg->max_smooth ||
      !batch->counts)
    return noalloc_fail(GS_ERR_SHAPE, "gs_forward_backward_noalloc: batch sizes outside the configuration");
  if (batch->R > 0 && (!batch->origin || !batch->dir || !batch->rgb || !batch->depth || !batch->t || !batch->cls))
    return noalloc_fail(GS_ERR_INVALID_ARG, "gs_forward_backward_noalloc: batch ray array is NULL");
  if (batch->P > 0 && (!batch->xs || !batch->eps || !batch->valid))
    return noalloc_fail(GS_ERR_INVALID_ARG, "gs_forward_backward_noalloc: batch smoothness array is NULL");
  if (batch->eik && (reinterpret_cast<uintptr_t>(batch->eik) & 15u))
    return noalloc_fail(GS_ERR_ALIGN, "gs_forward_backward_noalloc: batch eik is not 16-byte aligned");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return noalloc_fail(GS_ERR_CUDA, "gs_forward_backward_noalloc: no usable CUDA device");
  if (kRenderCtasPerSm * sms + kSmoothCtas > kNoAllocRows)
    return noalloc_fail(GS_ERR_UNSUPPORTED,
                        "gs_forward_backward_noalloc: the static scratch holds partial rows for at most 320 SMs");
  // The array's device address on the current device (its host-side name is only a stand-in).
  // Resolved on every call, so nothing cached can outlive a cudaDeviceReset; the first call
  // on a device may also load the module.
  float* scratch = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&scratch), g_noalloc_scratch) != cudaSuccess || !scratch)
    return noalloc_fail(GS_ERR_CUDA, "gs_forward_backward_noalloc: could not resolve the static scratch array");

  // a context on the stack whose workspace points into the static array (no allocation)
  gs_ctx c;
  c.cfg = *cfg;
  long long off = 0;
  for (int l = 0; l < GS_LEVELS; ++l) {
    for (int a = 0; a < 3; ++a) c.grid.dims[l][a] = cfg->dims[l][a];
    c.grid.voxel[l] = cfg->voxel[l];
    c.grid.inv_voxel[l] = 1.0f / cfg->voxel[l];
    c.grid.off[l] = off;
    off += (long long)cfg->dims[l][0] * cfg->dims[l][1] * cfg->dims[l][2] * GS_FEAT;
  }
  for (int a = 0; a < 3; ++a) c.grid.origin[a] = cfg->origin[a];
  c.grid.n_grid = off;
  c.device = dev;
  c.num_sms = sms;
  c.render_ctas = kRenderCtasPerSm * sms;
  c.max_n = N;
  c.loss_part = scratch;
  c.mlp_part = scratch + (size_t)kNoAllocRows * kLossPad;
  c.default_dloss = scratch + (size_t)kNoAllocRows * (kLossPad + kMlpPad);
  c.status = reinterpret_cast<int*>(c.default_dloss + 8);  // device-side check word
  const float* dl = dloss ? dloss : c.default_dloss;
  cudaStream_t st = (cudaStream_t)stream;
  noalloc_begin_kernel<<<1, 32, 0, st>>>(c.default_dloss, c.status);
  if (cudaGetLastError() != cudaSuccess)
    return noalloc_fail(GS_ERR_CUDA, "gs_forward_backward_noalloc: launch failed");
  if (batch->R > 0 && gs_launch_render(&c, theta, nullptr, batch, dl, grad, nullptr, nullptr, nullptr, 3, st) != GS_OK)
    return noalloc_fail(GS_ERR_CUDA, "gs_forward_backward_noalloc: render launch failed");
  if (gs_launch_smooth(&c, theta, batch, dl, grad, 3, st) != GS_OK)
    return noalloc_fail(GS_ERR_CUDA, "gs_forward_backward_noalloc: smoothness launch failed");
  // combine the rows written by this call: render CTAs (if any rays), then smoothness CTAs
  c.n_parts = (batch->R > 0 ? c.render_ctas : 0) + (batch->P > 0 ? kSmoothCtas : 0);
  if (batch->R == 0) {
    c.loss_part += (size_t)c.render_ctas * kLossPad;
    c.mlp_part += (size_t)c.render_ctas * kMlpPad;
  }
  if (gs_launch_finalize(&c, batch, loss, grad, 3, st) != GS_OK)
    return noalloc_fail(GS_ERR_CUDA, "gs_forward_backward_noalloc: finalize launch failed");
  noalloc_end_kernel<<<1, 32, 0, st>>>(c.status, loss);
  if (cudaGetLastError() != cudaSuccess)
    return noalloc_fail(GS_ERR_CUDA, "gs_forward_backward_noalloc: launch failed");
  return GS_OK;
}
