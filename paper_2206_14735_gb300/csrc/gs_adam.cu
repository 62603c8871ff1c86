// Dense Adam (Kingma & Ba) over the flat parameter vector with the per-group learning rates
// of Sec. 4 (grids 1e-2, decoders 1e-3).  One streaming pass reads theta, grad, m, v and
// writes theta, m, v, grad = 0 (and optionally a bfloat16 copy of the grid): 32 bytes per
// parameter, bound by HBM bandwidth.
#include <cuda_bf16.h>

#include "gs_internal.h"

namespace gs {

struct AdamArgs {
  float4 *p, *g, *m, *v;
  long long n4, ngrid4;
  float step_grid, step_mlp;  // lr / (1 - beta1^t)
  float inv_sqrt_bc2;         // 1 / sqrt(1 - beta2^t)
  float b1, b2, eps;
  uint2* bf16;                // 4 bf16 per grid float4, or null
};

__device__ __forceinline__ float adam1(float& p, float g, float& m, float& v, const AdamArgs& a, float step) {
  m = fmaf(a.b1, m, (1.0f - a.b1) * g);
  v = fmaf(a.b2, v, (1.0f - a.b2) * g * g);
  p -= step * m / (sqrtf(v) * a.inv_sqrt_bc2 + a.eps);
  return p;
}

__global__ void __launch_bounds__(256) adam_kernel(AdamArgs a) {
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n4; i += (long long)gridDim.x * blockDim.x) {
    float4 p = __ldcs(a.p + i), g = __ldcs(a.g + i), m = __ldcs(a.m + i), v = __ldcs(a.v + i);
    const bool grid = i < a.ngrid4;
    const float step = grid ? a.step_grid : a.step_mlp;
    adam1(p.x, g.x, m.x, v.x, a, step);
    adam1(p.y, g.y, m.y, v.y, a, step);
    adam1(p.z, g.z, m.z, v.z, a, step);
    adam1(p.w, g.w, m.w, v.w, a, step);
    a.p[i] = p;
    __stcs(a.m + i, m);
    __stcs(a.v + i, v);
    // the gradient is left zero for the next step; entries no sample touched are zero already
    if (g.x != 0.f || g.y != 0.f || g.z != 0.f || g.w != 0.f) __stcs(a.g + i, zero);
    if (a.bf16 != nullptr && grid) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(p.x, p.y), hi = __floats2bfloat162_rn(p.z, p.w);
      uint2 o;
      o.x = *reinterpret_cast<const unsigned*>(&lo);
      o.y = *reinterpret_cast<const unsigned*>(&hi);
      a.bf16[i] = o;
    }
  }
}

}  // namespace gs

using namespace gs;

gs_status gs_launch_adam(float* theta, float* grad, float* m, float* v, long long n, long long n_grid, int t,
                         float lr_grid, float lr_mlp, float b1, float b2, float eps, uint16_t* bf16, int num_sms,
                         cudaStream_t st) {
  AdamArgs a;
  a.p = reinterpret_cast<float4*>(theta);
  a.g = reinterpret_cast<float4*>(grad);
  a.m = reinterpret_cast<float4*>(m);
  a.v = reinterpret_cast<float4*>(v);
  a.n4 = n / 4;
  a.ngrid4 = n_grid / 4;
  const double bc1 = 1.0 - pow((double)b1, (double)t), bc2 = 1.0 - pow((double)b2, (double)t);
  a.step_grid = (float)(lr_grid / bc1);
  a.step_mlp = (float)(lr_mlp / bc1);
  a.inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
  a.b1 = b1;
  a.b2 = b2;
  a.eps = eps;
  a.bf16 = reinterpret_cast<uint2*>(bf16);
  long long blocks = (a.n4 + 255) / 256;
  const long long cap = (long long)num_sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  adam_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
