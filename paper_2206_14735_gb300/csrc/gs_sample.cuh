// Ray generation and sample classes shared by the plain sampler and the proposal sampler
// (Sec. 3.2-3.3), in explicitly rounded binary32.
#pragma once
#include "gs_internal.h"

namespace gs {

struct FramesDev {
  int F, H, W;
  const uint8_t* rgb;
  const float* depth;
  const float* c2w;
  float fx, fy, cx, cy;
};

// pixel -> (o, r, I, D); r has unit camera-z so the ray parameter is z-depth
__device__ __forceinline__ void pixel_ray(const FramesDev& fr, long long pix, float o[3], float r[3], float rgb[3],
                                          float* D) {
  const long long hw = (long long)fr.H * fr.W;
  const long long f = pix / hw, rem = pix - f * hw;
  const int v = (int)(rem / fr.W), u = (int)(rem - (long long)v * fr.W);
  const float dx = __fdiv_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), fr.cx), fr.fx);
  const float dy = __fdiv_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), fr.cy), fr.fy);
  const float* P = fr.c2w + 12 * f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[a] = __fadd_rn(__fadd_rn(__fmul_rn(P[4 * a + 0], dx), __fmul_rn(P[4 * a + 1], dy)), P[4 * a + 2]);
    o[a] = P[4 * a + 3];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) rgb[j] = __fdiv_rn((float)fr.rgb[3 * pix + j], 255.0f);
  *D = fr.depth[pix];
}

__device__ __forceinline__ int sample_class(float D, float t, float trunc) {
  if (!(D > 0.0f)) return CLS_NONE;
  const float b = __fsub_rn(D, t);
  if (fabsf(b) <= trunc) return CLS_TR;
  if (b > trunc) return CLS_FS;
  return CLS_NONE;
}

__device__ __forceinline__ void block_add_counts(int* counts, int a, int b, int c) {
  a = __reduce_add_sync(0xffffffffu, a);
  b = __reduce_add_sync(0xffffffffu, b);
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) {
    if (a) atomicAdd(counts + 0, a);
    if (b) atomicAdd(counts + 1, b);
    if (c) atomicAdd(counts + 2, c);
  }
}

}  // namespace gs
