// Device-side building blocks of the GO-Surf step shared by the kernels of this library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gosurf.h"

namespace gs {

constexpr int kLevels = GS_LEVELS;
constexpr int kFeat = GS_FEAT;
constexpr int kZ = kLevels * kFeat;  // 16-d geometry feature (Sec. 3.1)
constexpr int kH1 = 32, kOut = 16, kHF = 15, kH2 = 32, kRGB = 3;

// decoder block offsets inside the flat parameter vector (header layout)
constexpr int oW1 = 0, ob1 = oW1 + kH1 * kZ, oW2 = ob1 + kH1, ob2 = oW2 + kOut * kH1, oW3 = ob2 + kOut,
              ob3 = oW3 + kH2 * kHF, oW4 = ob3 + kH2, ob4 = oW4 + kRGB * kH2, oKappa = ob4 + kRGB;
static_assert(oKappa + 1 == GS_MLP_PARAMS, "decoder layout");

// Shared-memory copy of the decoders: W3 is padded to 32x16 so every row is float4 aligned.
constexpr int sW1 = 0, sb1 = 512, sW2 = 544, sb2 = 1056, sW3 = 1072, sb3 = 1584, sW4 = 1616, sb4 = 1712,
              sKappa = 1716, kSmemMlp = 1720;

enum { CLS_NONE = GS_CLS_NONE, CLS_TR = GS_CLS_TR, CLS_FS = GS_CLS_FS };

struct GridDesc {
  int dims[kLevels][3];
  float voxel[kLevels];
  float inv_voxel[kLevels];
  float origin[3];
  long long off[kLevels];  // float offset of each level in theta
  long long n_grid;
};

// ------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) keyed counter generator
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
__device__ __forceinline__ uint64_t draw_prefix(uint64_t seed, uint64_t stream, uint64_t step, uint64_t index) {
  return sm64(sm64(sm64(sm64(seed) ^ stream) ^ step) ^ index);
}
__device__ __forceinline__ uint64_t draw_slot(uint64_t prefix, uint64_t slot) { return sm64(prefix ^ slot); }
// 24 random bits scaled by 2^-24: an exact binary32 value in [0, 1)
__device__ __forceinline__ float unif24(uint64_t h) { return __fmul_rn((float)(uint32_t)(h >> 40), 0x1p-24f); }

// ------------------------------------------------------------------------------------
// cells of the multi-level grid (Sec. 3.1; Supp. Sec. 1)
// ------------------------------------------------------------------------------------
struct Cell {
  long long vtx;  // flat index of the base vertex (x fastest)
  float f[3];     // in-cell coordinates
  unsigned clamped;  // bit a set when axis a was clamped to the grid box
  int idx[3];     // base vertex per axis
};

// Cell of x at level l: u = (x - origin) / v decided in binary32 (round-to-nearest),
// clamped to [0, n-1], base = min(floor(u), n-2), f = u - base.
__device__ __forceinline__ Cell locate(const GridDesc& g, int l, const float x[3]) {
  Cell c;
  c.clamped = 0;
  int idx[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = g.dims[l][a];
    float u = __fdiv_rn(__fsub_rn(x[a], g.origin[a]), g.voxel[l]);
    if (u < 0.0f) {
      u = 0.0f;
      c.clamped |= 1u << a;
    } else if (u > (float)(n - 1)) {
      u = (float)(n - 1);
      c.clamped |= 1u << a;
    }
    int i = (int)floorf(u);
    i = min(i, n - 2);
    idx[a] = i;
    c.f[a] = __fsub_rn(u, (float)i);
  }
  c.vtx = ((long long)idx[2] * g.dims[l][1] + idx[1]) * g.dims[l][0] + idx[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) c.idx[a] = idx[a];
  return c;
}

// corner c = 4*bx + 2*by + bz  ->  vertex offset
__device__ __forceinline__ long long corner_offset(const GridDesc& g, int l, int c) {
  return ((c >> 2) & 1) + ((c >> 1) & 1) * (long long)g.dims[l][0] +
         (c & 1) * (long long)g.dims[l][0] * g.dims[l][1];
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4scale(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ void f4fma(float4& acc, float s, float4 b) {
  acc.x = fmaf(s, b.x, acc.x);
  acc.y = fmaf(s, b.y, acc.y);
  acc.z = fmaf(s, b.z, acc.z);
  acc.w = fmaf(s, b.w, acc.w);
}

// trilinear weights of the 8 corners
// Sum over the partial rows p = w, w + 8, ... < nparts of part[p stride + i] (a column of
// per-CTA partial rows): eight loads in flight, four partial sums combined in a fixed order,
// so the result does not depend on timing.
__device__ __forceinline__ float column_sum8(const float* __restrict__ part, size_t stride, int i, int w,
                                            int nparts) {
  float s[4] = {0.f, 0.f, 0.f, 0.f};
  int k = 0;
#pragma unroll 8
  for (int p = w; p < nparts; p += 8, ++k) s[k & 3] += part[(size_t)p * stride + i];
  return (s[0] + s[1]) + (s[2] + s[3]);
}

__device__ __forceinline__ void corner_weights(const float f[3], float w[8]) {
  const float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
  const float w00 = gx * gy, w01 = gx * f[1], w10 = f[0] * gy, w11 = f[0] * f[1];
  w[0] = w00 * gz;
  w[1] = w00 * f[2];
  w[2] = w01 * gz;
  w[3] = w01 * f[2];
  w[4] = w10 * gz;
  w[5] = w10 * f[2];
  w[6] = w11 * gz;
  w[7] = w11 * f[2];
}

// d w_c / d f_a, zero on clamped axes (Supp. Eq. coeff_jacobian)
__device__ __forceinline__ void corner_weight_grads(const float f[3], unsigned clamped, float dw[8][3]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int bx = (c >> 2) & 1, by = (c >> 1) & 1, bz = c & 1;
    const float wx = bx ? f[0] : 1.0f - f[0], wy = by ? f[1] : 1.0f - f[1], wz = bz ? f[2] : 1.0f - f[2];
    const float sx = bx ? 1.0f : -1.0f, sy = by ? 1.0f : -1.0f, sz = bz ? 1.0f : -1.0f;
    dw[c][0] = (clamped & 1u) ? 0.0f : sx * wy * wz;
    dw[c][1] = (clamped & 2u) ? 0.0f : wx * sy * wz;
    dw[c][2] = (clamped & 4u) ? 0.0f : wx * wy * sz;
  }
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// binary32 sample position x = o + d r (no contraction)
__device__ __forceinline__ void sample_pos(const float o[3], const float r[3], float t, float x[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[a], __fmul_rn(t, r[a]));
}

// z = [f_0(x), ..., f_3(x)]: the four levels' trilinear features, coarse to fine
__device__ __forceinline__ void grid_z(const GridDesc& g, const float* __restrict__ theta, const float x[3],
                                       float (&z)[kZ]) {
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell c = locate(g, l, x);
    float w[8];
    corner_weights(c.f, w);
    const float4* lv = reinterpret_cast<const float4*>(theta + g.off[l]);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f4fma(acc, w[k], __ldg(lv + c.vtx + corner_offset(g, l, k)));
    z[4 * l] = acc.x;
    z[4 * l + 1] = acc.y;
    z[4 * l + 2] = acc.z;
    z[4 * l + 3] = acc.w;
  }
}

// phi(x) in FP32 on CUDA cores: trilinear features of the 4 levels, then the SDF decoder's
// first output; sm holds W1 at sW1, b1 at sb1, row 0 of W2 at sW2 and b2[0] at sb2
__device__ __forceinline__ float sdf_at(const GridDesc& g, const float* __restrict__ theta, const float* sm,
                                        const float x[3]) {
  float z[kZ];
  grid_z(g, theta, x, z);
  float phi = sm[sb2];
#pragma unroll 8
  for (int j = 0; j < kH1; ++j) {
    float s = sm[sb1 + j];
#pragma unroll
    for (int k = 0; k < kZ; ++k) s = fmaf(sm[sW1 + j * 16 + k], z[k], s);
    phi = fmaf(sm[sW2 + j], fmaxf(s, 0.f), phi);
  }
  return phi;
}

// d z_l / d x (4 features x 3 axes) at level l, and the cell (for the scatter)
__device__ __forceinline__ Cell level_jacobian(const GridDesc& g, const float* __restrict__ theta, int l,
                                               const float y[3], float4 (&dl)[3], float (&dw)[8][3]) {
  const Cell c = locate(g, l, y);
  corner_weight_grads(c.f, c.clamped, dw);
  const float4* base = reinterpret_cast<const float4*>(theta + g.off[l]);
  dl[0] = dl[1] = dl[2] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 v = __ldg(base + c.vtx + corner_offset(g, l, k));
    f4fma(dl[0], dw[k][0], v);
    f4fma(dl[1], dw[k][1], v);
    f4fma(dl[2], dw[k][2], v);
  }
  const float iv = g.inv_voxel[l];
#pragma unroll
  for (int a = 0; a < 3; ++a) dl[a] = f4scale(dl[a], iv);
  return c;
}

// warp reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace gs
