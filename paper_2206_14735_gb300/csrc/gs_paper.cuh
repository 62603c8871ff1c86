// The paper's architecture (Sec. 3.1 Eq. SDF_MLP and Eq. COLOR_MLP, "Architecture Details"):
// layout of its decoder block and the FP32 evaluation of phi(x) on CUDA cores, shared by the
// render, smoothness, Eikonal, query, importance-sampler and lattice kernels of this model.
#pragma once
#include "gs_device.cuh"

namespace gs {
namespace paper {

constexpr int kH = 32;              // neurons per hidden layer
constexpr int kC = GS_COLOUR_FEAT;  // colour features
constexpr int kU = kC + 3;          // colour decoder input [W_beta(x), d]

// decoder block offsets in the flat parameter vector (header layout)
constexpr int A_gW1 = 0, A_gb1 = A_gW1 + kH * kZ, A_gW2 = A_gb1 + kH, A_gb2 = A_gW2 + kH * kH, A_gw3 = A_gb2 + kH,
              A_gb3 = A_gw3 + kH, A_cW1 = A_gb3 + 1, A_cb1 = A_cW1 + kH * kU, A_cW2 = A_cb1 + kH,
              A_cb2 = A_cW2 + kH * kH, A_cW3 = A_cb2 + kH, A_cb3 = A_cW3 + 3 * kH, A_kappa = A_cb3 + 3;
static_assert(A_kappa + 1 == GS_PAPER_MLP_PARAMS, "paper decoder layout");

// shared-memory copy: the matrices whose rows are read as float4 (gW1, gW2, gw3, cW2, cW3)
// start on 16-byte boundaries
constexpr int S_gW1 = 0, S_gb1 = 512, S_gW2 = 544, S_gb2 = 1568, S_gw3 = 1600, S_gb3 = 1632, S_cW1 = 1636,
              S_cb1 = 1924, S_cW2 = 1956, S_cb2 = 2980, S_cW3 = 3012, S_cb3 = 3108, S_kappa = 3111, kSm = 3112;
static_assert(S_gW2 % 4 == 0 && S_gw3 % 4 == 0 && S_cW2 % 4 == 0 && S_cW3 % 4 == 0, "float4 rows");
constexpr int kPart = 3112;  // per-CTA decoder-gradient partial row (>= GS_PAPER_MLP_PARAMS)

constexpr int kGeo = A_gb3 + 1;  // geometry decoder floats: same offsets in the flat block and in shared memory
static_assert(S_gW1 == A_gW1 && S_gb1 == A_gb1 && S_gW2 == A_gW2 && S_gb2 == A_gb2 && S_gw3 == A_gw3 &&
                  S_gb3 == A_gb3,
              "geometry decoder copied as one block");
constexpr int kGeoPad = (kGeo + 3) / 4 * 4;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// the geometry decoder (kGeo floats of the block at mlp) into shared memory sg
__device__ __forceinline__ void load_geometry_decoder(const float* __restrict__ mlp, float* sg) {
  for (int i = threadIdx.x; i < kGeoPad; i += blockDim.x) sg[i] = i < kGeo ? mlp[i] : 0.f;
}

// phi(x) = gw3 . relu(gW2 relu(gW1 z + gb1) + gb2) + gb3 with z the four levels' trilinear
// features at x (binary32 cell decisions as everywhere); sg from load_geometry_decoder; hs
// (may be nullptr) 32 floats of the calling thread's shared scratch for the hidden layer
__device__ __forceinline__ float phi_at(const GridDesc& g, const float* __restrict__ theta, const float* sg,
                                        const float x[3], float* hs = nullptr) {
  float z[kZ];
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
  float hr[kH];
  float* h = hs != nullptr ? hs : hr;  // the caller's shared scratch keeps the 32 values out of registers
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float y = sg[S_gb1 + j];
#pragma unroll
    for (int k4 = 0; k4 < 4; ++k4) {
      const float4 w = ld4(sg + S_gW1 + j * kZ + 4 * k4);
      y = fmaf(w.x, z[4 * k4], y);
      y = fmaf(w.y, z[4 * k4 + 1], y);
      y = fmaf(w.z, z[4 * k4 + 2], y);
      y = fmaf(w.w, z[4 * k4 + 3], y);
    }
    h[j] = fmaxf(y, 0.f);
  }
  float p = sg[S_gb3];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float y = sg[S_gb2 + j];
#pragma unroll
    for (int k = 0; k < kH; ++k) y = fmaf(sg[S_gW2 + j * kH + k], h[k], y);
    p = fmaf(sg[S_gw3 + j], fmaxf(y, 0.f), p);
  }
  return p;
}

}  // namespace paper
}  // namespace gs
