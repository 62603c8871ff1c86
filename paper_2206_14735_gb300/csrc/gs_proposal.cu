// Learned proposal sampler (an addition to the method: it cuts the samples per ray).
//
// [near, far] is split into 32 equal bins, one per lane of a warp.  For the centre of its
// bin a lane evaluates the proposal network on the two coarsest grid levels' features and
// the unit ray direction; a warp softmax gives the ray's bin distribution p.  Sampling
// inverts the CDF of the mixture 0.95 p + 0.05 / 32 at stratified targets (binary32 with
// explicit rounding, bit-reproducible for a given p).  Training bins the main model's
// rendering weights per ray and back-propagates the cross entropy through the network.
#include <algorithm>

#include <cuda_bf16.h>

#include "gs_sample.cuh"
#include "gs_tc.cuh"

namespace gs {

constexpr int kPB = GS_PROP_BINS;  // bins = lanes
constexpr int kPIn = 11, kPH = 32;
constexpr int pW1 = 0, pb1 = pW1 + kPH * kPIn, pW2 = pb1 + kPH, pb2 = pW2 + kPH * kPH, pw3 = pb2 + kPH,
              pb3 = pw3 + kPH;
static_assert(pb3 + 1 == GS_PROP_PARAMS, "proposal parameter layout");
static_assert(kPB == 32, "one lane per bin");
constexpr int kPropWarps = 4;
constexpr int kPropPad = 1476;                   // shared copy of the parameters (padded)
constexpr int kPropPart = 1480;                  // partial row: gradient | loss sum | rays used
constexpr int kRow = 140;                        // staged bin row: (pad) | a1 | dy1 | a2 | u | dl
constexpr int rA1 = 32, rDy1 = 64, rA2 = 96, rU = 128, rDl = 139;
constexpr float kMix = 0.05f / 32.0f;            // exact (power-of-two divisor)

__device__ __forceinline__ float prop_width(float near_m, float far_m) {
  return __fdiv_rn(__fsub_rn(far_m, near_m), (float)kPB);
}
__device__ __forceinline__ float prop_edge(float near_m, float width, int b) {
  return __fadd_rn(near_m, __fmul_rn((float)b, width));
}

// network input of this lane's bin: features of levels 0 and 1 at the bin centre, unit direction
__device__ __forceinline__ void prop_input(const GridDesc& g, const float* __restrict__ theta, const float o[3],
                                           const float r[3], float tc, float u[kPIn]) {
  float x[3];
  sample_pos(o, r, tc, x);
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const Cell c = locate(g, l, x);
    float w[8];
    corner_weights(c.f, w);
    const float4* base = reinterpret_cast<const float4*>(theta + g.off[l]);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f4fma(acc, w[k], __ldg(base + c.vtx + corner_offset(g, l, k)));
    u[4 * l] = acc.x;
    u[4 * l + 1] = acc.y;
    u[4 * l + 2] = acc.z;
    u[4 * l + 3] = acc.w;
  }
  const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[0], r[0]), __fmul_rn(r[1], r[1])), __fmul_rn(r[2], r[2])));
#pragma unroll
  for (int a = 0; a < 3; ++a) u[8 + a] = __fdiv_rn(r[a], n);
}

// logit of one bin; a1, a2 = the two ReLU layers' outputs
__device__ __forceinline__ float prop_mlp(const float* sq, const float u[kPIn], float a1[kPH], float a2[kPH]) {
#pragma unroll
  for (int j = 0; j < kPH; ++j) {
    float s = sq[pb1 + j];
#pragma unroll
    for (int k = 0; k < kPIn; ++k) s = fmaf(sq[pW1 + j * kPIn + k], u[k], s);
    a1[j] = fmaxf(s, 0.f);
  }
#pragma unroll
  for (int j = 0; j < kPH; ++j) {
    float s = sq[pb2 + j];
#pragma unroll
    for (int k = 0; k < kPH; ++k) s = fmaf(sq[pW2 + j * kPH + k], a1[k], s);
    a2[j] = fmaxf(s, 0.f);
  }
  float l = sq[pb3];
#pragma unroll
  for (int k = 0; k < kPH; ++k) l = fmaf(sq[pw3 + k], a2[k], l);
  return l;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// sum that every lane sees with the same rounding (lane 0's butterfly result)
__device__ __forceinline__ float warp_sum_bcast(float v) { return __shfl_sync(0xffffffffu, warp_sum(v), 0); }

// --------------------------------------------------------------------------------------
// sampling
// --------------------------------------------------------------------------------------
struct PropSampleArgs {
  FramesDev fr;
  GridDesc g;
  const float* theta;
  const float* q;
  const float* pdf_in;
  float* pdf_out;
  uint64_t seed;
  uint32_t step;
  int R, N, Ng;
  float near_m, far_m, guide_half, trunc;
  long long* pix;
  float *o, *r, *rgb, *D, *t;
  uint8_t* cls;
  int* counts;
};

// Given ray i's bin distribution pb (lane = bin): the inverse-CDF draws of the mixture
// 0.95 p + 0.05 / 32 at stratified targets and the depth-guided samples, sorted, with their
// classes (the whole warp calls it)
__device__ __forceinline__ void prop_draw(const PropSampleArgs& a, int i, float pb, float D, float width, int lane,
                                          int& ntr, int& nfs) {
  if (a.pdf_out != nullptr) a.pdf_out[(size_t)i * kPB + lane] = pb;
  // mixture and its running sums in bin order
  const float pp = __fadd_rn(__fmul_rn(0.95f, pb), kMix);
  float C = 0.0f;
#pragma unroll
  for (int j = 0; j < kPB; ++j) {
    const float v = __shfl_sync(0xffffffffu, pp, j);
    if (j <= lane) C = __fadd_rn(C, v);
  }
  const float total = __shfl_sync(0xffffffffu, C, kPB - 1);
  const int ng = (D > 0.0f && a.Ng > 0) ? a.Ng : 0;
  const int K = a.N - ng;
  const uint64_t pre2 = draw_prefix(a.seed, 2, a.step, (uint64_t)i);
  // lane k < K: inverse-CDF draw k; K <= k < N: guided sample k - K; others: +inf (sorted last)
  float target = 0.0f;
  if (lane < K) {
    const float uu = unif24(draw_slot(pre2, 1 + (uint64_t)lane));
    target = __fmul_rn(__fdiv_rn(__fadd_rn((float)lane, uu), (float)K), total);
  }
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < kPB; ++j) cnt += (__shfl_sync(0xffffffffu, C, j) <= target) ? 1 : 0;
  const int b = min(cnt, kPB - 1);
  float lo = __shfl_sync(0xffffffffu, C, max(b - 1, 0));
  if (b == 0) lo = 0.0f;
  const float ppb = __shfl_sync(0xffffffffu, pp, b);
  float tv = INFINITY;
  if (lane < K) {
    const float e0 = prop_edge(a.near_m, width, b), e1 = prop_edge(a.near_m, width, b + 1);
    const float x = __fadd_rn(e0, __fmul_rn(__fdiv_rn(__fsub_rn(target, lo), ppb), width));
    tv = fminf(fmaxf(x, e0), e1);
  } else if (lane < a.N) {
    const int j = lane - K;
    const float uu = unif24(draw_slot(pre2, 1 + (uint64_t)K + (uint64_t)j));
    const float gstep = __fdiv_rn(__fmul_rn(2.0f, a.guide_half), (float)ng);
    const float g0 = __fsub_rn(D, a.guide_half);
    tv = __fadd_rn(g0, __fmul_rn(__fadd_rn((float)j, uu), gstep));
  }
  // bitonic sort of the warp's 32 values, ascending
#pragma unroll
  for (int k2 = 2; k2 <= 32; k2 <<= 1)
#pragma unroll
    for (int j = k2 >> 1; j > 0; j >>= 1) {
      const float other = __shfl_xor_sync(0xffffffffu, tv, j);
      const bool asc = (lane & k2) == 0, low = (lane & j) == 0;
      tv = (low == asc) ? fminf(tv, other) : fmaxf(tv, other);
    }
  if (lane < a.N) {
    a.t[(size_t)i * a.N + lane] = tv;
    const int c = sample_class(D, tv, a.trunc);
    a.cls[(size_t)i * a.N + lane] = (uint8_t)c;
    ntr += c == CLS_TR;
    nfs += c == CLS_FS;
  }
}

__global__ void __launch_bounds__(kPropWarps * 32) prop_sample_kernel(PropSampleArgs a) {
  __shared__ __align__(16) float sq[kPropPad];
  if (a.pdf_in == nullptr)
    for (int i = threadIdx.x; i < GS_PROP_PARAMS; i += blockDim.x) sq[i] = a.q[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float width = prop_width(a.near_m, a.far_m);
  const long long npix = (long long)a.fr.F * a.fr.H * a.fr.W;
  int nd = 0, ntr = 0, nfs = 0;
  for (int i = blockIdx.x * kPropWarps + warp; i < a.R; i += gridDim.x * kPropWarps) {
    // the ray: the plain sampler's draw for ray i
    const uint64_t pre = draw_prefix(a.seed, 0, a.step, (uint64_t)i);
    const long long px = (long long)(draw_slot(pre, 0) % (uint64_t)npix);
    float o[3], r[3], rgb[3], D;
    pixel_ray(a.fr, px, o, r, rgb, &D);
    if (lane == 0) {
      a.pix[i] = px;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        a.o[3 * i + k] = o[k];
        a.r[3 * i + k] = r[k];
        a.rgb[3 * i + k] = rgb[k];
      }
      a.D[i] = D;
      nd += D > 0.0f;
    }
    // bin distribution p (lane = bin)
    float pb;
    if (a.pdf_in != nullptr) {
      pb = a.pdf_in[(size_t)i * kPB + lane];
    } else {
      const float tc = __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)lane, 0.5f), width));
      float u[kPIn], a1[kPH], a2[kPH];
      prop_input(a.g, a.theta, o, r, tc, u);
      const float l = prop_mlp(sq, u, a1, a2);
      const float e = expf(l - warp_max(l));
      pb = __fdiv_rn(e, warp_sum_bcast(e));
    }
    prop_draw(a, i, pb, D, width, lane, ntr, nfs);
  }
  block_add_counts(a.counts, nd, ntr, nfs);
}

// --------------------------------------------------------------------------------------
// training: binned weights -> cross entropy -> gradient of the network
// --------------------------------------------------------------------------------------
struct PropBwdArgs {
  GridDesc g;
  const float* theta;
  const float* q;
  int R, N;
  const float *o, *r, *t, *w;
  float near_m, far_m;
  float* part;  // [gridDim.x][kPropPart]
};

__global__ void __launch_bounds__(kPropWarps * 32, 1) prop_backward_kernel(PropBwdArgs a) {
  extern __shared__ __align__(16) float dsm[];
  float* sq = dsm;                                  // [kPropPad]
  float* hist = sq + kPropPad;                      // [kPropWarps][32]
  float* wacc = hist + kPropWarps * 32;             // [kPropWarps][kPropPart], transposed matrix blocks
  float* stage = wacc + kPropWarps * kPropPart;     // [kPropWarps][32][kRow]
  for (int i = threadIdx.x; i < kPropPad; i += blockDim.x) sq[i] = i < GS_PROP_PARAMS ? a.q[i] : 0.f;
  for (int i = threadIdx.x; i < kPropWarps * kPropPart; i += blockDim.x) wacc[i] = 0.f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* hw = hist + warp * 32;
  float* st = stage + (size_t)warp * 32 * kRow;
  // this warp's accumulator: dW2 and dW1 stored column-major ([k][j], lane j owns row j) so
  // that the lanes' updates fall in distinct banks; then b1, b2, w3, b3, loss, rays
  float* aW2 = wacc + warp * kPropPart;
  float* aW1 = aW2 + kPH * kPH;
  float* aB = aW1 + kPIn * kPH;  // b1[32] | b2[32] | w3[32] | b3 | loss | rays
  const float width = prop_width(a.near_m, a.far_m);
  const float tc = __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)lane, 0.5f), width));

  for (int i = blockIdx.x * kPropWarps + warp; i < a.R; i += gridDim.x * kPropWarps) {
    hw[lane] = 0.f;
    __syncwarp();
    for (int s = lane; s < a.N; s += 32) {
      const float tt = a.t[(size_t)i * a.N + s];
      const int b = min(max((int)floorf(__fdiv_rn(__fsub_rn(tt, a.near_m), width)), 0), kPB - 1);
      atomicAdd(hw + b, a.w[(size_t)i * a.N + s]);
    }
    __syncwarp();
    const float h = hw[lane];
    const float S = warp_sum_bcast(h);
    if (!(S >= 1e-3f)) continue;  // too little weight on this ray to be a target
    float* row = st + lane * kRow;
    {  // forward of this lane's bin and the adjoint dl = p - hh; stage a1, a2, u, dl, dy1
      const float o[3] = {a.o[3 * i], a.o[3 * i + 1], a.o[3 * i + 2]};
      const float r[3] = {a.r[3 * i], a.r[3 * i + 1], a.r[3 * i + 2]};
      float u[kPIn], a1[kPH], a2[kPH];
      prop_input(a.g, a.theta, o, r, tc, u);
      const float l = prop_mlp(sq, u, a1, a2);
      const float mx = warp_max(l);
      const float e = expf(l - mx);
      const float se = warp_sum_bcast(e);
      const float p = e / se, logp = l - mx - logf(se);
      const float hh = h / S;
      const float ce = -warp_sum_bcast(hh * logp);
      const float dl = p - hh;
      if (lane == 0) {
        aB[3 * kPH + 1] += ce;
        aB[3 * kPH + 2] += 1.f;
      }
#pragma unroll
      for (int k = 0; k < kPH; ++k) {
        row[rA1 + k] = a1[k];
        row[rA2 + k] = a2[k];
      }
#pragma unroll
      for (int k = 0; k < kPIn; ++k) row[rU + k] = u[k];
      row[rDl] = dl;
#pragma unroll 4
      for (int k = 0; k < kPH; ++k) {  // dy1_k = [a1_k > 0] sum_j W2[j][k] dy2_j, dy2_j = [a2_j > 0] dl w3_j
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kPH; ++j) s = fmaf(sq[pW2 + j * kPH + k], row[rA2 + j] > 0.f ? dl * sq[pw3 + j] : 0.f, s);
        row[rDy1 + k] = row[rA1 + k] > 0.f ? s : 0.f;
      }
    }
    __syncwarp();
    {  // sums over the warp's 32 bin rows: lane j owns row j of dW2 and dW1, entry j of b1, b2, w3
      const float w3j = sq[pw3 + lane];
      float gW2[kPH], gW1[kPIn], gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
#pragma unroll
      for (int k = 0; k < kPH; ++k) gW2[k] = 0.f;
#pragma unroll
      for (int k = 0; k < kPIn; ++k) gW1[k] = 0.f;
#pragma unroll 2
      for (int s2 = 0; s2 < 32; ++s2) {
        const float* rw = st + s2 * kRow;
        const float dl = rw[rDl], a2j = rw[rA2 + lane];
        const float d2 = a2j > 0.f ? dl * w3j : 0.f, d1 = rw[rDy1 + lane];
#pragma unroll
        for (int k = 0; k < kPH; ++k) gW2[k] = fmaf(d2, rw[rA1 + k], gW2[k]);
#pragma unroll
        for (int k = 0; k < kPIn; ++k) gW1[k] = fmaf(d1, rw[rU + k], gW1[k]);
        gb2 += d2;
        gb1 += d1;
        gw3 = fmaf(dl, a2j, gw3);
        gb3 += dl;
      }
#pragma unroll
      for (int k = 0; k < kPH; ++k) aW2[k * kPH + lane] += gW2[k];
#pragma unroll
      for (int k = 0; k < kPIn; ++k) aW1[k * kPH + lane] += gW1[k];
      aB[lane] += gb1;
      aB[kPH + lane] += gb2;
      aB[2 * kPH + lane] += gw3;
      if (lane == 0) aB[3 * kPH] += gb3;
    }
    __syncwarp();
  }
  __syncthreads();
  // block row in the parameter layout: sum of the warps' accumulators
  for (int e = threadIdx.x; e < kPropPart; e += blockDim.x) {
    int src;  // position of parameter e in a warp accumulator
    if (e < pb1) src = kPH * kPH + (e % kPIn) * kPH + e / kPIn;              // W1[j][k] at aW1[k][j]
    else if (e < pW2) src = kPH * kPH + kPIn * kPH + (e - pb1);              // b1
    else if (e < pb2) src = ((e - pW2) % kPH) * kPH + (e - pW2) / kPH;       // W2[j][k] at aW2[k][j]
    else if (e < pw3) src = kPH * kPH + kPIn * kPH + kPH + (e - pb2);        // b2
    else if (e < pb3) src = kPH * kPH + kPIn * kPH + 2 * kPH + (e - pw3);    // w3
    else if (e < GS_PROP_PARAMS + 2) src = kPH * kPH + kPIn * kPH + 3 * kPH + (e - pb3);  // b3, loss, rays
    else src = -1;
    float v = 0.f;
    if (src >= 0)
#pragma unroll
      for (int q = 0; q < kPropWarps; ++q) v += wacc[q * kPropPart + src];
    a.part[(size_t)blockIdx.x * kPropPart + e] = v;
  }
}

// the partial rows summed in a fixed order (block b: entries [32 b, 32 b + 32), warp w rows
// w, w + 8, ..., then the 8 warps' sums in order); scaled by 1 / (rays used)
__global__ void __launch_bounds__(256) prop_finalize_kernel(const float* part, int rows, float* grad, float* ce) {
  __shared__ float sp[8][33], sn[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  sp[wid][lane] = i < GS_PROP_PARAMS + 1 ? column_sum8(part, kPropPart, i, wid, rows) : 0.f;
  const float nw = column_sum8(part, kPropPart, GS_PROP_PARAMS + 1, wid, rows);  // rays used
  if (lane == 0) sn[wid] = nw;
  __syncthreads();
  if (wid == 0 && i < GS_PROP_PARAMS + 1) {
    float s = 0.f, n = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      s += sp[k][lane];
      n += sn[k];
    }
    if (i < GS_PROP_PARAMS) {
      if (n > 0.f) grad[i] += s / n;
    } else if (ce != nullptr) {
      ce[0] = n > 0.f ? s / n : 0.f;
      ce[1] = n;
    }
  }
}

// --------------------------------------------------------------------------------------
// BF16 form: the network's two hidden layers, and in training the first layer's adjoint, as
// tcgen05 products on the tensor core (bfloat16 operands, FP32 accumulation).  A CTA is one
// tile group of 4 warps; warp w takes one ray and its lanes the 32 bins, so the group's four
// rays fill the 128 rows of an M = 128 tile.  Biases, ReLUs, the output layer (32 -> 1), the
// softmax, the cross entropy and the weight-gradient sums stay on CUDA cores in FP32.
// --------------------------------------------------------------------------------------
constexpr int kTcK1 = 16;                                              // layer-1 K: 11 inputs padded
constexpr uint32_t kTcA = 128u * 32u * 2u;                             // A tile, K <= 32
constexpr uint32_t kTcW1 = 32u * kTcK1 * 2u, kTcW2 = 32u * 32u * 2u;   // weight tiles
constexpr uint32_t kTcWeights = kTcW1 + 2u * kTcW2;                    // W1, W2, W2^T
constexpr int kTcF = 100;                                              // FP32: b1 | b2 | w3 | b3
constexpr uint32_t kPropMbarLimit = 1u << 20;                          // bounded MMA wait (~2 s)

// a row of K bfloat16 values (round to nearest even) of a K-major no-swizzle tile
template <int K>
__device__ __forceinline__ void tc_store_row(uint8_t* tile, int row, const float* v) {
  constexpr uint32_t sbo = (uint32_t)(K * 2 / 16) * 128u;
#pragma unroll
  for (int c = 0; c < K / 8; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[8 * c + 2 * q], v[8 * c + 2 * q + 1]);
      w[q] = *reinterpret_cast<const uint32_t*>(&b);
    }
    *reinterpret_cast<uint4*>(tile + tc::core_offset((uint32_t)row, (uint32_t)c, 128u, sbo)) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}
// one element (n, k) of a K-major weight tile [N][K]
template <int K>
__device__ __forceinline__ void tc_store_w(uint8_t* tile, int n, int k, float v) {
  constexpr uint32_t sbo = (uint32_t)(K * 2 / 16) * 128u;
  *reinterpret_cast<__nv_bfloat16*>(tile + tc::core_offset((uint32_t)n, (uint32_t)(k / 8), 128u, sbo) +
                                    (uint32_t)(k % 8) * 2u) = __float2bfloat16_rn(v);
}
// the rows are written; thread 0 issues D[128][32] = A[128][K] B[32][K]^T and waits (bounded),
// then every thread may read its row.  false (for every thread) if the MMA never completed.
template <int K>
__device__ __forceinline__ bool tc_phase(uint32_t tcol, const uint8_t* A, const uint8_t* B, uint64_t* mbar,
                                         uint32_t& phase, int* abort) {
  constexpr uint32_t sbo = (uint32_t)(K * 2 / 16) * 128u;
  constexpr uint32_t idesc = tc::instr_desc(tc::KIND_BF16, 128, 32);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < K / 16; ++st) {
      const uint32_t off = (uint32_t)st * 256u;  // two 16-byte core-matrix columns per K step
      tc::mma_bf16(tcol, tc::smem_desc(tc::smem_u32(A) + off, 128u, sbo), tc::smem_desc(tc::smem_u32(B) + off, 128u, sbo),
                   idesc, st > 0 ? 1u : 0u);
    }
    tc::mma_commit(mbar);
    if (!tc::mbar_wait(mbar, phase, kPropMbarLimit)) *reinterpret_cast<volatile int*>(abort) = 1;
  }
  phase ^= 1u;
  __syncthreads();
  tc::fence_after_sync();
  return *reinterpret_cast<volatile int*>(abort) == 0;
}

// weight tiles (W1 [32][16], W2 [32][32] and, for training, W2^T) and the FP32 vectors
__device__ __forceinline__ void tc_load_weights(const float* __restrict__ q, uint8_t* tW1, uint8_t* tW2, uint8_t* tW2T,
                                                float* fb) {
  for (int e = threadIdx.x; e < 32 * kTcK1; e += blockDim.x) {
    const int n = e / kTcK1, k = e % kTcK1;
    tc_store_w<kTcK1>(tW1, n, k, k < kPIn ? q[pW1 + n * kPIn + k] : 0.f);
  }
  for (int e = threadIdx.x; e < kPH * kPH; e += blockDim.x) {
    const int n = e / kPH, k = e % kPH;
    tc_store_w<kPH>(tW2, n, k, q[pW2 + n * kPH + k]);
    if (tW2T != nullptr) tc_store_w<kPH>(tW2T, n, k, q[pW2 + k * kPH + n]);
  }
  for (int e = threadIdx.x; e < kTcF; e += blockDim.x)
    fb[e] = e < 32 ? q[pb1 + e] : (e < 64 ? q[pb2 + e - 32] : (e < 96 ? q[pw3 + e - 64] : (e == 96 ? q[pb3] : 0.f)));
}

// layers 1 and 2 of this thread's row through the tensor core: a1 (ReLU output of layer 1)
// and the logit; false if an MMA never completed
__device__ __forceinline__ bool tc_forward(uint32_t tcol, uint8_t* tA, const uint8_t* tW1, const uint8_t* tW2,
                                           const float* fb, const float (&u)[kTcK1], float (&a1)[kPH], float (&a2)[kPH],
                                           float& logit, uint64_t* mbar, uint32_t& phase, int* abort) {
  const int row = threadIdx.x, warp = threadIdx.x >> 5;
  const uint32_t lane_addr = tcol + ((uint32_t)(32 * warp) << 16);
  tc_store_row<kTcK1>(tA, row, u);
  if (!tc_phase<kTcK1>(tcol, tA, tW1, mbar, phase, abort)) return false;
  tc::tmem_ld32(lane_addr, a1);
  tc::tmem_ld_wait();
#pragma unroll
  for (int j = 0; j < kPH; ++j) a1[j] = fmaxf(a1[j] + fb[j], 0.f);
  tc_store_row<kPH>(tA, row, a1);
  if (!tc_phase<kPH>(tcol, tA, tW2, mbar, phase, abort)) return false;
  tc::tmem_ld32(lane_addr, a2);
  tc::tmem_ld_wait();
  float l = fb[96];
#pragma unroll
  for (int j = 0; j < kPH; ++j) {
    a2[j] = fmaxf(a2[j] + fb[32 + j], 0.f);
    l = fmaf(fb[64 + j], a2[j], l);
  }
  logit = l;
  return true;
}

size_t prop_sample_tc_smem() { return kTcA + kTcWeights + kTcF * sizeof(float) + 64 + 1024; }

__global__ void __launch_bounds__(128) prop_sample_tc_kernel(PropSampleArgs a, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* tA = base;
  uint8_t* tW1 = tA + kTcA;
  uint8_t* tW2 = tW1 + kTcW1;
  float* fb = reinterpret_cast<float*>(tW2 + 2u * kTcW2);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(fb + kTcF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* abort = reinterpret_cast<int*>(tslot + 1);
  tc_load_weights(a.q, tW1, tW2, nullptr, fb);
  if (threadIdx.x == 0) {
    tc::mbar_init(mbar, 1);
    tc::fence_mbar_init();
    *abort = 0;
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 32);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tcol = *tslot;
  uint32_t phase = 0;
  bool alive = true;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float width = prop_width(a.near_m, a.far_m);
  const long long npix = (long long)a.fr.F * a.fr.H * a.fr.W;
  const float tc = __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)lane, 0.5f), width));
  int nd = 0, ntr = 0, nfs = 0;
  for (int quad = blockIdx.x; quad * 4 < a.R && alive; quad += gridDim.x) {
    const int i = quad * 4 + warp;
    const bool has = i < a.R;
    float o[3] = {0.f, 0.f, 0.f}, r[3] = {0.f, 0.f, 1.f}, rgb[3], D = 0.f;
    if (has) {  // the ray: the plain sampler's draw for ray i
      const uint64_t pre = draw_prefix(a.seed, 0, a.step, (uint64_t)i);
      const long long px = (long long)(draw_slot(pre, 0) % (uint64_t)npix);
      pixel_ray(a.fr, px, o, r, rgb, &D);
      if (lane == 0) {
        a.pix[i] = px;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          a.o[3 * i + k] = o[k];
          a.r[3 * i + k] = r[k];
          a.rgb[3 * i + k] = rgb[k];
        }
        a.D[i] = D;
        nd += D > 0.0f;
      }
    }
    float u[kTcK1];
#pragma unroll
    for (int k = 0; k < kTcK1; ++k) u[k] = 0.f;
    if (has) prop_input(a.g, a.theta, o, r, tc, u);
    float a1[kPH], a2[kPH], l;
    if (!(alive = tc_forward(tcol, tA, tW1, tW2, fb, u, a1, a2, l, mbar, phase, abort))) break;
    if (!has) continue;  // warp-uniform
    const float e = expf(l - warp_max(l));
    const float pb = __fdiv_rn(e, warp_sum_bcast(e));
    prop_draw(a, i, pb, D, width, lane, ntr, nfs);
  }
  if (!alive && threadIdx.x == 0) {
    atomicOr(status, kStatusProposal);
    tc::mbar_wait(mbar, phase ^ 1u, kPropMbarLimit);  // let an MMA in flight finish
  }
  block_add_counts(a.counts, nd, ntr, nfs);
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tcol, 32);
  }
}

size_t prop_backward_tc_smem() {
  return kTcA + kTcWeights + kTcF * sizeof(float) + 64 +
         sizeof(float) * (4 * 32 + 4 * kPropPart + 4 * 32 * kRow) + 1024;
}

__global__ void __launch_bounds__(128) prop_backward_tc_kernel(PropBwdArgs a, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* tA = base;
  uint8_t* tW1 = tA + kTcA;
  uint8_t* tW2 = tW1 + kTcW1;
  uint8_t* tW2T = tW2 + kTcW2;
  float* fb = reinterpret_cast<float*>(tW2T + kTcW2);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(fb + kTcF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* abort = reinterpret_cast<int*>(tslot + 1);
  float* hist = reinterpret_cast<float*>(mbar + 8);  // [4][32]
  float* wacc = hist + 4 * 32;                       // [4][kPropPart]
  float* stage = wacc + 4 * kPropPart;               // [4][32][kRow]
  tc_load_weights(a.q, tW1, tW2, tW2T, fb);
  for (int i = threadIdx.x; i < 4 * kPropPart; i += blockDim.x) wacc[i] = 0.f;
  if (threadIdx.x == 0) {
    tc::mbar_init(mbar, 1);
    tc::fence_mbar_init();
    *abort = 0;
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 32);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tcol = *tslot;
  uint32_t phase = 0;
  bool alive = true;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lane_addr = tcol + ((uint32_t)(32 * warp) << 16);
  float* hw = hist + warp * 32;
  float* st = stage + (size_t)warp * 32 * kRow;
  float* aW2 = wacc + warp * kPropPart;
  float* aW1 = aW2 + kPH * kPH;
  float* aB = aW1 + kPIn * kPH;  // b1[32] | b2[32] | w3[32] | b3 | loss | rays
  const float width = prop_width(a.near_m, a.far_m);
  const float tc = __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)lane, 0.5f), width));

  for (int quad = blockIdx.x; quad * 4 < a.R && alive; quad += gridDim.x) {
    const int i = quad * 4 + warp;
    const bool has = i < a.R;
    hw[lane] = 0.f;
    __syncwarp();
    if (has)
      for (int s2 = lane; s2 < a.N; s2 += 32) {
        const float tt = a.t[(size_t)i * a.N + s2];
        const int b = min(max((int)floorf(__fdiv_rn(__fsub_rn(tt, a.near_m), width)), 0), kPB - 1);
        atomicAdd(hw + b, a.w[(size_t)i * a.N + s2]);
      }
    __syncwarp();
    const float h = hw[lane];
    const float S = warp_sum_bcast(h);
    const bool valid = has && S >= 1e-3f;  // warp-uniform: too little weight on a ray makes no target
    float u[kTcK1];
#pragma unroll
    for (int k = 0; k < kTcK1; ++k) u[k] = 0.f;
    if (valid) {
      const float o[3] = {a.o[3 * i], a.o[3 * i + 1], a.o[3 * i + 2]};
      const float r[3] = {a.r[3 * i], a.r[3 * i + 1], a.r[3 * i + 2]};
      prop_input(a.g, a.theta, o, r, tc, u);
    }
    float a1[kPH], a2[kPH], l;
    if (!(alive = tc_forward(tcol, tA, tW1, tW2, fb, u, a1, a2, l, mbar, phase, abort))) break;
    // softmax, cross entropy against the binned weights, dL/dlogit = p - h / S
    const float mx = warp_max(l);
    const float e = expf(l - mx);
    const float se = warp_sum_bcast(e);
    const float p = e / se, logp = l - mx - logf(se);
    const float hh = valid ? h / S : 0.f;
    const float ce = -warp_sum_bcast(hh * logp);
    const float dl = valid ? p - hh : 0.f;
    if (valid && lane == 0) {
      aB[3 * kPH + 1] += ce;
      aB[3 * kPH + 2] += 1.f;
    }
    // layer-2 adjoint on CUDA cores, layer-1 adjoint dA1 = d2 W2 on the tensor core
    float d2[kPH];
#pragma unroll
    for (int j = 0; j < kPH; ++j) d2[j] = a2[j] > 0.f ? dl * fb[64 + j] : 0.f;
    tc_store_row<kPH>(tA, threadIdx.x, d2);
    if (!(alive = tc_phase<kPH>(tcol, tA, tW2T, mbar, phase, abort))) break;
    float d1[kPH];
    tc::tmem_ld32(lane_addr, d1);
    tc::tmem_ld_wait();
    if (!valid) continue;  // warp-uniform
    float* row = st + lane * kRow;
#pragma unroll
    for (int k = 0; k < kPH; ++k) {
      row[rA1 + k] = a1[k];
      row[rDy1 + k] = a1[k] > 0.f ? d1[k] : 0.f;
      row[rA2 + k] = a2[k];
    }
#pragma unroll
    for (int k = 0; k < kPIn; ++k) row[rU + k] = u[k];
    row[rDl] = dl;
    __syncwarp();
    {  // sums over the warp's 32 bin rows: lane j owns row j of dW2 and dW1, entry j of b1, b2, w3
      const float w3j = fb[64 + lane];
      float gW2[kPH], gW1[kPIn], gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
#pragma unroll
      for (int k = 0; k < kPH; ++k) gW2[k] = 0.f;
#pragma unroll
      for (int k = 0; k < kPIn; ++k) gW1[k] = 0.f;
#pragma unroll 2
      for (int s2 = 0; s2 < 32; ++s2) {
        const float* rw = st + s2 * kRow;
        const float dls = rw[rDl], a2j = rw[rA2 + lane];
        const float dd2 = a2j > 0.f ? dls * w3j : 0.f, dd1 = rw[rDy1 + lane];
#pragma unroll
        for (int k = 0; k < kPH; ++k) gW2[k] = fmaf(dd2, rw[rA1 + k], gW2[k]);
#pragma unroll
        for (int k = 0; k < kPIn; ++k) gW1[k] = fmaf(dd1, rw[rU + k], gW1[k]);
        gb2 += dd2;
        gb1 += dd1;
        gw3 = fmaf(dls, a2j, gw3);
        gb3 += dls;
      }
#pragma unroll
      for (int k = 0; k < kPH; ++k) aW2[k * kPH + lane] += gW2[k];
#pragma unroll
      for (int k = 0; k < kPIn; ++k) aW1[k * kPH + lane] += gW1[k];
      aB[lane] += gb1;
      aB[kPH + lane] += gb2;
      aB[2 * kPH + lane] += gw3;
      if (lane == 0) aB[3 * kPH] += gb3;
    }
    __syncwarp();
  }
  if (!alive && threadIdx.x == 0) {
    atomicOr(status, kStatusProposal);
    tc::mbar_wait(mbar, phase ^ 1u, kPropMbarLimit);  // let an MMA in flight finish
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tcol, 32);
  }
  // block row in the parameter layout: sum of the warps' accumulators (as prop_backward_kernel)
  for (int e = threadIdx.x; e < kPropPart; e += blockDim.x) {
    int src;
    if (e < pb1) src = kPH * kPH + (e % kPIn) * kPH + e / kPIn;
    else if (e < pW2) src = kPH * kPH + kPIn * kPH + (e - pb1);
    else if (e < pb2) src = ((e - pW2) % kPH) * kPH + (e - pW2) / kPH;
    else if (e < pw3) src = kPH * kPH + kPIn * kPH + kPH + (e - pb2);
    else if (e < pb3) src = kPH * kPH + kPIn * kPH + 2 * kPH + (e - pw3);
    else if (e < GS_PROP_PARAMS + 2) src = kPH * kPH + kPIn * kPH + 3 * kPH + (e - pb3);
    else src = -1;
    float v = 0.f;
    if (src >= 0)
#pragma unroll
      for (int q2 = 0; q2 < 4; ++q2) v += wacc[q2 * kPropPart + src];
    a.part[(size_t)blockIdx.x * kPropPart + e] = v;
  }
}

size_t prop_backward_smem() {
  return sizeof(float) * (kPropPad + kPropWarps * 32 + kPropWarps * kPropPart + kPropWarps * 32 * kRow);
}

}  // namespace gs

using namespace gs;

int gs_prop_part_rows(int num_sms) { return 2 * num_sms; }
size_t gs_prop_part_floats(int num_sms) { return (size_t)gs_prop_part_rows(num_sms) * kPropPart; }

gs_status gs_launch_prop_sample(const gs_ctx* ctx, const float* theta, const float* q, const gs_frames* f,
                                uint64_t seed, uint32_t step, const float* pdf_in, float* pdf_out, const gs_batch* b,
                                cudaStream_t st) {
  if (cudaMemsetAsync(b->counts, 0, 4 * sizeof(int), st) != cudaSuccess) return GS_ERR_CUDA;
  if (b->R > 0) {
    PropSampleArgs a;
    a.fr = FramesDev{f->F, f->H, f->W, f->rgb, f->depth, f->c2w, f->fx, f->fy, f->cx, f->cy};
    a.g = ctx->grid;
    a.theta = theta;
    a.q = q;
    a.pdf_in = pdf_in;
    a.pdf_out = pdf_out;
    a.seed = seed;
    a.step = step;
    a.R = b->R;
    a.N = b->N;
    a.Ng = ctx->cfg.prop_guided;
    a.near_m = ctx->cfg.near_m;
    a.far_m = ctx->cfg.far_m;
    a.guide_half = ctx->cfg.guide_half;
    a.trunc = ctx->cfg.trunc;
    a.pix = (long long*)b->pix;
    a.o = b->origin;
    a.r = b->dir;
    a.rgb = b->rgb;
    a.D = b->depth;
    a.t = b->t;
    a.cls = b->cls;
    a.counts = b->counts;
    const int blocks = (int)std::min<long long>(((long long)b->R + kPropWarps - 1) / kPropWarps, 8LL * ctx->num_sms);
    if (ctx->cfg.precision == GS_PREC_BF16 && pdf_in == nullptr) {  // the network on the tensor core
      const size_t smem = prop_sample_tc_smem();
      if (cudaFuncSetAttribute(prop_sample_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return GS_ERR_CUDA;
      prop_sample_tc_kernel<<<blocks, 128, smem, st>>>(a, ctx->status);
    } else {
      prop_sample_kernel<<<blocks, kPropWarps * 32, 0, st>>>(a);
    }
    if (cudaPeekAtLastError() != cudaSuccess) return GS_ERR_CUDA;
  }
  return gs_launch_sample_smooth(ctx, f, seed, step, b, st);
}

gs_status gs_launch_prop_backward(const gs_ctx* ctx, const float* theta, const float* q, const gs_batch* b,
                                  float* grad, float* ce, cudaStream_t st) {
  const int rows = gs_prop_part_rows(ctx->num_sms);
  const int blocks = (int)std::min<long long>(std::max<long long>(((long long)b->R + kPropWarps - 1) / kPropWarps, 1),
                                              rows);
  PropBwdArgs a;
  a.g = ctx->grid;
  a.theta = theta;
  a.q = q;
  a.R = b->R;
  a.N = b->N;
  a.o = b->origin;
  a.r = b->dir;
  a.t = b->t;
  a.w = b->w;
  a.near_m = ctx->cfg.near_m;
  a.far_m = ctx->cfg.far_m;
  a.part = ctx->prop_part;
  if (ctx->cfg.precision == GS_PREC_BF16) {  // the network and its first layer's adjoint on the tensor core
    const size_t smem = prop_backward_tc_smem();
    if (cudaFuncSetAttribute(prop_backward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GS_ERR_CUDA;
    prop_backward_tc_kernel<<<blocks, 128, smem, st>>>(a, ctx->status);
  } else {
    const size_t smem = prop_backward_smem();
    if (cudaFuncSetAttribute(prop_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GS_ERR_CUDA;
    prop_backward_kernel<<<blocks, kPropWarps * 32, smem, st>>>(a);
  }
  prop_finalize_kernel<<<(GS_PROP_PARAMS + 1 + 31) / 32, 256, 0, st>>>(ctx->prop_part, blocks, grad, ce);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
