// The paper's architecture (Sec. 3.1 Eq. SDF_MLP and Eq. COLOR_MLP, "Architecture Details"):
// geometry features V_theta(x) from the four grid levels, colour features W_beta(x) (h_c = 6)
// from a separate grid on the finest level's vertices, phi = f_omega(V_theta(x)) and
// c = g_gamma(W_beta(x), d) with d the unit viewing direction, both decoders with two hidden
// layers of 32.  Rendering, losses and the smoothness term are those of the workload's model.
//
// Kernels here (FP32 on CUDA cores; the render pass is the tensor-core kernel of
// gs_paper_tc.cuh):
//   paper_smooth_kernel  the smoothness term on S_g and its second-order adjoint, one lane per
//                        evaluation (x or x + eps of 16 points per warp);
//   paper_combine_kernel per-CTA partial rows combined in a fixed order (losses in FP64).
#include "gs_internal.h"
#include "gs_paper.cuh"

namespace gs {
namespace paper {

// One block of the decoder: its range in the flat vector, its start in shared memory, and
// (matrices with 32 rows) its column count.  The gradient accumulators of those matrices
// are kept transposed in shared memory (entry (j, k) at k * 32 + j) so that lane j, which
// sums row j, touches bank j.
struct Block {
  int a, n, s, cols;
};
__constant__ Block kBlocks[13] = {{A_gW1, 512, S_gW1, kZ}, {A_gb1, 32, S_gb1, 0},  {A_gW2, 1024, S_gW2, kH},
                                  {A_gb2, 32, S_gb2, 0},   {A_gw3, 32, S_gw3, 0},  {A_gb3, 1, S_gb3, 0},
                                  {A_cW1, 288, S_cW1, kU}, {A_cb1, 32, S_cb1, 0},  {A_cW2, 1024, S_cW2, kH},
                                  {A_cb2, 32, S_cb2, 0},   {A_cW3, 96, S_cW3, 0},  {A_cb3, 3, S_cb3, 0},
                                  {A_kappa, 1, S_kappa, 0}};

__device__ __forceinline__ void copy_decoder(const float* __restrict__ mlp, float* sW) {
  for (int i = threadIdx.x; i < kSm; i += blockDim.x) sW[i] = 0.f;
  __syncthreads();
  for (int b = 0; b < 13; ++b)
    for (int i = threadIdx.x; i < kBlocks[b].n; i += blockDim.x) sW[kBlocks[b].s + i] = mlp[kBlocks[b].a + i];
}

// shared accumulator index of flat decoder entry i (inverse of the transposed storage)
__device__ __forceinline__ int acc_index(int i) {
  for (int b = 0; b < 13; ++b) {
    const Block k = kBlocks[b];
    if (i >= k.a && i < k.a + k.n) {
      const int r = i - k.a;
      return k.cols ? k.s + (r % k.cols) * 32 + r / k.cols : k.s + r;
    }
  }
  return -1;
}

// Per-lane row of staged sample vectors.  Every field starts on a 16-byte boundary and the
// stride is 4 (mod 32) words, so a lane's float4 access to its own row and a float4 read of
// one row by the whole warp (broadcast) are both free of bank conflicts.
constexpr int kRow = 164;
constexpr int fZ = 0, fU = 16, fA1 = 28, fA2 = 60, fR1 = 92, fR2 = 124, fDP = 156;  // fDP: dpre[3], dphi
static_assert(kRow % 32 == 4 && fU % 4 == 0 && fA1 % 4 == 0 && fDP % 4 == 0, "row layout");
constexpr int kWarps = 4;  // warps per CTA
constexpr int kThreads = kWarps * 32;
constexpr size_t kSmemBytes = sizeof(float) * (2 * kSm + 8 + kWarps * 32 * kRow);
constexpr int kCtasPerSm = 2;  // CTAs per SM of the CUDA-core kernels here (sizes the partial rows)

struct Args {
  GridDesc g;            // geometry levels; g.n_grid = decoder block offset (after the colour grid)
  long long colour_off;  // float offset of the colour grid
  const float* theta;
  float* grad;
  const float *o, *r, *rgb, *D, *t;
  const uint8_t* cls;
  const float *xs, *eps;
  const uint8_t* valid;
  const int* counts;
  const float* dloss;
  float *rgb_hat, *d_hat, *wsum, *w_out;
  float* dz_out;                // [R][N][32] per-sample records for the pose gradient (may be nullptr)
  float *loss_part, *mlp_part;  // this kernel's first partial row
  int R, N, P, mode;
  float lam[5];
  float kappa_fs;
};

// lane j (row j of a 32-row matrix) sums delta_s[j] * act_s[k] over the warp's 32 staged
// samples for k < K (and delta_s[j] for the bias) and adds them to the CTA accumulators
template <int K, bool kBias>
__device__ __forceinline__ void outer_rows(const float* wr, int fd, int fa, float* acc_m, float* acc_b, int lane) {
  float acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.f;
  float ab = 0.f;
#pragma unroll 2
  for (int s = 0; s < 32; ++s) {
    const float* rs = wr + s * kRow;
    const float d = rs[fd + lane];
    ab += d;
#pragma unroll
    for (int k4 = 0; k4 < (K + 3) / 4; ++k4) {
      const float4 v = *reinterpret_cast<const float4*>(rs + fa + 4 * k4);
      acc[4 * k4] = fmaf(d, v.x, acc[4 * k4]);
      if (4 * k4 + 1 < K) acc[4 * k4 + 1 < K ? 4 * k4 + 1 : 0] = fmaf(d, v.y, acc[4 * k4 + 1 < K ? 4 * k4 + 1 : 0]);
      if (4 * k4 + 2 < K) acc[4 * k4 + 2 < K ? 4 * k4 + 2 : 0] = fmaf(d, v.z, acc[4 * k4 + 2 < K ? 4 * k4 + 2 : 0]);
      if (4 * k4 + 3 < K) acc[4 * k4 + 3 < K ? 4 * k4 + 3 : 0] = fmaf(d, v.w, acc[4 * k4 + 3 < K ? 4 * k4 + 3 : 0]);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) atomicAdd(acc_m + k * 32 + lane, acc[k]);
  if (kBias) atomicAdd(acc_b + lane, ab);
}


// geometry features z (4 levels x 4) and colour features cf (level-3 cell, 6) at x
__device__ __forceinline__ void gather(const Args& a, const float x[3], float z[kZ], float cf[kC]) {
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell c = locate(a.g, l, x);
    float w[8];
    corner_weights(c.f, w);
    const float4* lv = reinterpret_cast<const float4*>(a.theta + a.g.off[l]);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f4fma(acc, w[k], __ldg(lv + c.vtx + corner_offset(a.g, l, k)));
    z[4 * l] = acc.x;
    z[4 * l + 1] = acc.y;
    z[4 * l + 2] = acc.z;
    z[4 * l + 3] = acc.w;
    if (l == kLevels - 1) {
#pragma unroll
      for (int q = 0; q < kC; ++q) cf[q] = 0.f;
      const float2* cg = reinterpret_cast<const float2*>(a.theta + a.colour_off);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const long long v2 = (c.vtx + corner_offset(a.g, l, k)) * 3;  // 3 float2 per vertex
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float2 f = __ldg(cg + v2 + q);
          cf[2 * q] = fmaf(w[k], f.x, cf[2 * q]);
          cf[2 * q + 1] = fmaf(w[k], f.y, cf[2 * q + 1]);
        }
      }
    }
  }
}

__device__ __forceinline__ void write_partials(const Args& a, const float* sG, const float* sL) {
  float* row = a.mlp_part + (size_t)blockIdx.x * kPart;
  for (int i = threadIdx.x; i < kPart; i += blockDim.x) row[i] = i < GS_PAPER_MLP_PARAMS ? sG[acc_index(i)] : 0.f;
  if (threadIdx.x < kLossPad) a.loss_part[(size_t)blockIdx.x * kLossPad + threadIdx.x] = sL[threadIdx.x];
}

// One lane, one point y: g = grad_x phi(y) = sum_k p_k dz_k/dx for the geometry decoder,
// p = gW1^T pm, pm = m1 (.) gW2^T e, e = m2 (.) gw3 (masks m1, m2 of the two hidden layers);
// e and pm are staged in the lane's row (fields A2, A1) for grad_phi_adjoint.
__device__ __forceinline__ void grad_phi_fwd(const Args& a, const float* sW, float* my, const float y[3],
                                             unsigned& m1, unsigned& m2, float pz[kZ], float g[3]) {
    // z; the x-derivatives dz/dx are gathered again level by level where they are used
    // (keeping all 48 of them in registers beside the decoder sensitivities spills)
    float z[kZ];
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
      const Cell c = locate(a.g, l, y);
      float wv[8];
      corner_weights(c.f, wv);
      const float4* lv = reinterpret_cast<const float4*>(a.theta + a.g.off[l]);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 8; ++k) f4fma(acc, wv[k], __ldg(lv + c.vtx + corner_offset(a.g, l, k)));
      z[4 * l] = acc.x;
      z[4 * l + 1] = acc.y;
      z[4 * l + 2] = acc.z;
      z[4 * l + 3] = acc.w;
    }
    // forward masks; the layer-1 activations go through the lane's row (field R1, free until
    // grad_phi_adjoint) instead of 32 registers
    m1 = 0u;
    m2 = 0u;
#pragma unroll 1
    for (int j4 = 0; j4 < kH / 4; ++j4) {
      float hv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 4 * j4 + q;
        float v = sW[S_gb1 + j];
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const float4 wv = ld4(sW + S_gW1 + j * kZ + 4 * k4);
          v = fmaf(wv.x, z[4 * k4], v);
          v = fmaf(wv.y, z[4 * k4 + 1], v);
          v = fmaf(wv.z, z[4 * k4 + 2], v);
          v = fmaf(wv.w, z[4 * k4 + 3], v);
        }
        hv[q] = fmaxf(v, 0.f);
        m1 |= (v > 0.f ? 1u : 0u) << j;
      }
      st4(my + fR1 + 4 * j4, hv[0], hv[1], hv[2], hv[3]);
    }
#pragma unroll 1
    for (int j = 0; j < kH; ++j) {
      float v = sW[S_gb2 + j];
#pragma unroll
      for (int k4 = 0; k4 < 8; ++k4) {
        const float4 wv = ld4(sW + S_gW2 + j * kH + 4 * k4), hv = ld4(my + fR1 + 4 * k4);
        v = fmaf(wv.x, hv.x, v);
        v = fmaf(wv.y, hv.y, v);
        v = fmaf(wv.z, hv.z, v);
        v = fmaf(wv.w, hv.w, v);
      }
      m2 |= (v > 0.f ? 1u : 0u) << j;
    }
    // e = m2 (.) gw3 (row field A2), pm = m1 (.) gW2^T e (row field A1), p = gW1^T pm
    {
      float pm[kH];
#pragma unroll
      for (int k = 0; k < kH; ++k) pm[k] = 0.f;
#pragma unroll 1
      for (int j = 0; j < kH; ++j) {
        const float e = (m2 >> j) & 1u ? sW[S_gw3 + j] : 0.f;
#pragma unroll
        for (int k4 = 0; k4 < 8; ++k4) {
          const float4 wv = ld4(sW + S_gW2 + j * kH + 4 * k4);
          pm[4 * k4] = fmaf(wv.x, e, pm[4 * k4]);
          pm[4 * k4 + 1] = fmaf(wv.y, e, pm[4 * k4 + 1]);
          pm[4 * k4 + 2] = fmaf(wv.z, e, pm[4 * k4 + 2]);
          pm[4 * k4 + 3] = fmaf(wv.w, e, pm[4 * k4 + 3]);
        }
      }
#pragma unroll
      for (int k = 0; k < kZ; ++k) pz[k] = 0.f;
#pragma unroll
      for (int j = 0; j < kH; ++j) pm[j] = (m1 >> j) & 1u ? pm[j] : 0.f;
#pragma unroll
      for (int j4 = 0; j4 < kH / 4; ++j4) {
        const float4 w3 = ld4(sW + S_gw3 + 4 * j4);
        const int b = 4 * j4;
        st4(my + fA2 + b, (m2 >> b) & 1u ? w3.x : 0.f, (m2 >> (b + 1)) & 1u ? w3.y : 0.f,
            (m2 >> (b + 2)) & 1u ? w3.z : 0.f, (m2 >> (b + 3)) & 1u ? w3.w : 0.f);
        st4(my + fA1 + b, pm[b], pm[b + 1], pm[b + 2], pm[b + 3]);
      }
#pragma unroll
      for (int j = 0; j < kH; ++j) {
        const float pj = pm[j];
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const float4 wv = ld4(sW + S_gW1 + j * kZ + 4 * k4);
          pz[4 * k4] = fmaf(wv.x, pj, pz[4 * k4]);
          pz[4 * k4 + 1] = fmaf(wv.y, pj, pz[4 * k4 + 1]);
          pz[4 * k4 + 2] = fmaf(wv.z, pj, pz[4 * k4 + 2]);
          pz[4 * k4 + 3] = fmaf(wv.w, pj, pz[4 * k4 + 3]);
        }
      }
    }
    g[0] = g[1] = g[2] = 0.f;
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
      float4 dl[3];
      float dw[8][3];
      level_jacobian(a.g, a.theta, l, y, dl, dw);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        g[q] += pz[4 * l] * dl[q].x + pz[4 * l + 1] * dl[q].y + pz[4 * l + 2] * dl[q].z + pz[4 * l + 3] * dl[q].w;
    }
}

// The second-order adjoint (Supp. Sec. 1) of sum over the warp's lanes of a . grad_x phi(y)
// with respect to the grid and the geometry decoder: j_k = a . dz_k/dx, grid term
// p_{l,f} (1/v_l) (a . dw_c/df) (when do_grid), gW1 += pm j^T, gW2 += e vj^T,
// gw3 += m2 (.) gW2 vj with vj = m1 (.) gW1 j; biases get none.  Every lane of the warp
// calls it (a lane with av = 0 adds nothing); its row holds e and pm from grad_phi_fwd.
__device__ __forceinline__ void grad_phi_adjoint(const Args& a, const float* sW, float* sG, const float* wr, float* my,
                                                 int lane, const float y[3], bool do_grid, const float av[3],
                                                 unsigned m1, unsigned m2, const float pz[kZ]) {
    float jv[kZ];  // j_k = a . dz_k/dx
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
      float4 dl[3];
      float dw[8][3];
      level_jacobian(a.g, a.theta, l, y, dl, dw);
      jv[4 * l] = av[0] * dl[0].x + av[1] * dl[1].x + av[2] * dl[2].x;
      jv[4 * l + 1] = av[0] * dl[0].y + av[1] * dl[1].y + av[2] * dl[2].y;
      jv[4 * l + 2] = av[0] * dl[0].z + av[1] * dl[1].z + av[2] * dl[2].z;
      jv[4 * l + 3] = av[0] * dl[0].w + av[1] * dl[1].w + av[2] * dl[2].w;
    }
#pragma unroll
    for (int k4 = 0; k4 < kZ / 4; ++k4) st4(my + fZ + 4 * k4, jv[4 * k4], jv[4 * k4 + 1], jv[4 * k4 + 2], jv[4 * k4 + 3]);
    // vj = m1 (.) gW1 j (row field R1);  w3g = m2 (.) gW2 vj (row field R2)
    {
      float vj[kH];
#pragma unroll
      for (int j = 0; j < kH; ++j) {
        float v = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const float4 wv = ld4(sW + S_gW1 + j * kZ + 4 * k4);
          v = fmaf(wv.x, jv[4 * k4], v);
          v = fmaf(wv.y, jv[4 * k4 + 1], v);
          v = fmaf(wv.z, jv[4 * k4 + 2], v);
          v = fmaf(wv.w, jv[4 * k4 + 3], v);
        }
        vj[j] = (m1 >> j) & 1u ? v : 0.f;
      }
#pragma unroll
      for (int j4 = 0; j4 < kH / 4; ++j4) st4(my + fR1 + 4 * j4, vj[4 * j4], vj[4 * j4 + 1], vj[4 * j4 + 2], vj[4 * j4 + 3]);
#pragma unroll 1
      for (int j4 = 0; j4 < kH / 4; ++j4) {
        float vv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * j4 + q;
          float v = 0.f;
#pragma unroll
          for (int k4 = 0; k4 < 8; ++k4) {
            const float4 wv = ld4(sW + S_gW2 + j * kH + 4 * k4);
            v = fmaf(wv.x, vj[4 * k4], v);
            v = fmaf(wv.y, vj[4 * k4 + 1], v);
            v = fmaf(wv.z, vj[4 * k4 + 2], v);
            v = fmaf(wv.w, vj[4 * k4 + 3], v);
          }
          vv[q] = (m2 >> j) & 1u ? v : 0.f;
        }
        st4(my + fR2 + 4 * j4, vv[0], vv[1], vv[2], vv[3]);
      }
    }
    __syncwarp();
    outer_rows<kZ, false>(wr, fA1, fZ, sG + S_gW1, nullptr, lane);  // pm j^T
    outer_rows<kH, false>(wr, fA2, fR1, sG + S_gW2, nullptr, lane);  // e vj^T
    {
      float acc = 0.f;
#pragma unroll 8
      for (int sidx = 0; sidx < 32; ++sidx) acc += wr[sidx * kRow + fR2 + lane];
      atomicAdd(sG + S_gw3 + lane, acc);
    }
    __syncwarp();
    // grid term
    if (do_grid) {
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        const Cell c = locate(a.g, l, y);
        float dw[8][3];
        corner_weight_grads(c.f, c.clamped, dw);
        const float4 p4 = make_float4(pz[4 * l], pz[4 * l + 1], pz[4 * l + 2], pz[4 * l + 3]);
        float4* gl = reinterpret_cast<float4*>(a.grad + a.g.off[l]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float ad = (av[0] * dw[k][0] + av[1] * dw[k][1] + av[2] * dw[k][2]) * a.g.inv_voxel[l];
          atomicAdd(gl + c.vtx + corner_offset(a.g, l, k), f4scale(p4, ad));
        }
      }
    }
}

// Smoothness term on S_g (Sec. 3.3 Eq. smoothness_loss) and its second-order adjoint
// (Supp. Sec. 1) for the two-hidden-layer geometry decoder.  Lane l of a warp evaluates
// point 16 * group + (l & 15) at x (l < 16) or x + eps (l >= 16):
//   g = grad_x phi = sum_k p_k dz_k/dx, p = gW1^T (m1 (.) gW2^T (m2 (.) gw3)).
// The adjoint a = dL/dg gives the grid term p_{l,f} (1/v_l) (a . dw_c/df) and the decoder
// terms gW1 += pm j^T, gW2 += e vj^T, gw3 += m2 (.) gW2 vj with j_k = a . dz_k/dx,
// pm = m1 (.) gW2^T e, e = m2 (.) gw3, vj = m1 (.) gW1 j (biases get none).
__global__ void __launch_bounds__(kThreads, 1) paper_smooth_kernel(Args a) {
  extern __shared__ __align__(16) float smem[];
  float* sW = smem;
  float* sG = sW + kSm;
  float* sL = sG + kSm;
  float* rows = sL + 8;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* wr = rows + wid * 32 * kRow;
  float* my = wr + lane * kRow;
  copy_decoder(a.theta + a.g.n_grid, sW);
  for (int i = threadIdx.x; i < kSm; i += blockDim.x) sG[i] = 0.f;
  if (threadIdx.x < 8) sL[threadIdx.x] = 0.f;
  __syncthreads();
  const bool bwd = (a.mode & 2) != 0;
  const int n_g = a.counts[3];
  const float w4 = a.dloss[4] + a.lam[4] * a.dloss[5];
  const int ev = lane >> 4;
  float lsum = 0.f;
  for (int grp = blockIdx.x * kWarps + wid; grp * 16 < a.P; grp += gridDim.x * kWarps) {
    const int p = grp * 16 + (lane & 15);
    const bool ok = p < a.P && a.valid[p] != 0;
    float y[3] = {0.f, 0.f, 0.f};
    if (ok) {
#pragma unroll
      for (int q = 0; q < 3; ++q) y[q] = ev ? __fadd_rn(a.xs[3 * p + q], a.eps[3 * p + q]) : a.xs[3 * p + q];
    }
    unsigned m1, m2;
    float pz[kZ], g[3];
    grad_phi_fwd(a, sW, my, y, m1, m2, pz, g);
    float dg[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float other = __shfl_xor_sync(0xffffffffu, g[q], 16);
      dg[q] = ev ? other - g[q] : g[q] - other;  // g(x) - g(x + eps) on both lanes
    }
    if (ok && ev == 0) lsum += dg[0] * dg[0] + dg[1] * dg[1] + dg[2] * dg[2];
    if (!bwd) continue;
    float av[3] = {0.f, 0.f, 0.f};
    if (ok && n_g > 0) {
      const float sc = (ev ? -2.f : 2.f) * w4 / (float)n_g;
#pragma unroll
      for (int q = 0; q < 3; ++q) av[q] = sc * dg[q];
    }
    grad_phi_adjoint(a, sW, sG, wr, my, lane, y, ok && n_g > 0, av, m1, m2, pz);
  }
  const float v = warp_sum(lsum);
  if (lane == 0) atomicAdd(sL + 4, v);
  __syncthreads();
  write_partials(a, sG, sL);
}

// phi(x) and (grad != nullptr) grad_x phi(x) of the geometry decoder, one thread per point
__global__ void __launch_bounds__(128) paper_query_kernel(GridDesc g, const float* __restrict__ theta,
                                                          const float* __restrict__ xq, int P, float* sdf,
                                                          float* grad) {
  __shared__ __align__(16) float sg[kGeoPad];
  __shared__ float hs[128][kH + 1];  // each thread's layer-1 activations (stride 33: conflict-free)
  load_geometry_decoder(theta + g.n_grid, sg);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  float* h = hs[threadIdx.x];
  const float x[3] = {xq[3 * i], xq[3 * i + 1], xq[3 * i + 2]};
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
  // phi = gw3 . relu(gW2 h + gb2) + gb3 with h = relu(gW1 z + gb1); for the gradient also
  // p = gW1^T (m1 (.) gW2^T (m2 (.) gw3)) and grad = sum over levels of (dz_l/dx)^T p_l
  unsigned m1 = 0u;
#pragma unroll 4
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
    m1 |= (y > 0.f ? 1u : 0u) << j;
  }
  float phi = sg[S_gb3];
  float pm[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) pm[k] = 0.f;
#pragma unroll 1
  for (int j = 0; j < kH; ++j) {
    float y = sg[S_gb2 + j];
#pragma unroll
    for (int k = 0; k < kH; ++k) y = fmaf(sg[S_gW2 + j * kH + k], h[k], y);
    phi = fmaf(sg[S_gw3 + j], fmaxf(y, 0.f), phi);
    if (grad) {
      const float e = y > 0.f ? sg[S_gw3 + j] : 0.f;
#pragma unroll
      for (int k = 0; k < kH; ++k) pm[k] = fmaf(sg[S_gW2 + j * kH + k], e, pm[k]);
    }
  }
  sdf[i] = phi;
  if (!grad) return;
  float pz[kZ];
#pragma unroll
  for (int k = 0; k < kZ; ++k) pz[k] = 0.f;
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    const float pj = (m1 >> j) & 1u ? pm[j] : 0.f;
#pragma unroll
    for (int k = 0; k < kZ; ++k) pz[k] = fmaf(sg[S_gW1 + j * kZ + k], pj, pz[k]);
  }
  float gr[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    float4 dl[3];
    float dw[8][3];
    level_jacobian(g, theta, l, x, dl, dw);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      gr[c] += pz[4 * l] * dl[c].x + pz[4 * l + 1] * dl[c].y + pz[4 * l + 2] * dl[c].z + pz[4 * l + 3] * dl[c].w;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) grad[3 * i + c] = gr[c];
}

// Reverse mode of the SDF query with respect to the parameters (the double backward of
// grad_x phi, Supp. Sec. 1): grad += sum_p dsdf_p d phi(x_p)/d theta + dgrad_p . d grad_x phi(x_p)/d theta.
// One lane per point.  The second term is the second-order adjoint of the smoothness and
// Eikonal kernels; the first the geometry decoder's backward pass (its input and hidden
// layers staged in the rows) and the adjoint of the gathers.  Colour parameters get nothing.
__global__ void __launch_bounds__(kThreads, 1) paper_query_backward_kernel(Args a, const float* __restrict__ xq, int P,
                                                                            const float* __restrict__ dsdf,
                                                                            const float* __restrict__ dgrad) {
  extern __shared__ __align__(16) float smem[];
  float* sW = smem;
  float* sG = sW + kSm;
  float* sL = sG + kSm;
  float* rows = sL + 8;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* wr = rows + wid * 32 * kRow;
  float* my = wr + lane * kRow;
  copy_decoder(a.theta + a.g.n_grid, sW);
  for (int i = threadIdx.x; i < kSm; i += blockDim.x) sG[i] = 0.f;
  if (threadIdx.x < 8) sL[threadIdx.x] = 0.f;
  __syncthreads();
  for (int base = (blockIdx.x * kWarps + wid) * 32; base < P; base += gridDim.x * kWarps * 32) {  // warp-uniform
    const int p = base + lane;
    const bool ok = p < P;
    float y[3] = {0.f, 0.f, 0.f};
    if (ok) {
#pragma unroll
      for (int c = 0; c < 3; ++c) y[c] = xq[3 * p + c];
    }
    if (dgrad) {  // second-order term
      unsigned m1, m2;
      float pz[kZ], g[3];
      grad_phi_fwd(a, sW, my, y, m1, m2, pz, g);
      float av[3] = {0.f, 0.f, 0.f};
      if (ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c) av[c] = dgrad[3 * p + c];
      }
      grad_phi_adjoint(a, sW, sG, wr, my, lane, y, ok, av, m1, m2, pz);
    }
    if (dsdf) {  // first-order term: phi = gw3 . a2 + gb3, a2 = relu(gW2 a1 + gb2), a1 = relu(gW1 z + gb1)
      float z[kZ], cf[kC];
      gather(a, y, z, cf);
      float h[kH];
#pragma unroll
      for (int j = 0; j < kH; ++j) {
        float v = sW[S_gb1 + j];
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const float4 w = ld4(sW + S_gW1 + j * kZ + 4 * k4);
          v = fmaf(w.x, z[4 * k4], v);
          v = fmaf(w.y, z[4 * k4 + 1], v);
          v = fmaf(w.z, z[4 * k4 + 2], v);
          v = fmaf(w.w, z[4 * k4 + 3], v);
        }
        h[j] = fmaxf(v, 0.f);
      }
      const float dp = ok ? dsdf[p] : 0.f;
      __syncwarp();  // the second-order products have read every row
#pragma unroll
      for (int k4 = 0; k4 < kZ / 4; ++k4) st4(my + fZ + 4 * k4, z[4 * k4], z[4 * k4 + 1], z[4 * k4 + 2], z[4 * k4 + 3]);
#pragma unroll
      for (int j4 = 0; j4 < kH / 4; ++j4) st4(my + fA1 + 4 * j4, h[4 * j4], h[4 * j4 + 1], h[4 * j4 + 2], h[4 * j4 + 3]);
#pragma unroll 1
      for (int j4 = 0; j4 < kH / 4; ++j4) {  // a2 and, in its place, dy2 = m2 (.) gw3 dphi
        float a2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * j4 + q;
          float v = sW[S_gb2 + j];
#pragma unroll
          for (int k4 = 0; k4 < 8; ++k4) {
            const float4 w = ld4(sW + S_gW2 + j * kH + 4 * k4);
            v = fmaf(w.x, h[4 * k4], v);
            v = fmaf(w.y, h[4 * k4 + 1], v);
            v = fmaf(w.z, h[4 * k4 + 2], v);
            v = fmaf(w.w, h[4 * k4 + 3], v);
          }
          a2[q] = fmaxf(v, 0.f);
        }
        st4(my + fR1 + 4 * j4, a2[0], a2[1], a2[2], a2[3]);
        const float4 w3 = ld4(sW + S_gw3 + 4 * j4);
        st4(my + fA2 + 4 * j4, a2[0] > 0.f ? w3.x * dp : 0.f, a2[1] > 0.f ? w3.y * dp : 0.f,
            a2[2] > 0.f ? w3.z * dp : 0.f, a2[3] > 0.f ? w3.w * dp : 0.f);
      }
      st4(my + fR2, dp, 0.f, 0.f, 0.f);
      __syncwarp();
      {  // gw3 (lane = column), gb3
        float ag = 0.f, bg = 0.f;
#pragma unroll 4
        for (int sidx = 0; sidx < 32; ++sidx) {
          const float* rs = wr + sidx * kRow;
          ag = fmaf(rs[fR2], rs[fR1 + lane], ag);
          bg += rs[fR2];
        }
        atomicAdd(sG + S_gw3 + lane, ag);
        if (lane == 0) atomicAdd(sG + S_gb3, bg);
      }
      outer_rows<kH, true>(wr, fA2, fA1, sG + S_gW2, sG + S_gb2, lane);
      __syncwarp();
      {  // dy1 = m1 (.) gW2^T dy2 over a1
        float acc[kH];
#pragma unroll
        for (int q = 0; q < kH; ++q) acc[q] = 0.f;
#pragma unroll 1
        for (int j4 = 0; j4 < kH / 4; ++j4) {
          const float4 dy4 = ld4(my + fA2 + 4 * j4);
          const float dys[4] = {dy4.x, dy4.y, dy4.z, dy4.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int k4 = 0; k4 < 8; ++k4) {
              const float4 wv = ld4(sW + S_gW2 + (4 * j4 + q) * kH + 4 * k4);
              acc[4 * k4] = fmaf(wv.x, dys[q], acc[4 * k4]);
              acc[4 * k4 + 1] = fmaf(wv.y, dys[q], acc[4 * k4 + 1]);
              acc[4 * k4 + 2] = fmaf(wv.z, dys[q], acc[4 * k4 + 2]);
              acc[4 * k4 + 3] = fmaf(wv.w, dys[q], acc[4 * k4 + 3]);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < kH; ++q) h[q] = h[q] > 0.f ? acc[q] : 0.f;
#pragma unroll
        for (int j4 = 0; j4 < kH / 4; ++j4) st4(my + fA1 + 4 * j4, h[4 * j4], h[4 * j4 + 1], h[4 * j4 + 2], h[4 * j4 + 3]);
      }
      __syncwarp();
      outer_rows<kZ, true>(wr, fA1, fZ, sG + S_gW1, sG + S_gb1, lane);
      if (ok && dp != 0.f) {  // dz = gW1^T dy1 into the four levels
        float dz[kZ];
#pragma unroll
        for (int q = 0; q < kZ; ++q) dz[q] = 0.f;
#pragma unroll 4
        for (int j = 0; j < kH; ++j) {
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            const float4 wv = ld4(sW + S_gW1 + j * kZ + 4 * k4);
            dz[4 * k4] = fmaf(wv.x, h[j], dz[4 * k4]);
            dz[4 * k4 + 1] = fmaf(wv.y, h[j], dz[4 * k4 + 1]);
            dz[4 * k4 + 2] = fmaf(wv.z, h[j], dz[4 * k4 + 2]);
            dz[4 * k4 + 3] = fmaf(wv.w, h[j], dz[4 * k4 + 3]);
          }
        }
#pragma unroll
        for (int l = 0; l < kLevels; ++l) {
          const Cell c = locate(a.g, l, y);
          float wv[8];
          corner_weights(c.f, wv);
          float4* gl = reinterpret_cast<float4*>(a.grad + a.g.off[l]);
          const float4 d4 = make_float4(dz[4 * l], dz[4 * l + 1], dz[4 * l + 2], dz[4 * l + 3]);
#pragma unroll
          for (int k = 0; k < 8; ++k) atomicAdd(gl + c.vtx + corner_offset(a.g, l, k), f4scale(d4, wv[k]));
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  write_partials(a, sG, sL);
}

// combine the per-CTA partial rows: decoder gradients in a fixed order into gmlp, losses
// in FP64 normalised by the set sizes (rgb: R, depth: rays with D > 0, sdf: |S_tr|,
// fs: |S_fs|, smooth: valid points) with the weighted total
__global__ void __launch_bounds__(256) paper_combine_kernel(const float* loss_part, const float* mlp_part,
                                                            int nparts, const int* counts, int R, float l0, float l1,
                                                            float l2, float l3, float l4, float* loss, float* gmlp) {
  // decoder gradients: block b owns entries [32b, 32b + 32); warp w sums rows w, w + 8, ...,
  // then warp 0 adds the 8 warps' sums in a fixed order
  __shared__ float part[8][33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  if (gmlp) {
    part[wid][lane] = i < GS_PAPER_MLP_PARAMS ? column_sum8(mlp_part, kPart, i, wid, nparts) : 0.f;
    __syncthreads();
    if (wid == 0 && i < GS_PAPER_MLP_PARAMS) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) t += part[k][lane];
      gmlp[i] += t;
    }
  }
  if (loss && blockIdx.x == 0 && threadIdx.x < 32) {
    double sk[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int p = lane; p < nparts; p += 32)
#pragma unroll
      for (int k = 0; k < 5; ++k) sk[k] += (double)loss_part[(size_t)p * kLossPad + k];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sk[k] += __shfl_xor_sync(0xffffffffu, sk[k], off);
    if (lane == 0) {
      const double den[5] = {(double)R, (double)counts[0], (double)counts[1], (double)counts[2], (double)counts[3]};
      const double lam[5] = {l0, l1, l2, l3, l4};
      double tot = 0.0;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const double v = den[k] > 0 ? sk[k] / den[k] : 0.0;
        loss[k] = (float)v;
        tot += lam[k] * v;
      }
      loss[5] = (float)tot;
    }
  }
}

}  // namespace paper
}  // namespace gs

using namespace gs;

int gs_paper_part_rows(int num_sms) { return paper::kCtasPerSm * num_sms + kSmoothCtas; }
size_t gs_paper_part_floats(int num_sms) { return (size_t)gs_paper_part_rows(num_sms) * paper::kPart; }

gs_status gs_launch_paper(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* grad,
                          float* loss, float* rgb_hat, float* d_hat, float* wsum, int mode, cudaStream_t st) {
  using namespace paper;
  Args a{};
  a.g = ctx->grid;
  a.colour_off = ctx->colour_off;
  a.theta = theta;
  a.grad = grad;
  a.o = b->origin;
  a.r = b->dir;
  a.rgb = b->rgb;
  a.D = b->depth;
  a.t = b->t;
  a.cls = b->cls;
  a.xs = b->xs;
  a.eps = b->eps;
  a.valid = b->valid;
  a.counts = b->counts;
  a.dloss = dloss;
  a.rgb_hat = rgb_hat;
  a.d_hat = d_hat;
  a.wsum = wsum;
  a.w_out = b->w;
  a.dz_out = b->dz;
  a.R = b->R;
  a.N = b->N;
  a.P = b->P;
  a.mode = mode;
  for (int k = 0; k < 5; ++k) a.lam[k] = ctx->cfg.lam[k];
  a.kappa_fs = ctx->cfg.kappa_fs;
  const int render_ctas = ctx->num_sms;  // the tensor-core render kernel: one CTA per SM
  int nparts = 0;
  float* first_loss = ctx->paper_loss_part;
  float* first_mlp = ctx->paper_part;
  // The smoothness kernel is independent of the render kernel (its own partial rows, atomics
  // into grad): on the side stream, forked before the render launch and joined before the
  // combine, it runs on the SMs that the render kernel's last ray-quads leave idle.
  const bool fork = b->R > 0 && b->P > 0;
  if (fork && (cudaEventRecord(ctx->ev_fork, st) != cudaSuccess ||
               cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0) != cudaSuccess))
    return GS_ERR_CUDA;
  if (b->R > 0) {
    const gs_status s = gs_launch_paper_tc(ctx, theta, b, dloss, grad, rgb_hat, d_hat, wsum, mode,
                                           ctx->paper_loss_part, ctx->paper_part, render_ctas, st);
    if (s != GS_OK) return s;
    nparts += render_ctas;
  }
  if (b->P > 0) {
    static bool attr = false;
    if (!attr) {
      if (cudaFuncSetAttribute(paper_smooth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
          cudaSuccess)
        return GS_ERR_CUDA;
      attr = true;
    }
    a.loss_part = ctx->paper_loss_part + (size_t)render_ctas * kLossPad;
    a.mlp_part = ctx->paper_part + (size_t)render_ctas * kPart;
    paper_smooth_kernel<<<kSmoothCtas, kThreads, kSmemBytes, fork ? ctx->side : st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return GS_ERR_CUDA;
    if (fork && (cudaEventRecord(ctx->ev_join, ctx->side) != cudaSuccess ||
                 cudaStreamWaitEvent(st, ctx->ev_join, 0) != cudaSuccess))
      return GS_ERR_CUDA;
    if (b->R == 0) {
      first_loss = a.loss_part;
      first_mlp = a.mlp_part;
    }
    nparts += kSmoothCtas;
  }
  if (nparts == 0) {
    // an empty batch: losses 0, gradient unchanged
    if (mode & 1) {
      if (cudaMemsetAsync(loss, 0, sizeof(float) * GS_NUM_LOSS, st) != cudaSuccess) return GS_ERR_CUDA;
    }
    return GS_OK;
  }
  const float* l = ctx->cfg.lam;
  paper_combine_kernel<<<(GS_PAPER_MLP_PARAMS + 31) / 32, 256, 0, st>>>(
      first_loss, first_mlp, nparts, b->counts, b->R, l[0], l[1], l[2], l[3], l[4], (mode & 1) ? loss : nullptr,
      (mode & 2) ? grad + ctx->grid.n_grid : nullptr);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_paper_eikonal(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss,
                                  float* loss, float* grad, cudaStream_t st) {
  return gs_launch_eikonal_paper_tc(ctx, theta, b, dloss, loss, grad, st);  // csrc/gs_eikonal.cu
}

gs_status gs_launch_paper_query_backward(const gs_ctx* ctx, const float* theta, const float* x, int P,
                                         const float* dsdf, const float* dgrad, float* grad, cudaStream_t st) {
  using namespace paper;
  if (P == 0 || (!dsdf && !dgrad)) return GS_OK;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(paper_query_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes) != cudaSuccess)
      return GS_ERR_CUDA;
    attr = true;
  }
  Args a{};
  a.g = ctx->grid;
  a.colour_off = ctx->colour_off;
  a.theta = theta;
  a.grad = grad;
  a.loss_part = ctx->paper_loss_part;
  a.mlp_part = ctx->paper_part;
  const int want = (P + kWarps * 32 - 1) / (kWarps * 32);
  const int ctas = want < 2 * ctx->num_sms ? want : 2 * ctx->num_sms;  // within the render kernel's partial rows
  paper_query_backward_kernel<<<ctas, kThreads, kSmemBytes, st>>>(a, x, P, dsdf, dgrad);
  if (cudaPeekAtLastError() != cudaSuccess) return GS_ERR_CUDA;
  const float* l = ctx->cfg.lam;
  paper_combine_kernel<<<(GS_PAPER_MLP_PARAMS + 31) / 32, 256, 0, st>>>(
      ctx->paper_loss_part, ctx->paper_part, ctas, nullptr, 0, l[0], l[1], l[2], l[3], l[4], nullptr,
      grad + ctx->grid.n_grid);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_paper_query(const gs_ctx* ctx, const float* theta, const float* x, int P, float* sdf, float* grad,
                                cudaStream_t st) {
  if (P > 0) paper::paper_query_kernel<<<(P + 127) / 128, 128, 0, st>>>(ctx->grid, theta, x, P, sdf, grad);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
