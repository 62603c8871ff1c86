// SDF-gradient smoothness term (Sec. 3.3, Eq. smoothness_loss) and its second-order adjoint
// (Supp. Sec. 1): L_smooth = mean_p || grad phi(x_p) - grad phi(x_p + eps_p) ||^2 over S_g.
//
// grad_x phi = sum_l (1/v_l) J_l(x)^T p_l with p = d phi/d z = W1^T (m (.) W2[0,:]^T), m the
// ReLU mask (the decoder is piecewise linear, so p does not depend on z almost everywhere).
// For an adjoint a = dL/d(grad phi) at a point y:
//   d/d theta_{l,c,k} = p_{l,k} (1/v_l) (a . dw_c/df)       (Supp. Eq. second_order_theta)
//   d/d W1 = (m (.) W2[0,:]) j^T,  d/d W2[0,:] = m (.) (W1 j), j_k = a . d z_k / d x.
// One lane per point; a warp stages its 32 points' vectors and reduces the decoder
// gradients as 4x4 tiles, as the render kernel does.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

constexpr int kSmoothWarps = 2;  // static shared memory stays under 48 KB
constexpr int kSt = 84;  // staged row: mw2[32] | j[16] | u[32] (+4 pad), stride = 20 mod 32 banks
constexpr int sMw2 = 0, sJ = 32, sU = 48;

struct SmoothRunArgs {
  GridDesc g;
  const float* theta;
  int P;
  const float *xs, *eps;
  const uint8_t* valid;
  const int* counts;
  const float* dloss;
  float lam4;
  float* grad;
  float* loss_part;  // rows for this kernel's CTAs
  float* mlp_part;
};

__device__ __forceinline__ float4 ldv(const float* p) { return *reinterpret_cast<const float4*>(p); }

// z at y (all levels), values only
__device__ __forceinline__ void features_only(const GridDesc& g, const float* __restrict__ theta, const float y[3],
                                              float z[kZ]) {
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell c = locate(g, l, y);
    float w[8];
    corner_weights(c.f, w);
    const float4* base = reinterpret_cast<const float4*>(theta + g.off[l]);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f4fma(acc, w[k], __ldg(base + c.vtx + corner_offset(g, l, k)));
    z[4 * l] = acc.x;
    z[4 * l + 1] = acc.y;
    z[4 * l + 2] = acc.z;
    z[4 * l + 3] = acc.w;
  }
}
// ReLU mask m (bit j = unit j on), m (.) W2[0,:], and p = d phi / d z
__device__ __forceinline__ unsigned phi_sensitivity(const float* sm, const float z[kZ], float mw2[kH1], float p[kZ]) {
  unsigned mask = 0;
#pragma unroll
  for (int j = 0; j < kH1; ++j) {
    float s = sm[sb1 + j];
#pragma unroll
    for (int k = 0; k < kZ; ++k) s = fmaf(sm[sW1 + j * 16 + k], z[k], s);
    mw2[j] = s > 0.f ? sm[sW2 + j] : 0.f;
    mask |= (s > 0.f ? 1u : 0u) << j;
  }
#pragma unroll
  for (int k = 0; k < kZ; ++k) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kH1; ++j) s = fmaf(sm[sW1 + j * 16 + k], mw2[j], s);
    p[k] = s;
  }
  return mask;
}

// layer-1 ReLU output a1 = max(W1 z + b1, 0) of the SDF decoder
__device__ __forceinline__ void sdf_layer1(const float* sm, const float z[kZ], float a1[kH1]) {
#pragma unroll
  for (int j = 0; j < kH1; ++j) {
    float s = sm[sb1 + j];
#pragma unroll
    for (int k = 0; k < kZ; ++k) s = fmaf(sm[sW1 + j * 16 + k], z[k], s);
    a1[j] = fmaxf(s, 0.f);
  }
}

template <bool FWD, bool BWD>
__global__ void __launch_bounds__(kSmoothWarps * 32, 1) smooth_kernel(SmoothRunArgs a) {
  __shared__ __align__(16) float sm[kSmemMlp];
  __shared__ __align__(16) float acc[kMlpPad + kLossPad];
  __shared__ __align__(16) float stage[kSmoothWarps][32 * kSt];
  const float* mlp = a.theta + a.g.n_grid;
  for (int i = threadIdx.x; i < kSmemMlp; i += blockDim.x) {
    float v = 0.0f;
    if (i < sb1) v = mlp[oW1 + i];
    else if (i < sW2) v = mlp[ob1 + i - sb1];
    else if (i < sb2) v = mlp[oW2 + i - sW2];
    sm[i] = v;
  }
  for (int i = threadIdx.x; i < kMlpPad + kLossPad; i += blockDim.x) acc[i] = 0.0f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* st = stage[warp];
  const int n_g = a.counts[3];
  const float k_sm = n_g > 0 ? (a.dloss[4] + a.lam4 * a.dloss[5]) * 2.0f / (float)n_g : 0.0f;
  float l_sm = 0.f;

  // one lane per gradient evaluation: lanes 2q and 2q+1 evaluate point q at x and x + eps
#pragma unroll 1
  for (int base = (blockIdx.x * kSmoothWarps + warp) * 16; base < a.P; base += gridDim.x * kSmoothWarps * 16) {
    const int p = base + (lane >> 1), e = lane & 1;
    const bool valid = p < a.P && a.valid[p];
    float y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) y[k] = valid ? (e == 0 ? a.xs[3 * p + k] : __fadd_rn(a.xs[3 * p + k], a.eps[3 * p + k])) : 0.f;
    float pz[kZ], mw2[kH1];
    unsigned mask;
    {
      float z[kZ];
      features_only(a.g, a.theta, y, z);
      mask = phi_sensitivity(sm, z, mw2, pz);
    }
    float gq[3] = {0.f, 0.f, 0.f};  // grad_x phi = sum_l (dz_l/dx)^T p_l
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
      float4 dl[3];
      float dw[8][3];
      level_jacobian(a.g, a.theta, l, y, dl, dw);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        gq[q] += pz[4 * l] * dl[q].x + pz[4 * l + 1] * dl[q].y + pz[4 * l + 2] * dl[q].z + pz[4 * l + 3] * dl[q].w;
    }
    float dg[3];  // g(x) - g(x + eps), on both lanes of the pair
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float other = __shfl_xor_sync(0xffffffffu, gq[q], 1);
      dg[q] = e == 0 ? gq[q] - other : other - gq[q];
    }
    if (FWD && valid && e == 0) l_sm += dg[0] * dg[0] + dg[1] * dg[1] + dg[2] * dg[2];
    if constexpr (!BWD) continue;
    const float sgn = e == 0 ? 1.f : -1.f;
    const float av[3] = {valid ? sgn * k_sm * dg[0] : 0.f, valid ? sgn * k_sm * dg[1] : 0.f,
                         valid ? sgn * k_sm * dg[2] : 0.f};
    // per level: j_l = a . dz_l/dx, and the direct term d/d theta_{l,c,k} = p_{l,k} (1/v_l) (a . dw_c/df)
    float jv[kZ];
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
      float4 dl[3];
      float dw[8][3];
      const Cell c = level_jacobian(a.g, a.theta, l, y, dl, dw);
      jv[4 * l] = av[0] * dl[0].x + av[1] * dl[1].x + av[2] * dl[2].x;
      jv[4 * l + 1] = av[0] * dl[0].y + av[1] * dl[1].y + av[2] * dl[2].y;
      jv[4 * l + 2] = av[0] * dl[0].z + av[1] * dl[1].z + av[2] * dl[2].z;
      jv[4 * l + 3] = av[0] * dl[0].w + av[1] * dl[1].w + av[2] * dl[2].w;
      if (valid) {
        const float iv = a.g.inv_voxel[l];
        const float4 p4 = make_float4(pz[4 * l], pz[4 * l + 1], pz[4 * l + 2], pz[4 * l + 3]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float ad = (av[0] * dw[k][0] + av[1] * dw[k][1] + av[2] * dw[k][2]) * iv;
          atomicAdd(reinterpret_cast<float4*>(a.grad + a.g.off[l]) + c.vtx + corner_offset(a.g, l, k), f4scale(p4, ad));
        }
      }
    }
    float* row = st + lane * kSt;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(row + sMw2 + 4 * q) = make_float4(mw2[4 * q], mw2[4 * q + 1], mw2[4 * q + 2], mw2[4 * q + 3]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(row + sJ + 4 * q) = make_float4(jv[4 * q], jv[4 * q + 1], jv[4 * q + 2], jv[4 * q + 3]);
    // d/d W2[0][j] = m_j (W1 j)_j
#pragma unroll
    for (int j = 0; j < kH1; ++j) {
      float u = 0.f;
      if ((mask >> j) & 1u) {
#pragma unroll
        for (int k = 0; k < kZ; ++k) u = fmaf(sm[sW1 + j * 16 + k], jv[k], u);
      }
      row[sU + j] = u;
    }
    __syncwarp();
    {  // dW1[32][16] += mw2 (x) j over the warp's 32 evaluations
      const int i0 = 4 * (lane >> 2), j0 = 4 * (lane & 3);
      float t[4][4] = {};
#pragma unroll 4
      for (int s2 = 0; s2 < 32; ++s2) {
        const float4 av4 = ldv(st + s2 * kSt + sMw2 + i0), bv4 = ldv(st + s2 * kSt + sJ + j0);
        const float ar[4] = {av4.x, av4.y, av4.z, av4.w}, br[4] = {bv4.x, bv4.y, bv4.z, bv4.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int q = 0; q < 4; ++q) t[x][q] = fmaf(ar[x], br[q], t[x][q]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(acc + oW1 + (i0 + x) * kZ + j0 + q, t[x][q]);
      float u = 0.f;  // dW2[0][lane] += sum_s u_s[lane]
#pragma unroll 4
      for (int s2 = 0; s2 < 32; ++s2) u += st[s2 * kSt + sU + lane];
      atomicAdd(acc + oW2 + lane, u);
    }
    __syncwarp();
  }
  if (FWD) {
    l_sm = warp_sum(l_sm);
    if (lane == 0) atomicAdd(acc + kMlpPad + 4, l_sm);
  }
  __syncthreads();
  if (threadIdx.x < kLossPad) a.loss_part[(size_t)blockIdx.x * kLossPad + threadIdx.x] = acc[kMlpPad + threadIdx.x];
  for (int i = threadIdx.x; i < kMlpPad; i += blockDim.x) a.mlp_part[(size_t)blockIdx.x * kMlpPad + i] = acc[i];
}

// ------------------------------------------------------------------------------------
// Reverse mode of the SDF query: grad += sum_p dsdf_p d phi(x_p)/d theta
//                                        + dgrad_p . d grad_x phi(x_p)/d theta.
// First order (Sec. 3.1): d phi/d z = p, so the grid gets p_{l,f} w_c and the decoder the
// usual dense-layer terms.  Second order (Supp. Sec. 1, as in the smoothness adjoint): with
// a = dgrad_p and j_k = a . d z_k/d x, the grid gets p_{l,f} (1/v_l)(a . d w_c/d f) and the
// decoder d/d W1 = (m (.) W2[0,:]) j^T, d/d W2[0,:] = m (.) (W1 j).  Combined per point:
//   dW1 += (m (.) W2[0,:]) (dsdf z + j)^T,  db1 += dsdf (m (.) W2[0,:]),
//   dW2[0,:] += dsdf a1 + m (.) (W1 j),     db2[0] += dsdf.
// One lane per point; the decoder gradients are reduced per warp as in the smoothness kernel.
// ------------------------------------------------------------------------------------
struct QueryBwdArgs {
  GridDesc g;
  const float* theta;
  const float* x;
  int P;
  const float* dsdf;   // [P] or nullptr
  const float* dgrad;  // [P][3] or nullptr
  float* grad;
};

__global__ void __launch_bounds__(kSmoothWarps * 32) query_backward_kernel(QueryBwdArgs a) {
  __shared__ __align__(16) float sm[kSmemMlp];
  __shared__ __align__(16) float acc[kH1 * kZ + kH1 + kH1 + 4];  // dW1 | db1 | dW2[0,:] | db2[0]
  __shared__ __align__(16) float stage[kSmoothWarps][32 * kSt];
  constexpr int aW1 = 0, ab1 = kH1 * kZ, aW2 = ab1 + kH1, ab2 = aW2 + kH1, kAcc = ab2 + 4;
  const float* mlp = a.theta + a.g.n_grid;
  for (int i = threadIdx.x; i < kSmemMlp; i += blockDim.x) {
    float v = 0.0f;
    if (i < sb1) v = mlp[oW1 + i];
    else if (i < sW2) v = mlp[ob1 + i - sb1];
    else if (i < sb2) v = mlp[oW2 + i - sW2];
    sm[i] = v;
  }
  for (int i = threadIdx.x; i < kAcc; i += blockDim.x) acc[i] = 0.0f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* st = stage[warp];
  float db2 = 0.f;
  for (int base = (blockIdx.x * kSmoothWarps + warp) * 32; base < a.P; base += gridDim.x * kSmoothWarps * 32) {
    const int p = base + lane;
    const bool valid = p < a.P;
    float y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) y[k] = valid ? a.x[3 * p + k] : 0.f;
    const float ds = (valid && a.dsdf) ? a.dsdf[p] : 0.f;
    float av[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) av[k] = (valid && a.dgrad) ? a.dgrad[3 * p + k] : 0.f;
    float z[kZ], a1[kH1], mw2[kH1], pz[kZ];
    features_only(a.g, a.theta, y, z);
    sdf_layer1(sm, z, a1);
    const unsigned mask = phi_sensitivity(sm, z, mw2, pz);
    float jv[kZ];
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
      float4 dl[3];
      float dw[8][3], w[8];
      const Cell c = level_jacobian(a.g, a.theta, l, y, dl, dw);
      corner_weights(c.f, w);
      jv[4 * l] = av[0] * dl[0].x + av[1] * dl[1].x + av[2] * dl[2].x;
      jv[4 * l + 1] = av[0] * dl[0].y + av[1] * dl[1].y + av[2] * dl[2].y;
      jv[4 * l + 2] = av[0] * dl[0].z + av[1] * dl[1].z + av[2] * dl[2].z;
      jv[4 * l + 3] = av[0] * dl[0].w + av[1] * dl[1].w + av[2] * dl[2].w;
      if (valid) {
        const float iv = a.g.inv_voxel[l];
        const float4 p4 = make_float4(pz[4 * l], pz[4 * l + 1], pz[4 * l + 2], pz[4 * l + 3]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float coef = ds * w[k] + (av[0] * dw[k][0] + av[1] * dw[k][1] + av[2] * dw[k][2]) * iv;
          atomicAdd(reinterpret_cast<float4*>(a.grad + a.g.off[l]) + c.vtx + corner_offset(a.g, l, k), f4scale(p4, coef));
        }
      }
    }
    float* row = st + lane * kSt;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(row + sMw2 + 4 * q) = make_float4(mw2[4 * q], mw2[4 * q + 1], mw2[4 * q + 2], mw2[4 * q + 3]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(row + sJ + 4 * q) =
          make_float4(fmaf(ds, z[4 * q], jv[4 * q]), fmaf(ds, z[4 * q + 1], jv[4 * q + 1]),
                      fmaf(ds, z[4 * q + 2], jv[4 * q + 2]), fmaf(ds, z[4 * q + 3], jv[4 * q + 3]));
#pragma unroll
    for (int j = 0; j < kH1; ++j) {
      float u = 0.f;
      if ((mask >> j) & 1u) {
#pragma unroll
        for (int k = 0; k < kZ; ++k) u = fmaf(sm[sW1 + j * 16 + k], jv[k], u);
      }
      row[sU + j] = fmaf(ds, a1[j], u);
    }
    row[80] = ds;
    db2 += ds;
    __syncwarp();
    {  // dW1[32][16] += mw2 (x) (ds z + j) over the warp's 32 points; dW2[0][lane], db1[lane]
      const int i0 = 4 * (lane >> 2), j0 = 4 * (lane & 3);
      float t[4][4] = {};
#pragma unroll 4
      for (int s2 = 0; s2 < 32; ++s2) {
        const float4 av4 = ldv(st + s2 * kSt + sMw2 + i0), bv4 = ldv(st + s2 * kSt + sJ + j0);
        const float ar[4] = {av4.x, av4.y, av4.z, av4.w}, br[4] = {bv4.x, bv4.y, bv4.z, bv4.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int q = 0; q < 4; ++q) t[x][q] = fmaf(ar[x], br[q], t[x][q]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(acc + aW1 + (i0 + x) * kZ + j0 + q, t[x][q]);
      float u = 0.f, b = 0.f;
#pragma unroll 4
      for (int s2 = 0; s2 < 32; ++s2) {
        u += st[s2 * kSt + sU + lane];
        b = fmaf(st[s2 * kSt + 80], st[s2 * kSt + sMw2 + lane], b);
      }
      atomicAdd(acc + aW2 + lane, u);
      atomicAdd(acc + ab1 + lane, b);
    }
    __syncwarp();
  }
  db2 = warp_sum(db2);
  if (lane == 0) atomicAdd(acc + ab2, db2);
  __syncthreads();
  float* gm = a.grad + a.g.n_grid;
  for (int i = threadIdx.x; i < kAcc; i += blockDim.x) {
    const float v = acc[i];
    if (v == 0.f) continue;
    if (i < ab1) atomicAdd(gm + oW1 + i, v);
    else if (i < aW2) atomicAdd(gm + ob1 + i - ab1, v);
    else if (i < ab2) atomicAdd(gm + oW2 + i - aW2, v);  // row 0 of W2
    else if (i == ab2) atomicAdd(gm + ob2, v);
  }
}

}  // namespace gs

using namespace gs;

gs_status gs_launch_query_backward(const gs_ctx* ctx, const float* theta, const float* x, int P, const float* dsdf,
                                   const float* dgrad, float* grad, cudaStream_t st) {
  if (P <= 0 || (!dsdf && !dgrad)) return GS_OK;
  QueryBwdArgs a;
  a.g = ctx->grid;
  a.theta = theta;
  a.x = x;
  a.P = P;
  a.dsdf = dsdf;
  a.dgrad = dgrad;
  a.grad = grad;
  const int per = kSmoothWarps * 32;
  const int blocks = (int)std::min<long long>(((long long)P + per - 1) / per, 8LL * ctx->num_sms);
  query_backward_kernel<<<blocks, per, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_smooth(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* grad,
                           int mode, cudaStream_t st) {
  if (b->P <= 0) return GS_OK;
  SmoothRunArgs a;
  a.g = ctx->grid;
  a.theta = theta;
  a.P = b->P;
  a.xs = b->xs;
  a.eps = b->eps;
  a.valid = b->valid;
  a.counts = b->counts;
  a.dloss = dloss;
  a.lam4 = ctx->cfg.lam[4];
  a.grad = grad;
  a.loss_part = ctx->loss_part + (size_t)ctx->render_ctas * kLossPad;
  a.mlp_part = ctx->mlp_part + (size_t)ctx->render_ctas * kMlpPad;
  if (mode == 1) smooth_kernel<true, false><<<kSmoothCtas, kSmoothWarps * 32, 0, st>>>(a);
  else if (mode == 2) smooth_kernel<false, true><<<kSmoothCtas, kSmoothWarps * 32, 0, st>>>(a);
  else smooth_kernel<true, true><<<kSmoothCtas, kSmoothWarps * 32, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
