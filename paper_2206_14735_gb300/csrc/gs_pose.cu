// Camera-pose refinement (Sec. 3.4: the optimised parameters include the poses; Sec. 4: a
// translation t in R^3 and nu in so(3) per frame, learning rate 5e-4).
//
// Frame f's pose is its given camera-to-world [R0 | t0] corrected by xi_f = (dt, nu):
// R = R0 Exp(nu) (Rodrigues), t = t0 + dt.  A ray's samples x_s = o + d_s r move with the pose
// (o = t, r = R d, d the pixel's camera direction with unit z), their depths d_s do not, so
// with g_s = dL/dx_s = sum_l (d z_l / d x)^T dL/dz_l (dL/dz from the backward pass):
//   dL/d dt = sum over the frame's rays of sum_s g_s,
//   dL/d nu = J_r(nu)^T [d]_x R^T sum_s d_s g_s,
// J_r the right Jacobian of Exp: I - (1 - cos a)/a^2 [nu]_x + (a - sin a)/a^3 [nu]_x^2, a = |nu|.
#include <algorithm>

#include "gs_sample.cuh"

namespace gs {

// E = Exp(nu), J = J_r(nu) (series below |nu| = 1e-2, where the closed forms lose digits in FP32)
__device__ __forceinline__ void so3_exp_jr(const float nu[3], float E[3][3], float J[3][3]) {
  const float a2 = nu[0] * nu[0] + nu[1] * nu[1] + nu[2] * nu[2], a = sqrtf(a2);
  const float K[3][3] = {{0.f, -nu[2], nu[1]}, {nu[2], 0.f, -nu[0]}, {-nu[1], nu[0], 0.f}};
  float K2[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) K2[i][j] = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
  float s1, s2, j1, j2;
  if (a < 1e-2f) {
    s1 = 1.f - a2 / 6.f;
    s2 = 0.5f - a2 / 24.f;
    j1 = 0.5f - a2 / 24.f;
    j2 = 1.f / 6.f - a2 / 120.f;
  } else {
    s1 = sinf(a) / a;
    s2 = (1.f - cosf(a)) / a2;
    j1 = s2;
    j2 = (a - sinf(a)) / (a2 * a);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float I = i == j ? 1.f : 0.f;
      E[i][j] = I + s1 * K[i][j] + s2 * K2[i][j];
      J[i][j] = I - j1 * K[i][j] + j2 * K2[i][j];
    }
}

__global__ void pose_apply_kernel(const float* __restrict__ c2w0, const float* __restrict__ xi, int F,
                                  float* __restrict__ c2w) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  float E[3][3], J[3][3];
  const float nu[3] = {xi[6 * f + 3], xi[6 * f + 4], xi[6 * f + 5]};
  so3_exp_jr(nu, E, J);
  const float* P = c2w0 + 12 * f;
  float* Q = c2w + 12 * f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[4 * i + j] = P[4 * i] * E[0][j] + P[4 * i + 1] * E[1][j] + P[4 * i + 2] * E[2][j];
    Q[4 * i + 3] = P[4 * i + 3] + xi[6 * f + i];
  }
}

struct PoseBwdArgs {
  FramesDev fr;  // the refined poses (c2w) the batch was sampled with
  GridDesc g;
  long long colour_off;  // paper architecture: float offset of the colour grid
  const float* theta;
  const float* xi;
  int R, N;
  const long long* pix;
  const float *o, *r, *t, *dz;
  float* pose_grad;  // [F][6] (+=)
};

// one warp per ray: lanes over its samples, then lane 0 turns the ray's sums into the frame's
// six pose derivatives.  kPaper (the paper's architecture): each sample's record holds 32
// floats, dL/dz (16), dL/dW_beta(x) (6) and dL/d(viewing direction) (3); the colour grid's
// x-derivative adds to g_s, and the direction r/|r| = R d/|d| adds dL/d(direction) / |d| to
// the rotation's moment.
template <bool kPaper>
__global__ void __launch_bounds__(128) pose_backward_kernel(PoseBwdArgs a) {
  constexpr int kRec = kPaper ? 32 : kZ;  // floats per sample record
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.R; i += (gridDim.x * blockDim.x) >> 5) {
    const float o[3] = {a.o[3 * i], a.o[3 * i + 1], a.o[3 * i + 2]};
    const float r[3] = {a.r[3 * i], a.r[3 * i + 1], a.r[3 * i + 2]};
    float go[3] = {0.f, 0.f, 0.f}, gr[3] = {0.f, 0.f, 0.f}, gd[3] = {0.f, 0.f, 0.f};
    for (int k = lane; k < a.N; k += 32) {
      const float tk = a.t[(size_t)i * a.N + k];
      float x[3];
      sample_pos(o, r, tk, x);
      const float4* dzk = reinterpret_cast<const float4*>(a.dz + ((size_t)i * a.N + k) * kRec);
      float gx[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        float4 dl[3];
        float dw[8][3];
        const Cell c = level_jacobian(a.g, a.theta, l, x, dl, dw);
        const float4 d4 = dzk[l];
#pragma unroll
        for (int q = 0; q < 3; ++q) gx[q] += dl[q].x * d4.x + dl[q].y * d4.y + dl[q].z * d4.z + dl[q].w * d4.w;
        if (kPaper && l == kLevels - 1) {  // colour grid on the finest level's cell
          const float4 c0 = dzk[4], c1 = dzk[5];
          const float dcf[6] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y};
          gd[0] += c1.z;
          gd[1] += c1.w;
          gd[2] += dzk[6].x;
          const float2* cg = reinterpret_cast<const float2*>(a.theta + a.colour_off);
          const float iv = a.g.inv_voxel[l];
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const long long v2 = (c.vtx + corner_offset(a.g, l, cc)) * 3;
            float sf = 0.f;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
              const float2 f2 = __ldg(cg + v2 + e);
              sf = fmaf(f2.x, dcf[2 * e], sf);
              sf = fmaf(f2.y, dcf[2 * e + 1], sf);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) gx[q] = fmaf(sf * iv, dw[cc][q], gx[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        go[q] += gx[q];
        gr[q] = fmaf(tk, gx[q], gr[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      go[q] = warp_sum(go[q]);
      gr[q] = warp_sum(gr[q]);
      if (kPaper) gd[q] = warp_sum(gd[q]);
    }
    if (lane == 0) {
      const long long hw = (long long)a.fr.H * a.fr.W;
      const long long p = a.pix[i], f = p / hw, rem = p - f * hw;
      const int v = (int)(rem / a.fr.W), u = (int)(rem - (long long)v * a.fr.W);
      const float d[3] = {((float)u + 0.5f - a.fr.cx) / a.fr.fx, ((float)v + 0.5f - a.fr.cy) / a.fr.fy, 1.f};
      if (kPaper) {
        const float inv_dn = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int q = 0; q < 3; ++q) gr[q] = fmaf(gd[q], inv_dn, gr[q]);
      }
      const float* Q = a.fr.c2w + 12 * f;
      float Rt[3];  // R^T gr
#pragma unroll
      for (int q = 0; q < 3; ++q) Rt[q] = Q[q] * gr[0] + Q[4 + q] * gr[1] + Q[8 + q] * gr[2];
      const float w[3] = {d[1] * Rt[2] - d[2] * Rt[1], d[2] * Rt[0] - d[0] * Rt[2], d[0] * Rt[1] - d[1] * Rt[0]};
      float E[3][3], J[3][3];
      const float nu[3] = {a.xi[6 * f + 3], a.xi[6 * f + 4], a.xi[6 * f + 5]};
      so3_exp_jr(nu, E, J);
      float* gp = a.pose_grad + 6 * f;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        atomicAdd(gp + q, go[q]);
        atomicAdd(gp + 3 + q, J[0][q] * w[0] + J[1][q] * w[1] + J[2][q] * w[2]);
      }
    }
  }
}

}  // namespace gs

using namespace gs;

gs_status gs_launch_pose_apply(const float* c2w0, const float* xi, int F, float* c2w, cudaStream_t st) {
  if (F > 0) pose_apply_kernel<<<(F + 127) / 128, 128, 0, st>>>(c2w0, xi, F, c2w);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_pose_backward(const gs_ctx* ctx, const float* theta, const gs_frames* f, const float* xi,
                                  const gs_batch* b, float* pose_grad, cudaStream_t st) {
  if (b->R <= 0) return GS_OK;
  PoseBwdArgs a;
  a.fr = FramesDev{f->F, f->H, f->W, f->rgb, f->depth, f->c2w, f->fx, f->fy, f->cx, f->cy};
  a.g = ctx->grid;
  a.colour_off = ctx->colour_off;
  a.theta = theta;
  a.xi = xi;
  a.R = b->R;
  a.N = b->N;
  a.pix = (const long long*)b->pix;
  a.o = b->origin;
  a.r = b->dir;
  a.t = b->t;
  a.dz = b->dz;
  a.pose_grad = pose_grad;
  const int blocks = (int)std::min<long long>(((long long)b->R * 32 + 127) / 128, 16LL * ctx->num_sms);
  if (ctx->cfg.arch == GS_ARCH_PAPER) pose_backward_kernel<true><<<blocks, 128, 0, st>>>(a);
  else pose_backward_kernel<false><<<blocks, 128, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
