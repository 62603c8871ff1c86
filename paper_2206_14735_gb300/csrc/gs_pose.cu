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

#include "gs_paper.cuh"
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

// the camera direction d of pixel p (unit z; the frame index in f)
__device__ __forceinline__ void pixel_dir(const FramesDev& fr, long long p, long long& f, float d[3]) {
  const long long hw = (long long)fr.H * fr.W;
  f = p / hw;
  const long long rem = p - f * hw;
  const int v = (int)(rem / fr.W), u = (int)(rem - (long long)v * fr.W);
  d[0] = ((float)u + 0.5f - fr.cx) / fr.fx;
  d[1] = ((float)v + 0.5f - fr.cy) / fr.fy;
  d[2] = 1.f;
}

// frame f's six derivatives from a ray's sums go = sum_s g_s and gr = sum_s d_s g_s:
// dL/d dt += go, dL/d nu += J_r(nu)^T [d]_x R^T gr
__device__ __forceinline__ void add_frame_pose_grad(const FramesDev& fr, const float* xi, float* pose_grad, long long f,
                                                    const float d[3], const float go[3], const float gr[3]) {
  const float* Q = fr.c2w + 12 * f;
  float Rt[3];  // R^T gr
#pragma unroll
  for (int q = 0; q < 3; ++q) Rt[q] = Q[q] * gr[0] + Q[4 + q] * gr[1] + Q[8 + q] * gr[2];
  const float w[3] = {d[1] * Rt[2] - d[2] * Rt[1], d[2] * Rt[0] - d[0] * Rt[2], d[0] * Rt[1] - d[1] * Rt[0]};
  float E[3][3], J[3][3];
  const float nu[3] = {xi[6 * f + 3], xi[6 * f + 4], xi[6 * f + 5]};
  so3_exp_jr(nu, E, J);
  float* gp = pose_grad + 6 * f;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    atomicAdd(gp + q, go[q]);
    atomicAdd(gp + 3 + q, J[0][q] * w[0] + J[1][q] * w[1] + J[2][q] * w[2]);
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
      long long f;
      float d[3];
      pixel_dir(a.fr, a.pix[i], f, d);
      if (kPaper) {
        const float inv_dn = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int q = 0; q < 3; ++q) gr[q] = fmaf(gd[q], inv_dn, gr[q]);
      }
      add_frame_pose_grad(a.fr, a.xi, a.pose_grad, f, d, go, gr);
    }
  }
}

// ---- the Eikonal term's pose derivative (x-Hessian of phi) ---------------------------------
// L_eik = mean over the free-space samples of (1 - |g_s|)^2, g_s = grad_x phi(x_s), and the
// samples x_s = o + d_s r move with the pose (depths and classes fixed).  phi = f(z(x)) with f
// piecewise linear (ReLU decoders), so within the ReLU region of x_s, g_s = sum_l J_l^T p_l
// with p = d phi/d z fixed and d g_s / d x_s = H_s = sum_{l,k} p_{l,k} Hess_x z_{l,k}: the
// x-Hessian of a trilinear interpolation has a zero diagonal and the off-diagonal entries
// h_ab = (1 / v_l^2) sum_c theta_c d^2 w_c / (d f_a d f_b) (Supp. Sec. 1: h12, h13, h23),
// zero along a clamped axis.  With a_s = dL/d g_s = dscale (-2 (1 - |g_s|) g_s / (|g_s| n_fs)),
// the sample's position gradient is H_s a_s, summed per ray into the frame's six derivatives
// as for the other terms.

// decoder floats the sensitivity reads, from the start of the decoder block: the workload's
// W1, b1 and row 0 of W2; the paper's gW1, gb1, gW2, gb2, gw3
template <bool kPaper>
constexpr int kSensFloats = kPaper ? paper::S_gb3 : oW2 + kH1;

// p = d phi / d z at z (sd: the decoder floats above in shared memory; hs: 64 floats of the
// calling thread's shared scratch for the paper decoder's hidden layers)
template <bool kPaper>
__device__ __forceinline__ void dphi_dz(const float* sd, const float z[kZ], float* hs, float p[kZ]) {
  float e[kH1];  // d phi / d (layer-1 output), masked
  if constexpr (!kPaper) {
#pragma unroll
    for (int j = 0; j < kH1; ++j) {
      float y = sd[ob1 + j];
#pragma unroll
      for (int k = 0; k < kZ; ++k) y = fmaf(sd[oW1 + j * kZ + k], z[k], y);
      e[j] = y > 0.f ? sd[oW2 + j] : 0.f;
    }
  } else {
    unsigned m1 = 0;
#pragma unroll
    for (int j = 0; j < paper::kH; ++j) {
      float y = sd[paper::S_gb1 + j];
#pragma unroll
      for (int k = 0; k < kZ; ++k) y = fmaf(sd[paper::S_gW1 + j * kZ + k], z[k], y);
      hs[j] = fmaxf(y, 0.f);
      m1 |= (y > 0.f ? 1u : 0u) << j;
    }
    float* e2 = hs + paper::kH;  // masked d phi / d (layer-2 output)
#pragma unroll 1
    for (int j = 0; j < paper::kH; ++j) {
      float y = sd[paper::S_gb2 + j];
      const float* wr = sd + paper::S_gW2 + j * paper::kH;
#pragma unroll
      for (int k = 0; k < paper::kH; ++k) y = fmaf(wr[k], hs[k], y);
      e2[j] = y > 0.f ? sd[paper::S_gw3 + j] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < paper::kH; ++i) {
      float v = 0.f;
#pragma unroll
      for (int j = 0; j < paper::kH; ++j) v = fmaf(sd[paper::S_gW2 + j * paper::kH + i], e2[j], v);
      e[i] = ((m1 >> i) & 1u) ? v : 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < kZ; ++k) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kH1; ++j) s = fmaf(sd[oW1 + j * kZ + k], e[j], s);
    p[k] = s;
  }
}

struct EikPoseArgs {
  FramesDev fr;
  GridDesc g;
  const float* theta;
  const float* xi;
  int R, N;
  const long long* pix;
  const float *o, *r, *t;
  const uint8_t* cls;
  const int* counts;   // counts[2] = |S_fs|
  const float* dloss;  // [1] or nullptr (1)
  float* pose_grad;    // [F][6] (+=)
  // the batch's deferred Eikonal records (written by the Eikonal call on this batch): plane l of
  // sample s holds p_l / v_l, so the sensitivity is read instead of computed; nullptr: computed
  const float4* eik;
  long long eik_stride;
};

// one warp per ray, lanes over its samples (free-space ones only), then lane 0 adds the
// ray's sums to its frame's six derivatives
template <bool kPaper>
__global__ void __launch_bounds__(128) eikonal_pose_kernel(EikPoseArgs a) {
  __shared__ __align__(16) float sd[kSensFloats<kPaper>];
  __shared__ __align__(16) float sp[128][kZ];           // this thread's p, read level by level
  __shared__ float sh[kPaper ? 128 : 1][kPaper ? 65 : 1];  // the paper decoder's hidden layers
  const float* mlp = a.theta + a.g.n_grid;
  for (int i = threadIdx.x; i < kSensFloats<kPaper>; i += blockDim.x) sd[i] = mlp[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int n_fs = a.counts[2];
  const float kscale = n_fs > 0 ? (a.dloss != nullptr ? a.dloss[0] : 1.f) * -2.f / (float)n_fs : 0.f;
  float* myp = sp[threadIdx.x];
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.R; i += (gridDim.x * blockDim.x) >> 5) {
    const float o[3] = {a.o[3 * i], a.o[3 * i + 1], a.o[3 * i + 2]};
    const float r[3] = {a.r[3 * i], a.r[3 * i + 1], a.r[3 * i + 2]};
    float go[3] = {0.f, 0.f, 0.f}, gr[3] = {0.f, 0.f, 0.f};
    for (int k = lane; k < a.N; k += 32) {
      if (a.cls[(size_t)i * a.N + k] != CLS_FS) continue;
      const float tk = a.t[(size_t)i * a.N + k];
      float x[3];
      sample_pos(o, r, tk, x);
      if (a.eik != nullptr) {  // q_l = p_l / v_l from the records
        const float4* rec = a.eik + (size_t)i * a.N + k;
#pragma unroll
        for (int l = 0; l < kLevels; ++l) *reinterpret_cast<float4*>(myp + 4 * l) = __ldg(rec + l * a.eik_stride);
      } else {
        float z[kZ], p[kZ];
#pragma unroll
        for (int l = 0; l < kLevels; ++l) {
          const Cell c = locate(a.g, l, x);
          float w[8];
          corner_weights(c.f, w);
          const float4* lv = reinterpret_cast<const float4*>(a.theta + a.g.off[l]);
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 8; ++q) f4fma(acc, w[q], __ldg(lv + c.vtx + corner_offset(a.g, l, q)));
          z[4 * l] = acc.x;
          z[4 * l + 1] = acc.y;
          z[4 * l + 2] = acc.z;
          z[4 * l + 3] = acc.w;
        }
        dphi_dz<kPaper>(sd, z, kPaper ? sh[threadIdx.x] : nullptr, p);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<float4*>(myp + 4 * q) = make_float4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
      }
      // g = sum_l J_l^T p_l and the Hessian's entries h01, h02, h12, from each level's corners
      float gx[3] = {0.f, 0.f, 0.f}, h01 = 0.f, h02 = 0.f, h12 = 0.f;
#pragma unroll 1
      for (int l = 0; l < kLevels; ++l) {
        const Cell c = locate(a.g, l, x);
        const float4* lv = reinterpret_cast<const float4*>(a.theta + a.g.off[l]);
        const float4 p4 = *reinterpret_cast<const float4*>(myp + 4 * l);
        float4 d0 = make_float4(0.f, 0.f, 0.f, 0.f), d1 = d0, d2 = d0, e01 = d0, e02 = d0, e12 = d0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int bx = (q >> 2) & 1, by = (q >> 1) & 1, bz = q & 1;
          const float wx = bx ? c.f[0] : 1.f - c.f[0], wy = by ? c.f[1] : 1.f - c.f[1], wz = bz ? c.f[2] : 1.f - c.f[2];
          const float sx = bx ? 1.f : -1.f, sy = by ? 1.f : -1.f, sz = bz ? 1.f : -1.f;
          const float4 v = __ldg(lv + c.vtx + corner_offset(a.g, l, q));
          f4fma(d0, sx * wy * wz, v);
          f4fma(d1, wx * sy * wz, v);
          f4fma(d2, wx * wy * sz, v);
          f4fma(e01, sx * sy * wz, v);
          f4fma(e02, sx * wy * sz, v);
          f4fma(e12, wx * sy * sz, v);
        }
        // the records hold p_l already divided by v_l
        const float iv = a.eik != nullptr ? 1.f : a.g.inv_voxel[l];
        const float iv2 = a.eik != nullptr ? a.g.inv_voxel[l] : iv * iv;
        const bool cx = c.clamped & 1u, cy = c.clamped & 2u, cz = c.clamped & 4u;
        const float dot0 = d0.x * p4.x + d0.y * p4.y + d0.z * p4.z + d0.w * p4.w;
        const float dot1 = d1.x * p4.x + d1.y * p4.y + d1.z * p4.z + d1.w * p4.w;
        const float dot2 = d2.x * p4.x + d2.y * p4.y + d2.z * p4.z + d2.w * p4.w;
        if (!cx) gx[0] = fmaf(dot0, iv, gx[0]);
        if (!cy) gx[1] = fmaf(dot1, iv, gx[1]);
        if (!cz) gx[2] = fmaf(dot2, iv, gx[2]);
        if (!cx && !cy) h01 = fmaf(e01.x * p4.x + e01.y * p4.y + e01.z * p4.z + e01.w * p4.w, iv2, h01);
        if (!cx && !cz) h02 = fmaf(e02.x * p4.x + e02.y * p4.y + e02.z * p4.z + e02.w * p4.w, iv2, h02);
        if (!cy && !cz) h12 = fmaf(e12.x * p4.x + e12.y * p4.y + e12.z * p4.z + e12.w * p4.w, iv2, h12);
      }
      const float nrm = sqrtf(gx[0] * gx[0] + gx[1] * gx[1] + gx[2] * gx[2]);
      if (!(nrm > 0.f)) continue;
      const float kk = kscale * (1.f - nrm) / nrm;
      const float av[3] = {kk * gx[0], kk * gx[1], kk * gx[2]};
      const float dx[3] = {h01 * av[1] + h02 * av[2], h01 * av[0] + h12 * av[2], h02 * av[0] + h12 * av[1]};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        go[q] += dx[q];
        gr[q] = fmaf(tk, dx[q], gr[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      go[q] = warp_sum(go[q]);
      gr[q] = warp_sum(gr[q]);
    }
    if (lane == 0) {
      long long f;
      float d[3];
      pixel_dir(a.fr, a.pix[i], f, d);
      add_frame_pose_grad(a.fr, a.xi, a.pose_grad, f, d, go, gr);
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

gs_status gs_launch_eikonal_pose_backward(const gs_ctx* ctx, const float* theta, const gs_frames* f, const float* xi,
                                          const gs_batch* b, const float* dloss, float* pose_grad, cudaStream_t st) {
  if (b->R <= 0) return GS_OK;
  EikPoseArgs a;
  a.fr = FramesDev{f->F, f->H, f->W, f->rgb, f->depth, f->c2w, f->fx, f->fy, f->cx, f->cy};
  a.g = ctx->grid;
  a.theta = theta;
  a.xi = xi;
  a.R = b->R;
  a.N = b->N;
  a.pix = (const long long*)b->pix;
  a.o = b->origin;
  a.r = b->dir;
  a.t = b->t;
  a.cls = b->cls;
  a.counts = b->counts;
  a.dloss = dloss;
  a.pose_grad = pose_grad;
  a.eik = reinterpret_cast<const float4*>(b->eik);
  a.eik_stride = (long long)b->R * b->N;
  const int blocks = (int)std::min<long long>(((long long)b->R * 32 + 127) / 128, 16LL * ctx->num_sms);
  if (ctx->cfg.arch == GS_ARCH_PAPER) eikonal_pose_kernel<true><<<blocks, 128, 0, st>>>(a);
  else eikonal_pose_kernel<false><<<blocks, 128, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
