// Fused per-ray pass of one GO-Surf step: multi-level trilinear gather (Sec. 3.1), geometry
// and colour decoders, NeuS compositing (Sec. 3.2), the rgb / depth / sdf / free-space
// losses (Sec. 3.2-3.4) and, in the same pass, their reverse mode down to the grid
// features and decoder weights.
//
// Mapping: a persistent grid of one CTA per SM; each warp owns one ray at a time and its
// lanes own the samples 32*j + lane (chunk j).  The compositing transmittance is a warp
// product scan with a carry across chunks; its adjoint is a reversed warp scan of affine
// maps.  Decoder weight gradients are sums over samples: each chunk stages its per-sample
// vectors in shared memory and every lane reduces a 4x4 tile of each weight matrix over the
// chunk's 32 samples, then adds the tile into the CTA's shared accumulator.  Grid gradients
// are scattered with 16-byte vector atomics (the coarsest level accumulates in shared
// memory first).
#pragma once
#include "gs_internal.h"

namespace gs {

constexpr int kRenderWarps = 6;
constexpr int kStage = 164;  // floats per staged sample row (row stride = 4 mod 32 banks)
// staged row layout
constexpr int stDpre = 0, stA2 = 4, stH = 36, stDy2 = 52, stA1 = 84, stDout = 116, stDy1 = 132;
constexpr int kLvl0MaxVerts = 512;  // keeps the largest configuration under 227 KB of shared memory

struct RenderArgs {
  GridDesc g;
  const float* theta;
  int R, N;
  const float *o, *r, *rgb, *D, *t;
  const uint8_t* cls;
  const int* counts;
  const float* dloss;
  float lam[5];
  float kappa_fs;
  float* grad;
  float* loss_part;
  float* mlp_part;
  float *rgb_hat, *d_hat, *wsum;
  int lvl0_staged;
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// arr[j] for a runtime j without forcing the register array into local memory
template <int N>
__device__ __forceinline__ float pick(const float (&arr)[N], int j) {
  float v = arr[0];
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (q == j) v = arr[q];
  return v;
}

// z = [V^0(x), .., V^3(x)]: trilinear interpolation at every level, concatenated coarse->fine
__device__ __forceinline__ void gather(const GridDesc& g, const float* __restrict__ theta, const float4* lvl0,
                                       const float x[3], float z[kZ]) {
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell c = locate(g, l, x);
    float w[8];
    corner_weights(c.f, w);
    float4 v[8];
    if (l == 0 && lvl0 != nullptr) {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = lvl0[c.vtx + corner_offset(g, l, k)];
    } else {
      const float4* base = reinterpret_cast<const float4*>(theta + g.off[l]);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldg(base + c.vtx + corner_offset(g, l, k));
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f4fma(acc, w[k], v[k]);
    z[4 * l + 0] = acc.x;
    z[4 * l + 1] = acc.y;
    z[4 * l + 2] = acc.z;
    z[4 * l + 3] = acc.w;
  }
}

// geometry decoder 16 -> 32 (ReLU) -> 16 (phi, h_1..h_15); colour decoder 15 -> 32 (ReLU) -> 3 (sigmoid)
__device__ __forceinline__ void decode(const float* __restrict__ sm, const float z[kZ], float a1[kH1], float out[kOut],
                                       float a2[kH2], float c[kRGB]) {
#pragma unroll
  for (int j = 0; j < kH1; ++j) {
    float s = sm[sb1 + j];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 wv = ld4(sm + sW1 + j * 16 + 4 * q);
      s = fmaf(wv.x, z[4 * q], s);
      s = fmaf(wv.y, z[4 * q + 1], s);
      s = fmaf(wv.z, z[4 * q + 2], s);
      s = fmaf(wv.w, z[4 * q + 3], s);
    }
    a1[j] = fmaxf(s, 0.0f);
  }
#pragma unroll
  for (int j = 0; j < kOut; ++j) {
    float s = sm[sb2 + j];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 wv = ld4(sm + sW2 + j * 32 + 4 * q);
      s = fmaf(wv.x, a1[4 * q], s);
      s = fmaf(wv.y, a1[4 * q + 1], s);
      s = fmaf(wv.z, a1[4 * q + 2], s);
      s = fmaf(wv.w, a1[4 * q + 3], s);
    }
    out[j] = s;
  }
#pragma unroll
  for (int j = 0; j < kH2; ++j) {
    float s = sm[sb3 + j];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 wv = ld4(sm + sW3 + j * 16 + 4 * q);  // padded column 15 is zero
      s = fmaf(wv.x, out[1 + 4 * q], s);
      s = fmaf(wv.y, out[2 + 4 * q], s);
      s = fmaf(wv.z, out[3 + 4 * q], s);
      if (q < 3) s = fmaf(wv.w, out[4 + 4 * q], s);
    }
    a2[j] = fmaxf(s, 0.0f);
  }
#pragma unroll
  for (int j = 0; j < kRGB; ++j) {
    float s = sm[sb4 + j];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 wv = ld4(sm + sW4 + j * 32 + 4 * q);
      s = fmaf(wv.x, a2[4 * q], s);
      s = fmaf(wv.y, a2[4 * q + 1], s);
      s = fmaf(wv.z, a2[4 * q + 2], s);
      s = fmaf(wv.w, a2[4 * q + 3], s);
    }
    c[j] = sigmoidf_(s);
  }
}

// acc[4][4] = sum over the chunk's 32 staged samples of A[s][i0..i0+3] (x) B[s][j0..j0+3]
__device__ __forceinline__ void tile_sum(const float* A, int lda, const float* B, int ldb, float acc[4][4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
  for (int s = 0; s < 32; ++s) {
    const float4 av = ld4(A + s * lda), bv = ld4(B + s * ldb);
    const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ar[a], br[b], acc[a][b]);
  }
}

// reduce the decoder-weight gradients of one staged chunk into the CTA accumulator
__device__ __forceinline__ void chunk_weight_grads(const float* stage, const float* zc, float* acc, int lane) {
  float t[4][4];
  {  // dW1[32][16] += dy1 (x) z
    const int i0 = 4 * (lane >> 2), j0 = 4 * (lane & 3);
    tile_sum(stage + stDy1 + i0, kStage, zc + j0, kZ, t);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) atomicAdd(acc + oW1 + (i0 + a) * kZ + j0 + b, t[a][b]);
  }
  {  // dW2[16][32] += dout (x) a1
    const int i0 = 4 * (lane >> 3), j0 = 4 * (lane & 7);
    tile_sum(stage + stDout + i0, kStage, stage + stA1 + j0, kStage, t);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) atomicAdd(acc + oW2 + (i0 + a) * kH1 + j0 + b, t[a][b]);
  }
  {  // dW3[32][15] += dy2 (x) h
    const int i0 = 4 * (lane >> 2), j0 = 4 * (lane & 3);
    tile_sum(stage + stDy2 + i0, kStage, stage + stH + j0, kStage, t);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (j0 + b < kHF) atomicAdd(acc + oW3 + (i0 + a) * kHF + j0 + b, t[a][b]);
  }
  // dW4[3][32] += dpre (x) a2 (column `lane`), and the four bias vectors
  float w4[3] = {0.f, 0.f, 0.f}, db1 = 0.f, db2 = 0.f, db3 = 0.f, db4 = 0.f;
#pragma unroll 4
  for (int s = 0; s < 32; ++s) {
    const float* row = stage + s * kStage;
    const float a2v = row[stA2 + lane];
    w4[0] = fmaf(row[stDpre + 0], a2v, w4[0]);
    w4[1] = fmaf(row[stDpre + 1], a2v, w4[1]);
    w4[2] = fmaf(row[stDpre + 2], a2v, w4[2]);
    db1 += row[stDy1 + lane];
    db3 += row[stDy2 + lane];
    db2 += row[stDout + (lane & 15)];
    db4 += row[stDpre + (lane & 3)];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) atomicAdd(acc + oW4 + j * kH2 + lane, w4[j]);
  atomicAdd(acc + ob1 + lane, db1);
  atomicAdd(acc + ob3 + lane, db3);
  if (lane < 16) atomicAdd(acc + ob2 + lane, db2);
  if (lane < 3) atomicAdd(acc + ob4 + lane, db4);
}

template <int NCH, bool FWD, bool BWD>
__global__ void __launch_bounds__(kRenderWarps * 32, 1) render_kernel(RenderArgs a) {
  extern __shared__ __align__(16) float smem[];
  float* sm = smem;                       // decoders [kSmemMlp]
  float* acc = sm + kSmemMlp;             // decoder gradient accumulator [kMlpPad]
  float* lacc = acc + kMlpPad;            // loss sums [8]
  float* lvl0 = lacc + kLossPad;          // coarsest level values (staged) [n0*4]
  const int n0 = a.g.dims[0][0] * a.g.dims[0][1] * a.g.dims[0][2];
  const int n0f = a.lvl0_staged ? n0 * 4 : 0;
  float* lvl0g = lvl0 + n0f;              // coarsest level gradient [n0*4] (BWD)
  float* wbase = lvl0g + (BWD ? n0f : 0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* zbuf = wbase + warp * (NCH * 32 * kZ + 32 * kStage);  // [NCH*32][16]
  float* stage = zbuf + NCH * 32 * kZ;                          // [32][kStage]

  // ---- CTA set-up: decoders, accumulators, coarsest level ----
  const float* mlp = a.theta + a.g.n_grid;
  for (int i = threadIdx.x; i < kSmemMlp; i += blockDim.x) {
    float v = 0.0f;
    if (i < sb1) v = mlp[oW1 + i];
    else if (i < sW2) v = mlp[ob1 + i - sb1];
    else if (i < sb2) v = mlp[oW2 + i - sW2];
    else if (i < sW3) v = mlp[ob2 + i - sb2];
    else if (i < sb3) {
      const int j = (i - sW3) >> 4, k = (i - sW3) & 15;
      v = k < kHF ? mlp[oW3 + j * kHF + k] : 0.0f;
    } else if (i < sW4) v = mlp[ob3 + i - sb3];
    else if (i < sb4) v = mlp[oW4 + i - sW4];
    else if (i < sb4 + 3) v = mlp[ob4 + i - sb4];
    else if (i == sKappa) v = mlp[oKappa];
    sm[i] = v;
  }
  for (int i = threadIdx.x; i < kMlpPad + kLossPad; i += blockDim.x) acc[i] = 0.0f;
  for (int i = threadIdx.x; i < n0f; i += blockDim.x) {
    lvl0[i] = a.theta[a.g.off[0] + i];
    if (BWD) lvl0g[i] = 0.0f;
  }
  __syncthreads();
  const float4* lvl0v = a.lvl0_staged ? reinterpret_cast<const float4*>(lvl0) : nullptr;

  const int N = a.N;
  const float s_sharp = expf(sm[sKappa]);
  // loss-term weights and set sizes (Sec. 3.4 normalisations)
  float wt[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) wt[k] = a.dloss[k] + a.lam[k] * a.dloss[5];
  const int n_d = a.counts[0], n_tr = a.counts[1], n_fs = a.counts[2];
  const float k_rgb = wt[0] * 2.0f / (float)a.R;
  const float k_d = n_d > 0 ? wt[1] / (float)n_d : 0.0f;
  const float k_sdf = n_tr > 0 ? wt[2] / (float)n_tr : 0.0f;
  const float k_fs = n_fs > 0 ? wt[3] / (float)n_fs : 0.0f;

  float l_rgb = 0.f, l_d = 0.f, l_sdf = 0.f, l_fs = 0.f, g_kappa = 0.f;
  const int gwarp = blockIdx.x * kRenderWarps + warp, nwarps = gridDim.x * kRenderWarps;

  for (int ray = gwarp; ray < a.R; ray += nwarps) {
    const float o[3] = {a.o[3 * ray], a.o[3 * ray + 1], a.o[3 * ray + 2]};
    const float r[3] = {a.r[3 * ray], a.r[3 * ray + 1], a.r[3 * ray + 2]};
    const float D = a.D[ray];
    float tt[NCH], ph[NCH], col[NCH][3];
    // ---- forward: gather + decoders per sample ----
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int si = 32 * j + lane;
      float* zs = zbuf + si * kZ;
      if (si < N) {
        tt[j] = a.t[(size_t)ray * N + si];
        float x[3], z[kZ];
        sample_pos(o, r, tt[j], x);
        gather(a.g, a.theta, lvl0v, x, z);
        float a1[kH1], out[kOut], a2[kH2];
        decode(sm, z, a1, out, a2, col[j]);
        ph[j] = out[0];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<float4*>(zs + 4 * q) = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
      } else {
        tt[j] = 0.f;
        ph[j] = 0.f;
        col[j][0] = col[j][1] = col[j][2] = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) *reinterpret_cast<float4*>(zs + 4 * q) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    // ---- NeuS opacity, transmittance, weights (Sec. 3.2) ----
    float Ph[NCH], PhN[NCH], al[NCH], T[NCH], w[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) Ph[j] = (32 * j + lane < N) ? sigmoidf_(s_sharp * ph[j]) : 0.f;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      float nx = __shfl_down_sync(0xffffffffu, Ph[j], 1);
      const float nx0 = (j + 1 < NCH) ? __shfl_sync(0xffffffffu, Ph[j + 1 < NCH ? j + 1 : j], 0) : 0.f;
      if (lane == 31) nx = nx0;
      PhN[j] = nx;
      const int si = 32 * j + lane;
      float q = 0.f;
      if (si < N - 1) q = (Ph[j] - nx) / fmaxf(Ph[j], 1e-6f);
      al[j] = q > 0.f ? q : 0.f;
    }
    float carry = 1.0f;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      float inc = 1.0f - al[j];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc *= y;
      }
      float exc = __shfl_up_sync(0xffffffffu, inc, 1);
      if (lane == 0) exc = 1.0f;
      T[j] = carry * exc;
      carry *= __shfl_sync(0xffffffffu, inc, 31);
      w[j] = T[j] * al[j];
    }
    float ch[3] = {0.f, 0.f, 0.f}, dh = 0.f, ws = 0.f;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
#pragma unroll
      for (int k = 0; k < 3; ++k) ch[k] = fmaf(w[j], col[j][k], ch[k]);
      dh = fmaf(w[j], tt[j], dh);
      ws += w[j];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) ch[k] = warp_sum(ch[k]);
    dh = warp_sum(dh);
    ws = warp_sum(ws);
    const float I[3] = {a.rgb[3 * ray], a.rgb[3 * ray + 1], a.rgb[3 * ray + 2]};
    // ---- losses (Sec. 3.2-3.4) ----
    if (FWD) {
      if (lane == 0) {
        float e2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) e2 = fmaf(I[k] - ch[k], I[k] - ch[k], e2);
        l_rgb += e2;
        if (D > 0.f) l_d += fabsf(D - dh);
        if (a.rgb_hat) {
          a.rgb_hat[3 * ray] = ch[0];
          a.rgb_hat[3 * ray + 1] = ch[1];
          a.rgb_hat[3 * ray + 2] = ch[2];
        }
        if (a.d_hat) a.d_hat[ray] = dh;
        if (a.wsum) a.wsum[ray] = ws;
      }
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int si = 32 * j + lane;
        if (si >= N) continue;
        const int cl = a.cls[(size_t)ray * N + si];
        const float b = __fsub_rn(D, tt[j]);
        if (cl == CLS_TR) l_sdf += fabsf(ph[j] - b);
        else if (cl == CLS_FS) l_fs += fmaxf(fmaxf(0.f, expf(-a.kappa_fs * ph[j]) - 1.0f), ph[j] - b);
      }
    }
    if constexpr (!BWD) continue;

    // ---- adjoint of compositing: dL/dalpha_k = T_k (e_k - U_k) ----
    float gc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) gc[k] = k_rgb * (ch[k] - I[k]);
    const float gd = (D > 0.f) ? k_d * ((dh > D) ? 1.f : (dh < D ? -1.f : 0.f)) : 0.f;
    float e[NCH], U[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) e[j] = gc[0] * col[j][0] + gc[1] * col[j][1] + gc[2] * col[j][2] + gd * tt[j];
    float cA = 0.f, cB = 1.f;
#pragma unroll
    for (int j = NCH - 1; j >= 0; --j) {
      float A = al[j] * e[j], B = 1.0f - al[j];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float A2 = __shfl_down_sync(0xffffffffu, A, off), B2 = __shfl_down_sync(0xffffffffu, B, off);
        if (lane + off < 32) {
          A = fmaf(B, A2, A);
          B *= B2;
        }
      }
      float eA = __shfl_down_sync(0xffffffffu, A, 1), eB = __shfl_down_sync(0xffffffffu, B, 1);
      if (lane == 31) {
        eA = 0.f;
        eB = 1.f;
      }
      U[j] = fmaf(eB, cA, eA);
      const float A0 = __shfl_sync(0xffffffffu, A, 0), B0 = __shfl_sync(0xffffffffu, B, 0);
      cA = fmaf(B0, cA, A0);
      cB *= B0;
    }
    // dalpha -> dPhi (own and successor) -> dphi, dkappa
    float dnext_prev = 0.f;  // lane 31 value of the previous chunk
    float dphi[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int si = 32 * j + lane;
      const float dal = T[j] * (e[j] - U[j]);
      float dself = 0.f, dnext = 0.f;
      if (si < N - 1) {
        const float den = fmaxf(Ph[j], 1e-6f);
        if (Ph[j] - PhN[j] > 0.f) {
          dnext = -dal / den;
          dself = (Ph[j] > 1e-6f) ? dal * PhN[j] / (Ph[j] * Ph[j]) : dal * 1e6f;
        }
      }
      float recv = __shfl_up_sync(0xffffffffu, dnext, 1);
      const float last = __shfl_sync(0xffffffffu, dnext, 31);
      if (lane == 0) recv = dnext_prev;
      dnext_prev = last;
      const float dPh = dself + recv;
      const float dsig = Ph[j] * (1.0f - Ph[j]);
      float d = dPh * s_sharp * dsig;
      if (si < N) {
        g_kappa = fmaf(dPh * dsig * s_sharp, ph[j], g_kappa);
        const int cl = a.cls[(size_t)ray * N + si];
        const float b = __fsub_rn(D, tt[j]);
        if (cl == CLS_TR) {
          const float df = ph[j] - b;
          d += k_sdf * (df > 0.f ? 1.f : (df < 0.f ? -1.f : 0.f));
        } else if (cl == CLS_FS) {
          const float ex = expf(-a.kappa_fs * ph[j]) - 1.0f, lin = ph[j] - b;
          int arg = 0;
          float top = 0.f;
          if (ex > top) {
            top = ex;
            arg = 1;
          }
          if (lin > top) arg = 2;
          d += k_fs * (arg == 1 ? -a.kappa_fs * (ex + 1.0f) : (arg == 2 ? 1.0f : 0.0f));
        }
      } else {
        d = 0.f;
      }
      dphi[j] = d;
    }

    // ---- decoder adjoints, weight-gradient reduction and grid scatter, chunk by chunk ----
#pragma unroll 1
    for (int j = 0; j < NCH; ++j) {
      const int si = 32 * j + lane;
      const bool valid = si < N;
      const float wj = pick(w, j);
      const float* zs = zbuf + si * kZ;
      float z[kZ];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = ld4(zs + 4 * q);
        z[4 * q] = v.x;
        z[4 * q + 1] = v.y;
        z[4 * q + 2] = v.z;
        z[4 * q + 3] = v.w;
      }
      float a1[kH1], out[kOut], a2[kH2], c[3];
      decode(sm, z, a1, out, a2, c);
      float* row = stage + lane * kStage;
      // colour decoder
      float dpre[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) dpre[k] = valid ? wj * gc[k] * c[k] * (1.0f - c[k]) : 0.f;
      *reinterpret_cast<float4*>(row + stDpre) = make_float4(dpre[0], dpre[1], dpre[2], 0.f);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(row + stA2 + 4 * q) = make_float4(a2[4 * q], a2[4 * q + 1], a2[4 * q + 2], a2[4 * q + 3]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(row + stH + 4 * q) =
            make_float4(out[1 + 4 * q], out[2 + 4 * q], out[3 + 4 * q], q < 3 ? out[4 + 4 * q] : 0.f);
      float dy2[kH2];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 w0 = ld4(sm + sW4 + 4 * q), w1 = ld4(sm + sW4 + 32 + 4 * q), w2 = ld4(sm + sW4 + 64 + 4 * q);
        const float d0 = w0.x * dpre[0] + w1.x * dpre[1] + w2.x * dpre[2];
        const float d1 = w0.y * dpre[0] + w1.y * dpre[1] + w2.y * dpre[2];
        const float d2 = w0.z * dpre[0] + w1.z * dpre[1] + w2.z * dpre[2];
        const float d3 = w0.w * dpre[0] + w1.w * dpre[1] + w2.w * dpre[2];
        dy2[4 * q] = a2[4 * q] > 0.f ? d0 : 0.f;
        dy2[4 * q + 1] = a2[4 * q + 1] > 0.f ? d1 : 0.f;
        dy2[4 * q + 2] = a2[4 * q + 2] > 0.f ? d2 : 0.f;
        dy2[4 * q + 3] = a2[4 * q + 3] > 0.f ? d3 : 0.f;
        *reinterpret_cast<float4*>(row + stDy2 + 4 * q) = make_float4(dy2[4 * q], dy2[4 * q + 1], dy2[4 * q + 2], dy2[4 * q + 3]);
      }
      // dout = [dphi, dh], dh = W3^T dy2
      float dout[kOut];
      dout[0] = pick(dphi, j);
#pragma unroll
      for (int k = 1; k < kOut; ++k) dout[k] = 0.f;
#pragma unroll
      for (int jj = 0; jj < kH2; ++jj) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 wv = ld4(sm + sW3 + jj * 16 + 4 * q);
          dout[1 + 4 * q] = fmaf(wv.x, dy2[jj], dout[1 + 4 * q]);
          dout[2 + 4 * q] = fmaf(wv.y, dy2[jj], dout[2 + 4 * q]);
          dout[3 + 4 * q] = fmaf(wv.z, dy2[jj], dout[3 + 4 * q]);
          if (q < 3) dout[4 + 4 * q] = fmaf(wv.w, dy2[jj], dout[4 + 4 * q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(row + stDout + 4 * q) = make_float4(dout[4 * q], dout[4 * q + 1], dout[4 * q + 2], dout[4 * q + 3]);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(row + stA1 + 4 * q) = make_float4(a1[4 * q], a1[4 * q + 1], a1[4 * q + 2], a1[4 * q + 3]);
      // dy1 = (W2^T dout) masked
      float dy1[kH1];
#pragma unroll
      for (int k = 0; k < kH1; ++k) dy1[k] = 0.f;
#pragma unroll
      for (int jj = 0; jj < kOut; ++jj) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 wv = ld4(sm + sW2 + jj * 32 + 4 * q);
          dy1[4 * q] = fmaf(wv.x, dout[jj], dy1[4 * q]);
          dy1[4 * q + 1] = fmaf(wv.y, dout[jj], dy1[4 * q + 1]);
          dy1[4 * q + 2] = fmaf(wv.z, dout[jj], dy1[4 * q + 2]);
          dy1[4 * q + 3] = fmaf(wv.w, dout[jj], dy1[4 * q + 3]);
        }
      }
#pragma unroll
      for (int k = 0; k < kH1; ++k) dy1[k] = a1[k] > 0.f ? dy1[k] : 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(row + stDy1 + 4 * q) = make_float4(dy1[4 * q], dy1[4 * q + 1], dy1[4 * q + 2], dy1[4 * q + 3]);
      // dz = W1^T dy1
      float dz[kZ];
#pragma unroll
      for (int k = 0; k < kZ; ++k) dz[k] = 0.f;
#pragma unroll
      for (int jj = 0; jj < kH1; ++jj) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 wv = ld4(sm + sW1 + jj * 16 + 4 * q);
          dz[4 * q] = fmaf(wv.x, dy1[jj], dz[4 * q]);
          dz[4 * q + 1] = fmaf(wv.y, dy1[jj], dz[4 * q + 1]);
          dz[4 * q + 2] = fmaf(wv.z, dy1[jj], dz[4 * q + 2]);
          dz[4 * q + 3] = fmaf(wv.w, dy1[jj], dz[4 * q + 3]);
        }
      }
      __syncwarp();
      chunk_weight_grads(stage, zbuf + 32 * j * kZ, acc, lane);
      __syncwarp();
      // scatter dL/dz into the 8 corners of the sample's cell at every level
      if (valid) {
        float x[3];
        sample_pos(o, r, pick(tt, j), x);
#pragma unroll
        for (int l = 0; l < kLevels; ++l) {
          const Cell cc = locate(a.g, l, x);
          float wc[8];
          corner_weights(cc.f, wc);
          const float4 g4 = make_float4(dz[4 * l], dz[4 * l + 1], dz[4 * l + 2], dz[4 * l + 3]);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const long long vtx = cc.vtx + corner_offset(a.g, l, k);
            const float4 v = f4scale(g4, wc[k]);
            if (l == 0 && a.lvl0_staged) {
              float* p = lvl0g + 4 * vtx;
              atomicAdd(p, v.x);
              atomicAdd(p + 1, v.y);
              atomicAdd(p + 2, v.z);
              atomicAdd(p + 3, v.w);
            } else {
              atomicAdd(reinterpret_cast<float4*>(a.grad + a.g.off[l]) + vtx, v);
            }
          }
        }
      }
    }
  }

  // ---- CTA epilogue: loss partials, decoder-gradient partials, coarsest-level flush ----
  if (FWD) {
    l_rgb = warp_sum(l_rgb);
    l_d = warp_sum(l_d);
    l_sdf = warp_sum(l_sdf);
    l_fs = warp_sum(l_fs);
    if (lane == 0) {
      atomicAdd(lacc + 0, l_rgb);
      atomicAdd(lacc + 1, l_d);
      atomicAdd(lacc + 2, l_sdf);
      atomicAdd(lacc + 3, l_fs);
    }
  }
  if (BWD) {
    g_kappa = warp_sum(g_kappa);
    if (lane == 0) atomicAdd(acc + oKappa, g_kappa);
  }
  __syncthreads();
  if (threadIdx.x < kLossPad) a.loss_part[(size_t)blockIdx.x * kLossPad + threadIdx.x] = lacc[threadIdx.x];
  for (int i = threadIdx.x; i < kMlpPad; i += blockDim.x) a.mlp_part[(size_t)blockIdx.x * kMlpPad + i] = acc[i];
  if (BWD)
    for (int i = threadIdx.x; i < n0f; i += blockDim.x) {
      const float v = lvl0g[i];
      if (v != 0.0f) atomicAdd(a.grad + a.g.off[0] + i, v);
    }
}

template <int NCH>
static size_t render_smem(const GridDesc& g, bool staged, bool bwd) {
  const int n0 = g.dims[0][0] * g.dims[0][1] * g.dims[0][2];
  const size_t f = kSmemMlp + kMlpPad + kLossPad + (staged ? (size_t)n0 * 4 * (bwd ? 2 : 1) : 0) +
                   (size_t)kRenderWarps * (NCH * 32 * kZ + 32 * kStage);
  return f * sizeof(float);
}

template <int NCH, bool FWD, bool BWD>
static gs_status launch_t(const gs_ctx* ctx, RenderArgs& a, cudaStream_t st) {
  const size_t smem = render_smem<NCH>(ctx->grid, a.lvl0_staged, BWD);
  auto k = render_kernel<NCH, FWD, BWD>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GS_ERR_CUDA;
  k<<<ctx->render_ctas, kRenderWarps * 32, smem, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

template <int NCH>
gs_status launch_n(const gs_ctx* ctx, RenderArgs& a, int mode, cudaStream_t st) {
  if (mode == 1) return launch_t<NCH, true, false>(ctx, a, st);
  if (mode == 2) return launch_t<NCH, false, true>(ctx, a, st);
  return launch_t<NCH, true, true>(ctx, a, st);
}

}  // namespace gs
