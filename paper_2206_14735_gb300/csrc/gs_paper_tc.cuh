// The paper's architecture (Sec. 3.1 Eq. SDF_MLP and Eq. COLOR_MLP, "Architecture Details") in
// one fused per-ray pass with both decoders on the tcgen05 tensor cores: phi = f_omega(V(x))
// with f_omega 16 -> 32 -> 32 -> 1, c = g_gamma(W_beta(x), d) with g_gamma 9 -> 32 -> 32 -> 3,
// NeuS compositing and the losses of Sec. 3.2-3.4, then their reverse mode down to both grids
// and every decoder weight.
//
// Mapping (as in the compact decoder's kernel).  A group of 4 warps owns one M = 128 tile:
// warp w renders one ray and its 32-sample chunk j fills rows 32 w .. 32 w + 31.  The two
// decoders are independent given their inputs, so each layer of both runs as one phase of two
// products (geometry on the tile Ag, colour on Ac):
//   forward  F1: [Z | U] -> H1 (K = 16),  F2: [A1 | R1] -> H2 (K = 32); the 32 -> 1 and
//            32 -> 3 output layers on CUDA cores;
//   reverse  (the forward recomputed: F1, F2), B1: [dY2 | dQ2] -> [dA1 | dR1] (K = 32),
//            B2: [dY1 | dQ1] -> [dZ | dU] (K = 32), each with the weight-gradient products
//            D[64][32] (+)= sum over the tile's samples of [x | 1]^T dy (MN-major operands,
//            accumulated in tensor memory over all of the group's tiles) issued by a second
//            thread; the output layers' gradients on CUDA cores.
// Operands are split into three bfloat16 parts with the six leading part products accumulated
// in FP32 (two parts and three products in the weight-gradient products), as in the compact
// kernel's FP32 form.  Activations are stored by the forward pass (156 floats per sample) and
// read back by the reverse pass, or recomputed there (no store).  Grid gradients: the geometry
// levels through the compact kernel's scatter (which also adds the deferred Eikonal records of
// the free-space samples), the colour grid (6 floats per finest-level vertex) with one 16-byte
// and one 8-byte reduction per corner; samples whose vectors are exactly zero issue none.
#pragma once
#include "gs_paper.cuh"
#include "gs_render_tc.cuh"

namespace gs {
namespace ptc {

using paper::kC;
using paper::kH;
using paper::kU;
using P3 = PrecBF16x3;

// weight (B) tiles {N, K}:
//   0 gW1 32x16 | 1 cW1 32x16 (cols 9.. zero) | 2 gW2 32x32 | 3 cW2 32x32
//   4 gW2^T 32x32 | 5 cW2^T 32x32 | 6 gW1^T 16x32 | 7 cW1^T 16x32 (rows 9.. zero)
__host__ __device__ constexpr int tN(int i) { return i < 6 ? 32 : 16; }
__host__ __device__ constexpr int tK(int i) { return i < 2 ? 16 : 32; }
__host__ __device__ constexpr uint32_t tOff(int i) {
  uint32_t o = 0;
  for (int k = 0; k < i; ++k) o += (uint32_t)(tN(k) * tK(k) * 2);
  return o;
}
constexpr uint32_t kTW = tOff(8);  // one bfloat16 part of all eight tiles

// per group: A tiles Ag | Ac (3 parts of 128 x 32 each) | partner tiles Bg | Bc (2 parts of
// 128 x 40 each: [a1 | 1], [r1 | 1] in B1, [z | 1], [u | 1] in B2) | mbarriers.  The M = 64
// reads of a partner tile run up to 383 bytes past its last part: into the next tile, the
// group's barriers and the next group (or, for the last group, the weight tiles).
constexpr uint32_t kAP = 128u * 32u * 2u;  // one part of an A tile
constexpr uint32_t kBP = 128u * 40u * 2u;  // one part of a partner tile
constexpr uint32_t oAg = 0, oAc = 3 * kAP, oBg = 6 * kAP, oBc = oBg + 2 * kBP, oBar = oBc + 2 * kBP;
constexpr uint32_t kPGroupBytes = oBar + 128;
constexpr int kPGroups = 2;  // tensor memory: 2 groups x 192 columns
constexpr int kPThreads = kPGroups * kGroupThreads;

// tensor-memory columns of a group: phase outputs (geometry 0.., colour 32.. or 16..), then
// the weight-gradient accumulators (M = 64 layout: row m in lane 32 (m / 16) + m % 16)
constexpr uint32_t cG = 0, cC = 32, cCb = 16, cWg2 = 64, cWc2 = 96, cWg1 = 128, cWc1 = 160, kPCols = 192;
constexpr uint32_t kPTmem = 512;
static_assert(kPGroups * kPCols <= kPTmem, "tensor-memory columns");

// FP32 scalars of the decoders in shared memory
constexpr int sc_gb1 = 0, sc_gb2 = 32, sc_gw3 = 64, sc_gb3 = 96, sc_cb1 = 100, sc_cb2 = 132, sc_cW3 = 164,
              sc_cb3 = 260, sc_kappa = 263, kScal = 264;
// per-group CUDA-core gradient accumulators: gw3 | gb3 | cW3 | cb3 | kappa
constexpr int ga_gw3 = 0, ga_gb3 = 32, ga_cW3 = 36, ga_cb3 = 132, ga_kappa = 135, kGAcc = 136;
// output-layer staging row of a lane: dpre[3] | dphi | a2[32] | r2[32] (stride 4 mod 32 words)
constexpr int kOr = 68;
static_assert(4u * 32u * kOr * 4u <= 2u * 3u * kAP, "output-layer staging fits in the A tiles");
static_assert(4u * kScatterStage * 4u <= 3u * kAP, "scatter staging fits in Ag");

struct PaperTcArgs {
  CUtensorMap tmap;      // the finest geometry level for the forward pass's tile::gather4 loads
  GridDesc g;            // geometry levels; g.n_grid = decoder block offset (after the colour grid)
  long long colour_off;  // float offset of the colour grid (a multiple of 4)
  const float* theta;
  float* grad;
  const float *o, *r, *rgb, *D, *t;
  const uint8_t* cls;
  const int* counts;
  const float* dloss;
  float lam[5];
  float kappa_fs;
  float *rgb_hat, *d_hat, *wsum, *w_out;
  float* dz_out;                // [R][N][32] per-sample records for the pose gradient (may be nullptr)
  float *loss_part, *mlp_part;  // this kernel's partial rows, one per CTA
  int R, N;
  int* status;  // kStatusPaperRender: a tensor-core phase did not complete
  // deferred Eikonal records ([5][R N] float4 planes) of the free-space samples, added to their
  // geometry scatter; nullptr: none
  const float4* eik;
  long long eik_stride;
  // stored activations: field f of sample s = rr N + si in component f % 4 of
  // ((float4*)store)[(f / 4) store_stride + s]; written by forward passes, read by backward
  // passes in place of the gathers and the two recomputed phases; nullptr: recompute
  float* store;
  long long store_stride;
};

// fields of one stored sample: z[16] | cf[6], phi, 0 | c[3], 0 | a1[32] | r1[32] | a2[32] | r2[32]
constexpr int kQz = 0, kQu = 16, kQc = 24, kQa1 = 28, kQr1 = 60, kQa2 = 92, kQr2 = 124, kQFields = 156;
static_assert(kQFields == kPaperStoreFloatsPerSample, "the store holds every field");

__device__ __forceinline__ void red_add_f2(float* p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// The gather of z (4 levels x 4) and the colour features cf (the finest cell, 6 per vertex) at
// x.  The finest level's geometry corners come through the TMA: one tile::gather4 per sample
// (rows (y,z), (y+1,z), (y,z+1), (y+1,z+1) of the level's 2D view, 2 vertices each: 128 B)
// into a slot in the half of an A plane that the 16-column z and u tiles leave free, which
// nothing else uses between the reverse pass of one chunk and the F1 epilogue of the next.
// The colour corners (24 bytes each) and the coarse levels (a warp's samples share their cells)
// come by plain loads meanwhile.  Every thread of the group takes part in every round (the
// byte count is fixed); lanes without a sample get zeros.
constexpr uint32_t kGatherBytes = 128u * 128u;  // per group and round
__device__ __forceinline__ uint8_t* geo_slot(uint8_t* gmem, int gt) {  // warp w: the free half of A plane w
  return gmem + (uint32_t)(gt >> 5) * kAP + kAP / 2 + (uint32_t)(gt & 31) * 128u;
}

__device__ __forceinline__ void gather_fwd(const PaperTcArgs& a, Group& G, uint8_t* gmem, const float x[3], bool valid,
                                           float z[kZ], float cf[kC]) {
  constexpr int l = kLevels - 1;
  const Cell c = locate(a.g, l, x);
  const int nx = a.g.dims[l][0], ny = a.g.dims[l][1];
  uint8_t* gs = geo_slot(gmem, G.gt);
  {
    tc::fence_smem_async();  // earlier generic accesses to the slot before the asynchronous write
    const int r0 = c.idx[2] * ny + c.idx[1];
    tc::tma_gather4(tc::smem_u32(gs), &a.tmap, 4 * c.idx[0], r0, r0 + 1, r0 + ny, r0 + ny + 1, G.mbar_tma);
  }
  const float f0 = c.f[0], f1 = c.f[1], f2 = c.f[2];
#pragma unroll
  for (int i = 0; i < kC; ++i) cf[i] = 0.f;
  if (valid) {
    const float* cg = a.theta + a.colour_off;
#pragma unroll
    for (int k = 0; k < 8; ++k) {  // corner k: vertex (x + (k & 1), y + (k >> 1 & 1), z + (k >> 2))
      const long long v = c.vtx + (k & 1) + (long long)((k >> 1) & 1) * nx + (long long)(k >> 2) * nx * ny;
      // its 24 bytes lie in the 16-byte aligned 32-byte window that starts at them (even v) or 8
      // bytes before them (odd v): two loads and selects, no branch, so that the loads of all
      // corners are in flight together (past the last vertex the window reads the decoder block)
      const bool odd = (v & 1) != 0;
      const float4* q = reinterpret_cast<const float4*>(cg + 6 * v - (odd ? 2 : 0));
      const float4 A = __ldg(q), B = __ldg(q + 1);
      const float e[6] = {odd ? A.z : A.x, odd ? A.w : A.y, odd ? B.x : A.z,
                          odd ? B.y : A.w, odd ? B.z : B.x, odd ? B.w : B.y};
      const float w = (((k & 1) ? f0 : 1.0f - f0) * ((k & 2) ? f1 : 1.0f - f1)) * ((k & 4) ? f2 : 1.0f - f2);
#pragma unroll
      for (int i = 0; i < kC; ++i) cf[i] = fmaf(w, e[i], cf[i]);
    }
    coarse_gather(a.g, a.theta, x, z);
  }
  if (!tc::mbar_wait(G.mbar_tma, G.phase_tma, kMbarLimit)) *reinterpret_cast<volatile int*>(G.abort) = 1;
  G.phase_tma ^= 1u;
  if (G.gt == 0) tc::mbar_arrive_expect_tx(G.mbar_tma, kGatherBytes);  // armed for the next round
  if (!valid) {
#pragma unroll
    for (int k = 0; k < kZ; ++k) z[k] = 0.f;
    return;
  }
  // geometry: 16-byte chunk c8 = vertex (x + (c8 & 1)) of row c8 >> 1, order rotated by lane
  const int lane = G.gt & 31;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c8 = (k + lane) & 7;
    const int bx = c8 & 1, by = (c8 >> 1) & 1, bz = c8 >> 2;
    const float w = ((bx ? f0 : 1.0f - f0) * (by ? f1 : 1.0f - f1)) * (bz ? f2 : 1.0f - f2);
    f4fma(s, w, *reinterpret_cast<const float4*>(gs + c8 * 16));
  }
  z[4 * l] = s.x;
  z[4 * l + 1] = s.y;
  z[4 * l + 2] = s.z;
  z[4 * l + 3] = s.w;
}

// colour-grid gradient of one sample: corner k of the finest cell += w_k dcf
__device__ __forceinline__ void scatter_colour(const PaperTcArgs& a, const float x[3], const float dcf[kC]) {
  const int l = kLevels - 1;
  const Cell c = locate(a.g, l, x);
  float w[8];
  corner_weights(c.f, w);
  float* cg = a.grad + a.colour_off;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const long long v = c.vtx + corner_offset(a.g, l, k);
    float* p = cg + 6 * v;
    float e[6];
#pragma unroll
    for (int q = 0; q < kC; ++q) e[q] = w[k] * dcf[q];
    if ((v & 1) == 0) {
      red_add_f4(reinterpret_cast<float4*>(p), make_float4(e[0], e[1], e[2], e[3]));
      red_add_f2(p + 4, e[4], e[5]);
    } else {
      red_add_f2(p, e[0], e[1]);
      red_add_f4(reinterpret_cast<float4*>(p + 2), make_float4(e[2], e[3], e[4], e[5]));
    }
  }
}

template <int N>
__device__ __forceinline__ int pick_cls(const int (&v)[N], int j) {
  int c = v[0];
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (q == j) c = v[q];
  return c;
}

// rows written by every thread of the group -> thread 0 issues `mma` and commits to G.mbar;
// with `dw`, thread 32 issues the weight-gradient products and commits them to G.mbar_dw
template <class F, class Fdw>
__device__ __forceinline__ void phase2(Group& G, F mma, Fdw dw, bool with_dw) {
  tc::fence_smem_async();
  tc::fence_before_sync();
  group_sync(G.g);
  tc::fence_after_sync();
  if (G.gt == 0) {
    mma();
    tc::mma_commit(G.mbar);
  } else if (with_dw && G.gt == 32) {
    dw();
    tc::mma_commit(G.mbar_dw);
  }
  if (with_dw) G.dw_pending = true;
}

// D[128][N] = A[128][K] B[N][K]^T over the six leading part products (A parts kAP apart,
// B parts kTW apart)
template <int N, int K>
__device__ __forceinline__ void mma3(uint32_t d, const uint8_t* a0, const uint8_t* b0) {
  issue_mma<P3, N, K>(d, tc::smem_u32(a0), tc::smem_u32(b0), kTW);
}

// the forward-only instantiation ends each ray-quad before its reverse pass, which the front
// end reports as unreachable code there
#pragma nv_diag_suppress 128
template <int NCH, bool FWD, bool BWD>
__global__ void __launch_bounds__(kPThreads, 1) paper_tc_kernel(const __grid_constant__ PaperTcArgs a) {
  using namespace paper;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* wt = base + kPGroups * kPGroupBytes;  // the eight weight tiles, 3 parts
  float* sc = reinterpret_cast<float*>(wt + 3 * kTW);
  float* gacc = sc + kScal;                      // [kPGroups][kGAcc]
  float* lacc = gacc + kPGroups * kGAcc;         // loss sums [8]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(lacc + 8);

  const int tid = threadIdx.x, gi = tid / kGroupThreads, gt = tid % kGroupThreads, warp_g = gt >> 5,
            lane = tid & 31;
  uint8_t* gmem = base + gi * kPGroupBytes;
  uint8_t* Ag = gmem + oAg;
  uint8_t* Ac = gmem + oAc;
  uint8_t* Bg = gmem + oBg;
  uint8_t* Bc = gmem + oBc;
  Group G;
  G.a = Ag;
  G.b = Bg;
  G.mbar = reinterpret_cast<uint64_t*>(gmem + oBar);
  G.mbar_dw = G.mbar + 1;
  G.mbar_tma = G.mbar + 2;
  G.abort = reinterpret_cast<int*>(G.mbar + 3);
  G.phase = G.phase_dw = G.phase_tma = 0;
  G.dw_pending = false;
  G.g = gi;
  G.gt = gt;

  // ---- CTA set-up: weight tiles, scalars, accumulators, barriers, tensor memory ----
  const float* mlp = a.theta + a.g.n_grid;
  for (int m = 0; m < 8; ++m) {
    const int Nn = tN(m), K = tK(m);
    for (int e = tid; e < Nn * K; e += blockDim.x) {
      const int n = e / K, k = e % K;
      float v = 0.f;
      switch (m) {
        case 0: v = mlp[A_gW1 + n * kZ + k]; break;
        case 1: v = k < kU ? mlp[A_cW1 + n * kU + k] : 0.f; break;
        case 2: v = mlp[A_gW2 + n * kH + k]; break;
        case 3: v = mlp[A_cW2 + n * kH + k]; break;
        case 4: v = mlp[A_gW2 + k * kH + n]; break;
        case 5: v = mlp[A_cW2 + k * kH + n]; break;
        case 6: v = mlp[A_gW1 + k * kZ + n]; break;
        default: v = n < kU ? mlp[A_cW1 + k * kU + n] : 0.f; break;
      }
      store_w<P3>(wt + tOff(m), kTW, K, n, k, v);
    }
  }
  for (int i = tid; i < kScal; i += blockDim.x) {
    float v = 0.f;
    if (i < sc_gb2) v = mlp[A_gb1 + i];
    else if (i < sc_gw3) v = mlp[A_gb2 + i - sc_gb2];
    else if (i < sc_gb3) v = mlp[A_gw3 + i - sc_gw3];
    else if (i == sc_gb3) v = mlp[A_gb3];
    else if (i >= sc_cb1 && i < sc_cb2) v = mlp[A_cb1 + i - sc_cb1];
    else if (i >= sc_cb2 && i < sc_cW3) v = mlp[A_cb2 + i - sc_cb2];
    else if (i >= sc_cW3 && i < sc_cb3) v = mlp[A_cW3 + i - sc_cW3];
    else if (i >= sc_cb3 && i < sc_kappa) v = mlp[A_cb3 + i - sc_cb3];
    else if (i == sc_kappa) v = mlp[A_kappa];
    sc[i] = v;
  }
  for (int i = tid; i < kPGroups * kGAcc + 8; i += blockDim.x) gacc[i] = 0.f;  // and lacc
  if (gt == 0) {
    tc::mbar_init(G.mbar, 1);
    tc::mbar_init(G.mbar_dw, 1);
    tc::mbar_init(G.mbar_tma, 1);
    tc::fence_mbar_init();
    tc::mbar_arrive_expect_tx(G.mbar_tma, kGatherBytes);  // armed for the first round
    *G.abort = 0;
  }
  if (tid < 32) tc::tmem_alloc(tslot, kPTmem);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  G.tcol = *tslot + (uint32_t)(gi * kPCols);
  const float s_sharp = expf(sc[sc_kappa]);
  float* ga = gacc + gi * kGAcc;

  const int N = a.N;
  float wt5[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) wt5[k] = a.dloss[k] + a.lam[k] * a.dloss[5];
  const int n_d = a.counts[0], n_tr = a.counts[1], n_fs = a.counts[2];
  const float k_rgb = a.R > 0 ? wt5[0] * 2.0f / (float)a.R : 0.f;
  const float k_d = n_d > 0 ? wt5[1] / (float)n_d : 0.0f;
  const float k_sdf = n_tr > 0 ? wt5[2] / (float)n_tr : 0.0f;
  const float k_fs = n_fs > 0 ? wt5[3] / (float)n_fs : 0.0f;
  float l_rgb = 0.f, l_d = 0.f, l_sdf = 0.f, l_fs = 0.f, g_kappa = 0.f;
  const int row = gt;
  bool alive = true, dw_acc = false;
  // this lane's column of the output layers' gradients: gw3[lane], cW3[.][lane]; gb3, cb3 (lanes < 4)
  float og = 0.f, oc[3] = {0.f, 0.f, 0.f}, ob = 0.f;

  for (int quad = blockIdx.x * kPGroups + gi; quad * 4 < a.R && alive; quad += gridDim.x * kPGroups) {
    const int ray = quad * 4 + warp_g;
    const bool has_ray = ray < a.R;
    const int rr = has_ray ? ray : 0;
    const float o[3] = {a.o[3 * rr], a.o[3 * rr + 1], a.o[3 * rr + 2]};
    const float r[3] = {a.r[3 * rr], a.r[3 * rr + 1], a.r[3 * rr + 2]};
    const float D = has_ray ? a.D[rr] : 0.f;
    const float I[3] = {a.rgb[3 * rr], a.rgb[3 * rr + 1], a.rgb[3 * rr + 2]};
    float dvw[3];  // the unit viewing direction, the colour decoder's last three inputs
    {
      const float rn = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
#pragma unroll
      for (int q = 0; q < 3; ++q) dvw[q] = r[q] / rn;
    }
    float tt[NCH], ph[NCH], col[NCH][3];
    int clv[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      const int si = 32 * q + lane;
      const bool in = has_ray && si < N;
      tt[q] = in ? a.t[(size_t)rr * N + si] : 0.f;
      clv[q] = in ? (int)a.cls[(size_t)rr * N + si] : 0;
    }

    // ================= forward: gather, then F1 and F2 per chunk =================
#pragma unroll 1
    for (int j = 0; j < NCH && alive; ++j) {
      const int si = 32 * j + lane;
      const bool valid = has_ray && si < N;
      const float t = pick_tc(tt, j);
      float4* sp = a.store != nullptr ? reinterpret_cast<float4*>(a.store) + (size_t)rr * N + si : nullptr;
      const long long ss = a.store_stride;
      if (!FWD && sp != nullptr) {  // stored by the forward pass: phi and c only
        const float4 u4 = valid ? sp[(kQu / 4 + 1) * ss] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 c4 = valid ? sp[(kQc / 4) * ss] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < NCH; ++q)
          if (q == j) {
            ph[q] = u4.z;
            col[q][0] = c4.x;
            col[q][1] = c4.y;
            col[q][2] = c4.z;
          }
        continue;
      }
      const bool put = FWD && sp != nullptr && valid;
      float cfs[8];  // the colour features, phi and a zero: stored fields kQu..kQu + 7
      {
        float z[kZ], u[16];
        {
          float x[3];
          sample_pos(o, r, t, x);
          gather_fwd(a, G, gmem, x, valid, z, u);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) u[kC + q] = dvw[q];
#pragma unroll
        for (int k = kU; k < 16; ++k) u[k] = 0.f;
        dw_wait(G);  // the previous chunk's weight-gradient products have read the tiles
        store_row_planes<3, 16, kAP>(Ag, row, z);
        store_row_planes<3, 16, kAP>(Ac, row, u);
        if (put) put_fields<kQz, 16>(sp, ss, z);
#pragma unroll
        for (int k = 0; k < kC; ++k) cfs[k] = u[k];
      }
      phase2(G, [&] {
        mma3<32, 16>(G.tcol + cG, Ag, wt + tOff(0));
        mma3<32, 16>(G.tcol + cC, Ac, wt + tOff(1));
      }, [] {}, false);
      if (!(alive = mma_phase_wait(G))) break;
      {
        float v[32];
        tc::tmem_ld32(lane_addr(G, cG, warp_g), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + sc[sc_gb1 + k], 0.f);
        store_row_planes<3, 32, kAP>(Ag, row, v);
        if (put) put_fields<kQa1, 32>(sp, ss, v);
        tc::tmem_ld32(lane_addr(G, cC, warp_g), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + sc[sc_cb1 + k], 0.f);
        store_row_planes<3, 32, kAP>(Ac, row, v);
        if (put) put_fields<kQr1, 32>(sp, ss, v);
      }
      phase2(G, [&] {
        mma3<32, 32>(G.tcol + cG, Ag, wt + tOff(2));
        mma3<32, 32>(G.tcol + cC, Ac, wt + tOff(3));
      }, [] {}, false);
      if (!(alive = mma_phase_wait(G))) break;
      float phi, c3[3];
      {
        float v[32];
        tc::tmem_ld32(lane_addr(G, cG, warp_g), v);
        tc::tmem_ld_wait();
        phi = sc[sc_gb3];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          v[k] = fmaxf(v[k] + sc[sc_gb2 + k], 0.f);
          phi = fmaf(sc[sc_gw3 + k], v[k], phi);
        }
        if (put) put_fields<kQa2, 32>(sp, ss, v);
        tc::tmem_ld32(lane_addr(G, cC, warp_g), v);
        tc::tmem_ld_wait();
        float pre[3] = {sc[sc_cb3], sc[sc_cb3 + 1], sc[sc_cb3 + 2]};
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          v[k] = fmaxf(v[k] + sc[sc_cb2 + k], 0.f);
#pragma unroll
          for (int i = 0; i < 3; ++i) pre[i] = fmaf(sc[sc_cW3 + 32 * i + k], v[k], pre[i]);
        }
        if (put) put_fields<kQr2, 32>(sp, ss, v);
#pragma unroll
        for (int i = 0; i < 3; ++i) c3[i] = sigmoidf_(pre[i]);
        if (put) {
          cfs[6] = phi;
          cfs[7] = 0.f;
          put_fields<kQu, 8>(sp, ss, cfs);
          const float c4[4] = {c3[0], c3[1], c3[2], 0.f};
          put_fields<kQc, 4>(sp, ss, c4);
        }
      }
#pragma unroll
      for (int q = 0; q < NCH; ++q)
        if (q == j) {
          ph[q] = valid ? phi : 0.f;
          col[q][0] = valid ? c3[0] : 0.f;
          col[q][1] = valid ? c3[1] : 0.f;
          col[q][2] = valid ? c3[2] : 0.f;
        }
    }
    if (!alive) break;

    // ================= NeuS opacity, transmittance, weights (Sec. 3.2) =================
    float Ph[NCH], PhN[NCH], al[NCH], T[NCH], w[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) Ph[j] = (has_ray && 32 * j + lane < N) ? sigmoidf_(s_sharp * ph[j]) : 0.f;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      float nx = __shfl_down_sync(0xffffffffu, Ph[j], 1);
      const float nx0 = (j + 1 < NCH) ? __shfl_sync(0xffffffffu, Ph[j + 1 < NCH ? j + 1 : j], 0) : 0.f;
      if (lane == 31) nx = nx0;
      PhN[j] = nx;
      float q = 0.f;
      if (has_ray && 32 * j + lane < N - 1) q = (Ph[j] - nx) / fmaxf(Ph[j], 1e-6f);
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
    if (FWD && a.w_out != nullptr && has_ray) {
#pragma unroll
      for (int j = 0; j < NCH; ++j)
        if (32 * j + lane < N) a.w_out[(size_t)ray * N + 32 * j + lane] = w[j];
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
    if (FWD && has_ray) {
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
        if (32 * j + lane >= N) continue;
        const int cl = clv[j];
        const float b = __fsub_rn(D, tt[j]);
        if (cl == CLS_TR) l_sdf += fabsf(ph[j] - b);
        else if (cl == CLS_FS) l_fs += fmaxf(fmaxf(0.f, expf(-a.kappa_fs * ph[j]) - 1.0f), ph[j] - b);
      }
    }
    if constexpr (!BWD) continue;

    // ================= adjoint of compositing: dL/dalpha_k = T_k (e_k - U_k) =================
    float gc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) gc[k] = has_ray ? k_rgb * (ch[k] - I[k]) : 0.f;
    const float gd = (has_ray && D > 0.f) ? k_d * ((dh > D) ? 1.f : (dh < D ? -1.f : 0.f)) : 0.f;
    float e[NCH], U[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) e[j] = gc[0] * col[j][0] + gc[1] * col[j][1] + gc[2] * col[j][2] + gd * tt[j];
    float cA = 0.f;
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
    }
    float dnext_prev = 0.f;
    float dphi[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const bool valid = has_ray && 32 * j + lane < N;
      const float dal = T[j] * (e[j] - U[j]);
      float dself = 0.f, dnext = 0.f;
      if (valid && 32 * j + lane < N - 1) {
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
      if (valid) {
        g_kappa = fmaf(dPh * dsig * s_sharp, ph[j], g_kappa);
        const int cl = clv[j];
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

    // ================= reverse, chunk by chunk: the stored activations (or F1, F2 again), B1, B2, scatter =================
#pragma unroll 1
    for (int j = 0; j < NCH && alive; ++j) {
      const int si = 32 * j + lane;
      const bool valid = has_ray && si < N;
      const float t = pick_tc(tt, j);
      float x[3];
      sample_pos(o, r, t, x);
      const float4* spr = a.store != nullptr ? reinterpret_cast<const float4*>(a.store) + (size_t)rr * N + si : nullptr;
      float z[kZ], u[16];
      uint32_t m1 = 0, mr1 = 0, m2 = 0, mr2 = 0;
      // output layers on CUDA cores: [dpre | dphi | a2 | r2] staged per lane in the A tiles
      float* ost = reinterpret_cast<float*>(Ag) + warp_g * (32 * kOr);
      float* orow = ost + lane * kOr;
      if (spr != nullptr) {  // stored by the forward pass: no gather and no forward phases
        const long long ss = a.store_stride;
        dw_wait(G);  // the previous chunk's weight-gradient products have read the tiles
        get_fields<kQz, 16>(spr, ss, valid, z);
        {
          float c8[8];
          get_fields<kQu, 8>(spr, ss, valid, c8);
#pragma unroll
          for (int k = 0; k < kC; ++k) u[k] = c8[k];
        }
        float v[32], pb[40];
        get_fields<kQa1, 32>(spr, ss, valid, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          m1 |= (v[k] > 0.f ? 1u : 0u) << k;
          pb[k] = v[k];
        }
        pb[32] = 1.f;  // ones column: the bias gradient lands in row 32
#pragma unroll
        for (int k = 33; k < 40; ++k) pb[k] = 0.f;
        store_row_planes<2, 40, kBP>(Bg, row, pb);
        get_fields<kQr1, 32>(spr, ss, valid, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          mr1 |= (v[k] > 0.f ? 1u : 0u) << k;
          pb[k] = v[k];
        }
        store_row_planes<2, 40, kBP>(Bc, row, pb);
        get_fields<kQa2, 32>(spr, ss, valid, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) m2 |= (v[k] > 0.f ? 1u : 0u) << k;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(orow + 4 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        get_fields<kQr2, 32>(spr, ss, valid, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) mr2 |= (v[k] > 0.f ? 1u : 0u) << k;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(orow + 36 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        dw_wait(G);  // the previous chunk's weight-gradient products have read the tiles the gather lands in
        gather_fwd(a, G, gmem, x, valid, z, u);
#pragma unroll
        for (int q = 0; q < 3; ++q) u[kC + q] = dvw[q];
#pragma unroll
        for (int k = kU; k < 16; ++k) u[k] = 0.f;
        store_row_planes<3, 16, kAP>(Ag, row, z);
        store_row_planes<3, 16, kAP>(Ac, row, u);
        phase2(G, [&] {
          mma3<32, 16>(G.tcol + cG, Ag, wt + tOff(0));
          mma3<32, 16>(G.tcol + cC, Ac, wt + tOff(1));
        }, [] {}, false);
        if (!(alive = mma_phase_wait(G))) break;
        {
          float v[32], pb[40];
          tc::tmem_ld32(lane_addr(G, cG, warp_g), v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            v[k] = fmaxf(v[k] + sc[sc_gb1 + k], 0.f);
            m1 |= (v[k] > 0.f ? 1u : 0u) << k;
            pb[k] = v[k];
          }
          pb[32] = 1.f;  // ones column: the bias gradient lands in row 32
#pragma unroll
          for (int k = 33; k < 40; ++k) pb[k] = 0.f;
          store_row_planes<3, 32, kAP>(Ag, row, v);
          store_row_planes<2, 40, kBP>(Bg, row, pb);
          tc::tmem_ld32(lane_addr(G, cC, warp_g), v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            v[k] = fmaxf(v[k] + sc[sc_cb1 + k], 0.f);
            mr1 |= (v[k] > 0.f ? 1u : 0u) << k;
            pb[k] = v[k];
          }
          store_row_planes<3, 32, kAP>(Ac, row, v);
          store_row_planes<2, 40, kBP>(Bc, row, pb);
        }
        phase2(G, [&] {
          mma3<32, 32>(G.tcol + cG, Ag, wt + tOff(2));
          mma3<32, 32>(G.tcol + cC, Ac, wt + tOff(3));
        }, [] {}, false);
        if (!(alive = mma_phase_wait(G))) break;
        float v[32];
        tc::tmem_ld32(lane_addr(G, cG, warp_g), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          v[k] = fmaxf(v[k] + sc[sc_gb2 + k], 0.f);
          m2 |= (v[k] > 0.f ? 1u : 0u) << k;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(orow + 4 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        tc::tmem_ld32(lane_addr(G, cC, warp_g), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          v[k] = fmaxf(v[k] + sc[sc_cb2 + k], 0.f);
          mr2 |= (v[k] > 0.f ? 1u : 0u) << k;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(orow + 36 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) u[kC + q] = dvw[q];
#pragma unroll
      for (int k = kU; k < 16; ++k) u[k] = 0.f;
      float dpre[3];
      const float dph = valid ? pick_tc(dphi, j) : 0.f;
      {
        const float wj = pick_tc(w, j);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          float cj = col[0][i];
#pragma unroll
          for (int q = 1; q < NCH; ++q)
            if (q == j) cj = col[q][i];
          dpre[i] = valid ? wj * gc[i] * cj * (1.0f - cj) : 0.f;
        }
        *reinterpret_cast<float4*>(orow) = make_float4(dpre[0], dpre[1], dpre[2], dph);
      }
      __syncwarp();
#pragma unroll 4
      for (int s2 = 0; s2 < 32; ++s2) {  // lane = column: gw3[lane], cW3[.][lane]; gb3, cb3 in lanes < 4
        const float* r2 = ost + s2 * kOr;
        const float4 d4 = *reinterpret_cast<const float4*>(r2);
        og = fmaf(d4.w, r2[4 + lane], og);
        const float rv = r2[36 + lane];
        oc[0] = fmaf(d4.x, rv, oc[0]);
        oc[1] = fmaf(d4.y, rv, oc[1]);
        oc[2] = fmaf(d4.z, rv, oc[2]);
        ob += r2[lane & 3];
      }
      group_sync(G.g);  // every warp has read its staged rows before the tiles are rewritten
      {
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = ((m2 >> k) & 1u) ? sc[sc_gw3 + k] * dph : 0.f;  // dy2
        store_row_planes<3, 32, kAP>(Ag, row, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {  // dq2 = m(r2) (.) cW3^T dpre
          const float d = fmaf(dpre[0], sc[sc_cW3 + k], fmaf(dpre[1], sc[sc_cW3 + 32 + k], dpre[2] * sc[sc_cW3 + 64 + k]));
          v[k] = ((mr2 >> k) & 1u) ? d : 0.f;
        }
        store_row_planes<3, 32, kAP>(Ac, row, v);
      }
      // B1: dA1 = dY2 gW2, dR1 = dQ2 cW2; dW2^T, db2 (+)= [a1 | 1]^T dY2 and the colour's
      phase2(G, [&] {
        mma3<32, 32>(G.tcol + cG, Ag, wt + tOff(4));
        mma3<32, 32>(G.tcol + cC, Ac, wt + tOff(5));
      }, [&] {
        issue_mma_dw<2, 3, 2, 32>(G.tcol + cWg2, tc::smem_u32(Bg), kBP, 5u * 128u, tc::smem_u32(Ag), kAP, 4u * 128u,
                                  dw_acc);
        issue_mma_dw<2, 3, 2, 32>(G.tcol + cWc2, tc::smem_u32(Bc), kBP, 5u * 128u, tc::smem_u32(Ac), kAP, 4u * 128u,
                                  dw_acc);
      }, true);
      if (!(alive = mma_phase_wait(G))) break;
      {
        float v[32], v2[32];
        tc::tmem_ld32(lane_addr(G, cG, warp_g), v);
        tc::tmem_ld32(lane_addr(G, cC, warp_g), v2);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          v[k] = ((m1 >> k) & 1u) ? v[k] : 0.f;     // dy1
          v2[k] = ((mr1 >> k) & 1u) ? v2[k] : 0.f;  // dq1
        }
        dw_wait(G);  // the weight-gradient products of B1 have read the tiles
        store_row_planes<3, 32, kAP>(Ag, row, v);
        store_row_planes<3, 32, kAP>(Ac, row, v2);
        float pb[24];
#pragma unroll
        for (int k = 0; k < kZ; ++k) pb[k] = z[k];
        pb[16] = 1.f;
#pragma unroll
        for (int k = 17; k < 24; ++k) pb[k] = 0.f;
        store_row_planes<2, 24, kBP>(Bg, row, pb);
#pragma unroll
        for (int k = 0; k < 16; ++k) pb[k] = k < kU ? u[k] : (k == kU ? 1.f : 0.f);
        store_row_planes<2, 16, kBP>(Bc, row, pb);
      }
      // B2: dZ = dY1 gW1, dU = dQ1 cW1; dW1, db1 (+)= [z | 1]^T dY1 and the colour's [u | 1]^T dQ1
      phase2(G, [&] {
        mma3<16, 32>(G.tcol + cG, Ag, wt + tOff(6));
        mma3<16, 32>(G.tcol + cCb, Ac, wt + tOff(7));
      }, [&] {
        issue_mma_dw<2, 3, 2, 32>(G.tcol + cWg1, tc::smem_u32(Bg), kBP, 3u * 128u, tc::smem_u32(Ag), kAP, 4u * 128u,
                                  dw_acc);
        issue_mma_dw<2, 3, 2, 32>(G.tcol + cWc1, tc::smem_u32(Bc), kBP, 2u * 128u, tc::smem_u32(Ac), kAP, 4u * 128u,
                                  dw_acc);
      }, true);
      if (!(alive = mma_phase_wait(G))) break;
      dw_acc = true;
      float dz[16], du[16];
      tc::tmem_ld16(lane_addr(G, cG, warp_g), dz);
      tc::tmem_ld16(lane_addr(G, cCb, warp_g), du);
      tc::tmem_ld_wait();
      dw_wait(G);  // the scatter's staging rows overwrite the tiles
      const float4* er = a.eik != nullptr && valid && pick_cls(clv, j) == CLS_FS ? a.eik + (size_t)rr * N + si : nullptr;
      scatter_dz(a.g, a.grad, x, dz, valid, reinterpret_cast<float*>(Ag) + warp_g * kScatterStage, er, a.eik_stride);
      if (valid) {
        if (du[0] != 0.f || du[1] != 0.f || du[2] != 0.f || du[3] != 0.f || du[4] != 0.f || du[5] != 0.f)
          scatter_colour(a, x, du);  // a zero vector adds nothing
        if (a.dz_out != nullptr) {  // the sample's record: dz (16), dcf (6), d direction (3), zeros (7)
          float4* rec = reinterpret_cast<float4*>(a.dz_out + ((size_t)rr * N + si) * 32);
#pragma unroll
          for (int q = 0; q < 4; ++q) rec[q] = make_float4(dz[4 * q], dz[4 * q + 1], dz[4 * q + 2], dz[4 * q + 3]);
          rec[4] = make_float4(du[0], du[1], du[2], du[3]);
          rec[5] = make_float4(du[4], du[5], du[6], du[7]);
          rec[6] = make_float4(du[8], 0.f, 0.f, 0.f);
          rec[7] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      group_sync(G.g);  // every warp is done with its staging rows before the tiles are rewritten
    }
  }

  // ---- epilogue: loss sums, decoder-gradient partial row, tensor memory ----
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
    if (lane == 0) atomicAdd(ga + ga_kappa, g_kappa);
    atomicAdd(ga + ga_gw3 + lane, og);
#pragma unroll
    for (int i = 0; i < 3; ++i) atomicAdd(ga + ga_cW3 + 32 * i + lane, oc[i]);
    if (lane < 3) atomicAdd(ga + ga_cb3 + lane, ob);
    else if (lane == 3) atomicAdd(ga + ga_gb3, ob);
  }
  if (!alive && gt == 0) {
    atomicOr(a.status, kStatusPaperRender);
    tc::mbar_wait(G.mbar, G.phase ^ 1u, kMbarLimit);  // let an MMA in flight finish
  }
  dw_wait(G);
  tc::fence_before_sync();
  __syncthreads();
  float* prow = reinterpret_cast<float*>(base);  // the CTA's partial row, over group 0's tiles
  for (int i = tid; i < kPart; i += blockDim.x) prow[i] = 0.f;
  __syncthreads();
  tc::fence_after_sync();
  if (BWD && alive && dw_acc && *reinterpret_cast<volatile int*>(G.abort) == 0) {
    // warp w holds rows 16 w .. 16 w + 15 of every M = 64 product in its lanes 0..15
    const int m = 16 * warp_g + lane;
    float d[32];
    tc::tmem_ld32(lane_addr(G, cWg2, warp_g), d);  // [a1 | 1]^T dY2
    tc::tmem_ld_wait();
    if (lane < 16 && m <= 32)
#pragma unroll
      for (int n = 0; n < 32; ++n) atomicAdd(prow + (m < 32 ? A_gW2 + n * kH + m : A_gb2 + n), d[n]);
    tc::tmem_ld32(lane_addr(G, cWc2, warp_g), d);  // [r1 | 1]^T dQ2
    tc::tmem_ld_wait();
    if (lane < 16 && m <= 32)
#pragma unroll
      for (int n = 0; n < 32; ++n) atomicAdd(prow + (m < 32 ? A_cW2 + n * kH + m : A_cb2 + n), d[n]);
    tc::tmem_ld32(lane_addr(G, cWg1, warp_g), d);  // [z | 1]^T dY1
    tc::tmem_ld_wait();
    if (lane < 16 && m <= kZ)
#pragma unroll
      for (int n = 0; n < 32; ++n) atomicAdd(prow + (m < kZ ? A_gW1 + n * kZ + m : A_gb1 + n), d[n]);
    tc::tmem_ld32(lane_addr(G, cWc1, warp_g), d);  // [u | 1]^T dQ1
    tc::tmem_ld_wait();
    if (lane < 16 && m <= kU)
#pragma unroll
      for (int n = 0; n < 32; ++n) atomicAdd(prow + (m < kU ? A_cW1 + n * kU + m : A_cb1 + n), d[n]);
  }
  __syncthreads();
  if (BWD) {
    for (int i = tid; i < kPGroups * kGAcc; i += blockDim.x) {
      const int k = i % kGAcc;
      const float v = gacc[i];
      int dst;
      if (k < ga_gb3) dst = A_gw3 + k;
      else if (k == ga_gb3) dst = A_gb3;
      else if (k < ga_cW3) continue;
      else if (k < ga_cb3) dst = A_cW3 + k - ga_cW3;
      else if (k < ga_kappa) dst = A_cb3 + k - ga_cb3;
      else dst = A_kappa;
      atomicAdd(prow + dst, v);
    }
  }
  __syncthreads();
  for (int i = tid; i < kPart; i += blockDim.x) a.mlp_part[(size_t)blockIdx.x * kPart + i] = prow[i];
  if (tid < kLossPad) a.loss_part[(size_t)blockIdx.x * kLossPad + tid] = tid < 4 ? lacc[tid] : 0.f;
  if (tid < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*tslot, kPTmem);
  }
}
#pragma nv_diag_default 128

inline size_t paper_tc_smem() {
  return 1024 + (size_t)kPGroups * kPGroupBytes + 3 * kTW + sizeof(float) * (kScal + kPGroups * kGAcc + 8) + 16;
}
static_assert(kPGroups * kPGroupBytes + 3 * kTW + sizeof(float) * (kScal + kPGroups * kGAcc + 8) + 16 + 1024 <=
                  227u * 1024u,
              "shared memory per CTA");
static_assert(paper::kPart * 4 <= 3 * kAP, "the partial row fits in group 0's geometry tile");

template <int NCH>
gs_status launch_paper_tc(const PaperTcArgs& a, int mode, int ctas, cudaStream_t st) {
  const size_t smem = paper_tc_smem();
  auto k = mode == 1 ? paper_tc_kernel<NCH, true, false>
                     : (mode == 2 ? paper_tc_kernel<NCH, false, true> : paper_tc_kernel<NCH, true, true>);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GS_ERR_CUDA;
  k<<<ctas, kPThreads, smem, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace ptc
}  // namespace gs
