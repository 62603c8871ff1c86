// Eikonal term (Sec. 3.3 Eq. eikonal_loss, normalised as in Sec. 3.4) with the decoder's
// contractions on the tcgen05 tensor cores.
//
// L_eik = mean over the batch's free-space samples S_fs of (1 - |g|)^2, g = grad_x phi(x_s),
// x_s = o + d_s r.  With the compact geometry decoder phi = w2 . relu(W1 z + b1) + b2[0]
// (w2 = row 0 of W2) and m the 0/1 ReLU mask of the sample:
//   p = d phi / d z = W1^T (m (.) w2) = V^T m,   V = diag(w2) W1,
//   g = sum_l (1/v_l) J_l^T p_l,                  J_l = d z_l / d f (trilinear, Supp. Sec. 1).
// The decoder is piecewise linear, so p does not depend on z between kinks.  The adjoint
// a = k (1 - |g|) g / |g| (k = -2 dloss / |S_fs|; 0 where |g| = 0) reaches
//   the grid:    d/d theta_{l,c,k} = p_{l,k} (1/v_l) (a . dw_c / df)    (Supp. Sec. 1)
//   the decoder: with j_k = a . d z_k / d x and C = sum_s m_s j_s^T (32 x 16),
//                d/d W1 = diag(w2) C  and  d/d W2[0,j] = sum_k W1[j,k] C[j,k]
// (the sum over samples of (m (.) w2) j^T and of m (.) (W1 j)); b1, b2 and the other rows
// of W2 get nothing.
//
// Mapping.  A compaction pass lists the batch's free-space samples (in sample order within
// blocks of 1024).  A CTA holds kEtGroups groups of 4 warps; a group owns one M = 128 tile
// whose row 32 w + i is lane i of warp w, takes every (number of groups)-th run of 128 listed
// samples, loads the next tile's list entries and rays while the current one runs, and for
// each tile runs:
//   1. on CUDA cores: the 4 levels' 8 corners give z and J (kept in registers),
//   2. H = Z W1^T on the tensor core (three bfloat16 parts per operand, six part products:
//      FP32-grade), the mask m = [H + b1 > 0] on CUDA cores,
//   3. P = M V on the tensor core (M is exact in bfloat16; three parts of V),
//   4. g, |g|, a and j on CUDA cores; C += M^T J on the tensor core (M = 64 layout, MN-major
//      operands, three parts of J), accumulated over all of the group's tiles in tensor
//      memory and issued by a second thread while the grid scatter runs,
//   5. the grid scatter: the two coarse levels summed over runs of equal cells in the warp's
//      staging rows first (one 16-byte reduction per corner and run), the fine levels with
//      one 16-byte reduction per corner and sample.  With the batch's Eikonal records the
//      scatter is deferred instead: each free-space sample's p_l / v_l and a are written
//      there, and the render kernel's backward pass adds the term to the corner vectors it
//      reduces anyway.  The scatter's reductions are what bounds this kernel (the L2 takes
//      about 3e10 16-byte reductions per second, and the fine levels need 16 per sample),
//      so the deferred form leaves it the gathers and the tensor-core phases.
// The loss is summed per CTA and combined in FP64 by the last CTA to finish.
#include <algorithm>

#include "gs_paper.cuh"
#include "gs_render_tc.cuh"

namespace gs {
namespace {

constexpr int kEtGroups = 4;                  // 16 warps per SM at one CTA per SM
constexpr int kEtThreads = kEtGroups * kGroupThreads;
constexpr int kEtRunLevels = 2;               // levels scattered after a run reduction
constexpr int kEtSt = 36;                     // staging row: 8 corner vectors | run key | pad
constexpr uint32_t kZPlane = 128u * kZ * 2u;  // Z tile (K = 16), one bfloat16 part
constexpr uint32_t kMTile = 128u * kH1 * 2u;  // mask tile (K = 32), exact in bfloat16
constexpr uint32_t kJPlane = 128u * kZ * 2u;  // j tile (K = 16), one bfloat16 part
constexpr uint32_t kStageBytes = 4u * 32u * kEtSt * 4u;
// per group: Z (3 parts) | M | J (3 parts) | staging rows.  The M = 64 reads of the mask tile
// run up to 512 bytes past its end, into the J tile (rows 32.. of C, which are not used).
constexpr uint32_t oZ = 0, oM = oZ + 3u * kZPlane, oJ = oM + kMTile, oS = oJ + 3u * kJPlane;
constexpr uint32_t kEtGroupBytes = oS + kStageBytes;
constexpr uint32_t kW1Plane = kH1 * kZ * 2u;  // B of H = Z W1^T: {N = 32, K = 16}
constexpr uint32_t kVPlane = kZ * kH1 * 2u;   // B of P = M V: {N = 16, K = 32}
constexpr uint32_t oW1t = kEtGroups * kEtGroupBytes, oVt = oW1t + 3u * kW1Plane, oMisc = oVt + 3u * kVPlane;
// tensor-memory columns of a group: H (N = 32), P (N = 16), C (M = 64 layout, N = 16)
constexpr uint32_t cH = 0, cP = 32, cC = 48, kEtCols = 64;
constexpr uint32_t kEtTmem = 256;  // a power of two >= kEtGroups * kEtCols
static_assert(kEtGroups * kEtCols <= kEtTmem, "tensor-memory columns");

struct EtMisc {
  float b1[kH1];
  float w2[kH1];
  float dacc[kH1 * kZ + kH1];  // dW1 | dW2[0,:]
  float lsum[kEtGroups * 4];
  uint64_t mbar[kEtGroups];
  uint64_t mbar_dw[kEtGroups];
  uint64_t mbar_unused;
  int abort[kEtGroups];
  uint32_t tslot;
  int last;
};
constexpr size_t kEtSmem = oMisc + sizeof(EtMisc) + 1024;  // + alignment of the base
static_assert(kEtSmem <= 227u * 1024u, "shared memory per CTA");

struct EikArgs {
  GridDesc g;
  const float* theta;
  long long S;  // R * N samples
  int N;
  const float *o, *r, *t;
  const int* list;     // the free-space samples' indices (compaction pass), *list_n of them
  const int* list_n;
  const int* counts;   // counts[2] = |S_fs|
  const float* dloss;  // [1]
  float* loss;         // [1] or nullptr
  float* grad;         // nullptr: loss only
  float* part;         // [gridDim.x] per-CTA loss sums
  unsigned* ticket;    // 0 between calls
  int* status;         // kStatusEikonal: a tensor-core phase did not complete
  float4* eik;         // deferred grid term: [5][S] records of the free-space samples; nullptr: scatter here
};

// Compaction of the free-space samples: CTA b lists those among samples [1024 b, 1024 b + 1024)
// in sample order at an offset taken with one atomic per CTA (the CTAs' blocks land in any
// order), so consecutive entries are mostly consecutive samples of one ray.
constexpr int kCompactThreads = 256;
__global__ void __launch_bounds__(kCompactThreads) eik_compact_kernel(const uint8_t* __restrict__ cls, long long S,
                                                                      int* count, int* list) {
  __shared__ int wsum[kCompactThreads / 32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long s0 = ((long long)blockIdx.x * kCompactThreads + threadIdx.x) * 4;
  bool fs[4];
  int c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    fs[k] = s0 + k < S && cls[s0 + k] == CLS_FS;
    c += fs[k] ? 1 : 0;
  }
  int incl = c;  // inclusive scan over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
#pragma unroll
    for (int w = 0; w < kCompactThreads / 32; ++w) {
      const int t = wsum[w];
      wsum[w] = tot;
      tot += t;
    }
    base = tot > 0 ? atomicAdd(count, tot) : 0;
  }
  __syncthreads();
  int pos = base + wsum[warp] + incl - c;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (fs[k]) list[pos++] = (int)(s0 + k);
}

// D[128][N] (+)= sum of the part products A_i B_j^T (i < APL, j < BPL, i + j < SUM), smallest
// first; A [128][K] and B [N][K] K-major without swizzle, parts `a_plane` / `b_plane` apart
template <int APL, int BPL, int SUM, int N, int K>
__device__ __forceinline__ void et_mma(uint32_t d, uint32_t a0, uint32_t a_plane, uint32_t b0, uint32_t b_plane) {
  constexpr uint32_t sbo = (uint32_t)(K * 2 / 16) * 128u;
  constexpr uint32_t idesc = tc::instr_desc(tc::KIND_BF16, 128, N);
  bool first = true;
#pragma unroll
  for (int s = 0; s < K / 16; ++s) {
    const uint32_t off = (uint32_t)s * 256u;
#pragma unroll
    for (int sum = SUM - 1; sum >= 0; --sum)
#pragma unroll
      for (int i = 0; i <= sum; ++i) {
        const int j = sum - i;
        if (i >= APL || j >= BPL) continue;
        tc::mma_bf16(d, tc::smem_desc(a0 + i * a_plane + off, 128u, sbo), tc::smem_desc(b0 + j * b_plane + off, 128u, sbo),
                     idesc, first ? 0u : 1u);
        first = false;
      }
  }
}

// rows written by every thread of the group -> thread 0 issues `mma` and commits to G.mbar
template <class F>
__device__ __forceinline__ void et_phase(Group& G, F mma) {
  tc::fence_smem_async();
  tc::fence_before_sync();
  group_sync(G.g);
  tc::fence_after_sync();
  if (G.gt == 0) {
    mma();
    tc::mma_commit(G.mbar);
  }
}

// The Eikonal term's grid part at this lane's point y: corner c of level l += p_{l,k} (1/v_l)
// (a . dw_c/df) (Supp. Sec. 1).  Every lane of the warp calls it (act false: nothing added);
// the coarse levels are summed over runs of equal cells first: lane r stages its 8 corner
// vectors as row r of `st` (this warp's 32 x kEtSt floats), lane c walks the rows summing
// component c (corner c / 4, feature c % 4), and at the end of a run the 4 lanes of a corner
// pass their sums to the first, which adds the corner's vector with one 16-byte reduction;
// the fine levels take one 16-byte reduction per corner.
__device__ __forceinline__ void eik_grid_scatter(const GridDesc& g, float* grad, const float y[3], const float p[kZ],
                                                 const float av[3], bool act, float* st, int lane) {
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell c = locate(g, l, y);
    float dw[8][3];
    corner_weight_grads(c.f, c.clamped, dw);
    const float iv = g.inv_voxel[l];
    const float4 p4 = make_float4(p[4 * l], p[4 * l + 1], p[4 * l + 2], p[4 * l + 3]);
    if (l < kEtRunLevels) {
      float* srow = st + lane * kEtSt;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float ad = (av[0] * dw[k][0] + av[1] * dw[k][1] + av[2] * dw[k][2]) * iv;
        *reinterpret_cast<float4*>(srow + 4 * k) = f4scale(p4, ad);
      }
      srow[32] = __int_as_float(act ? (int)c.vtx : -1);
      __syncwarp();
      const long long coff = corner_offset(g, l, lane >> 2);
      float4* gl = reinterpret_cast<float4*>(grad + g.off[l]);
      int key = __float_as_int(st[32]);
      float sum = 0.f;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        sum += st[r * kEtSt + lane];
        const int nk = r < 31 ? __float_as_int(st[(r + 1) * kEtSt + 32]) : -2;
        if (nk != key) {  // warp-uniform: every lane reads the same keys
          const float s1 = __shfl_down_sync(0xffffffffu, sum, 1);
          const float s2 = __shfl_down_sync(0xffffffffu, sum, 2);
          const float s3 = __shfl_down_sync(0xffffffffu, sum, 3);
          if (key >= 0 && (lane & 3) == 0) red_add_f4(gl + (long long)key + coff, make_float4(sum, s1, s2, s3));
          sum = 0.f;
          key = nk;
        }
      }
      __syncwarp();
    } else if (act) {
      float4* gl = reinterpret_cast<float4*>(grad + g.off[l]) + c.vtx;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float ad = (av[0] * dw[k][0] + av[1] * dw[k][1] + av[2] * dw[k][2]) * iv;
        red_add_f4(gl + corner_offset(g, l, k), f4scale(p4, ad));
      }
    }
  }
}

__global__ void __launch_bounds__(kEtThreads, 1) eikonal_tc_kernel(EikArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  EtMisc& ms = *reinterpret_cast<EtMisc*>(base + oMisc);
  uint8_t* W1t = base + oW1t;
  uint8_t* Vt = base + oVt;
  const float* mlp = a.theta + a.g.n_grid;
  for (int i = threadIdx.x; i < kH1 * kZ; i += blockDim.x) {
    const int j = i / kZ, k = i % kZ;
    const float w = mlp[oW1 + i];
    store_w<PrecBF16x3>(W1t, kW1Plane, kZ, j, k, w);                           // B[n = j][k] = W1[j][k]
    store_w<PrecBF16x3>(Vt, kVPlane, kH1, k, j, __fmul_rn(mlp[oW2 + j], w));  // B[n = k][j] = w2_j W1[j][k]
  }
  for (int i = threadIdx.x; i < kH1; i += blockDim.x) {
    ms.b1[i] = mlp[ob1 + i];
    ms.w2[i] = mlp[oW2 + i];
  }
  for (int i = threadIdx.x; i < kH1 * kZ + kH1; i += blockDim.x) ms.dacc[i] = 0.f;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int g = 0; g < kEtGroups; ++g) {
      tc::mbar_init(&ms.mbar[g], 1);
      tc::mbar_init(&ms.mbar_dw[g], 1);
      ms.abort[g] = 0;
    }
    tc::fence_mbar_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(&ms.tslot, kEtTmem);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = warp >> 2, warp_g = warp & 3;
  uint8_t* gb = base + gi * kEtGroupBytes;
  Group G;
  G.a = gb + oZ;
  G.b = gb + oJ;
  G.mbar = &ms.mbar[gi];
  G.mbar_dw = &ms.mbar_dw[gi];
  G.mbar_tma = &ms.mbar_unused;
  G.abort = &ms.abort[gi];
  G.tcol = ms.tslot + gi * kEtCols;
  G.phase = G.phase_dw = G.phase_tma = 0;
  G.dw_pending = false;
  G.g = gi;
  G.gt = threadIdx.x & (kGroupThreads - 1);
  const int row = G.gt;
  uint8_t* Zt = gb + oZ;
  uint8_t* Mt = gb + oM;
  uint8_t* Jt = gb + oJ;
  float* st = reinterpret_cast<float*>(gb + oS) + warp_g * 32 * kEtSt;
  const bool bwd = a.grad != nullptr;
  const int n_fs = a.counts[2];
  const float k_eik = n_fs > 0 ? a.dloss[0] * -2.0f / (float)n_fs : 0.0f;
  const int n_list = *a.list_n;
  float l_eik = 0.f;
  bool alive = true, dw_acc = false;

  // Static schedule: group gg takes tiles gg, gg + ng, ... of 128 listed samples (row r of a
  // tile is entry 128 tile + r).  The next tile's list entry and ray are loaded while this
  // tile runs: the entry before the gather, the ray after it.
  const int ng = (int)gridDim.x * kEtGroups;
  const int gg = (int)blockIdx.x * kEtGroups + gi;
  auto entry = [&](int tile) { return tile * 128 + row < n_list ? __ldg(a.list + tile * 128 + row) : -1; };
  int s_nx = entry(gg);
  float o_nx[3] = {0.f, 0.f, 0.f}, r_nx[3] = {0.f, 0.f, 0.f}, t_nx = 0.f;
  auto ray_of = [&](int s, float (&o3)[3], float (&r3)[3], float& t) {
    if (s < 0) return;
    const int i = s / a.N;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o3[k] = __ldg(a.o + 3 * i + k);
      r3[k] = __ldg(a.r + 3 * i + k);
    }
    t = __ldg(a.t + s);
  };
  ray_of(s_nx, o_nx, r_nx, t_nx);
#pragma unroll 1
  for (int tile = gg; tile * 128 < n_list; tile += ng) {  // group-uniform
    const int s_cur = s_nx;
    const bool valid = s_cur >= 0;
    float y[3] = {0.f, 0.f, 0.f};
    if (valid) sample_pos(o_nx, r_nx, t_nx, y);
    s_nx = entry(tile + ng);
    // ---- 1. z and J = d z / d x (1/v_l folded in) from one pass over each level's corners ----
    float4 J[kLevels][3];
    {
      Cell cs[kLevels];
#pragma unroll
      for (int l = 0; l < kLevels; ++l) cs[l] = locate(a.g, l, y);
      float z[kZ];
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        const Cell c = cs[l];
        float w[8], dw[8][3];
        corner_weights(c.f, w);
        corner_weight_grads(c.f, c.clamped, dw);
        const float4* lv = reinterpret_cast<const float4*>(a.theta + a.g.off[l]);
        float4 zz = make_float4(0.f, 0.f, 0.f, 0.f);
        J[l][0] = J[l][1] = J[l][2] = zz;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 v = __ldg(lv + c.vtx + corner_offset(a.g, l, k));
          f4fma(zz, w[k], v);
          f4fma(J[l][0], dw[k][0], v);
          f4fma(J[l][1], dw[k][1], v);
          f4fma(J[l][2], dw[k][2], v);
        }
        const float iv = a.g.inv_voxel[l];
#pragma unroll
        for (int d = 0; d < 3; ++d) J[l][d] = f4scale(J[l][d], iv);
        z[4 * l] = zz.x;
        z[4 * l + 1] = zz.y;
        z[4 * l + 2] = zz.z;
        z[4 * l + 3] = zz.w;
      }
      store_row_planes<3, kZ, kZPlane>(Zt, row, z);
    }
    ray_of(s_nx, o_nx, r_nx, t_nx);  // the next tile's ray, in flight during the tensor-core phases
    // ---- 2. H = Z W1^T; the mask ----
    et_phase(G, [&] { et_mma<3, 3, 3, kH1, kZ>(G.tcol + cH, tc::smem_u32(Zt), kZPlane, tc::smem_u32(W1t), kW1Plane); });
    if (!(alive = mma_phase_wait(G))) break;
    {
      float h[kH1];
      tc::tmem_ld32(lane_addr(G, cH, warp_g), h);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < kH1; ++j) h[j] = __fadd_rn(h[j], ms.b1[j]) > 0.f ? 1.f : 0.f;
      dw_wait(G);  // the mask and j tiles are free once the last C product has read them
      store_row_planes<1, kH1, kMTile>(Mt, row, h);
    }
    // ---- 3. P = M V ----
    et_phase(G, [&] { et_mma<1, 3, 3, kZ, kH1>(G.tcol + cP, tc::smem_u32(Mt), kMTile, tc::smem_u32(Vt), kVPlane); });
    if (!(alive = mma_phase_wait(G))) break;
    float p[kZ];
    tc::tmem_ld16(lane_addr(G, cP, warp_g), p);
    tc::tmem_ld_wait();
    // ---- 4. g, |g|, the adjoint a and j = a . dz/dx ----
    float gq[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float v = 0.f;
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        const float4 q4 = J[l][d];
        v += p[4 * l] * q4.x + p[4 * l + 1] * q4.y + p[4 * l + 2] * q4.z + p[4 * l + 3] * q4.w;
      }
      gq[d] = v;
    }
    const float nrm = __fsqrt_rn(gq[0] * gq[0] + gq[1] * gq[1] + gq[2] * gq[2]);
    if (valid) l_eik += (1.f - nrm) * (1.f - nrm);
    const float kk = bwd && valid && nrm > 0.f ? k_eik * (1.f - nrm) / nrm : 0.f;
    const float av[3] = {kk * gq[0], kk * gq[1], kk * gq[2]};
    if (a.eik != nullptr && valid) {
      // the deferred grid term's record: q_l = p_l / v_l, then (a, 0) (zero adjoint without grad)
      float4* rec = a.eik + s_cur;
#pragma unroll
      for (int l = 0; l < kLevels; ++l)
        rec[l * a.S] = f4scale(make_float4(p[4 * l], p[4 * l + 1], p[4 * l + 2], p[4 * l + 3]), a.g.inv_voxel[l]);
      rec[4 * a.S] = make_float4(av[0], av[1], av[2], 0.f);
    }
    if (bwd) {
      {
        float jv[kZ];
#pragma unroll
        for (int l = 0; l < kLevels; ++l) {
          const float4 d0 = J[l][0], d1 = J[l][1], d2 = J[l][2];
          jv[4 * l] = av[0] * d0.x + av[1] * d1.x + av[2] * d2.x;
          jv[4 * l + 1] = av[0] * d0.y + av[1] * d1.y + av[2] * d2.y;
          jv[4 * l + 2] = av[0] * d0.z + av[1] * d1.z + av[2] * d2.z;
          jv[4 * l + 3] = av[0] * d0.w + av[1] * d1.w + av[2] * d2.w;
        }
        store_row_planes<3, kZ, kJPlane>(Jt, row, jv);
      }
      // C += M^T J over the tile's 128 samples, issued by thread 32 of the group; the scatter
      // below runs meanwhile and the tiles are rewritten only after dw_wait
      tc::fence_smem_async();
      tc::fence_before_sync();
      group_sync(gi);
      tc::fence_after_sync();
      if (G.gt == 32) {
        issue_mma_dw<1, 3, 3, kZ>(G.tcol + cC, tc::smem_u32(Mt), kMTile, 4u * 128u, tc::smem_u32(Jt), kJPlane, 2u * 128u,
                                  dw_acc);
        tc::mma_commit(G.mbar_dw);
      }
      G.dw_pending = true;
      dw_acc = true;
      // ---- 5. grid scatter: p_{l,k} (1/v_l) (a . dw_c / df), here or (records) in the backward pass ----
      if (a.eik == nullptr) eik_grid_scatter(a.g, a.grad, y, p, av, kk != 0.f, st, lane);
    }
  }

  if (!alive && G.gt == 0) {
    atomicOr(a.status, kStatusEikonal);
    tc::mbar_wait(G.mbar, G.phase ^ 1u, kMbarLimit);  // let an MMA in flight finish
  }
  dw_wait(G);
  group_sync(gi);
  // ---- epilogue: C -> dW1 = diag(w2) C and dW2[0,:] = rowsum(W1 (.) C) ----
  if (bwd && alive && dw_acc && *reinterpret_cast<volatile int*>(G.abort) == 0) {
    float c[kZ];
    tc::tmem_ld16(lane_addr(G, cC, warp_g), c);  // warp w holds rows 16 w .. 16 w + 15 in lanes 0..15
    tc::tmem_ld_wait();
    const int m = 16 * warp_g + lane;
    if (lane < 16 && m < kH1) {
      float u = 0.f;
#pragma unroll
      for (int k = 0; k < kZ; ++k) {
        atomicAdd(&ms.dacc[m * kZ + k], ms.w2[m] * c[k]);
        u = fmaf(mlp[oW1 + m * kZ + k], c[k], u);
      }
      atomicAdd(&ms.dacc[kH1 * kZ + m], u);
    }
  }
  l_eik = warp_sum(l_eik);
  if (lane == 0) ms.lsum[warp] = l_eik;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(ms.tslot, kEtTmem);
  }
  if (bwd) {
    float* gm = a.grad + a.g.n_grid;
    for (int i = threadIdx.x; i < kH1 * kZ + kH1; i += blockDim.x) {
      const float v = ms.dacc[i];
      if (v == 0.f) continue;
      if (i < kH1 * kZ) atomicAdd(gm + oW1 + i, v);
      else atomicAdd(gm + oW2 + i - kH1 * kZ, v);  // row 0 of W2
    }
  }
  if (!a.loss) return;
  if (threadIdx.x == 0) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kEtThreads / 32; ++w) v += ms.lsum[w];
    a.part[blockIdx.x] = v;
    __threadfence();
    ms.last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!ms.last || warp != 0) return;
  __threadfence();
  double sum = 0.0;
  for (int b = lane; b < (int)gridDim.x; b += 32) sum += (double)__ldcg(a.part + b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    a.loss[0] = n_fs > 0 ? (float)(sum / (double)n_fs) : 0.0f;
    *a.ticket = 0u;  // ready for the next call
  }
}


// ------------------------------------------------------------------------------------
// The paper architecture's geometry decoder (two hidden layers): phi = gw3 . relu(gW2
// relu(gW1 z + gb1) + gb2) + gb3 with masks m1, m2 of the two layers.  Then
//   p = d phi / d z = gW1^T pm,  pm = m1 (.) P1,  P1 = V2^T m2,  V2 = diag(gw3) gW2,
// and the second-order adjoint of a . g (j = a . dz/dx) reaches the decoder as
//   d/d gW1 = sum_s pm j^T;  with vj = m1 (.) gW1 j and C2 = sum_s m2 vj^T (32 x 32):
//   d/d gW2 = diag(gw3) C2,  d/d gw3 = rowsum(gW2 (.) C2);  the biases get nothing.
// Per tile, five tensor-core phases: H1 = Z gW1^T, H2 = A1 gW2^T (masks), P1 = M2 V2,
// P = PM gW1, VJ = J gW1^T; C1 (+)= PM^T J and C2 (+)= M2^T VJ accumulate in tensor memory
// (M = 64 layout, MN-major operands).  The grid part as in the compact decoder's kernel
// (deferred records, or the scatter here, while the VJ phase runs).
// ------------------------------------------------------------------------------------
constexpr int kEpGroups = 3;  // 12 warps per SM
constexpr int kEpThreads = kEpGroups * kGroupThreads;
constexpr uint32_t kQ32 = 128u * 32u * 2u;  // one part of a K = 32 tile
constexpr uint32_t kQ16 = 128u * 16u * 2u;  // one part of a K = 16 tile
// per group: R1 (Z, then A1, then VJ: 3 parts; the coarse scatter's staging while VJ runs) |
// M2 (exact, 1 part) | PM (3 parts) | J (2 parts).  The M = 64 reads of M2 and PM run 512 bytes
// past a part's end, into the next part or tile.
constexpr uint32_t qR1 = 0, qM2 = 3 * kQ32, qPM = qM2 + kQ32, qJ = qPM + 3 * kQ32;
constexpr uint32_t kEpGroupBytes = qJ + 2 * kQ16;
static_assert(4u * 32u * kEtSt * 4u <= 3u * kQ32, "scatter staging fits in R1");
// weight tiles {N, K}: gW1 32x16 | gW2 32x32 | V2 {k, j} 32x32 | gW1^T {k, j} 16x32; 3 parts
constexpr uint32_t qW1 = 0, qW2 = qW1 + 32u * 16u * 2u, qV2 = qW2 + 32u * 32u * 2u, qW1T = qV2 + 32u * 32u * 2u,
                   kQW = qW1T + 16u * 32u * 2u;
constexpr uint32_t oQW = kEpGroups * kEpGroupBytes, oQMisc = oQW + 3 * kQW;
// tensor-memory columns of a group: phase outputs, C1 (N = 16), C2 (N = 32)
constexpr uint32_t eH = 0, eC1 = 32, eC2 = 48, kEpCols = 80;
static_assert(kEpGroups * kEpCols <= 256, "tensor-memory columns");

struct EpMisc {
  float b1[32];
  float b2[32];
  float lsum[kEpGroups * 4];
  uint64_t mbar[kEpGroups];
  uint64_t mbar_dw[kEpGroups];
  uint64_t mbar_unused;
  int abort[kEpGroups];
  uint32_t tslot;
  int last;
};
constexpr size_t kEpSmem = oQMisc + sizeof(EpMisc) + 1024;
static_assert(kEpSmem <= 227u * 1024u, "shared memory per CTA");

__global__ void __launch_bounds__(kEpThreads, 1) eikonal_paper_tc_kernel(EikArgs a) {
  using namespace paper;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  EpMisc& ms = *reinterpret_cast<EpMisc*>(base + oQMisc);
  uint8_t* W = base + oQW;
  const float* mlp = a.theta + a.g.n_grid;
  for (int i = threadIdx.x; i < kH * kZ; i += blockDim.x) {
    const int j = i / kZ, k = i % kZ;
    const float w = mlp[A_gW1 + i];
    store_w<PrecBF16x3>(W + qW1, kQW, kZ, j, k, w);   // B[n = j][k] = gW1[j][k]
    store_w<PrecBF16x3>(W + qW1T, kQW, kH, k, j, w);  // B[n = k][j] = gW1[j][k]
  }
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
    const int j = i / kH, k = i % kH;
    const float w = mlp[A_gW2 + i];
    store_w<PrecBF16x3>(W + qW2, kQW, kH, j, k, w);                              // B[n = j][k] = gW2[j][k]
    store_w<PrecBF16x3>(W + qV2, kQW, kH, k, j, __fmul_rn(mlp[A_gw3 + j], w));  // B[n = k][j] = gw3_j gW2[j][k]
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    ms.b1[i] = mlp[A_gb1 + i];
    ms.b2[i] = mlp[A_gb2 + i];
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int g = 0; g < kEpGroups; ++g) {
      tc::mbar_init(&ms.mbar[g], 1);
      tc::mbar_init(&ms.mbar_dw[g], 1);
      ms.abort[g] = 0;
    }
    tc::fence_mbar_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(&ms.tslot, 256);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = warp >> 2, warp_g = warp & 3;
  uint8_t* gb = base + gi * kEpGroupBytes;
  Group G;
  G.a = gb + qR1;
  G.b = gb + qPM;
  G.mbar = &ms.mbar[gi];
  G.mbar_dw = &ms.mbar_dw[gi];
  G.mbar_tma = &ms.mbar_unused;
  G.abort = &ms.abort[gi];
  G.tcol = ms.tslot + gi * kEpCols;
  G.phase = G.phase_dw = G.phase_tma = 0;
  G.dw_pending = false;
  G.g = gi;
  G.gt = threadIdx.x & (kGroupThreads - 1);
  const int row = G.gt;
  uint8_t* R1 = gb + qR1;
  uint8_t* M2 = gb + qM2;
  uint8_t* PM = gb + qPM;
  uint8_t* Jt = gb + qJ;
  float* st = reinterpret_cast<float*>(R1) + warp_g * 32 * kEtSt;
  const bool bwd = a.grad != nullptr;
  const int n_fs = a.counts[2];
  const float k_eik = n_fs > 0 ? a.dloss[0] * -2.0f / (float)n_fs : 0.0f;
  const int n_list = *a.list_n;
  float l_eik = 0.f;
  bool alive = true, dw_acc = false;

  const int ng = (int)gridDim.x * kEpGroups;
  const int gg = (int)blockIdx.x * kEpGroups + gi;
  auto entry = [&](int tile) { return tile * 128 + row < n_list ? __ldg(a.list + tile * 128 + row) : -1; };
  int s_nx = entry(gg);
  float o_nx[3] = {0.f, 0.f, 0.f}, r_nx[3] = {0.f, 0.f, 0.f}, t_nx = 0.f;
  auto ray_of = [&](int s, float (&o3)[3], float (&r3)[3], float& t) {
    if (s < 0) return;
    const int i = s / a.N;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o3[k] = __ldg(a.o + 3 * i + k);
      r3[k] = __ldg(a.r + 3 * i + k);
    }
    t = __ldg(a.t + s);
  };
  ray_of(s_nx, o_nx, r_nx, t_nx);
#pragma unroll 1
  for (int tile = gg; tile * 128 < n_list; tile += ng) {  // group-uniform
    const int s_cur = s_nx;
    const bool valid = s_cur >= 0;
    float y[3] = {0.f, 0.f, 0.f};
    if (valid) sample_pos(o_nx, r_nx, t_nx, y);
    s_nx = entry(tile + ng);
    float4 J[kLevels][3];
    {
      float z[kZ];
      Cell cs[kLevels];
#pragma unroll
      for (int l = 0; l < kLevels; ++l) cs[l] = locate(a.g, l, y);
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        const Cell c = cs[l];
        float w[8], dw[8][3];
        corner_weights(c.f, w);
        corner_weight_grads(c.f, c.clamped, dw);
        const float4* lv = reinterpret_cast<const float4*>(a.theta + a.g.off[l]);
        float4 zz = make_float4(0.f, 0.f, 0.f, 0.f);
        J[l][0] = J[l][1] = J[l][2] = zz;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 v = __ldg(lv + c.vtx + corner_offset(a.g, l, k));
          f4fma(zz, w[k], v);
          f4fma(J[l][0], dw[k][0], v);
          f4fma(J[l][1], dw[k][1], v);
          f4fma(J[l][2], dw[k][2], v);
        }
        const float iv = a.g.inv_voxel[l];
#pragma unroll
        for (int d = 0; d < 3; ++d) J[l][d] = f4scale(J[l][d], iv);
        z[4 * l] = zz.x;
        z[4 * l + 1] = zz.y;
        z[4 * l + 2] = zz.z;
        z[4 * l + 3] = zz.w;
      }
      dw_wait(G);  // the previous tile's C1, C2 products have read the tiles
      store_row_planes<3, kZ, kQ32>(R1, row, z);
    }
    ray_of(s_nx, o_nx, r_nx, t_nx);  // the next tile's ray, in flight during the tensor-core phases
    uint32_t m1 = 0;
    // ---- H1 = Z gW1^T: layer 1 ----
    et_phase(G, [&] { et_mma<3, 3, 3, kH, kZ>(G.tcol + eH, tc::smem_u32(R1), kQ32, tc::smem_u32(W + qW1), kQW); });
    if (!(alive = mma_phase_wait(G))) break;
    {
      float v[32];
      tc::tmem_ld32(lane_addr(G, eH, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < kH; ++j) {
        const float h = __fadd_rn(v[j], ms.b1[j]);
        m1 |= (h > 0.f ? 1u : 0u) << j;
        v[j] = fmaxf(h, 0.f);
      }
      store_row_planes<3, kH, kQ32>(R1, row, v);
    }
    // ---- H2 = A1 gW2^T: the mask of layer 2 ----
    et_phase(G, [&] { et_mma<3, 3, 3, kH, kH>(G.tcol + eH, tc::smem_u32(R1), kQ32, tc::smem_u32(W + qW2), kQW); });
    if (!(alive = mma_phase_wait(G))) break;
    uint32_t m2 = 0;
    {
      float v[32];
      tc::tmem_ld32(lane_addr(G, eH, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < kH; ++j) {
        const bool on = __fadd_rn(v[j], ms.b2[j]) > 0.f;
        m2 |= (on ? 1u : 0u) << j;
        v[j] = on ? 1.f : 0.f;
      }
      store_row_planes<1, kH, kQ32>(M2, row, v);
    }
    // ---- P1 = M2 V2, pm = m1 (.) P1 ----
    et_phase(G, [&] { et_mma<1, 3, 3, kH, kH>(G.tcol + eH, tc::smem_u32(M2), kQ32, tc::smem_u32(W + qV2), kQW); });
    if (!(alive = mma_phase_wait(G))) break;
    {
      float v[32];
      tc::tmem_ld32(lane_addr(G, eH, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < kH; ++j) v[j] = ((m1 >> j) & 1u) ? v[j] : 0.f;
      store_row_planes<3, kH, kQ32>(PM, row, v);
    }
    // ---- P = PM gW1: the sensitivity ----
    et_phase(G, [&] { et_mma<3, 3, 3, kZ, kH>(G.tcol + eH, tc::smem_u32(PM), kQ32, tc::smem_u32(W + qW1T), kQW); });
    if (!(alive = mma_phase_wait(G))) break;
    float p[kZ];
    tc::tmem_ld16(lane_addr(G, eH, warp_g), p);
    tc::tmem_ld_wait();
    float gq[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float v = 0.f;
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        const float4 q4 = J[l][d];
        v += p[4 * l] * q4.x + p[4 * l + 1] * q4.y + p[4 * l + 2] * q4.z + p[4 * l + 3] * q4.w;
      }
      gq[d] = v;
    }
    const float nrm = __fsqrt_rn(gq[0] * gq[0] + gq[1] * gq[1] + gq[2] * gq[2]);
    if (valid) l_eik += (1.f - nrm) * (1.f - nrm);
    const float kk = bwd && valid && nrm > 0.f ? k_eik * (1.f - nrm) / nrm : 0.f;
    const float av[3] = {kk * gq[0], kk * gq[1], kk * gq[2]};
    if (a.eik != nullptr && valid) {
      float4* rec = a.eik + s_cur;
#pragma unroll
      for (int l = 0; l < kLevels; ++l)
        rec[l * a.S] = f4scale(make_float4(p[4 * l], p[4 * l + 1], p[4 * l + 2], p[4 * l + 3]), a.g.inv_voxel[l]);
      rec[4 * a.S] = make_float4(av[0], av[1], av[2], 0.f);
    }
    if (!bwd) continue;
    {
      float jv[kZ];
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        const float4 d0 = J[l][0], d1 = J[l][1], d2 = J[l][2];
        jv[4 * l] = av[0] * d0.x + av[1] * d1.x + av[2] * d2.x;
        jv[4 * l + 1] = av[0] * d0.y + av[1] * d1.y + av[2] * d2.y;
        jv[4 * l + 2] = av[0] * d0.z + av[1] * d1.z + av[2] * d2.z;
        jv[4 * l + 3] = av[0] * d0.w + av[1] * d1.w + av[2] * d2.w;
      }
      store_row_planes<2, kZ, kQ16>(Jt, row, jv);
    }
    // ---- VJ = J gW1^T (vj = m1 (.) VJ); the grid scatter meanwhile ----
    et_phase(G, [&] { et_mma<2, 3, 3, kH, kZ>(G.tcol + eH, tc::smem_u32(Jt), kQ16, tc::smem_u32(W + qW1), kQW); });
    if (a.eik == nullptr) eik_grid_scatter(a.g, a.grad, y, p, av, kk != 0.f, st, lane);
    if (!(alive = mma_phase_wait(G))) break;  // its barrier also ends every warp's use of the staging rows
    {
      float v[32];
      tc::tmem_ld32(lane_addr(G, eH, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < kH; ++j) v[j] = ((m1 >> j) & 1u) ? v[j] : 0.f;
      store_row_planes<3, kH, kQ32>(R1, row, v);
    }
    // C1 += PM^T J and C2 += M2^T VJ, issued by thread 32 of the group
    tc::fence_smem_async();
    tc::fence_before_sync();
    group_sync(gi);
    tc::fence_after_sync();
    if (G.gt == 32) {
      issue_mma_dw<2, 2, 2, kZ>(G.tcol + eC1, tc::smem_u32(PM), kQ32, 4u * 128u, tc::smem_u32(Jt), kQ16, 2u * 128u,
                                dw_acc);
      issue_mma_dw<1, 3, 3, kH>(G.tcol + eC2, tc::smem_u32(M2), kQ32, 4u * 128u, tc::smem_u32(R1), kQ32, 4u * 128u,
                                dw_acc);
      tc::mma_commit(G.mbar_dw);
    }
    G.dw_pending = true;
    dw_acc = true;
  }

  if (!alive && G.gt == 0) {
    atomicOr(a.status, kStatusEikonal);
    tc::mbar_wait(G.mbar, G.phase ^ 1u, kMbarLimit);  // let an MMA in flight finish
  }
  dw_wait(G);
  group_sync(gi);
  // ---- epilogue: dgW1 = C1, dgW2 = diag(gw3) C2, dgw3 = rowsum(gW2 (.) C2) ----
  if (bwd && alive && dw_acc && *reinterpret_cast<volatile int*>(G.abort) == 0) {
    float c1[16], c2[32];
    tc::tmem_ld16(lane_addr(G, eC1, warp_g), c1);  // warp w holds rows 16 w .. 16 w + 15 in lanes 0..15
    tc::tmem_ld32(lane_addr(G, eC2, warp_g), c2);
    tc::tmem_ld_wait();
    const int m = 16 * warp_g + lane;
    if (lane < 16 && m < kH) {
      float* gm = a.grad + a.g.n_grid;
#pragma unroll
      for (int n = 0; n < kZ; ++n) atomicAdd(gm + A_gW1 + m * kZ + n, c1[n]);
      const float w3 = mlp[A_gw3 + m];
      float u = 0.f;
#pragma unroll
      for (int n = 0; n < kH; ++n) {
        atomicAdd(gm + A_gW2 + m * kH + n, w3 * c2[n]);
        u = fmaf(mlp[A_gW2 + m * kH + n], c2[n], u);
      }
      atomicAdd(gm + A_gw3 + m, u);
    }
  }
  l_eik = warp_sum(l_eik);
  if (lane == 0) ms.lsum[warp] = l_eik;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(ms.tslot, 256);
  }
  if (!a.loss) return;
  if (threadIdx.x == 0) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kEpThreads / 32; ++w) v += ms.lsum[w];
    a.part[blockIdx.x] = v;
    __threadfence();
    ms.last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!ms.last || warp != 0) return;
  __threadfence();
  double sum = 0.0;
  for (int b = lane; b < (int)gridDim.x; b += 32) sum += (double)__ldcg(a.part + b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    a.loss[0] = n_fs > 0 ? (float)(sum / (double)n_fs) : 0.0f;
    *a.ticket = 0u;  // ready for the next call
  }
}

}  // namespace
}  // namespace gs

using namespace gs;

// Arguments of both Eikonal kernels, and the compaction pass that lists the free-space samples
static gs_status eik_prepare(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* loss,
                             float* grad, EikArgs& a, cudaStream_t st) {
  a.g = ctx->grid;
  a.theta = theta;
  a.S = (long long)b->R * b->N;
  a.N = b->N;
  a.o = b->origin;
  a.r = b->dir;
  a.t = b->t;
  a.list = ctx->eik_list;
  a.list_n = ctx->eik_count;
  a.counts = b->counts;
  a.dloss = dloss;
  a.loss = loss;
  a.grad = grad;
  a.part = ctx->eik_part;
  a.ticket = ctx->eik_ticket;
  a.status = ctx->status;
  a.eik = reinterpret_cast<float4*>(b->eik);
  if (cudaMemsetAsync(ctx->eik_count, 0, sizeof(int), st) != cudaSuccess) return GS_ERR_CUDA;
  if (a.S > 0) {
    const long long per_cta = 4LL * kCompactThreads;
    eik_compact_kernel<<<(unsigned)((a.S + per_cta - 1) / per_cta), kCompactThreads, 0, st>>>(b->cls, a.S, ctx->eik_count,
                                                                                             ctx->eik_list);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_eikonal(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* loss,
                            float* grad, cudaStream_t st) {
  EikArgs a;
  if (eik_prepare(ctx, theta, b, dloss, loss, grad, a, st) != GS_OK) return GS_ERR_CUDA;
  const long long per = kEtThreads;
  const int blocks = (int)std::max<long long>(
      1, std::min<long long>((a.S + per - 1) / per, (long long)std::min(ctx->num_sms, ctx->eik_ctas)));
  if (cudaFuncSetAttribute(eikonal_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEtSmem) != cudaSuccess)
    return GS_ERR_CUDA;
  eikonal_tc_kernel<<<blocks, kEtThreads, kEtSmem, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_eikonal_paper_tc(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss,
                                     float* loss, float* grad, cudaStream_t st) {
  EikArgs a;
  if (eik_prepare(ctx, theta, b, dloss, loss, grad, a, st) != GS_OK) return GS_ERR_CUDA;
  const long long per = kEpThreads;
  const int blocks = (int)std::max<long long>(
      1, std::min<long long>((a.S + per - 1) / per, (long long)std::min(ctx->num_sms, ctx->eik_ctas)));
  if (cudaFuncSetAttribute(eikonal_paper_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEpSmem) !=
      cudaSuccess)
    return GS_ERR_CUDA;
  eikonal_paper_tc_kernel<<<blocks, kEpThreads, kEpSmem, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
