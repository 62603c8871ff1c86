// Fused per-ray pass of one GO-Surf step with the decoders on the tcgen05 tensor cores.
//
// What it computes (same as the paper's step, Sec. 3.1-3.4): multi-level trilinear gather,
// geometry and colour decoders, NeuS compositing, the rgb / depth / sdf / free-space losses
// and, in the same pass, their reverse mode down to every grid feature and decoder weight.
//
// Mapping.  A "group" of 4 warps owns one M = 128 tensor-core tile: warp w of the group
// renders one ray and its 32-sample chunk j fills tile rows 32w..32w+31, which are exactly
// the tensor-memory lanes that warp may read.  Each decoder layer of a chunk is one MMA
// phase: every thread writes its sample's activation row into the shared-memory A operand
// (K-major, no swizzle), one thread issues the MMA(s) against the shared-memory weight tile,
// the result lands in tensor memory and every thread reads its own row back with
// tcgen05.ld.  Forward: 4 phases per chunk.  Reverse: the forward is recomputed (4 phases)
// and the four activation adjoints run as 4 more phases; the decoder weight gradients are
// reduced on CUDA cores as 4x4 register tiles over the warp's 32 staged samples while the
// next MMA runs.  FP32 form: each operand is split into three bfloat16 parts and the six
// leading part products are accumulated in FP32 (FP32-grade accuracy on BF16 tensor cores).
// Compositing and its adjoint are warp scans over the ray's chunks, as in the CUDA-core
// design; grid gradients are scattered with 16-byte vector atomics (coarsest level first
// accumulated in shared memory).
#pragma once
#include "gs_internal.h"
#include <cuda.h>
#include <cuda_bf16.h>

#include "gs_tc.cuh"

namespace gs {

// Operand precisions.  Every operand is split into `planes` bfloat16 parts
// x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1): 24 significant
// bits) and a product is the sum of the part products with i + j < planes, accumulated in
// FP32 by the tensor core: 6 MMAs per K step give FP32-grade products (the dropped terms
// are below 2^-24 relative), 1 MMA per step is the plain BF16 form.
struct PrecBF16x3 {
  static constexpr int kind = tc::KIND_BF16;
  static constexpr int es = 2;      // bytes per operand element
  static constexpr int kmma = 16;   // K per MMA instruction
  static constexpr int planes = 3;
};
struct PrecBF16 {
  static constexpr int kind = tc::KIND_BF16;
  static constexpr int es = 2;
  static constexpr int kmma = 16;
  static constexpr int planes = 1;
};

constexpr int kKD = 16;  // padded K of the colour-output adjoint (3 real columns) = one bf16 K step

// weight (B) tiles: {N, K} of the 8 decoder contractions
//   0 W1  32x16 | 1 W2 16x32 | 2 W3 32x16 (col 15 zero) | 3 W4 16x32 (rows 3.. zero)
//   4 W4^T 32xKD (cols 3.. zero) | 5 W3^T 16x32 (row 15 zero) | 6 W2^T 32x16 | 7 W1^T 16x32
__host__ __device__ constexpr int wN(int i) { return (i == 0 || i == 2 || i == 4 || i == 6) ? 32 : 16; }
__host__ __device__ constexpr int wK(int i) { return i == 4 ? kKD : ((i == 0 || i == 2 || i == 6) ? 16 : 32); }
template <class P>
__host__ __device__ constexpr uint32_t wBytes(int i) { return (uint32_t)(wN(i) * wK(i) * P::es); }
template <class P>
__host__ __device__ constexpr uint32_t wOff(int i) {
  uint32_t o = 0;
  for (int k = 0; k < i; ++k) o += wBytes<P>(k);
  return o;
}
template <class P>
__host__ __device__ constexpr uint32_t wTotal() { return wOff<P>(8); }

// tensor-memory columns of one group: forward accumulators D1..D3 and the colour output X;
// the backward phases reuse D3 (N = 32) and D2 (N = 16) once those are consumed; the decoder
// weight gradients accumulate over all of the group's tiles in W1..W4 (M = 64 layout: row m
// in lane 32 (m / 16) + m % 16)
constexpr uint32_t cD1 = 0, cD2 = 32, cD3 = 48, cX = 80, cXb = cD3, cYb = cD2;
constexpr uint32_t cW1 = 96, cW2 = 120, cW3 = 136, cW4 = 152, kGroupCols = 160;
// tcgen05.alloc takes a power of two >= 32 columns
__host__ __device__ constexpr uint32_t tmem_cols(int groups) {
  uint32_t c = 32;
  while (c < (uint32_t)groups * kGroupCols) c <<= 1;
  return c;
}

constexpr int kGroupThreads = 128;
constexpr uint32_t kMbarLimit = 1u << 20;  // bounded MMA-completion wait (tries of up to 2 us: ~2 s)

template <class P>
struct TcLayout {
  static constexpr uint32_t a_bytes = 128u * 32u * P::es;  // one A operand plane, K <= 32
  // partner operand of the weight-gradient products (an activation tile of up to 40 columns);
  // 12 KB per plane keeps every M = 64 operand read inside the plane
  static constexpr uint32_t b_bytes = 12288u;
  static constexpr int b_planes = P::planes < 2 ? P::planes : 2;
  static constexpr uint32_t group_bytes = a_bytes * P::planes + b_bytes * b_planes + 128;  // + mbarrier, flag
};

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGroupThreads) : "memory");
}

// ---- operand rows ---------------------------------------------------------------------
// bf16 parts of x (round to nearest even; the differences are exact in binary32)
template <int PL>
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 (&p)[PL]) {
  float r = x;
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    p[i] = __float2bfloat16_rn(r);
    r = r - __bfloat162float(p[i]);
  }
}

// write K values as row `row` of a K-major no-swizzle tile, one plane per bf16 part; pairs
// of values are rounded together (one cvt.rn.bf16x2 per pair and part)
template <int NPL, int K, uint32_t PLANE_BYTES>
__device__ __forceinline__ void store_row_planes(uint8_t* planes, int row, const float* v) {
  constexpr uint32_t sbo = (uint32_t)(K * 2 / 16) * 128u;
  constexpr uint32_t plane_bytes = PLANE_BYTES;
  constexpr int kPl = NPL;
#pragma unroll
  for (int c = 0; c < K / 8; ++c) {
    float r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = v[8 * c + q];
    const uint32_t off = tc::core_offset((uint32_t)row, (uint32_t)c, 128u, sbo);
#pragma unroll
    for (int pl = 0; pl < kPl; ++pl) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(r[2 * q], r[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t*>(&b);
        if (pl + 1 < kPl) {
          r[2 * q] -= __uint_as_float(w[q] << 16);
          r[2 * q + 1] -= __uint_as_float(w[q] & 0xFFFF0000u);
        }
      }
      *reinterpret_cast<uint4*>(planes + pl * plane_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}
// a row of the A operand tile of the decoder phases
template <class P, int K>
__device__ __forceinline__ void store_row(uint8_t* planes, int row, const float* v) {
  static_assert(P::es == 2, "bf16 parts");
  store_row_planes<P::planes, K, 128u * 32u * P::es>(planes, row, v);
}

// one element of a weight tile (planes `wplane` bytes apart)
template <class P>
__device__ __forceinline__ void store_w(uint8_t* planes, uint32_t wplane, int K, int n, int k, float v) {
  const uint32_t sbo = (uint32_t)(K * P::es / 16) * 128u;
  const uint32_t off = tc::core_offset((uint32_t)n, (uint32_t)(k * P::es / 16), 128u, sbo) + (uint32_t)(k * P::es % 16);
  __nv_bfloat16 e[P::planes];
  split_bf16<P::planes>(v, e);
#pragma unroll
  for (int pl = 0; pl < P::planes; ++pl) *reinterpret_cast<__nv_bfloat16*>(planes + pl * wplane + off) = e[pl];
}

// D[128][N] (+)= A[128][K] * B[N][K]^T over the part products i + j < planes, one thread
template <class P, int N, int K>
__device__ __forceinline__ void issue_mma(uint32_t d, uint32_t a0, uint32_t b0, uint32_t wplane) {
  constexpr uint32_t sbo = (uint32_t)(K * P::es / 16) * 128u;
  constexpr uint32_t idesc = tc::instr_desc(P::kind, 128, N);
  constexpr uint32_t aplane = 128u * 32u * P::es;
  bool first = true;
#pragma unroll
  for (int s = 0; s < K / P::kmma; ++s) {
    const uint32_t off = (uint32_t)s * 256u;  // two 16-byte core-matrix columns per K step
    // smallest part products first
#pragma unroll
    for (int sum = P::planes - 1; sum >= 0; --sum)
#pragma unroll
      for (int i = 0; i <= sum; ++i) {
        const int jj = sum - i;
        tc::mma_bf16(d, tc::smem_desc(a0 + i * aplane + off, 128u, sbo),
                     tc::smem_desc(b0 + jj * wplane + off, 128u, sbo), idesc, first ? 0u : 1u);
        first = false;
      }
  }
}

// Decoder weight gradients on the tensor core: D[64][N] (+)= sum over the tile's 128 samples
// of A[s][m] B[s][n], both operands read MN-major from the sample-row tiles the phases write
// (core-matrix stride along K = the tile's row-group stride, along M/N = 128 bytes).  Part
// products i + j < SUM, i < APL, j < BPL, smallest first; `acc` false on the first tile.
template <int APL, int BPL, int SUM, int N>
__device__ __forceinline__ void issue_mma_dw(uint32_t d, uint32_t a0, uint32_t a_plane, uint32_t a_kstride,
                                             uint32_t b0, uint32_t b_plane, uint32_t b_kstride, bool acc) {
  constexpr uint32_t idesc = tc::instr_desc(tc::KIND_BF16, 64, N) | (1u << 15) | (1u << 16);
#pragma unroll 1
  for (int s = 0; s < 8; ++s) {  // K = 128 samples, 16 per MMA
    const uint32_t oa = (uint32_t)s * 2u * a_kstride, ob = (uint32_t)s * 2u * b_kstride;
#pragma unroll
    for (int sum = SUM - 1; sum >= 0; --sum)
#pragma unroll
      for (int i = 0; i <= sum; ++i) {
        const int j = sum - i;
        if (i >= APL || j >= BPL) continue;
        tc::mma_bf16(d, tc::smem_desc(a0 + i * a_plane + oa, a_kstride, 128u),
                     tc::smem_desc(b0 + j * b_plane + ob, b_kstride, 128u), idesc, acc ? 1u : 0u);
        acc = true;
      }
  }
}

// Part products kept in the weight-gradient MMAs: i + j < 2 in the FP32 form (relative error
// of a product below 2^-15, against the 1e-4 gradient tolerance), the single product in BF16.
template <class P>
constexpr int kDwSum = P::planes > 1 ? 2 : 1;

// per-group MMA machinery
struct Group {
  uint8_t* a;  // A operand planes
  uint8_t* b;  // partner planes of the weight-gradient products
  uint64_t* mbar;     // completion of the phase MMAs (issued by thread 0 of the group)
  uint64_t* mbar_dw;  // completion of the weight-gradient MMAs (issued by thread 32)
  uint64_t* mbar_tma; // completion of the fine-level TMA gathers (armed by thread 0)
  int* abort;
  uint32_t tcol;      // tensor-memory address of this group's column 0
  uint32_t phase;     // parity of the next completion on mbar
  uint32_t phase_dw;  // ... on mbar_dw
  uint32_t phase_tma; // ... on mbar_tma
  bool dw_pending;    // weight-gradient MMAs may still read the operand tiles
  int g, gt;
};

// A rows written by every thread -> one thread issues the MMA and commits
template <class P, int N, int K>
__device__ __forceinline__ void mma_phase_issue(Group& G, uint32_t dcol, const uint8_t* w, uint32_t wplane) {
  tc::fence_smem_async();
  tc::fence_before_sync();
  group_sync(G.g);
  tc::fence_after_sync();
  if (G.gt == 0) {
    issue_mma<P, N, K>(G.tcol + dcol, tc::smem_u32(G.a), tc::smem_u32(w), wplane);
    tc::mma_commit(G.mbar);
  }
}
// the same, and a second thread issues the weight-gradient products that read the same tiles
// and commits them to mbar_dw: the phase's result does not wait for them, and the operand
// tiles are rewritten only after dw_wait
template <class P, int N, int K, class Extra>
__device__ __forceinline__ void mma_phase_issue_dw(Group& G, uint32_t dcol, const uint8_t* w, uint32_t wplane,
                                                   Extra extra) {
  tc::fence_smem_async();
  tc::fence_before_sync();
  group_sync(G.g);
  tc::fence_after_sync();
  if (G.gt == 0) {
    issue_mma<P, N, K>(G.tcol + dcol, tc::smem_u32(G.a), tc::smem_u32(w), wplane);
    tc::mma_commit(G.mbar);
  } else if (G.gt == 32) {
    extra();
    tc::mma_commit(G.mbar_dw);
  }
  G.dw_pending = true;
}
// every thread of the group: bounded wait until the weight-gradient MMAs are done with the tiles
__device__ __forceinline__ void dw_wait(Group& G) {
  if (!G.dw_pending) return;
  if (!tc::mbar_wait(G.mbar_dw, G.phase_dw, kMbarLimit)) *reinterpret_cast<volatile int*>(G.abort) = 1;
  G.phase_dw ^= 1u;
  G.dw_pending = false;
  tc::fence_after_sync();
}
// the issuing thread waits for the MMA (bounded) while the other threads of the group park on
// the hardware barrier; false (for every thread) if it never completed
__device__ __forceinline__ bool mma_phase_wait(Group& G) {
  if (G.gt == 0 && !tc::mbar_wait(G.mbar, G.phase, kMbarLimit)) *reinterpret_cast<volatile int*>(G.abort) = 1;
  G.phase ^= 1u;
  group_sync(G.g);
  tc::fence_after_sync();
  return *reinterpret_cast<volatile int*>(G.abort) == 0;
}

__device__ __forceinline__ uint32_t lane_addr(const Group& G, uint32_t col, int warp_g) {
  return G.tcol + col + ((uint32_t)(32 * warp_g) << 16);
}

// ---- gather / scatter -------------------------------------------------------------------
// z = [V^0(x), .., V^3(x)] from the FP32 grid, or (BF16 form) from its bfloat16 copy
template <bool BF16GRID>
__device__ __forceinline__ void gather_z(const GridDesc& g, const float* __restrict__ theta,
                                         const uint16_t* __restrict__ theta_bf16, const float x[3], float z[kZ]) {
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell c = locate(g, l, x);
    float w[8];
    corner_weights(c.f, w);
    float4 v[8];
    if constexpr (BF16GRID) {
      const uint2* base = reinterpret_cast<const uint2*>(theta_bf16 + g.off[l]);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint2 u = __ldg(base + c.vtx + corner_offset(g, l, k));
        v[k] = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
      }
    } else {
      const float4* base = reinterpret_cast<const float4*>(theta + g.off[l]);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldg(base + c.vtx + corner_offset(g, l, k));
    }
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f4fma(s, w[k], v[k]);
    z[4 * l] = s.x;
    z[4 * l + 1] = s.y;
    z[4 * l + 2] = s.z;
    z[4 * l + 3] = s.w;
  }
}

// The finest kTmaLevels levels through the TMA: every thread of the group issues one
// tile::gather4 per level for its sample (rows (y,z), (y+1,z), (y,z+1), (y+1,z+1) of the
// level's 2D view, 2 vertices each) into a 128-byte slot.  The slots sit where the group's
// tiles are not written before the first decoder phase: the partner tile, then the gaps of the
// A planes that the 16-column z tile leaves free.
__device__ __forceinline__ uint32_t fine_slot(uint8_t* ga, uint8_t* gb, int lvl, int gt) {
  if (lvl == 0) return tc::smem_u32(gb + gt * 128);
  if (gt < 64) return tc::smem_u32(gb + 16384 + gt * 128);
  if (gt < 96) return tc::smem_u32(ga + 4096 + (gt - 64) * 128);
  return tc::smem_u32(ga + 12288 + (gt - 96) * 128);
}
constexpr int kTmaLevels = 1;  // the finest levels that go through the TMA (the rest: plain loads)
// host: the 2D view [nz ny][4 nx] of grid level l in theta, a box of 2 vertices x 4 features one
// row high (the tile::gather4 source of the finest level); false if the driver refused it
bool gs_encode_level_map(const gs_ctx* ctx, const float* theta, int l, CUtensorMap* m);
constexpr uint32_t kFineTmaBytes = 128u * kTmaLevels * 128u;  // per group and round: 128 samples x levels x 128 B

// issue both fine-level gathers of this thread's sample; returns the cells (for the weights)
__device__ __forceinline__ void fine_gather_issue(const GridDesc& g, const CUtensorMap* tmap, uint8_t* ga, uint8_t* gb,
                                                  int gt, uint64_t* mbar, const float x[3], Cell (&cs)[kTmaLevels]) {
  tc::fence_smem_async();  // earlier generic accesses to the slots before the asynchronous writes
#pragma unroll
  for (int q = 0; q < kTmaLevels; ++q) {
    const int l = kLevels - kTmaLevels + q;
    cs[q] = locate(g, l, x);
    const int ny = g.dims[l][1];
    const int r0 = cs[q].idx[2] * ny + cs[q].idx[1];
    tc::tma_gather4(fine_slot(ga, gb, q, gt), &tmap[q], 4 * cs[q].idx[0], r0, r0 + 1, r0 + ny, r0 + ny + 1, mbar);
  }
}
// z of the fine levels from this thread's slots (chunk order rotated by lane: no bank conflicts)
__device__ __forceinline__ void fine_gather_read(const uint8_t* ga, const uint8_t* gb, int gt,
                                                 const Cell (&cs)[kTmaLevels], float z[kZ]) {
  const int lane = gt & 31;
#pragma unroll
  for (int q = 0; q < kTmaLevels; ++q) {
    const int l = kLevels - kTmaLevels + q;
    const uint8_t* slot = q == 0 ? gb + gt * 128
                                 : (gt < 64 ? gb + 16384 + gt * 128
                                            : (gt < 96 ? ga + 4096 + (gt - 64) * 128 : ga + 12288 + (gt - 96) * 128));
    const float f0 = cs[q].f[0], f1 = cs[q].f[1], f2 = cs[q].f[2];
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = (k + lane) & 7;  // 16-byte chunk: row c >> 1 = (by, bz), x-vertex c & 1
      const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
      const float w = ((bx ? f0 : 1.0f - f0) * (by ? f1 : 1.0f - f1)) * (bz ? f2 : 1.0f - f2);
      f4fma(s, w, *reinterpret_cast<const float4*>(slot + c * 16));
    }
    z[4 * l] = s.x;
    z[4 * l + 1] = s.y;
    z[4 * l + 2] = s.z;
    z[4 * l + 3] = s.w;
  }
}
// the other levels by plain loads (a warp's samples share the coarse cells)
__device__ __forceinline__ void coarse_gather(const GridDesc& g, const float* __restrict__ theta, const float x[3],
                                              float z[kZ]) {
#pragma unroll
  for (int l = 0; l < kLevels - kTmaLevels; ++l) {
    const Cell c = locate(g, l, x);
    float w[8];
    corner_weights(c.f, w);
    const float4* base = reinterpret_cast<const float4*>(theta + g.off[l]);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f4fma(s, w[k], __ldg(base + c.vtx + corner_offset(g, l, k)));
    z[4 * l] = s.x;
    z[4 * l + 1] = s.y;
    z[4 * l + 2] = s.z;
    z[4 * l + 3] = s.w;
  }
}

// staging floats per warp of scatter_dz: 32 rows of 36 floats, then the 32 keys
constexpr int kScatterStage = 33 * 36;

// 16-byte vector reduction into global memory (fire and forget; the result is not read)
__device__ __forceinline__ void red_add_f4(float4* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

// Adjoint of the gather: dtheta_l[corner] += w_c dz_l.  A warp's lanes hold consecutive
// samples of one ray, so the cells they fall in are visited monotonically and equal cells form
// contiguous runs of lanes.  At the two coarse levels (long runs) the 8 weighted corner vectors
// are summed over each run through shared memory: every lane stages its 32 values as a row,
// lane c walks the 32 rows summing component c (corner c / 4, feature c % 4), and at the end of
// each run the four features of a corner are gathered into one lane, which issues one 16-byte
// reduction (8 per run).  At the fine levels, where runs are short, every lane issues its 8
// corners' 16-byte reductions directly (staging them there measured slower).
// `st`: this warp's kScatterStage floats of staging space.
// Deferred Eikonal term: `er` (nullptr for samples without one) points at the sample's record
// in plane 0 of the batch's Eikonal records (planes `es` float4 apart: q_l = p_l / v_l for the
// four levels, then the adjoint a); corner c of level l then also receives q_l (a . dw_c/df),
// the grid part of the Eikonal gradient (Supp. Sec. 1), in the same 16-byte reduction.
// PAIRED (the fine levels): lane pairs (2i, 2i + 1) take turns on each other's samples so
// that in one reduction instruction the pair adds a cell's two x-neighbouring corners of one
// sample, 32 contiguous bytes (one sector when the cell's x index is even): a quarter fewer
// L2 reduction requests for 18 shuffles per level and lane.
template <bool PAIRED = false>
__device__ __forceinline__ void scatter_dz(const GridDesc& g, float* grad, const float x[3], const float dz[kZ],
                                           bool valid, float* st, const float4* er = nullptr, long long es = 0) {
  const unsigned active = __ballot_sync(0xffffffffu, valid);
  if (active == 0) return;
  const int lane = threadIdx.x & 31;
  const bool eik_any = __any_sync(0xffffffffu, er != nullptr);
  float ea[3] = {0.f, 0.f, 0.f};
  if (er != nullptr) {
    const float4 a4 = __ldg(er + 4 * es);
    ea[0] = a4.x;
    ea[1] = a4.y;
    ea[2] = a4.z;
  }
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell cc = locate(g, l, x);
    float wc[8];
    corner_weights(cc.f, wc);
    const float4 g4 = valid ? make_float4(dz[4 * l], dz[4 * l + 1], dz[4 * l + 2], dz[4 * l + 3])
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float dd[8];  // a . dw_c/df (zero without a record)
#pragma unroll
    for (int k = 0; k < 8; ++k) dd[k] = 0.f;
    if (eik_any) {  // warp-uniform
      if (er != nullptr) q4 = __ldg(er + l * es);
      float dw[8][3];
      corner_weight_grads(cc.f, cc.clamped, dw);
#pragma unroll
      for (int k = 0; k < 8; ++k) dd[k] = ea[0] * dw[k][0] + ea[1] * dw[k][1] + ea[2] * dw[k][2];
    }
    float4* gl = reinterpret_cast<float4*>(grad + g.off[l]);
    if (l >= 2) {
      // a zero vector adds nothing: samples whose dL/dz_l is exactly zero (saturated opacity and
      // no active loss term) issue no reductions at the fine levels
      const bool nz = g4.x != 0.f || g4.y != 0.f || g4.z != 0.f || g4.w != 0.f || er != nullptr;
      if constexpr (PAIRED) {
        // corners k and k + 4 are the x-neighbours v and v + 1.  The even lane sends its
        // upper corner's vector and receives the odd lane's lower one; then the even lane adds
        // the lower corners (its own sample's, then its partner's) and the odd lane the upper
        // ones (its partner's, then its own), so each instruction covers one sample's pair.
        const bool odd = (lane & 1) != 0;
        const bool give = valid && nz;
        const long long pv = __shfl_xor_sync(0xffffffffu, cc.vtx, 1);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float4 lo4 = make_float4(0.f, 0.f, 0.f, 0.f), hi4 = lo4;
          if (give) {
            lo4 = f4scale(g4, wc[k]);
            hi4 = f4scale(g4, wc[k + 4]);
            if (eik_any) {
              f4fma(lo4, dd[k], q4);
              f4fma(hi4, dd[k + 4], q4);
            }
          }
          const float4 snd = odd ? lo4 : hi4;
          float4 rcv;
          rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, 1);
          rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, 1);
          rcv.z = __shfl_xor_sync(0xffffffffu, snd.z, 1);
          rcv.w = __shfl_xor_sync(0xffffffffu, snd.w, 1);
          const long long off = corner_offset(g, l, k);  // the lower corner; the upper one is + 1
          // first instruction: the even lane's sample; second: the odd lane's
          const long long v0 = (odd ? pv : cc.vtx) + off + (odd ? 1 : 0);
          const long long v1 = (odd ? cc.vtx : pv) + off + (odd ? 1 : 0);
          const float4 c0 = odd ? rcv : lo4, c1 = odd ? hi4 : rcv;
          if (c0.x != 0.f || c0.y != 0.f || c0.z != 0.f || c0.w != 0.f) red_add_f4(gl + v0, c0);
          if (c1.x != 0.f || c1.y != 0.f || c1.z != 0.f || c1.w != 0.f) red_add_f4(gl + v1, c1);
        }
      } else if (valid && nz) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          float4 cv = f4scale(g4, wc[k]);
          if (eik_any) f4fma(cv, dd[k], q4);
          red_add_f4(gl + cc.vtx + corner_offset(g, l, k), cv);
        }
      }
      continue;
    }
    const int key = valid ? (int)cc.vtx : -1;  // the coarse levels have fewer than 2^31 vertices
    const int next = __shfl_down_sync(0xffffffffu, key, 1);
    const unsigned ends = __ballot_sync(0xffffffffu, lane == 31 || next != key || key < 0);  // a run's last lane
    float* rw = st + lane * 36;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float4 cv = f4scale(g4, wc[k]);
      if (eik_any) f4fma(cv, dd[k], q4);
      *reinterpret_cast<float4*>(rw + 4 * k) = cv;
    }
    st[32 * 36 + lane] = __int_as_float(key);  // the keys after the rows
    __syncwarp();
    const long long coff = corner_offset(g, l, lane >> 2);
    float acc = 0.f;
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      acc += st[i * 36 + lane];
      if ((ends >> i) & 1u) {  // uniform: the run holding row i ends at row i
        const float a1 = __shfl_down_sync(0xffffffffu, acc, 1), a2 = __shfl_down_sync(0xffffffffu, acc, 2),
                    a3 = __shfl_down_sync(0xffffffffu, acc, 3);
        const int ki = __float_as_int(st[32 * 36 + i]);
        if ((lane & 3) == 0 && ki >= 0) red_add_f4(gl + (long long)ki + coff, make_float4(acc, a1, a2, a3));
        acc = 0.f;
      }
    }
    __syncwarp();
  }
}

template <int N>
__device__ __forceinline__ float pick_tc(const float (&arr)[N], int j) {
  float v = arr[0];
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (q == j) v = arr[q];
  return v;
}

// Stored activations come in groups of four fields, one float4 plane per group: field f of
// sample s sits in component f % 4 of ((float4*)store)[(f / 4) * ss + s], so a warp's 32
// consecutive samples read or write one 512-byte line per group.  sp points at sample s's
// element of plane 0.
template <int F0, int NF, int M>
__device__ __forceinline__ void put_fields(float4* sp, long long ss, const float (&v)[M]) {
  static_assert(F0 % 4 == 0 && NF % 4 == 0 && NF <= M, "whole groups of four fields");
#pragma unroll
  for (int q = 0; q < NF / 4; ++q) sp[(F0 / 4 + q) * ss] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
template <int F0, int NF, int M>
__device__ __forceinline__ void get_fields(const float4* sp, long long ss, bool get, float (&v)[M]) {
  static_assert(F0 % 4 == 0 && NF % 4 == 0 && NF <= M, "whole groups of four fields");
#pragma unroll
  for (int q = 0; q < NF / 4; ++q) {
    const float4 u = get ? __ldg(sp + (F0 / 4 + q) * ss) : make_float4(0.f, 0.f, 0.f, 0.f);
    v[4 * q] = u.x;
    v[4 * q + 1] = u.y;
    v[4 * q + 2] = u.z;
    v[4 * q + 3] = u.w;
  }
}

struct RenderTcArgs {
  GridDesc g;
  const float* theta;
  const uint16_t* theta_bf16;  // BF16 form: grid copy read by the gathers
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
  int* status;      // device status word (bit 1: an MMA never completed)
  // Stored activations (store mode): field f of sample s = rr * N + si in component f % 4 of
  // ((float4*)store)[(f / 4) * store_stride + s], one coalesced float4 plane per four fields.
  // Written by every forward pass, read by every backward pass in place of the gather and the
  // four recomputed decoder phases.  nullptr: recompute.
  float* store;
  long long store_stride;
  float* w_out;  // [R][N] rendering weights, written by forward passes when not nullptr
  float* dz_out; // [R][N][16] dL/dz of every sample, written by backward passes when not nullptr
  // deferred Eikonal records ([5][R][N] float4 planes, eik_stride = R N) of the free-space
  // samples, added to their grid scatter by backward passes; nullptr: none
  const float4* eik;
  long long eik_stride;
  // FP32 form: 2D views [nz * ny][nx * 4] of grid levels 2 and 3 for the TMA gathers (a box of
  // 2 vertices x 4 features; one tile::gather4 brings a cell's 8 corners)
  CUtensorMap tmap[2];
};

// fields of one stored sample: z[16] | a1 = ReLU layer-1 output [32] | (phi, h[15]) | a2 [32] | c[3], 0
constexpr int kFz = 0, kFa1 = 16, kFout = 48, kFa2 = 64, kFc = 96, kStoreFields = 100;
static_assert(kStoreFields == kStoreFloatsPerSample, "the store holds every field");

// colour c = sigmoid(W4 a2 + b4) on CUDA cores (3 outputs: too narrow for a tensor-core phase)
__device__ __forceinline__ void colour_out(const float* w4f, const float* b4, const float (&a2)[32], float (&c3)[3]) {
#pragma unroll
  for (int n = 0; n < 3; ++n) {
    float s = b4[n];
#pragma unroll
    for (int k = 0; k < 32; ++k) s = fmaf(w4f[32 * n + k], a2[k], s);
    c3[n] = sigmoidf_(s);
  }
}

// z of one chunk: every thread of the group takes part (the TMA round counts all 128 slots);
// invalid samples get z = 0
template <class P>
__device__ __forceinline__ void gather_chunk(Group& G, const RenderTcArgs& a, const float x[3], bool valid,
                                             float z[kZ]) {
  if constexpr (P::planes > 1) {  // FP32 form: fine levels through the TMA, coarse by plain loads
    Cell cs[kTmaLevels];
    fine_gather_issue(a.g, a.tmap + (2 - kTmaLevels), G.a, G.b, G.gt, G.mbar_tma, x, cs);
    if (valid) coarse_gather(a.g, a.theta, x, z);
    if (!tc::mbar_wait(G.mbar_tma, G.phase_tma, kMbarLimit)) *reinterpret_cast<volatile int*>(G.abort) = 1;
    G.phase_tma ^= 1u;
    if (G.gt == 0) tc::mbar_arrive_expect_tx(G.mbar_tma, kFineTmaBytes);  // armed for the next round
    fine_gather_read(G.a, G.b, G.gt, cs, z);
  } else if (valid) {
    gather_z<true>(a.g, a.theta, a.theta_bf16, x, z);
  }
  if (!valid) {
#pragma unroll
    for (int k = 0; k < kZ; ++k) z[k] = 0.f;
  }
}

// the forward-only instantiation ends each ray-quad before its reverse pass, which the front
// end reports as unreachable code there
#pragma nv_diag_suppress 128
template <class P, int NCH, int GR, bool FWD, bool BWD>
__global__ void __launch_bounds__(GR * kGroupThreads, 1) render_tc_kernel(const __grid_constant__ RenderTcArgs a) {
  using L = TcLayout<P>;
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr uint32_t wplane = wTotal<P>();  // one bf16 part of all weight tiles
  uint8_t* wt0 = smem;
  float* acc = reinterpret_cast<float*>(smem + wplane * P::planes);  // [kMlpPad] + loss [kLossPad]
  float* lacc = acc + kMlpPad;
  float* bias = lacc + kLossPad;  // b1[32] b2[16] b3[32] b4[4] kappa
  float* w4f = bias + 88;         // W4 [3][32] in FP32: the colour output layer runs on CUDA cores
  uint32_t* tslot = reinterpret_cast<uint32_t*>(w4f + 96);
  float* gacc = reinterpret_cast<float*>(tslot + 4);  // per-group decoder-gradient accumulators [GR][kMlpPad]
  uint8_t* gbase = reinterpret_cast<uint8_t*>(gacc + GR * kMlpPad);
  gbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gbase) + 1023) & ~uintptr_t(1023));

  const int tid = threadIdx.x, gi = tid / kGroupThreads, gt = tid % kGroupThreads, warp_g = gt >> 5,
            lane = tid & 31;
  uint8_t* gmem = gbase + (size_t)gi * L::group_bytes;
  Group G;
  G.a = gmem;
  G.b = gmem + L::a_bytes * P::planes;
  G.mbar = reinterpret_cast<uint64_t*>(gmem + L::a_bytes * P::planes + L::b_bytes * L::b_planes);
  G.mbar_dw = G.mbar + 1;
  G.mbar_tma = G.mbar + 2;
  G.abort = reinterpret_cast<int*>(G.mbar + 3);
  G.phase_dw = 0;
  G.phase_tma = 0;
  G.dw_pending = false;
  G.g = gi;
  G.gt = gt;
  G.phase = 0;

  // ---- CTA set-up: weight tiles, biases, accumulators, barriers, tensor memory ----
  const float* mlp = a.theta + a.g.n_grid;
  for (int m = 0; m < 8; ++m) {
    const int Nn = wN(m), K = wK(m);
    for (int e = tid; e < Nn * K; e += blockDim.x) {
      const int n = e / K, k = e % K;
      float v = 0.f;
      switch (m) {
        case 0: v = mlp[oW1 + n * kZ + k]; break;
        case 1: v = mlp[oW2 + n * kH1 + k]; break;
        case 2: v = k < kHF ? mlp[oW3 + n * kHF + k] : 0.f; break;
        case 3: v = n < kRGB ? mlp[oW4 + n * kH2 + k] : 0.f; break;
        case 4: v = k < kRGB ? mlp[oW4 + k * kH2 + n] : 0.f; break;
        case 5: v = n < kHF ? mlp[oW3 + k * kHF + n] : 0.f; break;
        case 6: v = mlp[oW2 + k * kH1 + n]; break;
        default: v = mlp[oW1 + k * kZ + n]; break;
      }
      store_w<P>(wt0 + wOff<P>(m), wplane, K, n, k, v);
    }
  }
  for (int i = tid; i < 96; i += blockDim.x) w4f[i] = mlp[oW4 + i];
  for (int i = tid; i < 88; i += blockDim.x) {
    float v = 0.f;
    if (i < 32) v = mlp[ob1 + i];
    else if (i < 48) v = mlp[ob2 + i - 32];
    else if (i < 80) v = mlp[ob3 + i - 48];
    else if (i < 83) v = mlp[ob4 + i - 80];
    else if (i == 84) v = mlp[oKappa];
    bias[i] = v;
  }
  for (int i = tid; i < kMlpPad + kLossPad; i += blockDim.x) acc[i] = 0.f;
  for (int i = tid; i < GR * kMlpPad; i += blockDim.x) gacc[i] = 0.f;
  if (gt == 0) {
    tc::mbar_init(G.mbar, 1);
    tc::mbar_init(G.mbar_dw, 1);
    tc::mbar_init(G.mbar_tma, 1);
    tc::fence_mbar_init();
    if (P::planes > 1) tc::mbar_arrive_expect_tx(G.mbar_tma, kFineTmaBytes);  // armed for the first round
    *G.abort = 0;
  }
  static_assert(tmem_cols(GR) <= 512, "tensor memory holds 512 columns");
  if (tid < 32) tc::tmem_alloc(tslot, tmem_cols(GR));
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  G.tcol = *tslot + (uint32_t)(gi * kGroupCols);
  const float* b1 = bias;
  const float* b2 = bias + 32;
  const float* b3 = bias + 48;
  const float* b4 = bias + 80;
  const float s_sharp = expf(bias[84]);
  float* macc = gacc + gi * kMlpPad;  // this group's decoder-gradient accumulator

  const int N = a.N;
  float wt[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) wt[k] = a.dloss[k] + a.lam[k] * a.dloss[5];
  const int n_d = a.counts[0], n_tr = a.counts[1], n_fs = a.counts[2];
  const float k_rgb = a.R > 0 ? wt[0] * 2.0f / (float)a.R : 0.f;
  const float k_d = n_d > 0 ? wt[1] / (float)n_d : 0.0f;
  const float k_sdf = n_tr > 0 ? wt[2] / (float)n_tr : 0.0f;
  const float k_fs = n_fs > 0 ? wt[3] / (float)n_fs : 0.0f;
  float l_rgb = 0.f, l_d = 0.f, l_sdf = 0.f, l_fs = 0.f, g_kappa = 0.f;
  const int row = gt;  // tile row of this thread's sample
  bool alive = true;
  bool dw_acc = false;  // the weight-gradient accumulators hold a first tile (accumulate from then on)
  float w4acc[3] = {0.f, 0.f, 0.f}, b4acc = 0.f;  // this warp's dW4[.][lane] and (lanes < 3) db4[lane]

  // ray-quads are dealt CTA-major (quad = round * G + CTA * GR + gi): when the quads do not
  // divide evenly, whole SMs finish a round early, and the smoothness kernel, launched beside
  // this one on another stream, runs there
  for (int quad = blockIdx.x * GR + gi; quad * 4 < a.R && alive; quad += gridDim.x * GR) {
    const int ray = quad * 4 + warp_g;
    const bool has_ray = ray < a.R;
    const int rr = has_ray ? ray : 0;
    const float o[3] = {a.o[3 * rr], a.o[3 * rr + 1], a.o[3 * rr + 2]};
    const float r[3] = {a.r[3 * rr], a.r[3 * rr + 1], a.r[3 * rr + 2]};
    const float D = has_ray ? a.D[rr] : 0.f;
    const float I[3] = {a.rgb[3 * rr], a.rgb[3 * rr + 1], a.rgb[3 * rr + 2]};
    float tt[NCH], ph[NCH], col[NCH][3];
    int clv[NCH];  // sample classes
    // every per-sample input of the ray up front: one memory round trip instead of one per chunk
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      const int si = 32 * q + lane;
      const bool in = has_ray && si < N;
      tt[q] = in ? a.t[(size_t)rr * N + si] : 0.f;
      clv[q] = in ? (int)a.cls[(size_t)rr * N + si] : 0;
    }

    // ================= forward: gather, then 4 decoder phases per chunk =================
#pragma unroll 1
    for (int j = 0; j < NCH && alive; ++j) {
      const int si = 32 * j + lane;
      const bool valid = has_ray && si < N;
      const float t = pick_tc(tt, j);
      float4* sp = a.store != nullptr ? reinterpret_cast<float4*>(a.store) + (size_t)rr * N + si : nullptr;
      const long long ss = a.store_stride;
      if (!FWD && sp != nullptr) {  // stored by the forward pass: no decoder phases here
        const float4 o4 = valid ? sp[(kFout / 4) * ss] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 c4 = valid ? sp[(kFc / 4) * ss] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < NCH; ++q)
          if (q == j) {
            tt[q] = t;
            ph[q] = o4.x;
            col[q][0] = c4.x;
            col[q][1] = c4.y;
            col[q][2] = c4.z;
          }
        continue;
      }
      const bool put = FWD && sp != nullptr && valid;
      float z[kZ];
      {
        float x[3];
        sample_pos(o, r, t, x);
        dw_wait(G);  // the TMA slots overlap the partner tile and the A planes
        gather_chunk<P>(G, a, x, valid, z);
      }
      store_row<P, 16>(G.a, row, z);
      mma_phase_issue<P, 32, 16>(G, cD1, wt0 + wOff<P>(0), wplane);
      if (put) put_fields<kFz, 16>(sp, ss, z);
      if (!(alive = mma_phase_wait(G))) break;
      float v[32];
      tc::tmem_ld32(lane_addr(G, cD1, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + b1[k], 0.f);
      store_row<P, 32>(G.a, row, v);
      mma_phase_issue<P, 16, 32>(G, cD2, wt0 + wOff<P>(1), wplane);
      if (put) put_fields<kFa1, 32>(sp, ss, v);
      if (!(alive = mma_phase_wait(G))) break;
      float u[16];
      tc::tmem_ld16(lane_addr(G, cD2, warp_g), u);
      tc::tmem_ld_wait();
      const float phi = u[0] + b2[0];
      float h[16];
#pragma unroll
      for (int k = 0; k < 15; ++k) h[k] = u[k + 1] + b2[k + 1];
      h[15] = 0.f;
      store_row<P, 16>(G.a, row, h);
      mma_phase_issue<P, 32, 16>(G, cD3, wt0 + wOff<P>(2), wplane);
      if (put) {
        float oh[16];
        oh[0] = phi;
#pragma unroll
        for (int k = 0; k < 15; ++k) oh[k + 1] = h[k];
        put_fields<kFout, 16>(sp, ss, oh);
      }
      if (!(alive = mma_phase_wait(G))) break;
      tc::tmem_ld32(lane_addr(G, cD3, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + b3[k], 0.f);
      if (put) put_fields<kFa2, 32>(sp, ss, v);
      float c3[3];
      colour_out(w4f, b4, v, c3);
      if (put) {
        const float c4[4] = {c3[0], c3[1], c3[2], 0.f};
        put_fields<kFc, 4>(sp, ss, c4);
      }
      // keep per-chunk values in registers (compile-time index via a selector loop)
#pragma unroll
      for (int q = 0; q < NCH; ++q)
        if (q == j) {
          tt[q] = t;
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
        const int si = 32 * j + lane;
        if (si >= N) continue;
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
      const int si = 32 * j + lane;
      const bool valid = has_ray && si < N;
      const float dal = T[j] * (e[j] - U[j]);
      float dself = 0.f, dnext = 0.f;
      if (valid && si < N - 1) {
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

    // ================= reverse, chunk by chunk: recompute, 4 adjoint phases =================
#pragma unroll 1
    for (int j = 0; j < NCH && alive; ++j) {
      const int si = 32 * j + lane;
      const bool valid = has_ray && si < N;
      const float t = pick_tc(tt, j);
      float x[3];
      sample_pos(o, r, t, x);
      const float4* sp = a.store != nullptr ? reinterpret_cast<const float4*>(a.store) + (size_t)rr * N + si : nullptr;
      const long long ss = a.store_stride;
      const bool get = sp != nullptr && valid;
      float z[kZ], v[32], h[16], u[16], c3[3];
      uint32_t mask2 = 0;
      if (sp != nullptr) {  // stored activations: z, a2, h and c now, a1 where it is used
        get_fields<kFz, 16>(sp, ss, get, z);
        get_fields<kFa2, 32>(sp, ss, get, v);
        float oh[16];
        get_fields<kFout, 16>(sp, ss, get, oh);
#pragma unroll
        for (int k = 0; k < 15; ++k) h[k] = oh[k + 1];
        h[15] = 0.f;
        float c4[4];
        get_fields<kFc, 4>(sp, ss, get, c4);
        c3[0] = c4[0];
        c3[1] = c4[1];
        c3[2] = c4[2];
      } else {
        dw_wait(G);
        gather_chunk<P>(G, a, x, valid, z);
        // recompute the decoders (the same four phases as the forward)
        store_row<P, 16>(G.a, row, z);
        mma_phase_issue<P, 32, 16>(G, cD1, wt0 + wOff<P>(0), wplane);
        if (!(alive = mma_phase_wait(G))) break;
        tc::tmem_ld32(lane_addr(G, cD1, warp_g), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + b1[k], 0.f);
        store_row<P, 32>(G.a, row, v);
        mma_phase_issue<P, 16, 32>(G, cD2, wt0 + wOff<P>(1), wplane);
        if (!(alive = mma_phase_wait(G))) break;
        tc::tmem_ld16(lane_addr(G, cD2, warp_g), u);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 15; ++k) h[k] = u[k + 1] + b2[k + 1];
        h[15] = 0.f;
        store_row<P, 16>(G.a, row, h);
        mma_phase_issue<P, 32, 16>(G, cD3, wt0 + wOff<P>(2), wplane);
        if (!(alive = mma_phase_wait(G))) break;
        tc::tmem_ld32(lane_addr(G, cD3, warp_g), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + b3[k], 0.f);
        colour_out(w4f, b4, v, c3);
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) mask2 |= (v[k] > 0.f ? 1u : 0u) << k;
      // colour output adjoint: dpre = w gc c (1 - c)
      const float wj = pick_tc(w, j);
      float dp[kKD];
#pragma unroll
      for (int k = 0; k < kKD; ++k) dp[k] = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) dp[k] = valid ? wj * gc[k] * c3[k] * (1.0f - c3[k]) : 0.f;
      dw_wait(G);  // no tensor-core product reads the tiles now: stage the colour layer's rows there
      // --- b4 on CUDA cores: da2 = dpre W4 (3 x 32); dW4, db4 (+)= sum over the warp's samples ---
      {
        // 4 warps x 32 rows x 36 floats = 18 KB from the A planes on (the A and partner planes
        // are contiguous and hold at least 20 KB in both forms)
        static_assert(L::a_bytes * P::planes + L::b_bytes * L::b_planes >= 4u * 32u * 36u * 4u, "staging space");
        float* st = reinterpret_cast<float*>(G.a) + warp_g * (32 * 36);  // row: dpre[3] | 0 | a2[32]
        float* rw = st + lane * 36;
        *reinterpret_cast<float4*>(rw) = make_float4(dp[0], dp[1], dp[2], 0.f);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(rw + 4 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
#pragma unroll 4
        for (int s2 = 0; s2 < 32; ++s2) {
          const float* r2 = st + s2 * 36;
          const float a2v = r2[4 + lane];
          w4acc[0] = fmaf(r2[0], a2v, w4acc[0]);
          w4acc[1] = fmaf(r2[1], a2v, w4acc[1]);
          w4acc[2] = fmaf(r2[2], a2v, w4acc[2]);
          b4acc += r2[lane & 3];
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 32; ++k) {  // dy2 = mask2 (.) (dpre W4)
          const float d = fmaf(dp[0], w4f[k], fmaf(dp[1], w4f[32 + k], dp[2] * w4f[64 + k]));
          v[k] = ((mask2 >> k) & 1u) ? d : 0.f;
        }
        group_sync(G.g);  // every warp has read its staged rows before the tiles are rewritten
      }
      store_row<P, 32>(G.a, row, v);
      h[15] = 1.f;  // ones column: the bias gradient db3 lands in column 15 of dW3
      store_row_planes<L::b_planes, 16, L::b_bytes>(G.b, row, h);
      // --- b3: dh = dy2 W3;  dW3, db3 (+)= dy2^T [h | 1] ---
      mma_phase_issue_dw<P, 16, 32>(G, cYb, wt0 + wOff<P>(5), wplane, [&] {
        issue_mma_dw<P::planes, L::b_planes, kDwSum<P>, 16>(G.tcol + cW3, tc::smem_u32(G.a), L::a_bytes, 4u * 128u,
                                                            tc::smem_u32(G.b), L::b_bytes, 2u * 128u, dw_acc);
      });
      if (!(alive = mma_phase_wait(G))) break;
      tc::tmem_ld16(lane_addr(G, cYb, warp_g), u);
      tc::tmem_ld_wait();
      float dout[16];
      dout[0] = valid ? pick_tc(dphi, j) : 0.f;
#pragma unroll
      for (int k = 1; k < 16; ++k) dout[k] = u[k - 1];
      dw_wait(G);
      store_row<P, 16>(G.a, row, dout);
      uint32_t mask1 = 0;
      {
        float ab[40];
        if (sp != nullptr) {
          get_fields<kFa1, 32>(sp, ss, get, ab);
        } else {
          float a1[32];
          tc::tmem_ld32(lane_addr(G, cD1, warp_g), a1);
          tc::tmem_ld_wait();
#pragma unroll
          for (int k = 0; k < 32; ++k) ab[k] = fmaxf(a1[k] + b1[k], 0.f);
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) mask1 |= (ab[k] > 0.f ? 1u : 0u) << k;
        ab[32] = 1.f;
#pragma unroll
        for (int k = 33; k < 40; ++k) ab[k] = 0.f;
        store_row_planes<L::b_planes, 40, L::b_bytes>(G.b, row, ab);
      }
      // --- b2: da1 = dout W2;  dW2^T, db2 (+)= [a1 | 1]^T dout ---
      mma_phase_issue_dw<P, 32, 16>(G, cXb, wt0 + wOff<P>(6), wplane, [&] {
        issue_mma_dw<L::b_planes, P::planes, kDwSum<P>, 16>(G.tcol + cW2, tc::smem_u32(G.b), L::b_bytes, 5u * 128u,
                                                            tc::smem_u32(G.a), L::a_bytes, 2u * 128u, dw_acc);
      });
      if (!(alive = mma_phase_wait(G))) break;
      tc::tmem_ld32(lane_addr(G, cXb, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = ((mask1 >> k) & 1u) ? v[k] : 0.f;  // dy1
      dw_wait(G);
      store_row<P, 32>(G.a, row, v);
      {
        float zb[24];
#pragma unroll
        for (int k = 0; k < 16; ++k) zb[k] = z[k];
        zb[16] = 1.f;
#pragma unroll
        for (int k = 17; k < 24; ++k) zb[k] = 0.f;
        store_row_planes<L::b_planes, 24, L::b_bytes>(G.b, row, zb);
      }
      // --- b1: dz = dy1 W1;  dW1, db1 (+)= dy1^T [z | 1] ---
      mma_phase_issue_dw<P, 16, 32>(G, cYb, wt0 + wOff<P>(7), wplane, [&] {
        issue_mma_dw<P::planes, L::b_planes, kDwSum<P>, 24>(G.tcol + cW1, tc::smem_u32(G.a), L::a_bytes, 4u * 128u,
                                                            tc::smem_u32(G.b), L::b_bytes, 3u * 128u, dw_acc);
      });
      if (!(alive = mma_phase_wait(G))) break;
      dw_acc = true;
      tc::tmem_ld16(lane_addr(G, cYb, warp_g), u);
      tc::tmem_ld_wait();
      if (a.dz_out != nullptr && valid) {  // dL/dz of this sample (camera-pose gradients)
        float4* dzo = reinterpret_cast<float4*>(a.dz_out + ((size_t)rr * N + si) * kZ);
#pragma unroll
        for (int q = 0; q < 4; ++q) dzo[q] = make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
      }
      dw_wait(G);  // the tiles' space holds the scatter's staging rows
      static_assert(L::a_bytes * P::planes + L::b_bytes * L::b_planes >= 4u * kScatterStage * 4u, "staging space");
      int clj = clv[0];
#pragma unroll
      for (int q = 1; q < NCH; ++q)
        if (q == j) clj = clv[q];
      const float4* er = a.eik != nullptr && valid && clj == CLS_FS ? a.eik + (size_t)rr * N + si : nullptr;
      scatter_dz<(P::planes == 1)>(a.g, a.grad, x, u, valid, reinterpret_cast<float*>(G.a) + warp_g * kScatterStage, er,
                                   a.eik_stride);
      group_sync(G.g);  // every warp is done with its rows before the tiles are rewritten
    }
  }

  // ---- epilogue: loss and decoder-gradient partials, coarsest level, tensor memory ----
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
    dw_wait(G);
    if (alive && dw_acc && *reinterpret_cast<volatile int*>(G.abort) == 0) {
      // the group's weight-gradient accumulators: warp w holds rows 16 w .. 16 w + 15 of every
      // M = 64 product in its lanes 0..15 (rows 32.. are the bias rows or unused)
      float d1[32], d2[32];
      tc::tmem_ld32(lane_addr(G, cW1, warp_g), d1);  // cW1 .. cW1 + 31: dW1 (24) | dW2^T (first 8)
      tc::tmem_ld32(lane_addr(G, cW1 + 32, warp_g), d2);  // dW2^T (last 8) | dW3 (16) | dW4^T (8)
      tc::tmem_ld_wait();
      const int m = 16 * warp_g + lane;  // D row held by this lane
      if (lane < 16 && m < 32) {
#pragma unroll
        for (int n = 0; n < 16; ++n) macc[oW1 + m * kZ + n] += d1[n];  // dW1[m][n]
        macc[ob1 + m] += d1[16];                                       // db1[m]
#pragma unroll
        for (int n = 0; n < 16; ++n) macc[oW2 + n * kH1 + m] += (n < 8 ? d1[24 + n] : d2[n - 8]);  // dW2[n][m]
#pragma unroll
        for (int n = 0; n < 15; ++n) macc[oW3 + m * kHF + n] += d2[8 + n];  // dW3[m][n]
        macc[ob3 + m] += d2[8 + 15];                                      // db3[m]
      } else if (lane == 0 && m == 32) {  // bias row of the transposed product
#pragma unroll
        for (int n = 0; n < 16; ++n) macc[ob2 + n] += (n < 8 ? d1[24 + n] : d2[n - 8]);
      }
    }
    // the colour layer's gradient, accumulated per warp on CUDA cores
#pragma unroll
    for (int n = 0; n < 3; ++n) atomicAdd(macc + oW4 + n * kH2 + lane, w4acc[n]);
    if (lane < 3) atomicAdd(macc + ob4 + lane, b4acc);
  }
  if (!alive && gt == 0) {
    atomicOr(a.status, 2);
    tc::mbar_wait(G.mbar, G.phase ^ 1u, kMbarLimit);  // let an MMA in flight finish
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < kLossPad) a.loss_part[(size_t)blockIdx.x * kLossPad + tid] = lacc[tid];
  for (int i = tid; i < kMlpPad; i += blockDim.x) {
    float v = acc[i];
#pragma unroll
    for (int q = 0; q < GR; ++q) v += gacc[q * kMlpPad + i];
    a.mlp_part[(size_t)blockIdx.x * kMlpPad + i] = v;
  }
  if (tid < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*tslot, tmem_cols(GR));
  }
}
#pragma nv_diag_default 128

template <class P, int GR>
size_t render_tc_smem() {
  using L = TcLayout<P>;
  size_t b = wTotal<P>() * P::planes + (kMlpPad + kLossPad + 88 + 96 + 4 + GR * kMlpPad) * 4;
  b = (b + 1023) & ~size_t(1023);
  return b + (size_t)GR * L::group_bytes + 1024;  // + alignment slack of the dynamic window
}

template <class P, int NCH, int GR, bool FWD, bool BWD>
gs_status launch_tc_t(const gs_ctx* ctx, RenderTcArgs& a, cudaStream_t st) {
  const size_t smem = render_tc_smem<P, GR>();
  auto k = render_tc_kernel<P, NCH, GR, FWD, BWD>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GS_ERR_CUDA;
  k<<<ctx->render_ctas, GR * kGroupThreads, smem, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

template <class P, int NCH>
gs_status launch_tc_n(const gs_ctx* ctx, RenderTcArgs& a, int mode, cudaStream_t st) {
  // tile groups in one CTA per SM; rays of 5 chunks keep more per-ray state in registers,
  // which only fits with 2 groups (255 registers per thread)
  constexpr int GR = NCH > 4 ? 2 : kRenderGroups;
  if (mode == 1) return launch_tc_t<P, NCH, GR, true, false>(ctx, a, st);
  if (mode == 2) return launch_tc_t<P, NCH, GR, false, true>(ctx, a, st);
  return launch_tc_t<P, NCH, GR, true, true>(ctx, a, st);
}

}  // namespace gs
