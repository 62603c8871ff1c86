// Hierarchical importance sampling (Sec. 3.2: starting from N_c coarse samples, 3 steps each
// add 12 samples drawn from the weights of the samples so far, as in NeuS; Sec. 4: N_c = 96,
// N_f = 36).
//
// The rays are those of the plain sampler for the same (seed, step).  One warp per ray:
//   1. N_c depths stratified over [near, far] (stream 3, slot 1 + k), phi at each;
//   2. per step: the NeuS opacities of the current samples with the model's s = exp(kappa)
//      (alpha_k = max((Phi_k - Phi_k+1) / max(Phi_k, 1e-6), 0), Phi = sigmoid(s phi)), the
//      transmittance by a product scan across the lanes, interval masses w_k + 1e-5 and their
//      running sums by an additive scan, then M stratified inverse-CDF draws u_j = (j + xi_j)/M
//      (stream 3, slot 1 + N_c + step M + j), each placed linearly inside its interval; phi at
//      the new depths; a rank merge into the sorted list (an existing depth first on ties);
//   3. classes by the bound b = D - t, as in the plain sampler.
// phi is the SDF decoder's first output (layer 1, ReLU, row 0 of layer 2; the paper's decoder:
// two hidden layers), its layers on the tensor cores (below).  The sample lists live in shared
// memory, double-buffered per warp.
#include <algorithm>

#include "gs_paper.cuh"
#include "gs_render_tc.cuh"
#include "gs_sample.cuh"

namespace gs {

constexpr int kImpMax = 160;     // samples per ray held (the render kernel takes up to 5 chunks of 32)
constexpr int kImpSeg = kImpMax / 32;  // consecutive intervals per lane in the scans

struct ImpArgs {
  FramesDev fr;
  GridDesc g;
  const float* theta;
  uint64_t seed;
  uint32_t step;
  int R, Nc, steps, M;
  float near_m, far_m, trunc;
  long long* pix;
  float *o, *r, *rgb, *D, *t;
  uint8_t* cls;
  int* counts;
};

// phi on the tcgen05 tensor cores.  A group of 4 warps samples 4 rays
// (warp w: ray 4 q + w); every phi evaluation is a round in which lane i of warp w fills row
// 32 w + i of an M = 128 tile: the coarse depths in rounds of 32 per ray, each step's draws in
// one round (lanes < M).  A round: the trilinear features z on CUDA cores, then H1 = Z W1^T on
// the tensor core (three bfloat16 parts per operand, six part products: FP32-grade); the
// workload's decoder finishes phi = W2[0,:] relu(H1 + b1) + b2[0] on CUDA cores, the paper's
// runs H2 = A1 gW2^T as a second phase and phi = gw3 . relu(H2 + gb2) + gb3.  Opacities,
// scans, draws and the rank merge stay per warp on CUDA cores as above.
constexpr int kItGroups = 4;
constexpr int kItThreads = kItGroups * kGroupThreads;
constexpr uint32_t kItA = 128u * 32u * 2u * 3u;  // a group's A tile: 3 parts of 128 x 32 (z, then a1)
constexpr uint32_t kItW1 = 32u * 16u * 2u, kItW2 = 32u * 32u * 2u;  // one part of W1 {32, 16}, gW2 {32, 32}
constexpr uint32_t oItW = kItGroups * kItA, oItScal = oItW + 3u * (kItW1 + kItW2);
constexpr uint32_t kItMbarLimit = 1u << 20;

template <bool kPaper>
__global__ void __launch_bounds__(kItThreads, 1) importance_tc_kernel(ImpArgs a, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ float ts[kItGroups * 4][2][kImpMax], ps[kItGroups * 4][2][kImpMax];
  __shared__ float cs[kItGroups * 4][kImpMax];
  __shared__ float tn[kItGroups * 4][32];
  __shared__ uint64_t mbar[kItGroups];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag[kItGroups];
  uint8_t* W1t = base + oItW;
  uint8_t* W2t = W1t + 3u * kItW1;
  float* sc = reinterpret_cast<float*>(base + oItScal);  // b1[32] | w2[32] | b2[32] | c0
  const float* mlp = a.theta + a.g.n_grid;
  // geometry decoder: workload (W1 [32][16], b1, W2 row 0, b2[0]) or paper (gW1, gb1, gW2, gb2, gw3, gb3)
  const int oW1_ = kPaper ? paper::A_gW1 : oW1, ob1_ = kPaper ? paper::A_gb1 : ob1;
  for (int i = threadIdx.x; i < kH1 * kZ; i += blockDim.x)
    store_w<PrecBF16x3>(W1t, kItW1, kZ, i / kZ, i % kZ, mlp[oW1_ + i]);
  if (kPaper)
    for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x)
      store_w<PrecBF16x3>(W2t, kItW2, 32, i / 32, i % 32, mlp[paper::A_gW2 + i]);
  for (int i = threadIdx.x; i < 97; i += blockDim.x) {
    float v = 0.f;
    if (i < 32) v = mlp[ob1_ + i];
    else if (i < 64) v = kPaper ? mlp[paper::A_gw3 + i - 32] : mlp[oW2 + i - 32];
    else if (i < 96) v = kPaper ? mlp[paper::A_gb2 + i - 64] : 0.f;
    else v = kPaper ? mlp[paper::A_gb3] : mlp[ob2];
    sc[i] = v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = warp >> 2, warp_g = warp & 3;
  Group G;
  G.a = base + gi * kItA;
  G.b = nullptr;
  G.mbar = &mbar[gi];
  G.mbar_dw = &mbar[gi];
  G.mbar_tma = &mbar[gi];
  G.abort = &abort_flag[gi];
  G.phase = G.phase_dw = G.phase_tma = 0;
  G.dw_pending = false;
  G.g = gi;
  G.gt = threadIdx.x & (kGroupThreads - 1);
  if (G.gt == 0) {
    tc::mbar_init(G.mbar, 1);
    tc::fence_mbar_init();
    *G.abort = 0;
  }
  if (threadIdx.x < 32) tc::tmem_alloc(&tslot, 128);
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  G.tcol = tslot + (uint32_t)(gi * 32);
  const int row = G.gt;
  bool alive = true;
  const float s_sharp = expf(mlp[kPaper ? paper::A_kappa : oKappa]);
  // one phi round of the whole group: this lane's point x (valid) or an idle row
  auto phi_round = [&](bool valid, const float x[3]) -> float {
    float z[kZ];
    if (valid) {
      grid_z(a.g, a.theta, x, z);
    } else {
#pragma unroll
      for (int k = 0; k < kZ; ++k) z[k] = 0.f;
    }
    store_row_planes<3, kZ, 128u * 32u * 2u>(G.a, row, z);
    mma_phase_issue<PrecBF16x3, 32, kZ>(G, 0, W1t, kItW1);
    if (!(alive = alive && mma_phase_wait(G))) return 0.f;
    float v[32];
    tc::tmem_ld32(lane_addr(G, 0, warp_g), v);
    tc::tmem_ld_wait();
    float phi = sc[96];
    if constexpr (!kPaper) {
#pragma unroll
      for (int j = 0; j < 32; ++j) phi = fmaf(sc[32 + j], fmaxf(v[j] + sc[j], 0.f), phi);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + sc[j], 0.f);
      store_row_planes<3, 32, 128u * 32u * 2u>(G.a, row, v);
      mma_phase_issue<PrecBF16x3, 32, 32>(G, 0, W2t, kItW2);
      if (!(alive = alive && mma_phase_wait(G))) return 0.f;
      tc::tmem_ld32(lane_addr(G, 0, warp_g), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 32; ++j) phi = fmaf(sc[32 + j], fmaxf(v[j] + sc[64 + j], 0.f), phi);
    }
    return phi;
  };
  int nd = 0, ntr = 0, nfs = 0;
  const int rounds = (a.Nc + 31) / 32;
  for (int quad = blockIdx.x * kItGroups + gi; quad * 4 < a.R && alive; quad += gridDim.x * kItGroups) {
    const int i = quad * 4 + warp_g;
    const bool has = i < a.R;  // a warp without a ray takes part in the rounds with idle rows
    float o[3] = {0.f, 0.f, 0.f}, r[3] = {0.f, 0.f, 1.f}, D = 0.f;
    if (has) {
      const uint64_t pre = draw_prefix(a.seed, 0, a.step, (uint64_t)i);
      const long long npix = (long long)a.fr.F * a.fr.H * a.fr.W;
      const long long p = (long long)(draw_slot(pre, 0) % (uint64_t)npix);
      float rgb[3];
      pixel_ray(a.fr, p, o, r, rgb, &D);
      if (lane == 0) {
        a.pix[i] = p;
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
    const uint64_t pre3 = draw_prefix(a.seed, 3, a.step, (uint64_t)i);
    // 1. coarse strata and phi there, 32 per round
    const float delta = __fdiv_rn(__fsub_rn(a.far_m, a.near_m), (float)a.Nc);
    for (int c = 0; c < rounds; ++c) {
      const int k = 32 * c + lane;
      const bool v = has && k < a.Nc;
      float tk = 0.f, x[3] = {0.f, 0.f, 0.f};
      if (v) {
        const float u = unif24(draw_slot(pre3, 1 + (uint64_t)k));
        tk = __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)k, u), delta));
        sample_pos(o, r, tk, x);
      }
      const float ph = phi_round(v, x);
      if (!alive) break;
      if (v) {
        ts[warp][0][k] = tk;
        ps[warp][0][k] = ph;
      }
    }
    if (!alive) break;
    __syncwarp();
    int n = a.Nc, cur = 0;
    for (int si = 0; si < a.steps && alive; ++si) {
      const float* Tc = ts[warp][cur];
      const float* Pc = ps[warp][cur];
      float* C = cs[warp];
      float tj = 0.f, x[3] = {0.f, 0.f, 0.f};
      if (has) {
        // 2a. opacities of this lane's intervals [k0, k0 + E) and their transmittance
        const int E = (n + 31) / 32, k0 = lane * E;
        float al[kImpSeg], prod = 1.f;
#pragma unroll
        for (int e = 0; e < kImpSeg; ++e) {
          const int k = k0 + e;
          al[e] = 0.f;
          if (e < E && k + 1 < n) {
            const float P0 = sigmoidf_(s_sharp * Pc[k]), P1 = sigmoidf_(s_sharp * Pc[k + 1]);
            al[e] = fmaxf((P0 - P1) / fmaxf(P0, 1e-6f), 0.f);
          }
          prod *= 1.f - al[e];
        }
        float incl = prod;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float v = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl *= v;
        }
        float T = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) T = 1.f;
        // 2b. interval masses w_k + 1e-5 and the mass left of each interval
        float mass[kImpSeg], msum = 0.f;
#pragma unroll
        for (int e = 0; e < kImpSeg; ++e) {
          const int k = k0 + e;
          mass[e] = (e < E && k + 1 < n) ? T * al[e] + 1e-5f : 0.f;
          T *= 1.f - al[e];
          msum += mass[e];
        }
        float inc = msum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float v = __shfl_up_sync(0xffffffffu, inc, off);
          if (lane >= off) inc += v;
        }
        const float tot = __shfl_sync(0xffffffffu, inc, 31);
        float left = inc - msum;
#pragma unroll
        for (int e = 0; e < kImpSeg; ++e) {
          const int k = k0 + e;
          if (e < E && k + 1 < n) C[k] = left;
          left += mass[e];
        }
        __syncwarp();
        // 2c. stratified inverse-CDF draws, placed linearly inside their interval
        if (lane < a.M) {
          const float xi = unif24(draw_slot(pre3, 1 + (uint64_t)a.Nc + (uint64_t)si * a.M + (uint64_t)lane));
          const float target = __fdiv_rn(__fadd_rn((float)lane, xi), (float)a.M) * tot;
          int lo = 0, hi = n - 2;  // the last interval whose left mass is <= target (C[0] = 0)
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (C[mid] <= target) lo = mid;
            else hi = mid - 1;
          }
          const float pk = (lo + 1 <= n - 2 ? C[lo + 1] : tot) - C[lo];
          const float f = pk > 0.f ? fminf(fmaxf((target - C[lo]) / pk, 0.f), 1.f) : 0.f;
          tj = fminf(fmaxf(Tc[lo] + f * (Tc[lo + 1] - Tc[lo]), Tc[lo]), Tc[lo + 1]);
          sample_pos(o, r, tj, x);
          tn[warp][lane] = tj;
        }
      }
      const float pj = phi_round(has && lane < a.M, x);
      if (!alive) break;
      __syncwarp();
      if (has) {
        // 2d. rank merge into the other buffer: an existing depth goes before equal new ones
        float* Tn = ts[warp][cur ^ 1];
        float* Pn = ps[warp][cur ^ 1];
        for (int k = lane; k < n; k += 32) {
          const float v = Tc[k];
          int c = 0;
          for (int j = 0; j < a.M; ++j) c += tn[warp][j] < v;
          Tn[k + c] = v;
          Pn[k + c] = Pc[k];
        }
        if (lane < a.M) {
          int lo = 0, hi = n;  // number of existing depths <= tj
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Tc[mid] <= tj) lo = mid + 1;
            else hi = mid;
          }
          Tn[lane + lo] = tj;
          Pn[lane + lo] = pj;
        }
      }
      __syncwarp();
      n += a.M;
      cur ^= 1;
    }
    if (!alive) break;
    // 3. output depths and classes
    if (has) {
      const int N = n;
      for (int k = lane; k < N; k += 32) {
        const float tk = ts[warp][cur][k];
        a.t[(size_t)i * N + k] = tk;
        const int c = sample_class(D, tk, a.trunc);
        a.cls[(size_t)i * N + k] = (uint8_t)c;
        ntr += c == CLS_TR;
        nfs += c == CLS_FS;
      }
    }
    __syncwarp();
  }
  if (!alive && G.gt == 0) {
    atomicOr(status, kStatusImportance);
    tc::mbar_wait(G.mbar, G.phase ^ 1u, kItMbarLimit);  // let an MMA in flight finish
  }
  block_add_counts(a.counts, nd, ntr, nfs);
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tslot, 128);
  }
}

inline size_t importance_tc_smem() { return 1024 + oItScal + 97 * sizeof(float); }

}  // namespace gs

using namespace gs;

gs_status gs_launch_importance(const gs_ctx* ctx, const float* theta, const gs_frames* f, uint64_t seed,
                               uint32_t step, const gs_batch* b, cudaStream_t st) {
  if (cudaMemsetAsync(b->counts, 0, 4 * sizeof(int), st) != cudaSuccess) return GS_ERR_CUDA;
  if (b->R > 0) {
    ImpArgs a;
    a.fr = FramesDev{f->F, f->H, f->W, f->rgb, f->depth, f->c2w, f->fx, f->fy, f->cx, f->cy};
    a.g = ctx->grid;
    a.theta = theta;
    a.seed = seed;
    a.step = step;
    a.R = b->R;
    a.Nc = ctx->cfg.imp_coarse;
    a.steps = ctx->cfg.imp_steps;
    a.M = ctx->cfg.imp_per_step;
    a.near_m = ctx->cfg.near_m;
    a.far_m = ctx->cfg.far_m;
    a.trunc = ctx->cfg.trunc;
    a.pix = (long long*)b->pix;
    a.o = b->origin;
    a.r = b->dir;
    a.rgb = b->rgb;
    a.D = b->depth;
    a.t = b->t;
    a.cls = b->cls;
    a.counts = b->counts;
    // phi on the tensor cores: one CTA of 4 groups (16 rays in flight) per SM
    const int blocks = (int)std::min<long long>(((long long)b->R + 4 * kItGroups - 1) / (4 * kItGroups), ctx->num_sms);
    const size_t smem = importance_tc_smem();
    if (ctx->cfg.arch == GS_ARCH_PAPER) {
      if (cudaFuncSetAttribute(importance_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return GS_ERR_CUDA;
      importance_tc_kernel<true><<<blocks, kItThreads, smem, st>>>(a, ctx->status);
    } else {
      if (cudaFuncSetAttribute(importance_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return GS_ERR_CUDA;
      importance_tc_kernel<false><<<blocks, kItThreads, smem, st>>>(a, ctx->status);
    }
    if (cudaPeekAtLastError() != cudaSuccess) return GS_ERR_CUDA;
  }
  return gs_launch_sample_smooth(ctx, f, seed, step, b, st);
}
