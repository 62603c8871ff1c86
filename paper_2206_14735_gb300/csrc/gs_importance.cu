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
// phi is the SDF decoder's first output evaluated on CUDA cores in FP32 (layer 1, ReLU, row 0
// of layer 2).  The sample lists live in shared memory, double-buffered per warp.
#include <algorithm>

#include "gs_paper.cuh"
#include "gs_sample.cuh"

namespace gs {

constexpr int kImpWarps = 4;     // rays per CTA
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

// kPaper: phi from the paper's two-hidden-layer geometry decoder (GS_ARCH_PAPER) instead of
// the workload's decoder
template <bool kPaper>
__global__ void __launch_bounds__(kImpWarps * 32, 3) importance_kernel(ImpArgs a) {
  // workload decoder: W1 | b1 | W2 row 0 | b2[0]; paper: the geometry decoder block
  __shared__ __align__(16) float sm[kPaper ? paper::kGeoPad : sb2 + 4];
  // paper decoder: each thread's hidden layer in shared memory (stride 33), not in registers
  __shared__ float hsc[kPaper ? kImpWarps * 32 : 1][kPaper ? 33 : 1];
  __shared__ float ts[kImpWarps][2][kImpMax], ps[kImpWarps][2][kImpMax];
  __shared__ float cs[kImpWarps][kImpMax];   // mass left of each interval (unnormalised)
  __shared__ float tn[kImpWarps][32];        // this step's new depths
  const float* mlp = a.theta + a.g.n_grid;
  if (kPaper) {
    paper::load_geometry_decoder(mlp, sm);
  } else {
    for (int i = threadIdx.x; i <= sb2; i += blockDim.x) {
      float v = 0.f;
      if (i < sb1) v = mlp[oW1 + i];
      else if (i < sW2) v = mlp[ob1 + i - sb1];
      else if (i < sW2 + kH1) v = mlp[oW2 + i - sW2];
      else if (i == sb2) v = mlp[ob2];
      sm[i] = v;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float s_sharp = expf(mlp[kPaper ? paper::A_kappa : oKappa]);
  int nd = 0, ntr = 0, nfs = 0;
  for (int i = blockIdx.x * kImpWarps + warp; i < a.R; i += gridDim.x * kImpWarps) {  // warp-uniform
    const uint64_t pre = draw_prefix(a.seed, 0, a.step, (uint64_t)i);
    const long long npix = (long long)a.fr.F * a.fr.H * a.fr.W;
    const long long p = (long long)(draw_slot(pre, 0) % (uint64_t)npix);
    float o[3], r[3], rgb[3], D;
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
    const uint64_t pre3 = draw_prefix(a.seed, 3, a.step, (uint64_t)i);
    // 1. coarse strata and phi there
    const float delta = __fdiv_rn(__fsub_rn(a.far_m, a.near_m), (float)a.Nc);
    for (int k = lane; k < a.Nc; k += 32) {
      const float u = unif24(draw_slot(pre3, 1 + (uint64_t)k));
      const float tk = __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)k, u), delta));
      float x[3];
      sample_pos(o, r, tk, x);
      ts[warp][0][k] = tk;
      ps[warp][0][k] = kPaper ? paper::phi_at(a.g, a.theta, sm, x, hsc[threadIdx.x]) : sdf_at(a.g, a.theta, sm, x);
    }
    __syncwarp();
    int n = a.Nc, cur = 0;
    for (int si = 0; si < a.steps; ++si) {
      const float* Tc = ts[warp][cur];
      const float* Pc = ps[warp][cur];
      float* C = cs[warp];
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
      float tj = 0.f, pj = 0.f;
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
        float x[3];
        sample_pos(o, r, tj, x);
        pj = kPaper ? paper::phi_at(a.g, a.theta, sm, x, hsc[threadIdx.x]) : sdf_at(a.g, a.theta, sm, x);
        tn[warp][lane] = tj;
      }
      __syncwarp();
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
      __syncwarp();
      n += a.M;
      cur ^= 1;
    }
    // 3. output depths and classes
    const int N = n;
    for (int k = lane; k < N; k += 32) {
      const float tk = ts[warp][cur][k];
      a.t[(size_t)i * N + k] = tk;
      const int c = sample_class(D, tk, a.trunc);
      a.cls[(size_t)i * N + k] = (uint8_t)c;
      ntr += c == CLS_TR;
      nfs += c == CLS_FS;
    }
    __syncwarp();
  }
  block_add_counts(a.counts, nd, ntr, nfs);
}

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
    const int blocks = (int)std::min<long long>(((long long)b->R + kImpWarps - 1) / kImpWarps, 16LL * ctx->num_sms);
    if (ctx->cfg.arch == GS_ARCH_PAPER) importance_kernel<true><<<blocks, kImpWarps * 32, 0, st>>>(a);
    else importance_kernel<false><<<blocks, kImpWarps * 32, 0, st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return GS_ERR_CUDA;
  }
  return gs_launch_sample_smooth(ctx, f, seed, step, b, st);
}
