// Ray batch sampling, sample placement and bound classes (Sec. 3.2-3.4), and the
// near-surface smoothness points S_g (Sec. 3.3).  Every value here is computed with
// explicitly rounded binary32 operations so that it is reproducible bit for bit.
#include "gs_sample.cuh"

namespace gs {

struct SampleArgs {
  FramesDev fr;
  uint64_t seed;
  uint32_t step;
  int R, Ns, Ng;
  float near_m, far_m, guide_half, trunc;
  long long* pix;
  float *o, *r, *rgb, *D, *t;
  uint8_t* cls;
  int* counts;
};

__global__ void __launch_bounds__(128) sample_rays_kernel(SampleArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int nd = 0, ntr = 0, nfs = 0;
  if (i < a.R) {
    const uint64_t pre = draw_prefix(a.seed, 0, a.step, (uint64_t)i);
    const long long npix = (long long)a.fr.F * a.fr.H * a.fr.W;
    const long long p = (long long)(draw_slot(pre, 0) % (uint64_t)npix);
    float o[3], r[3], rgb[3], D;
    pixel_ray(a.fr, p, o, r, rgb, &D);
    a.pix[i] = p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a.o[3 * i + k] = o[k];
      a.r[3 * i + k] = r[k];
      a.rgb[3 * i + k] = rgb[k];
    }
    a.D[i] = D;
    const int N = a.Ns + a.Ng;
    float* ti = a.t + (size_t)i * N;
    uint8_t* ci = a.cls + (size_t)i * N;
    if (D > 0.0f) {
      ++nd;
      // N_s strata of [near, far] and N_g strata of [D - g, D + g], merged by depth
      const float delta = __fdiv_rn(__fsub_rn(a.far_m, a.near_m), (float)a.Ns);
      const float gstep = __fdiv_rn(__fmul_rn(2.0f, a.guide_half), (float)a.Ng);
      const float g0 = __fsub_rn(D, a.guide_half);
      auto strat = [&](int k) {
        const float u = unif24(draw_slot(pre, 1 + (uint64_t)k));
        return __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)k, u), delta));
      };
      auto guided = [&](int k) {
        const float u = unif24(draw_slot(pre, 1 + (uint64_t)a.Ns + (uint64_t)k));
        return __fadd_rn(g0, __fmul_rn(__fadd_rn((float)k, u), gstep));
      };
      int ia = 0, ib = 0;
      float ta = a.Ns > 0 ? strat(0) : 0.0f, tb = a.Ng > 0 ? guided(0) : 0.0f;
      for (int k = 0; k < N; ++k) {
        float tk;
        if (ib >= a.Ng || (ia < a.Ns && ta <= tb)) {  // ties: stratified first
          tk = ta;
          ++ia;
          if (ia < a.Ns) ta = strat(ia);
        } else {
          tk = tb;
          ++ib;
          if (ib < a.Ng) tb = guided(ib);
        }
        ti[k] = tk;
        const int c = sample_class(D, tk, a.trunc);
        ci[k] = (uint8_t)c;
        ntr += c == CLS_TR;
        nfs += c == CLS_FS;
      }
    } else {
      const float delta = __fdiv_rn(__fsub_rn(a.far_m, a.near_m), (float)N);
      for (int k = 0; k < N; ++k) {
        const float u = unif24(draw_slot(pre, 1 + (uint64_t)k));
        ti[k] = __fadd_rn(a.near_m, __fmul_rn(__fadd_rn((float)k, u), delta));
        ci[k] = (uint8_t)CLS_NONE;
      }
    }
  }
  block_add_counts(a.counts, nd, ntr, nfs);
}

struct SmoothArgs {
  FramesDev fr;
  uint64_t seed;
  uint32_t step;
  int P;
  float trunc, delta_s;
  float *xs, *eps;
  uint8_t* valid;
  int* counts;
};

// S_g: back-projected observed depth of a random valid pixel (up to 8 draws) jittered by
// +-t per axis; eps of length delta_s in a direction drawn by rejection from [-1,1]^3.
__global__ void __launch_bounds__(128) sample_smooth_kernel(SmoothArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  int nv = 0;
  if (p < a.P) {
    const uint64_t pre = draw_prefix(a.seed, 1, a.step, (uint64_t)p);
    const long long npix = (long long)a.fr.F * a.fr.H * a.fr.W;
    long long px = -1;
    for (int tr = 0; tr < 8; ++tr) {
      const long long q = (long long)(draw_slot(pre, (uint64_t)tr) % (uint64_t)npix);
      if (a.fr.depth[q] > 0.0f) {
        px = q;
        break;
      }
    }
    if (px < 0) {
      a.valid[p] = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) a.xs[3 * p + k] = a.eps[3 * p + k] = 0.0f;
    } else {
      nv = 1;
      a.valid[p] = 1;
      float o[3], r[3], rgb[3], D;
      pixel_ray(a.fr, px, o, r, rgb, &D);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float u = unif24(draw_slot(pre, 16 + (uint64_t)k));
        const float base = __fadd_rn(o[k], __fmul_rn(D, r[k]));
        const float jit = __fmul_rn(a.trunc, __fsub_rn(__fmul_rn(2.0f, u), 1.0f));
        a.xs[3 * p + k] = __fadd_rn(base, jit);
      }
      float v[3] = {1.0f, 0.0f, 0.0f}, n2 = 1.0f;
      for (int tr = 0; tr < 16; ++tr) {
        float w[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
          w[k] = __fsub_rn(__fmul_rn(2.0f, unif24(draw_slot(pre, 32 + 3 * (uint64_t)tr + k))), 1.0f);
        const float q = __fadd_rn(__fadd_rn(__fmul_rn(w[0], w[0]), __fmul_rn(w[1], w[1])), __fmul_rn(w[2], w[2]));
        if (q >= 0.01f && q <= 1.0f) {
          v[0] = w[0];
          v[1] = w[1];
          v[2] = w[2];
          n2 = q;
          break;
        }
      }
      const float sc = __fdiv_rn(a.delta_s, __fsqrt_rn(n2));
#pragma unroll
      for (int k = 0; k < 3; ++k) a.eps[3 * p + k] = __fmul_rn(v[k], sc);
    }
  }
  nv = __reduce_add_sync(0xffffffffu, nv);
  if ((threadIdx.x & 31) == 0 && nv) atomicAdd(a.counts + 3, nv);
}

}  // namespace gs

using namespace gs;

gs_status gs_launch_sample_smooth(const gs_ctx* ctx, const gs_frames* f, uint64_t seed, uint32_t step,
                                  const gs_batch* b, cudaStream_t st) {
  FramesDev fr{f->F, f->H, f->W, f->rgb, f->depth, f->c2w, f->fx, f->fy, f->cx, f->cy};
  if (b->P > 0) {
    SmoothArgs s{fr, seed, step, b->P, ctx->cfg.trunc, ctx->cfg.delta_s, b->xs, b->eps, b->valid, b->counts};
    sample_smooth_kernel<<<(b->P + 127) / 128, 128, 0, st>>>(s);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_sample(const gs_ctx* ctx, const gs_frames* f, uint64_t seed, uint32_t step, const gs_batch* b,
                           cudaStream_t st) {
  FramesDev fr{f->F, f->H, f->W, f->rgb, f->depth, f->c2w, f->fx, f->fy, f->cx, f->cy};
  if (cudaMemsetAsync(b->counts, 0, 4 * sizeof(int), st) != cudaSuccess) return GS_ERR_CUDA;
  if (b->R > 0) {
    SampleArgs a{fr,     seed,   step,   b->R,   ctx->cfg.n_strat, ctx->cfg.n_guided, ctx->cfg.near_m,
                 ctx->cfg.far_m, ctx->cfg.guide_half, ctx->cfg.trunc, (long long*)b->pix, b->origin, b->dir,
                 b->rgb, b->depth, b->t, b->cls, b->counts};
    sample_rays_kernel<<<(b->R + 127) / 128, 128, 0, st>>>(a);
  }
  return gs_launch_sample_smooth(ctx, f, seed, step, b, st);
}
