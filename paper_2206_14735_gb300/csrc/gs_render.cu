// Loss / decoder-gradient combination, SDF query and cell lookup, and the dispatch of the
// fused render kernel over samples-per-ray (its instantiations live in gs_render_tc_n*.cu).
#include "gs_render_tc.cuh"

namespace gs {

extern template gs_status launch_tc_n<PrecBF16x3, 1>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16x3, 2>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16x3, 3>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16x3, 4>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16x3, 5>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16, 1>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16, 2>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16, 3>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16, 4>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
extern template gs_status launch_tc_n<PrecBF16, 5>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);

// ------------------------------------------------------------------------------------
// combine per-CTA partials: losses in FP64, decoder gradients in a fixed order
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) finalize_kernel(const float* loss_part, const float* mlp_part, int nparts,
                                                       const int* counts, int R, float l0, float l1, float l2,
                                                       float l3, float l4, float* loss, float* gmlp) {
  // decoder gradients: block b owns entries [32b, 32b + 32); warp w sums rows w, w + 8, ...,
  // then warp 0 adds the 8 warps' sums in a fixed order
  __shared__ float part[8][33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  if (gmlp) {
    part[wid][lane] = i < GS_MLP_PARAMS ? column_sum8(mlp_part, kMlpPad, i, wid, nparts) : 0.f;
    __syncthreads();
    if (wid == 0 && i < GS_MLP_PARAMS) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) t += part[k][lane];
      gmlp[i] += t;
    }
  }
  // losses (FP64): lane l of warp 0 sums rows l, l + 32, ... of every term, then a warp sum
  if (loss && blockIdx.x == 0 && threadIdx.x < 32) {
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int p = lane; p < nparts; p += 32)
#pragma unroll
      for (int k = 0; k < 5; ++k) s[k] += (double)loss_part[(size_t)p * kLossPad + k];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if (lane == 0) {
      const double den[5] = {(double)R, (double)counts[0], (double)counts[1], (double)counts[2], (double)counts[3]};
      const double lam[5] = {l0, l1, l2, l3, l4};
      double tot = 0.0;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const double v = den[k] > 0 ? s[k] / den[k] : 0.0;
        loss[k] = (float)v;
        tot += lam[k] * v;
      }
      loss[5] = (float)tot;
    }
  }
}

// ------------------------------------------------------------------------------------
// SDF query and cell lookup
// ------------------------------------------------------------------------------------
__global__ void query_kernel(GridDesc g, const float* __restrict__ theta, const float* __restrict__ xq, int P,
                             float* sdf, float* grad) {
  __shared__ __align__(16) float sm[kSmemMlp];
  const float* mlp = theta + g.n_grid;
  for (int i = threadIdx.x; i < kSmemMlp; i += blockDim.x) {
    float v = 0.0f;
    if (i < sb1) v = mlp[oW1 + i];
    else if (i < sW2) v = mlp[ob1 + i - sb1];
    else if (i < sb2) v = mlp[oW2 + i - sW2];
    else if (i < sW3) v = mlp[ob2 + i - sb2];
    else if (i < sb3) {
      const int j = (i - sW3) >> 4, k = (i - sW3) & 15;
      v = k < kHF ? mlp[oW3 + j * kHF + k] : 0.0f;
    }
    sm[i] = v;
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float x[3] = {xq[3 * p], xq[3 * p + 1], xq[3 * p + 2]};
  float z[kZ], dzdx[kZ][3];
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    const Cell c = locate(g, l, x);
    float w[8], dw[8][3];
    corner_weights(c.f, w);
    corner_weight_grads(c.f, c.clamped, dw);
    const float4* base = reinterpret_cast<const float4*>(theta + g.off[l]);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), ax = acc, ay = acc, az = acc;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float4 v = __ldg(base + c.vtx + corner_offset(g, l, k));
      f4fma(acc, w[k], v);
      f4fma(ax, dw[k][0], v);
      f4fma(ay, dw[k][1], v);
      f4fma(az, dw[k][2], v);
    }
    const float iv = g.inv_voxel[l];
    const float zz[4] = {acc.x, acc.y, acc.z, acc.w}, gx[4] = {ax.x, ax.y, ax.z, ax.w},
                gy[4] = {ay.x, ay.y, ay.z, ay.w}, gz[4] = {az.x, az.y, az.z, az.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      z[4 * l + k] = zz[k];
      dzdx[4 * l + k][0] = gx[k] * iv;
      dzdx[4 * l + k][1] = gy[k] * iv;
      dzdx[4 * l + k][2] = gz[k] * iv;
    }
  }
  float y1[kH1];
  float phi = sm[sb2];
#pragma unroll
  for (int j = 0; j < kH1; ++j) {
    float s = sm[sb1 + j];
#pragma unroll
    for (int k = 0; k < kZ; ++k) s = fmaf(sm[sW1 + j * 16 + k], z[k], s);
    y1[j] = s;
    phi = fmaf(sm[sW2 + j], fmaxf(s, 0.f), phi);
  }
  sdf[p] = phi;
  if (grad) {
    float gxyz[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kZ; ++k) {
      float pk = 0.f;  // d phi / d z_k = sum_j W1[j][k] [y1_j > 0] W2[0][j]
#pragma unroll
      for (int j = 0; j < kH1; ++j) pk = fmaf(sm[sW1 + j * 16 + k], y1[j] > 0.f ? sm[sW2 + j] : 0.f, pk);
#pragma unroll
      for (int q = 0; q < 3; ++q) gxyz[q] = fmaf(pk, dzdx[k][q], gxyz[q]);
    }
    grad[3 * p] = gxyz[0];
    grad[3 * p + 1] = gxyz[1];
    grad[3 * p + 2] = gxyz[2];
  }
}

__global__ void voxel_index_kernel(GridDesc g, const float* __restrict__ xq, int P, long long* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float x[3] = {xq[3 * p], xq[3 * p + 1], xq[3 * p + 2]};
#pragma unroll
  for (int l = 0; l < kLevels; ++l) out[(size_t)kLevels * p + l] = locate(g, l, x).vtx;
}

}  // namespace gs

using namespace gs;

// cuTensorMapEncodeTiled from the driver (the library links only the runtime)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// 2D view [nz * ny][nx * 4] of grid level l with a box of 2 vertices x 4 features, one row high
bool gs::gs_encode_level_map(const gs_ctx* ctx, const float* theta, int l, CUtensorMap* m) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const GridDesc& g = ctx->grid;
  const cuuint64_t dims[2] = {(cuuint64_t)g.dims[l][0] * 4, (cuuint64_t)g.dims[l][1] * g.dims[l][2]};
  const cuuint64_t strides[1] = {(cuuint64_t)g.dims[l][0] * 16};
  const cuuint32_t box[2] = {8, 1};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(theta + g.off[l]), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static_assert(kStatusRender == 2, "render_tc_kernel reports a bounded wait that ran out as bit 1 (value 2)");

gs_status gs_launch_render(const gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* b,
                           const float* dloss, float* grad, float* rgb_hat, float* d_hat, float* wsum, int mode,
                           cudaStream_t st) {
  RenderTcArgs a;
  a.g = ctx->grid;
  a.theta = theta;
  a.theta_bf16 = theta_bf16;
  a.R = b->R;
  a.N = b->N;
  a.o = b->origin;
  a.r = b->dir;
  a.rgb = b->rgb;
  a.D = b->depth;
  a.t = b->t;
  a.cls = b->cls;
  a.counts = b->counts;
  a.dloss = dloss;
  for (int k = 0; k < 5; ++k) a.lam[k] = ctx->cfg.lam[k];
  a.kappa_fs = ctx->cfg.kappa_fs;
  a.grad = grad;
  a.loss_part = ctx->loss_part;
  a.mlp_part = ctx->mlp_part;
  a.rgb_hat = rgb_hat;
  a.d_hat = d_hat;
  a.wsum = wsum;
  a.status = ctx->status;
  if (ctx->cfg.precision != GS_PREC_BF16)
    for (int q = 0; q < 2; ++q)
      if (!gs_encode_level_map(ctx, theta, 2 + q, &a.tmap[q])) return GS_ERR_CUDA;
  a.store = ctx->store;
  a.w_out = b->w;
  a.dz_out = b->dz;
  a.eik = reinterpret_cast<const float4*>(b->eik);
  a.eik_stride = (long long)b->R * b->N;
  a.store_stride = (long long)ctx->cfg.max_rays * ctx->max_n;
  const int nch = (b->N + 31) / 32;
  if (ctx->cfg.precision == GS_PREC_BF16) {
    switch (nch) {
      case 1: return launch_tc_n<PrecBF16, 1>(ctx, a, mode, st);
      case 2: return launch_tc_n<PrecBF16, 2>(ctx, a, mode, st);
      case 3: return launch_tc_n<PrecBF16, 3>(ctx, a, mode, st);
      case 4: return launch_tc_n<PrecBF16, 4>(ctx, a, mode, st);
      case 5: return launch_tc_n<PrecBF16, 5>(ctx, a, mode, st);
      default: return GS_ERR_UNSUPPORTED;
    }
  }
  switch (nch) {
    case 1: return launch_tc_n<PrecBF16x3, 1>(ctx, a, mode, st);
    case 2: return launch_tc_n<PrecBF16x3, 2>(ctx, a, mode, st);
    case 3: return launch_tc_n<PrecBF16x3, 3>(ctx, a, mode, st);
    case 4: return launch_tc_n<PrecBF16x3, 4>(ctx, a, mode, st);
    case 5: return launch_tc_n<PrecBF16x3, 5>(ctx, a, mode, st);
    default: return GS_ERR_UNSUPPORTED;
  }
}

gs_status gs_launch_finalize(const gs_ctx* ctx, const gs_batch* b, float* loss, float* grad, int mode,
                             cudaStream_t st) {
  const float* l = ctx->cfg.lam;
  float* gmlp = (mode & 2) ? grad + ctx->grid.n_grid : nullptr;
  float* lo = (mode & 1) ? loss : nullptr;
  finalize_kernel<<<(GS_MLP_PARAMS + 31) / 32, 256, 0, st>>>(ctx->loss_part, ctx->mlp_part, ctx->n_parts,
                                                                b->counts, b->R, l[0], l[1], l[2], l[3], l[4], lo,
                                                                gmlp);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_query(const gs_ctx* ctx, const float* theta, const float* x, int P, float* sdf, float* grad,
                          cudaStream_t st) {
  if (P > 0) query_kernel<<<(P + 127) / 128, 128, 0, st>>>(ctx->grid, theta, x, P, sdf, grad);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_launch_voxel_index(const gs_ctx* ctx, const float* x, int P, long long* out, cudaStream_t st) {
  if (P > 0) voxel_index_kernel<<<(P + 127) / 128, 128, 0, st>>>(ctx->grid, x, P, out);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
