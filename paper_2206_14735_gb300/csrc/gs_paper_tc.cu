// Launch of the paper architecture's tensor-core render kernel (gs_paper_tc.cuh); the kernel
// is instantiated per chunk count of the ray in gs_paper_tc_n{1..5}.cu.
#include "gs_paper_tc.cuh"

namespace gs {
namespace ptc {
extern template gs_status launch_paper_tc<1>(const PaperTcArgs&, int, int, cudaStream_t);
extern template gs_status launch_paper_tc<2>(const PaperTcArgs&, int, int, cudaStream_t);
extern template gs_status launch_paper_tc<3>(const PaperTcArgs&, int, int, cudaStream_t);
extern template gs_status launch_paper_tc<4>(const PaperTcArgs&, int, int, cudaStream_t);
extern template gs_status launch_paper_tc<5>(const PaperTcArgs&, int, int, cudaStream_t);
}  // namespace ptc
}  // namespace gs

using namespace gs;

gs_status gs_launch_paper_tc(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* grad,
                             float* rgb_hat, float* d_hat, float* wsum, int mode, float* loss_part, float* mlp_part,
                             int ctas, cudaStream_t st) {
  ptc::PaperTcArgs a;
  a.g = ctx->grid;
  a.colour_off = ctx->colour_off;
  a.theta = theta;
  a.grad = grad;
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
  a.rgb_hat = rgb_hat;
  a.d_hat = d_hat;
  a.wsum = wsum;
  a.w_out = b->w;
  a.dz_out = b->dz;
  a.loss_part = loss_part;
  a.mlp_part = mlp_part;
  a.R = b->R;
  a.N = b->N;
  a.status = ctx->status;
  a.eik = reinterpret_cast<const float4*>(b->eik);
  a.eik_stride = (long long)b->R * b->N;
  a.store = ctx->store;
  a.store_stride = (long long)ctx->cfg.max_rays * ctx->max_n;
  if (!gs_encode_level_map(ctx, theta, GS_LEVELS - 1, &a.tmap)) return GS_ERR_CUDA;
  switch ((b->N + 31) / 32) {
    case 1: return ptc::launch_paper_tc<1>(a, mode, ctas, st);
    case 2: return ptc::launch_paper_tc<2>(a, mode, ctas, st);
    case 3: return ptc::launch_paper_tc<3>(a, mode, ctas, st);
    case 4: return ptc::launch_paper_tc<4>(a, mode, ctas, st);
    case 5: return ptc::launch_paper_tc<5>(a, mode, ctas, st);
    default: return GS_ERR_UNSUPPORTED;
  }
}
