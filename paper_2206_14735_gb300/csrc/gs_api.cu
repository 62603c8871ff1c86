// C ABI entry points (include/gosurf.h): argument validation, context and workspace.
#include <cstdio>
#include <cstring>
#include <new>

#include "gs_internal.h"

namespace {

thread_local std::string g_err;  // errors raised before a context exists

gs_status fail(gs_ctx* ctx, gs_status s, const char* msg) {
  if (ctx) ctx->last_error = msg;
  else g_err = msg;
  return s;
}

gs_status cuda_fail(gs_ctx* ctx, const char* where) {
  const cudaError_t e = cudaGetLastError();
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return fail(ctx, GS_ERR_CUDA, buf);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

long long level_floats(const gs_config* c, int l) {
  return (long long)c->dims[l][0] * c->dims[l][1] * c->dims[l][2] * GS_FEAT;
}

int imp_samples(const gs_config* c) { return c->imp_coarse + c->imp_steps * c->imp_per_step; }

// colour grid floats of the paper architecture: 6 per finest-level vertex, padded to a multiple of 4
long long colour_floats(const gs_config* c) {
  const long long n = (long long)c->dims[3][0] * c->dims[3][1] * c->dims[3][2] * GS_COLOUR_FEAT;
  return (n + 3) / 4 * 4;
}


gs_status check_batch(gs_ctx* ctx, const gs_batch* b, bool need_smooth_arrays) {
  if (!b) return fail(ctx, GS_ERR_INVALID_ARG, "batch is NULL");
  if (b->R < 0 || b->R > ctx->cfg.max_rays) return fail(ctx, GS_ERR_SHAPE, "batch R outside [0, max_rays]");
  if (b->N != ctx->cfg.n_strat + ctx->cfg.n_guided && !(ctx->cfg.prop_samples > 0 && b->N == ctx->cfg.prop_samples) &&
      !(ctx->cfg.imp_coarse > 0 && b->N == imp_samples(&ctx->cfg)))
    return fail(ctx, GS_ERR_SHAPE, "batch N is neither n_strat + n_guided, prop_samples nor the importance sampler's");
  if (b->P < 0 || b->P > ctx->cfg.max_smooth) return fail(ctx, GS_ERR_SHAPE, "batch P outside [0, max_smooth]");
  if (!b->counts) return fail(ctx, GS_ERR_INVALID_ARG, "batch counts is NULL");
  if (b->R > 0 && (!b->origin || !b->dir || !b->rgb || !b->depth || !b->t || !b->cls))
    return fail(ctx, GS_ERR_INVALID_ARG, "batch ray array is NULL");
  if (b->R > 0 && need_smooth_arrays && !b->pix) return fail(ctx, GS_ERR_INVALID_ARG, "batch pix is NULL");
  if (b->P > 0 && (!b->xs || !b->eps || !b->valid)) return fail(ctx, GS_ERR_INVALID_ARG, "batch smoothness array is NULL");
  if (b->eik && (reinterpret_cast<uintptr_t>(b->eik) & 15u)) return fail(ctx, GS_ERR_ALIGN, "batch eik is not 16-byte aligned");
  return GS_OK;
}

gs_status check_frames(gs_ctx* ctx, const gs_frames* frames, const char* who) {
  std::string w(who);
  if (!frames || !frames->rgb || !frames->depth || !frames->c2w)
    return fail(ctx, GS_ERR_INVALID_ARG, (w + ": frames or a frame array is NULL").c_str());
  if (frames->F < 1 || frames->H < 1 || frames->W < 1) return fail(ctx, GS_ERR_SHAPE, (w + ": empty frames").c_str());
  if (!(frames->fx != 0.0f) || !(frames->fy != 0.0f))
    return fail(ctx, GS_ERR_INVALID_ARG, (w + ": zero focal length").c_str());
  return GS_OK;
}

}  // namespace

// Records a message for gs_last_error(NULL) (used by entry points that have no context).
void gs_set_thread_error(const char* msg) { g_err = msg; }

// Checks a configuration without touching the device.  Returns GS_OK, or the status and a
// message (without the caller's name) for the first violated rule.  gs_create and
// gs_forward_backward_noalloc share it, so both accept exactly the same configurations.
gs_status gs_check_config(const gs_config* cfg, const char** msg) {
  auto bad = [&](gs_status s, const char* m) { *msg = m; return s; };
  for (int l = 0; l < GS_LEVELS; ++l) {
    for (int a = 0; a < 3; ++a)
      if (cfg->dims[l][a] < 2) return bad(GS_ERR_INVALID_ARG, "every level needs >= 2 vertices per axis");
    if (!(cfg->voxel[l] > 0.0f)) return bad(GS_ERR_INVALID_ARG, "voxel size must be > 0");
  }
  for (int l = 0; l < 2; ++l)  // the coarse-level scatters key their runs by a 32-bit vertex index
    if (level_floats(cfg, l) / GS_FEAT >= (1LL << 31))
      return bad(GS_ERR_UNSUPPORTED, "levels 0 and 1 must have fewer than 2^31 vertices");
  const int N = cfg->n_strat + cfg->n_guided;
  if (cfg->n_strat < 1 || cfg->n_guided < 0 || N < 2) return bad(GS_ERR_INVALID_ARG, "need n_strat >= 1 and N >= 2");
  if (N > GS_MAX_SAMPLES) return bad(GS_ERR_UNSUPPORTED, "this build renders at most 160 samples per ray");
  if (cfg->imp_coarse != 0 &&
      (cfg->imp_coarse < 2 || cfg->imp_steps < 0 || cfg->imp_per_step < 1 || cfg->imp_per_step > 32 ||
       imp_samples(cfg) > GS_MAX_SAMPLES))
    return bad(GS_ERR_INVALID_ARG,
               "the importance sampler needs imp_coarse >= 2, 1 <= imp_per_step <= 32 and at most 160 samples");
  if (!(cfg->far_m > cfg->near_m) || !(cfg->trunc > 0.0f) || !(cfg->guide_half >= 0.0f))
    return bad(GS_ERR_INVALID_ARG, "bad near/far/trunc/guide_half");
  if (cfg->max_rays < 0 || cfg->max_smooth < 0) return bad(GS_ERR_INVALID_ARG, "negative batch bound");
  if (cfg->prop_samples != 0 &&
      (cfg->prop_samples < 2 || cfg->prop_samples > GS_PROP_BINS || cfg->prop_guided < 0 ||
       cfg->prop_guided >= cfg->prop_samples))
    return bad(GS_ERR_INVALID_ARG, "need 2 <= prop_samples <= 32 and 0 <= prop_guided < prop_samples");
  if (cfg->arch != GS_ARCH_COMPACT && cfg->arch != GS_ARCH_PAPER)
    return bad(GS_ERR_INVALID_ARG, "arch must be GS_ARCH_COMPACT or GS_ARCH_PAPER");
  if (cfg->arch == GS_ARCH_PAPER && cfg->precision != GS_PREC_FP32)
    return bad(GS_ERR_UNSUPPORTED, "GS_ARCH_PAPER runs in FP32");
  return GS_OK;
}

extern "C" {

int64_t gs_param_count(const gs_config* cfg, int64_t* n_grid) {
  if (!cfg) return -1;
  long long g = 0;
  for (int l = 0; l < GS_LEVELS; ++l) g += level_floats(cfg, l);
  if (cfg->arch == GS_ARCH_PAPER) g += colour_floats(cfg);
  if (n_grid) *n_grid = g;
  return g + (cfg->arch == GS_ARCH_PAPER ? GS_PAPER_MLP_PARAMS : GS_MLP_PARAMS);
}

gs_status gs_create(const gs_config* cfg, gs_ctx** out) {
  if (!cfg || !out) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_create: NULL argument");
  *out = nullptr;
  const char* why = nullptr;
  const gs_status cs = gs_check_config(cfg, &why);
  if (cs != GS_OK) return fail(nullptr, cs, (std::string("gs_create: ") + why).c_str());
  const int N = cfg->n_strat + cfg->n_guided;

  gs_ctx* c = new (std::nothrow) gs_ctx();
  if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_create: out of host memory");
  c->cfg = *cfg;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return cuda_fail(nullptr, "gs_create: no CUDA device");
  }
  gs::GridDesc& g = c->grid;
  long long off = 0;
  for (int l = 0; l < GS_LEVELS; ++l) {
    for (int a = 0; a < 3; ++a) g.dims[l][a] = cfg->dims[l][a];
    g.voxel[l] = cfg->voxel[l];
    g.inv_voxel[l] = 1.0f / cfg->voxel[l];
    g.off[l] = off;
    off += level_floats(cfg, l);
  }
  for (int a = 0; a < 3; ++a) g.origin[a] = cfg->origin[a];
  c->colour_off = off;
  if (cfg->arch == GS_ARCH_PAPER) off += colour_floats(cfg);
  g.n_grid = off;
  c->render_ctas = kRenderCtasPerSm * c->num_sms;
  c->n_parts = c->render_ctas + kSmoothCtas;
  c->eik_ctas = kEikCtasPerSm * c->num_sms;
  c->max_n = N;
  if (cfg->prop_samples > c->max_n) c->max_n = cfg->prop_samples;
  if (cfg->imp_coarse > 0 && imp_samples(cfg) > c->max_n) c->max_n = imp_samples(cfg);
  const float dl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
  if (cudaMalloc(&c->loss_part, sizeof(float) * kLossPad * c->n_parts) != cudaSuccess ||
      cudaMalloc(&c->mlp_part, sizeof(float) * kMlpPad * c->n_parts) != cudaSuccess ||
      cudaMalloc(&c->default_dloss, sizeof(float) * 8) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->eik_part, sizeof(float) * kEikCtasPerSm * c->num_sms) != cudaSuccess ||
      cudaMalloc(&c->eik_ticket, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->eik_ticket, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->eik_count, sizeof(int) * (4 + (size_t)cfg->max_rays * c->max_n)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaMemcpy(c->default_dloss, dl, sizeof(dl), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess ||
      (cfg->prop_samples > 0 &&
       cudaMalloc(&c->prop_part, sizeof(float) * gs_prop_part_floats(c->num_sms)) != cudaSuccess) ||
      (cfg->arch == GS_ARCH_PAPER &&
       (cudaMalloc(&c->paper_part, sizeof(float) * gs_paper_part_floats(c->num_sms)) != cudaSuccess ||
        cudaMalloc(&c->paper_loss_part, sizeof(float) * kLossPad * gs_paper_part_rows(c->num_sms)) != cudaSuccess)) ||
      (cfg->store_activations &&
       cudaMalloc(&c->store, c->store_bytes = (size_t)cfg->max_rays * c->max_n *
                                             (cfg->arch == GS_ARCH_PAPER ? kPaperStoreFloatsPerSample
                                                                         : kStoreFloatsPerSample) *
                                             sizeof(float)) !=
           cudaSuccess)) {
    gs_status s = cuda_fail(nullptr, "gs_create: workspace allocation");
    gs_destroy(c);
    return s;
  }
  c->eik_list = c->eik_count + 4;  // 16-byte aligned, after the count
  *out = c;
  return GS_OK;
}

void gs_destroy(gs_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->loss_part);
  cudaFree(ctx->mlp_part);
  cudaFree(ctx->default_dloss);
  cudaFree(ctx->status);
  cudaFree(ctx->store);
  cudaFree(ctx->prop_part);
  cudaFree(ctx->eik_part);
  cudaFree(ctx->eik_ticket);
  cudaFree(ctx->eik_count);
  cudaFree(ctx->paper_part);
  cudaFree(ctx->paper_loss_part);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  delete ctx;
}

gs_status gs_sample_rays(gs_ctx* ctx, const gs_frames* frames, uint64_t seed, uint32_t step, gs_batch* batch,
                         void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_sample_rays: ctx is NULL");
  gs_status fs = check_frames(ctx, frames, "gs_sample_rays");
  if (fs != GS_OK) return fs;
  gs_status s = check_batch(ctx, batch, true);
  if (s != GS_OK) return s;
  if (batch->N != ctx->cfg.n_strat + ctx->cfg.n_guided)
    return fail(ctx, GS_ERR_SHAPE, "gs_sample_rays: batch N != n_strat + n_guided");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  s = gs_launch_sample(ctx, frames, seed, step, batch, st);
  return s == GS_OK ? s : cuda_fail(ctx, "gs_sample_rays");
}

static gs_status render_common(gs_ctx* ctx, const char* who, const float* theta, const uint16_t* theta_bf16,
                               const gs_batch* batch, const float* dloss, float* loss, float* grad, float* rgb_hat,
                               float* d_hat, float* wsum, int mode, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "ctx is NULL");
  if (!theta) return fail(ctx, GS_ERR_INVALID_ARG, "theta is NULL");
  if (!aligned16(theta)) return fail(ctx, GS_ERR_ALIGN, "theta is not 16-byte aligned");
  if (ctx->cfg.precision == GS_PREC_BF16 && !theta_bf16)
    return fail(ctx, GS_ERR_INVALID_ARG, "the BF16 form needs theta_bf16 (the grid copy written by gs_adam_step)");
  if (ctx->cfg.precision == GS_PREC_BF16 && (reinterpret_cast<uintptr_t>(theta_bf16) & 7u))
    return fail(ctx, GS_ERR_ALIGN, "theta_bf16 is not 8-byte aligned");
  if ((mode & 1) && !loss) return fail(ctx, GS_ERR_INVALID_ARG, "loss is NULL");
  if ((mode & 2) && !grad) return fail(ctx, GS_ERR_INVALID_ARG, "grad is NULL");
  if ((mode & 2) && !aligned16(grad)) return fail(ctx, GS_ERR_ALIGN, "grad is not 16-byte aligned");
  gs_status s = check_batch(ctx, batch, false);
  if (s != GS_OK) return s;
  if (ctx->cfg.store_activations && mode == 2 && batch->R > 0 &&
      (ctx->store_R != batch->R || ctx->store_N != batch->N || ctx->store_t != batch->t))
    return fail(ctx, GS_ERR_INVALID_ARG,
                "store_activations: gs_backward needs a gs_forward of the same batch first (none, or another batch)");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  const float* dl = dloss ? dloss : ctx->default_dloss;
  if (ctx->cfg.arch == GS_ARCH_PAPER) {
    if (batch->dz && (reinterpret_cast<uintptr_t>(batch->dz) & 15u)) return fail(ctx, GS_ERR_ALIGN, "batch dz is not 16-byte aligned");
    if (gs_launch_paper(ctx, theta, batch, dl, grad, loss, rgb_hat, d_hat, wsum, mode, st) != GS_OK)
      return cuda_fail(ctx, who);
    if (ctx->cfg.store_activations && (mode & 1)) {
      ctx->store_R = batch->R;
      ctx->store_N = batch->N;
      ctx->store_t = batch->t;
    }
    return GS_OK;
  }
  // The smoothness kernel is independent of the render kernel (its own partial rows, atomics
  // into grad).  On a side stream that forks from the calling stream before the render launch,
  // and launched after it, it runs on the SMs that the render kernel's last ray-quads leave
  // idle.  The calling stream waits for it before the combine (a fork-join that stream
  // capture records as such).
  const bool fork = batch->R > 0 && batch->P > 0;
  if (fork && (cudaEventRecord(ctx->ev_fork, st) != cudaSuccess ||
               cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0) != cudaSuccess))
    return cuda_fail(ctx, who);
  if (batch->R > 0 &&
      gs_launch_render(ctx, theta, theta_bf16, batch, dl, grad, rgb_hat, d_hat, wsum, mode, st) != GS_OK)
    return cuda_fail(ctx, who);
  if (gs_launch_smooth(ctx, theta, batch, dl, grad, mode, fork ? ctx->side : st) != GS_OK) return cuda_fail(ctx, who);
  if (fork && (cudaEventRecord(ctx->ev_join, ctx->side) != cudaSuccess ||
               cudaStreamWaitEvent(st, ctx->ev_join, 0) != cudaSuccess))
    return cuda_fail(ctx, who);
  // partial rows: render CTAs (if any rays) then smoothness CTAs (if any points)
  gs_ctx tmp = *ctx;
  if (batch->R == 0 || batch->P == 0) {
    // only rows that this call wrote are combined
    tmp.n_parts = (batch->R > 0 ? ctx->render_ctas : 0) + (batch->P > 0 ? kSmoothCtas : 0);
    if (batch->R == 0) {
      tmp.loss_part = ctx->loss_part + (size_t)ctx->render_ctas * kLossPad;
      tmp.mlp_part = ctx->mlp_part + (size_t)ctx->render_ctas * kMlpPad;
    }
  }
  if (gs_launch_finalize(&tmp, batch, loss, grad, mode, st) != GS_OK) return cuda_fail(ctx, who);
  tmp.last_error.clear();
  if (ctx->cfg.store_activations && (mode & 1)) {
    ctx->store_R = batch->R;
    ctx->store_N = batch->N;
    ctx->store_t = batch->t;
  }
  return GS_OK;
}

gs_status gs_forward(gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* batch, float* loss,
                     float* rgb_hat, float* d_hat, float* wsum, void* stream) {
  return render_common(ctx, "gs_forward", theta, theta_bf16, batch, nullptr, loss, nullptr, rgb_hat, d_hat, wsum, 1,
                       stream);
}

gs_status gs_backward(gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* batch,
                      const float* dloss, float* grad, void* stream) {
  return render_common(ctx, "gs_backward", theta, theta_bf16, batch, dloss, nullptr, grad, nullptr, nullptr, nullptr,
                       2, stream);
}

gs_status gs_forward_backward(gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* batch,
                              const float* dloss, float* loss, float* grad, void* stream) {
  return render_common(ctx, "gs_forward_backward", theta, theta_bf16, batch, dloss, loss, grad, nullptr, nullptr,
                       nullptr, 3, stream);
}

gs_status gs_adam_step(gs_ctx* ctx, float* theta, float* grad, float* m, float* v, int64_t n, int64_t n_grid,
                       int32_t t, float lr_grid, float lr_mlp, float beta1, float beta2, float eps,
                       uint16_t* theta_bf16, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_adam_step: ctx is NULL");
  if (!theta || !grad || !m || !v) return fail(ctx, GS_ERR_INVALID_ARG, "gs_adam_step: NULL array");
  if (!aligned16(theta) || !aligned16(grad) || !aligned16(m) || !aligned16(v) ||
      (theta_bf16 && (reinterpret_cast<uintptr_t>(theta_bf16) & 7u)))
    return fail(ctx, GS_ERR_ALIGN, "gs_adam_step: arrays must be 16-byte aligned (bf16 copy 8-byte)");
  if (n < 0 || n_grid < 0 || n_grid > n || (n & 3) || (n_grid & 3))
    return fail(ctx, GS_ERR_SHAPE, "gs_adam_step: n and n_grid must be multiples of 4 with n_grid <= n");
  if (t < 1) return fail(ctx, GS_ERR_INVALID_ARG, "gs_adam_step: step count t must be >= 1");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_adam_step: bad beta or eps");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  if (n == 0) return GS_OK;
  if (gs_launch_adam(theta, grad, m, v, n, n_grid, t, lr_grid, lr_mlp, beta1, beta2, eps, theta_bf16, ctx->num_sms,
                     st) != GS_OK)
    return cuda_fail(ctx, "gs_adam_step");
  return GS_OK;
}

gs_status gs_query_sdf(gs_ctx* ctx, const float* theta, const float* x, int32_t P, float* sdf, float* grad,
                       void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_query_sdf: ctx is NULL");
  if (P < 0) return fail(ctx, GS_ERR_SHAPE, "gs_query_sdf: P < 0");
  if (P > 0 && (!theta || !x || !sdf)) return fail(ctx, GS_ERR_INVALID_ARG, "gs_query_sdf: NULL array");
  if (P > 0 && !aligned16(theta)) return fail(ctx, GS_ERR_ALIGN, "gs_query_sdf: theta is not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  const gs_status qs = ctx->cfg.arch == GS_ARCH_PAPER ? gs_launch_paper_query(ctx, theta, x, P, sdf, grad, st)
                                                      : gs_launch_query(ctx, theta, x, P, sdf, grad, st);
  if (qs != GS_OK) return cuda_fail(ctx, "gs_query_sdf");
  return GS_OK;
}

gs_status gs_proposal_sample(gs_ctx* ctx, const float* theta, const float* prop, const gs_frames* frames,
                             uint64_t seed, uint32_t step, const float* pdf_in, float* pdf_out, gs_batch* batch,
                             void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_proposal_sample: ctx is NULL");
  if (ctx->cfg.prop_samples <= 0) return fail(ctx, GS_ERR_UNSUPPORTED, "gs_proposal_sample: prop_samples is 0");
  gs_status s = check_frames(ctx, frames, "gs_proposal_sample");
  if (s != GS_OK) return s;
  s = check_batch(ctx, batch, true);
  if (s != GS_OK) return s;
  if (batch->N != ctx->cfg.prop_samples) return fail(ctx, GS_ERR_SHAPE, "gs_proposal_sample: batch N != prop_samples");
  if (batch->R > 0 && !pdf_in && (!theta || !prop))
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_proposal_sample: theta and prop are needed without pdf_in");
  if (batch->R > 0 && !pdf_in && !aligned16(theta)) return fail(ctx, GS_ERR_ALIGN, "gs_proposal_sample: theta is not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  s = gs_launch_prop_sample(ctx, theta, prop, frames, seed, step, pdf_in, pdf_out, batch, st);
  return s == GS_OK ? s : cuda_fail(ctx, "gs_proposal_sample");
}

gs_status gs_sample_importance(gs_ctx* ctx, const float* theta, const gs_frames* frames, uint64_t seed, uint32_t step,
                               gs_batch* batch, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_sample_importance: ctx is NULL");
  if (ctx->cfg.imp_coarse <= 0) return fail(ctx, GS_ERR_UNSUPPORTED, "gs_sample_importance: imp_coarse is 0");
  gs_status s = check_frames(ctx, frames, "gs_sample_importance");
  if (s != GS_OK) return s;
  s = check_batch(ctx, batch, true);
  if (s != GS_OK) return s;
  if (batch->N != imp_samples(&ctx->cfg))
    return fail(ctx, GS_ERR_SHAPE, "gs_sample_importance: batch N != imp_coarse + imp_steps * imp_per_step");
  if (batch->R > 0 && !theta) return fail(ctx, GS_ERR_INVALID_ARG, "gs_sample_importance: theta is NULL");
  if (batch->R > 0 && !aligned16(theta)) return fail(ctx, GS_ERR_ALIGN, "gs_sample_importance: theta is not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  s = gs_launch_importance(ctx, theta, frames, seed, step, batch, st);
  return s == GS_OK ? s : cuda_fail(ctx, "gs_sample_importance");
}

gs_status gs_proposal_backward(gs_ctx* ctx, const float* theta, const float* prop, const gs_batch* batch,
                               float* prop_grad, float* ce, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_proposal_backward: ctx is NULL");
  if (ctx->cfg.prop_samples <= 0) return fail(ctx, GS_ERR_UNSUPPORTED, "gs_proposal_backward: prop_samples is 0");
  gs_status s = check_batch(ctx, batch, false);
  if (s != GS_OK) return s;
  if (!theta || !prop || !prop_grad) return fail(ctx, GS_ERR_INVALID_ARG, "gs_proposal_backward: NULL array");
  if (batch->R > 0 && !batch->w) return fail(ctx, GS_ERR_INVALID_ARG, "gs_proposal_backward: batch w is NULL");
  if (!aligned16(theta)) return fail(ctx, GS_ERR_ALIGN, "gs_proposal_backward: theta is not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  s = gs_launch_prop_backward(ctx, theta, prop, batch, prop_grad, ce, st);
  return s == GS_OK ? s : cuda_fail(ctx, "gs_proposal_backward");
}

gs_status gs_query_sdf_backward(gs_ctx* ctx, const float* theta, const float* x, int32_t P, const float* dsdf,
                                const float* dgrad, float* grad, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_query_sdf_backward: ctx is NULL");
  if (P < 0) return fail(ctx, GS_ERR_SHAPE, "gs_query_sdf_backward: P < 0");
  if (P > 0 && (!theta || !x || !grad)) return fail(ctx, GS_ERR_INVALID_ARG, "gs_query_sdf_backward: NULL array");
  if (P > 0 && (!aligned16(theta) || !aligned16(grad)))
    return fail(ctx, GS_ERR_ALIGN, "gs_query_sdf_backward: theta or grad is not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  const gs_status bs = ctx->cfg.arch == GS_ARCH_PAPER
                           ? gs_launch_paper_query_backward(ctx, theta, x, P, dsdf, dgrad, grad, st)
                           : gs_launch_query_backward(ctx, theta, x, P, dsdf, dgrad, grad, st);
  if (bs != GS_OK) return cuda_fail(ctx, "gs_query_sdf_backward");
  return GS_OK;
}

gs_status gs_eikonal(gs_ctx* ctx, const float* theta, const gs_batch* batch, const float* dloss, float* loss,
                     float* grad, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_eikonal: ctx is NULL");
  if (!theta) return fail(ctx, GS_ERR_INVALID_ARG, "gs_eikonal: theta is NULL");
  if (!loss && !grad) return fail(ctx, GS_ERR_INVALID_ARG, "gs_eikonal: loss and grad are both NULL");
  if (!aligned16(theta) || (grad && !aligned16(grad)))
    return fail(ctx, GS_ERR_ALIGN, "gs_eikonal: theta or grad is not 16-byte aligned");
  gs_status s = check_batch(ctx, batch, false);
  if (s != GS_OK) return s;
  if ((long long)batch->R * batch->N > 0x7fffffffLL)
    return fail(ctx, GS_ERR_SHAPE, "gs_eikonal: R * N must stay below 2^31 (32-bit sample indices)");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  const float* dl = dloss ? dloss : ctx->default_dloss + 5;  // 1.0
  const gs_status es = ctx->cfg.arch == GS_ARCH_PAPER ? gs_launch_paper_eikonal(ctx, theta, batch, dl, loss, grad, st)
                                                      : gs_launch_eikonal(ctx, theta, batch, dl, loss, grad, st);
  if (es != GS_OK) return cuda_fail(ctx, "gs_eikonal");
  return GS_OK;
}

gs_status gs_pose_apply(gs_ctx* ctx, const float* c2w0, const float* xi, int32_t F, float* c2w, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_pose_apply: ctx is NULL");
  if (F < 0) return fail(ctx, GS_ERR_SHAPE, "gs_pose_apply: F < 0");
  if (F > 0 && (!c2w0 || !xi || !c2w)) return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_apply: NULL array");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  if (gs_launch_pose_apply(c2w0, xi, F, c2w, st) != GS_OK) return cuda_fail(ctx, "gs_pose_apply");
  return GS_OK;
}

gs_status gs_pose_backward(gs_ctx* ctx, const float* theta, const gs_frames* frames, const float* xi,
                           const gs_batch* batch, float* pose_grad, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_pose_backward: ctx is NULL");
  gs_status s = check_frames(ctx, frames, "gs_pose_backward");
  if (s != GS_OK) return s;
  s = check_batch(ctx, batch, true);
  if (s != GS_OK) return s;
  if (!theta || !xi || !pose_grad) return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_backward: NULL array");
  if (batch->R > 0 && !batch->dz) return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_backward: batch dz is NULL");
  if (!aligned16(theta) || (batch->dz && !aligned16(batch->dz)))
    return fail(ctx, GS_ERR_ALIGN, "gs_pose_backward: theta or batch dz is not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  if (gs_launch_pose_backward(ctx, theta, frames, xi, batch, pose_grad, st) != GS_OK)
    return cuda_fail(ctx, "gs_pose_backward");
  return GS_OK;
}

gs_status gs_eikonal_pose_backward(gs_ctx* ctx, const float* theta, const gs_frames* frames, const float* xi,
                                   const gs_batch* batch, const float* dloss, float* pose_grad, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_eikonal_pose_backward: ctx is NULL");
  gs_status s = check_frames(ctx, frames, "gs_eikonal_pose_backward");
  if (s != GS_OK) return s;
  s = check_batch(ctx, batch, true);
  if (s != GS_OK) return s;
  if (!theta || !xi || !pose_grad) return fail(ctx, GS_ERR_INVALID_ARG, "gs_eikonal_pose_backward: NULL array");
  if (!aligned16(theta)) return fail(ctx, GS_ERR_ALIGN, "gs_eikonal_pose_backward: theta is not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  if (gs_launch_eikonal_pose_backward(ctx, theta, frames, xi, batch, dloss, pose_grad, st) != GS_OK)
    return cuda_fail(ctx, "gs_eikonal_pose_backward");
  return GS_OK;
}

gs_status gs_extract_mesh(gs_ctx* ctx, const float* theta, const float* lo, float step, int32_t nx, int32_t ny,
                          int32_t nz, float iso, float* phi, float* tris, int64_t max_tris, int64_t* n_tris,
                          void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_extract_mesh: ctx is NULL");
  if (!theta || !lo || !phi || !n_tris) return fail(ctx, GS_ERR_INVALID_ARG, "gs_extract_mesh: NULL argument");
  if (max_tris < 0 || (max_tris > 0 && !tris)) return fail(ctx, GS_ERR_INVALID_ARG, "gs_extract_mesh: bad tris / max_tris");
  if (nx < 2 || ny < 2 || nz < 2 || !(step > 0.0f)) return fail(ctx, GS_ERR_SHAPE, "gs_extract_mesh: need nx, ny, nz >= 2 and step > 0");
  if (!aligned16(theta)) return fail(ctx, GS_ERR_ALIGN, "gs_extract_mesh: theta is not 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(n_tris) & 7u)) return fail(ctx, GS_ERR_ALIGN, "gs_extract_mesh: n_tris is not 8-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  if (gs_launch_mesh(ctx, theta, lo, step, nx, ny, nz, iso, phi, tris, max_tris,
                     reinterpret_cast<unsigned long long*>(n_tris), st) != GS_OK)
    return cuda_fail(ctx, "gs_extract_mesh");
  return GS_OK;
}

gs_status gs_voxel_index(gs_ctx* ctx, const float* x, int32_t P, int64_t* out, void* stream) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_voxel_index: ctx is NULL");
  if (P < 0) return fail(ctx, GS_ERR_SHAPE, "gs_voxel_index: P < 0");
  if (P > 0 && (!x || !out)) return fail(ctx, GS_ERR_INVALID_ARG, "gs_voxel_index: NULL array");
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  if (gs_launch_voxel_index(ctx, x, P, (long long*)out, st) != GS_OK) return cuda_fail(ctx, "gs_voxel_index");
  return GS_OK;
}

gs_status gs_sync_status(gs_ctx* ctx) {
  if (!ctx) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_sync_status: ctx is NULL");
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return cuda_fail(ctx, "gs_sync_status");
  int h = 0;
  if (cudaMemcpy(&h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail(ctx, "gs_sync_status");
  if (h != 0) {
    std::string m = "a bounded wait for tensor-core products ran out in:";
    if (h & kStatusRender) m += " render";
    if (h & kStatusProposal) m += " proposal";
    if (h & kStatusEikonal) m += " eikonal";
    if (h & kStatusPaperRender) m += " render (paper architecture)";
    if (h & kStatusImportance) m += " importance sampler";
    return fail(ctx, GS_ERR_DEVICE, m.c_str());
  }
  return GS_OK;
}

const char* gs_last_error(gs_ctx* ctx) { return ctx ? ctx->last_error.c_str() : g_err.c_str(); }

}  // extern "C"
