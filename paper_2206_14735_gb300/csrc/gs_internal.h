// Library-internal declarations: the context object and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "gosurf.h"
#include "gs_device.cuh"

constexpr int kMlpPad = 1688;     // per-CTA decoder-gradient partial row (>= GS_MLP_PARAMS, 16-B multiple)
constexpr int kLossPad = 8;       // per-CTA loss partial row
constexpr int kSmoothCtas = 128;  // CTAs of the smoothness kernel (fixed, so partial rows are known)
constexpr int kRenderCtasPerSm = 1;  // persistent render CTAs per SM
constexpr int kStoreFloatsPerSample = 100;  // stored activations: z 16, a1 32, (phi, h) 16, a2 32, c 3 + 1 pad
constexpr int kPaperStoreFloatsPerSample = 156;  // paper architecture: z 16, cf 6 + phi + pad, c 3 + pad, 4 x 32 hidden
constexpr int kRenderGroups = 3;     // tile groups (4 warps, 128 tensor-memory columns each) per render CTA
// Bits of the context's device status word: a kernel sets its bit when a bounded wait for its
// tensor-core products ran out (it then stops early; that call's outputs are incomplete)
constexpr int kStatusRender = 2, kStatusProposal = 4, kStatusEikonal = 8, kStatusPaperRender = 16,
              kStatusImportance = 32;
constexpr int kEikCtasPerSm = 4;     // CTAs of the Eikonal kernel per SM (one wave at 230 registers x 64 threads)

struct gs_ctx {
  gs_config cfg;
  gs::GridDesc grid;
  int device = 0;
  int num_sms = 0;
  int render_ctas = 0;  // persistent CTAs of the fused render kernel
  int n_parts = 0;      // render_ctas + kSmoothCtas
  int max_n = 0;        // most samples per ray of any batch form (sizes the activation store)
  float* loss_part = nullptr;
  float* mlp_part = nullptr;
  float* default_dloss = nullptr;  // (0,0,0,0,0,1)
  int* status = nullptr;
  float* store = nullptr;    // decoder activations kept by the forward pass (store_activations)
  size_t store_bytes = 0;
  int store_R = -1, store_N = -1;     // batch shape and depths pointer of the gs_forward that filled it
  const float* store_t = nullptr;
  float* prop_part = nullptr;        // proposal training partial rows (prop_samples > 0)
  int eik_ctas = 0;                  // largest grid of the Eikonal kernel
  float* eik_part = nullptr;         // its per-CTA loss sums
  unsigned* eik_ticket = nullptr;    // CTAs finished in the running call (0 between calls)
  int* eik_count = nullptr;          // free-space samples listed by the Eikonal call's compaction pass
  int* eik_list = nullptr;           // their sample indices [max_rays * max_n] (order kept within 1024)
  long long colour_off = 0;          // paper architecture: float offset of the colour grid
  float* paper_part = nullptr;       // paper architecture: per-CTA decoder-gradient partial rows
  float* paper_loss_part = nullptr;  // and loss partial rows
  cudaStream_t last_stream = nullptr;
  cudaStream_t side = nullptr;       // the smoothness kernel runs here beside the render kernel
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string last_error;
};

gs_status gs_launch_sample(const gs_ctx* ctx, const gs_frames* f, uint64_t seed, uint32_t step, const gs_batch* b,
                           cudaStream_t st);
// mode bit 1: forward outputs (loss partials, per-ray outputs), bit 2: backward (grad)
gs_status gs_launch_render(const gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* b,
                           const float* dloss, float* grad, float* rgb_hat, float* d_hat, float* wsum, int mode,
                           cudaStream_t st);
gs_status gs_launch_smooth(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* grad,
                           int mode, cudaStream_t st);
gs_status gs_launch_finalize(const gs_ctx* ctx, const gs_batch* b, float* loss, float* grad, int mode,
                             cudaStream_t st);
gs_status gs_launch_adam(float* theta, float* grad, float* m, float* v, long long n, long long n_grid, int t,
                         float lr_grid, float lr_mlp, float b1, float b2, float eps, uint16_t* bf16, int num_sms,
                         cudaStream_t st);
gs_status gs_launch_sample_smooth(const gs_ctx* ctx, const gs_frames* f, uint64_t seed, uint32_t step,
                                  const gs_batch* b, cudaStream_t st);
int gs_prop_part_rows(int num_sms);
size_t gs_prop_part_floats(int num_sms);
gs_status gs_launch_prop_sample(const gs_ctx* ctx, const float* theta, const float* q, const gs_frames* f,
                                uint64_t seed, uint32_t step, const float* pdf_in, float* pdf_out, const gs_batch* b,
                                cudaStream_t st);
gs_status gs_launch_prop_backward(const gs_ctx* ctx, const float* theta, const float* q, const gs_batch* b,
                                  float* grad, float* ce, cudaStream_t st);
gs_status gs_launch_importance(const gs_ctx* ctx, const float* theta, const gs_frames* f, uint64_t seed,
                               uint32_t step, const gs_batch* b, cudaStream_t st);
gs_status gs_launch_mesh(const gs_ctx* ctx, const float* theta, const float lo[3], float step, int nx, int ny, int nz,
                         float iso, float* phi, float* tris, long long max_tris, unsigned long long* n_tris,
                         cudaStream_t st);
gs_status gs_launch_pose_apply(const float* c2w0, const float* xi, int F, float* c2w, cudaStream_t st);
gs_status gs_launch_pose_backward(const gs_ctx* ctx, const float* theta, const gs_frames* f, const float* xi,
                                  const gs_batch* b, float* pose_grad, cudaStream_t st);
gs_status gs_launch_eikonal_pose_backward(const gs_ctx* ctx, const float* theta, const gs_frames* f, const float* xi,
                                          const gs_batch* b, const float* dloss, float* pose_grad, cudaStream_t st);
gs_status gs_launch_eikonal(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* loss,
                            float* grad, cudaStream_t st);
gs_status gs_launch_query_backward(const gs_ctx* ctx, const float* theta, const float* x, int P, const float* dsdf,
                                   const float* dgrad, float* grad, cudaStream_t st);
gs_status gs_launch_query(const gs_ctx* ctx, const float* theta, const float* x, int P, float* sdf, float* grad,
                          cudaStream_t st);
gs_status gs_launch_voxel_index(const gs_ctx* ctx, const float* x, int P, long long* out, cudaStream_t st);
void gs_set_thread_error(const char* msg);
// Host-side configuration rules shared by gs_create and gs_forward_backward_noalloc.
gs_status gs_check_config(const gs_config* cfg, const char** msg);
int gs_paper_part_rows(int num_sms);
size_t gs_paper_part_floats(int num_sms);
gs_status gs_launch_paper(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* grad,
                          float* loss, float* rgb_hat, float* d_hat, float* wsum, int mode, cudaStream_t st);
gs_status gs_launch_paper_tc(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss, float* grad,
                             float* rgb_hat, float* d_hat, float* wsum, int mode, float* loss_part, float* mlp_part,
                             int ctas, cudaStream_t st);
gs_status gs_launch_eikonal_paper_tc(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss,
                                     float* loss, float* grad, cudaStream_t st);
gs_status gs_launch_paper_eikonal(const gs_ctx* ctx, const float* theta, const gs_batch* b, const float* dloss,
                                  float* loss, float* grad, cudaStream_t st);
gs_status gs_launch_paper_query(const gs_ctx* ctx, const float* theta, const float* x, int P, float* sdf, float* grad,
                                cudaStream_t st);
gs_status gs_launch_paper_query_backward(const gs_ctx* ctx, const float* theta, const float* x, int P,
                                         const float* dsdf, const float* dgrad, float* grad, cudaStream_t st);
