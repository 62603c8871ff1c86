/*
 * gosurf.h -- C ABI of the GB300 (sm_103a) implementation of one GO-Surf optimisation step
 * (Wang, Bleja, Agapito: "GO-Surf: Neural Feature Grid Optimization for Fast, High-Fidelity
 * RGB-D Surface Reconstruction", arXiv 2206.14735).
 *
 * One step samples a batch of rays from posed RGB-D frames, decodes an SDF and a colour at
 * every sample from a four-level dense feature grid and two small decoders, renders colour
 * and depth with NeuS weights, evaluates the rgb / depth / truncated-SDF / free-space losses
 * and the SDF-gradient smoothness term (the Eikonal term through its own entry point),
 * back-propagates to every grid feature and decoder weight, and applies Adam.
 *
 * Conventions common to every entry point
 *   - Every pointer argument is a DEVICE pointer unless its comment says "host".  The caller
 *     owns all of them; the library never frees or keeps them past the call.
 *   - Device arrays of float / float4 data must be 16-byte aligned (GS_ERR_ALIGN otherwise).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls only
 *     enqueue work and return; argument errors are detected on the host and returned before
 *     anything is enqueued.  Errors raised on the device (bounds checks of debug builds) are
 *     recorded in the context and reported by gs_sync_status().
 *   - No call allocates device memory except gs_create (which sizes its workspace once).
 *   - A context serves one stream at a time and is not thread-safe.
 *
 * Parameter vector (one flat float32 array, "theta"), in this order:
 *   grid level l = 0 (coarsest) .. 3 (finest): dims[l][2] x dims[l][1] x dims[l][0] vertices
 *     stored z-major, x fastest, 4 features per vertex (one 16-byte vector per vertex);
 *   decoder block of GS_MLP_PARAMS floats: W1[32][16], b1[32], W2[16][32], b2[16],
 *     W3[32][15], b3[32], W4[3][32], b4[3], kappa (sharpness s = exp(kappa)).
 *   The gradient vector and the Adam moments use the same layout.
 *
 * The paper's architecture (gs_config.arch = GS_ARCH_PAPER; Sec. 3.1 Eq. SDF_MLP and
 * Eq. COLOR_MLP, "Architecture Details") has its own flat vector:
 *   grid levels 0..3 as above (geometry features V_theta);
 *   the colour grid W_beta: dims[3] vertices (those of the finest level), 6 features per
 *     vertex ([nz][ny][nx][6], 24 bytes per vertex), padded with zeros to a multiple of 4 floats;
 *   decoder block of GS_PAPER_MLP_PARAMS floats: geometry decoder gW1[32][16], gb1[32],
 *     gW2[32][32], gb2[32], gw3[32], gb3 (phi = gw3 . relu(gW2 relu(gW1 z + gb1) + gb2) + gb3);
 *     colour decoder cW1[32][9], cb1[32], cW2[32][32], cb2[32], cW3[3][32], cb3[3]
 *     (c = sigmoid(cW3 relu(cW2 relu(cW1 u + cb1) + cb2) + cb3), u = [W_beta(x), d] with d the
 *     unit viewing direction r/|r|); kappa.
 *   gs_param_count reports its size (not a multiple of 4: pad the arrays given to
 *   gs_adam_step to one; the padding entries keep a zero gradient).
 */
#ifndef GOSURF_H
#define GOSURF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_LEVELS 4
#define GS_FEAT 4
#define GS_MLP_PARAMS 1684
#define GS_MAX_SAMPLES 160 /* samples per ray of any batch (5 chunks of 32) */
#define GS_NUM_LOSS 6      /* rgb, depth, sdf, fs, smooth, total */
#define GS_PROP_BINS 32    /* bins of the learned proposal over [near_m, far_m] */
#define GS_PROP_PARAMS 1473 /* proposal network: W1[32][11], b1[32], W2[32][32], b2[32], w3[32], b3 */
#define GS_COLOUR_FEAT 6       /* colour features per vertex of the paper architecture's colour grid (h_c) */
#define GS_PAPER_MLP_PARAMS 3109 /* decoder block of the paper architecture (layout above) */

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* NULL pointer or out-of-range scalar */
  GS_ERR_SHAPE = 2,       /* sizes inconsistent with the context's configuration */
  GS_ERR_ALIGN = 3,       /* a device array is not 16-byte aligned */
  GS_ERR_CUDA = 4,        /* a CUDA runtime call failed (see gs_last_error) */
  GS_ERR_DEVICE = 5,      /* a device-side check failed in an earlier call */
  GS_ERR_UNSUPPORTED = 6  /* configuration outside what this build supports */
} gs_status;

/* Arithmetic forms of the render pass (gs_config.precision): */
#define GS_PREC_FP32 0 /* FP32 grid gathers; decoders on tensor cores with FP32-grade products */
#define GS_PREC_BF16 1 /* gathers from the bfloat16 grid copy; decoders in BF16 with FP32 accumulation */

/* Scene models (gs_config.arch): */
#define GS_ARCH_COMPACT 0 /* geometry decoder 16-32-16 ([phi, 15 geometric features]), colour decoder
                             15-32-3 fed the geometric features: the workload's model */
#define GS_ARCH_PAPER 1   /* the paper's (Sec. 3.1): colour grid W_beta at the finest level, colour decoder
                             fed W_beta(x) and the viewing direction, both decoders with two hidden layers
                             of 32.  Supported by gs_sample_rays, gs_sample_importance, gs_proposal_sample,
                             gs_proposal_backward, gs_forward, gs_backward, gs_forward_backward, gs_eikonal,
                             gs_query_sdf, gs_query_sdf_backward, gs_extract_mesh, gs_pose_apply,
                             gs_pose_backward and gs_adam_step (FP32; store_activations keeps 156 floats
                             per sample: z, W_beta(x), phi, c and the four hidden layers);
                             gs_forward_backward_noalloc returns GS_ERR_UNSUPPORTED */

/* Sample classes written by gs_sample_rays (Sec. 3.3): */
#define GS_CLS_NONE 0 /* no SDF supervision (behind the surface, or the ray has no depth) */
#define GS_CLS_TR 1   /* near surface, |D - d| <= t: truncated-SDF loss */
#define GS_CLS_FS 2   /* free space in front of the surface, D - d > t: free-space loss */

/* Scene and optimisation settings (host struct; values copied by gs_create). */
typedef struct gs_config {
  int32_t dims[GS_LEVELS][3]; /* vertex counts (nx, ny, nz) per level, level 0 coarsest (Sec. 3.1) */
  float voxel[GS_LEVELS];     /* voxel edge length per level, metres */
  float origin[3];            /* world position of vertex (0,0,0) of every level */
  int32_t n_strat;            /* stratified samples per ray over [near, far] */
  int32_t n_guided;           /* samples stratified over [D - g, D + g] when D > 0 */
  float near_m, far_m;        /* stratified range, metres */
  float guide_half;           /* g, metres */
  float trunc;                /* truncation distance t of the SDF bound, metres (Sec. 3.3) */
  float kappa_fs;             /* exponent scale of the free-space penalty (Sec. 3.3: 5) */
  float lam[5];               /* loss weights: rgb, depth, sdf, fs, smooth (Sec. 3.4) */
  int32_t max_rays;           /* largest ray batch any call will see (workspace sizing) */
  int32_t max_smooth;         /* largest smoothness point batch */
  float delta_s;              /* smoothness perturbation length, metres (Sec. 3.3) */
  int32_t precision;          /* GS_PREC_FP32 or GS_PREC_BF16 */
  int32_t store_activations;  /* 1: every forward pass writes each sample's decoder inputs and
                                 activations (z, ReLU outputs, SDF, geometric feature, colour:
                                 100 floats = 400 bytes per sample, max_rays x N samples, in
                                 float4 planes of four fields each, allocated by gs_create;
                                 GS_ARCH_PAPER: 156 floats) and every backward pass reads
                                 them instead of gathering
                                 again and recomputing the decoders; 0: the backward pass
                                 recomputes them (no memory) */
  int32_t prop_samples;       /* learned proposal sampler (not part of the paper): samples per
                                 ray of a proposal batch, 2..32; 0 disables gs_proposal_* */
  int32_t prop_guided;        /* of those, samples stratified over [D - g, D + g] when D > 0 */
  int32_t imp_coarse;         /* hierarchical importance sampler (Sec. 3.2): coarse samples per ray,
                                 >= 2; 0 disables gs_sample_importance */
  int32_t imp_steps;          /* importance steps (Sec. 4: 3) */
  int32_t imp_per_step;       /* samples added per step, 1..32 (Sec. 4: 12); batches of this sampler
                                 hold imp_coarse + imp_steps * imp_per_step <= 160 samples per ray */
  int32_t arch;               /* GS_ARCH_COMPACT or GS_ARCH_PAPER (the parameter layout follows it) */
} gs_config;

/* Posed RGB-D frames resident in device memory (Sec. 3: {I_t, D_t}, xi_t). */
typedef struct gs_frames {
  int32_t F, H, W;
  const uint8_t* rgb;  /* [F][H][W][3] */
  const float* depth;  /* [F][H][W], metres of z-depth, 0 = missing */
  const float* c2w;    /* [F][3][4] camera-to-world, OpenCV axes (x right, y down, z forward) */
  float fx, fy, cx, cy;
} gs_frames;

/* A ray batch; all arrays caller-allocated on the device. */
typedef struct gs_batch {
  int32_t R;       /* rays */
  int32_t N;       /* samples per ray = n_strat + n_guided */
  int32_t P;       /* smoothness points (may be 0) */
  int64_t* pix;    /* [R] flat pixel id f*H*W + v*W + u */
  float* origin;   /* [R][3] ray origin o */
  float* dir;      /* [R][3] ray direction r with unit camera-z (ray parameter = z-depth) */
  float* rgb;      /* [R][3] observed colour I[u,v] in [0,1] */
  float* depth;    /* [R] observed depth D[u,v] (0 = missing) */
  float* t;        /* [R][N] sample depths d_i, ascending */
  uint8_t* cls;    /* [R][N] GS_CLS_* */
  float* xs;       /* [P][3] smoothness points x */
  float* eps;      /* [P][3] perturbations (|eps| = delta_s) */
  uint8_t* valid;  /* [P] 1 if the point is used */
  int32_t* counts; /* [4] rays with D > 0, |S_tr|, |S_fs|, valid smoothness points */
  float* w;        /* [R][N] rendering weights w_i = T_i alpha_i, written by the forward passes
                      when not NULL; read by gs_proposal_backward */
  float* dz;       /* [R][N][16] dL/dz of every sample (the upstream gradient of its geometry
                      feature), written by the backward passes when not NULL; read by
                      gs_pose_backward.  GS_ARCH_PAPER: [R][N][32] per sample, dL/dz (16),
                      dL/dW_beta(x) (6), dL/d(viewing direction) (3), zeros (7) */
  float* eik;      /* NULL, or [5][R][N][4] (16-byte aligned) deferred Eikonal records, written
                      by gs_eikonal for the free-space samples and read by the next backward
                      pass over this batch (see gs_eikonal); plane k of sample s = r N + i at
                      ((float4*)eik)[k R N + s]: planes 0..3 p_l / v_l (level l's part of
                      d phi / d z over its voxel size), plane 4 (a, 0) with a the Eikonal
                      adjoint dL/d(grad_x phi).  Both architectures. */
} gs_batch;

typedef struct gs_ctx gs_ctx;

/* Creates a context for the current CUDA device and sizes its workspace for cfg->max_rays.
 * Returns GS_ERR_INVALID_ARG / GS_ERR_UNSUPPORTED for a bad configuration. */
gs_status gs_create(const gs_config* cfg, gs_ctx** out);
void gs_destroy(gs_ctx* ctx);

/* Host: number of floats in the flat parameter vector of cfg->arch; *n_grid (may be NULL)
 * receives the number of grid floats (geometry levels, and the padded colour grid of
 * GS_ARCH_PAPER) that precede the decoder block. */
int64_t gs_param_count(const gs_config* cfg, int64_t* n_grid);

/* Ray batch sampling (Sec. 3.4 "we sample a batch of R rays from all pixels across all
 * images, including pixels that have missing depth"), sample placement and the bound
 * classes of Sec. 3.3, plus the near-surface smoothness points S_g (Sec. 3.3, Eq.
 * smoothness_loss).  Pixels, jitters and perturbation directions come from SplitMix64 keyed
 * by (seed, stream, step, index, slot); every quantity is computed in binary32 with
 * round-to-nearest and no contraction, so results are reproducible bit for bit.
 * batch->R, N, P select the sizes; N must equal n_strat + n_guided.  The render entry
 * points also accept batches of N = prop_samples made by gs_proposal_sample and of
 * N = imp_coarse + imp_steps * imp_per_step made by gs_sample_importance. */
gs_status gs_sample_rays(gs_ctx* ctx, const gs_frames* frames, uint64_t seed, uint32_t step, gs_batch* batch,
                         void* stream);

/* Forward pass (Sec. 3.1-3.4): loss[6] = L_rgb, L_d, L_sdf, L_fs, L_smooth and the weighted
 * total sum_k lam_k L_k (device floats; per-CTA partial sums are combined in FP64).
 * theta_bf16: the bfloat16 copy of the grid that gs_adam_step writes; read by the gathers of
 * the BF16 form (required there), ignored (may be NULL) in the FP32 form.  The decoders always
 * read theta.  rgb_hat [R][3], d_hat [R], wsum [R] (sum of weights) may each be NULL. */
gs_status gs_forward(gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* batch, float* loss,
                     float* rgb_hat, float* d_hat, float* wsum, void* stream);

/* Backward pass: grad += d(sum_k dloss_k * out_k)/d theta, with out = the six outputs of
 * gs_forward and dloss [6] device floats (NULL = (0,0,0,0,0,1), the gradient of the total).
 * With store_activations the activations kept by the last gs_forward (or
 * gs_forward_backward) are read: that call must have seen the same theta and batch, and
 * GS_ERR_INVALID_ARG is returned when no forward pass of a batch with this R, N and t
 * pointer came first.  Otherwise everything is recomputed from theta.  Grid
 * gradients are accumulated with FP32 atomics (summation order not deterministic); decoder
 * gradients are reduced in a fixed order.  With batch->eik set, the grid gradient also
 * receives the deferred Eikonal term of every free-space sample (records written by
 * gs_eikonal on this batch before this call; see there). */
gs_status gs_backward(gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* batch,
                      const float* dloss, float* grad, void* stream);

/* Forward and backward in one pass over the batch (loss and grad as above).
 * With GS_ARCH_PAPER these three entry points evaluate the paper's architecture (layout at
 * the top of this file): the same losses, batch normalisations and smoothness term with
 * phi = f_omega(V_theta(x)) and c = g_gamma(W_beta(x), r/|r|), the gradient reaching the
 * geometry grid, the colour grid and both decoders; FP32 only; batch->dz receives the
 * 32-float records described at gs_batch. */
gs_status gs_forward_backward(gs_ctx* ctx, const float* theta, const uint16_t* theta_bf16, const gs_batch* batch,
                              const float* dloss, float* loss, float* grad, void* stream);

/* Adam (Kingma & Ba) over the n-entry flat vectors theta, grad, m, v with bias correction
 * for step t >= 1; entries [0, n_grid) use lr_grid, the rest lr_mlp (Sec. 4: 1e-2 for
 * grids, 1e-3 for decoders).  grad is set to zero.  theta_bf16 (may be NULL) receives a
 * round-to-nearest-even bfloat16 copy of the first n_grid entries. */
gs_status gs_adam_step(gs_ctx* ctx, float* theta, float* grad, float* m, float* v, int64_t n, int64_t n_grid,
                       int32_t t, float lr_grid, float lr_mlp, float beta1, float beta2, float eps,
                       uint16_t* theta_bf16, void* stream);

/* SDF query (Sec. 3.1 Eq. SDF_MLP; gradient per Supp. Eq. sdf_first_grad): sdf[P] and, if
 * grad != NULL, grad_x phi [P][3] at points x [P][3]. */
gs_status gs_query_sdf(gs_ctx* ctx, const float* theta, const float* x, int32_t P, float* sdf, float* grad,
                       void* stream);

/* Learned proposal sampler (an addition to the paper's method: it reduces the samples per
 * ray).  [near_m, far_m] is cut into GS_PROP_BINS equal bins; for the centre x_b of bin b a
 * network reads the features of the two coarsest grid levels and the unit ray direction,
 * u = [z_0(x_b), z_1(x_b), r/|r|], and gives one logit
 *   l_b = w3 . relu(W2 relu(W1 u + b1) + b2) + b3;   p = softmax_b(l).
 * prop: the GS_PROP_PARAMS floats in the order of the GS_PROP_PARAMS comment.
 *
 * gs_proposal_sample draws the same rays as gs_sample_rays for the same (seed, step) (and
 * the same smoothness points), then batch->N = prop_samples depths per ray from the
 * mixture pp = 0.95 p + 0.05 / GS_PROP_BINS: K = N - prop_guided inverse-CDF draws
 * u_k = (k + xi_k) / K (K = N when D <= 0), placed linearly inside their bin, plus
 * prop_guided samples stratified over [D - g, D + g] when D > 0; sorted ascending and
 * classified as in gs_sample_rays.  Binary32 with explicit rounding (bit-reproducible for a
 * given p).  pdf_in [R][GS_PROP_BINS] (may be NULL) replaces the network's p (then theta and
 * prop may be NULL); pdf_out (may be NULL) receives the p that was used. */
gs_status gs_proposal_sample(gs_ctx* ctx, const float* theta, const float* prop, const gs_frames* frames,
                             uint64_t seed, uint32_t step, const float* pdf_in, float* pdf_out, gs_batch* batch,
                             void* stream);

/* Hierarchical importance sampling (Sec. 3.2: from N_c coarse samples, 3 steps each add 12
 * samples drawn from the weights of the samples so far, as in NeuS; Sec. 4: N_c = 96,
 * N_f = 36).  The rays (pix, origin, dir, rgb, depth) and the smoothness points are those of
 * gs_sample_rays for the same (seed, step).  Per ray: imp_coarse depths stratified over
 * [near_m, far_m]; then imp_steps times: phi at the current samples (theta, FP32), the NeuS
 * weights w_k = T_k alpha_k of Sec. 3.2 Eq. volume_rendering_alpha with s = exp(kappa),
 * interval masses w_k + 1e-5 over [t_k, t_k+1], and imp_per_step stratified inverse-CDF
 * draws u_j = (j + xi_j) / imp_per_step, each placed linearly inside its interval and merged
 * into the sorted depths (an existing depth first on ties); classes as in gs_sample_rays.
 * batch->N must be imp_coarse + imp_steps * imp_per_step; needs imp_coarse > 0 in the
 * configuration (GS_ERR_UNSUPPORTED otherwise).  theta 16-byte aligned. */
gs_status gs_sample_importance(gs_ctx* ctx, const float* theta, const gs_frames* frames, uint64_t seed, uint32_t step,
                               gs_batch* batch, void* stream);

/* Training step of the proposal: for every ray the weights batch->w at the depths batch->t
 * (from a forward pass of the main model on this batch, any sampler) are summed per bin,
 * h_b, and normalised; rays with sum(h) < 1e-3 are skipped.  The loss is the mean over the
 * used rays of -sum_b (h_b / sum h) log p_b; the target is constant (no gradient reaches
 * theta).  prop_grad [GS_PROP_PARAMS] += the gradient w.r.t. prop; ce [2] (may be NULL)
 * receives (loss, rays used).  Needs prop_samples > 0 in the configuration. */
gs_status gs_proposal_backward(gs_ctx* ctx, const float* theta, const float* prop, const gs_batch* batch,
                               float* prop_grad, float* ce, void* stream);

/* Reverse mode of gs_query_sdf with respect to the parameters (the double backward of the
 * SDF gradient, Supp. Sec. 1): grad [n_params] += sum_p dsdf[p] d phi(x_p)/d theta
 * + dgrad[p] . d grad_x phi(x_p)/d theta, for device arrays x [P][3], dsdf [P] and dgrad
 * [P][3] (either may be NULL = zero).  theta and grad 16-byte aligned.  The points x are
 * constants (no gradient with respect to x).  Accumulates with atomics (order not fixed). */
gs_status gs_query_sdf_backward(gs_ctx* ctx, const float* theta, const float* x, int32_t P, const float* dsdf,
                                const float* dgrad, float* grad, void* stream);

/* Eikonal term (Sec. 3.3 Eq. eikonal_loss, on the free-space samples as Sec. 3.4 states):
 *   L_eik = (1 / |S_fs|) sum over the batch's samples of class GS_CLS_FS of (1 - |grad_x phi(x)|)^2,
 * x = o + d r formed in binary32 as in gs_forward, |S_fs| = batch->counts[2] (written by the
 * sampler); 0 when S_fs is empty.  The five losses of gs_forward do not include it: the
 * caller adds lam_eik L_eik (Sec. 4: lam_eik = 1) to its objective.
 * loss [1] (device, may be NULL) receives L_eik, reduced in FP64 over per-CTA partial sums.
 * grad (may be NULL; not both NULL) += dloss[0] dL_eik/dtheta with dloss [1] a device float
 * (NULL = 1): the second-order path of Supp. Sec. 1 (grid features through d z/d x, W1 and
 * row 0 of W2 through d phi/d z; the sub-gradient at grad_x phi = 0 is 0), accumulated with
 * atomics (order not fixed).  Reads the FP32 grid in every precision form.  Needs only the
 * batch's ray arrays (origin, dir, t, cls, counts).
 * Deferred grid term (batch->eik != NULL): the grid part of the gradient is not scattered
 * here; every free-space sample's record (p_l / v_l, a; a = 0 when grad is NULL) goes to
 * batch->eik instead, and the next gs_backward / gs_forward_backward over the same batch adds
 * p_l (1/v_l) (a . dw_c/df) to the corner vectors it scatters anyway (no reductions of its
 * own).  grad then holds the full gradient only after that backward pass; the decoder part
 * and the loss are written by this call as without records. */
gs_status gs_eikonal(gs_ctx* ctx, const float* theta, const gs_batch* batch, const float* dloss, float* loss,
                     float* grad, void* stream);

/* Mesh extraction (Sec. 4: meshes are extracted from phi on a 1 cm lattice by marching
 * cubes).  phi [nz][ny][nx] (device scratch, written) receives phi at the lattice points
 * lo + (i, j, k) * step (lo host float[3], binary32 positions, FP32 SDF).  Each lattice cell is
 * split into 6 tetrahedra around its corner-0-to-corner-7 diagonal (corner c at offset
 * (c & 1, (c >> 1) & 1, c >> 2)); a tetrahedron with 1 or 3 corners below iso yields one
 * triangle, with 2 below two, their vertices on its edges where the linear interpolation of
 * phi equals iso (interpolated from the endpoint of lower lattice index, so shared edges give
 * identical points: the mesh is closed wherever the surface stays inside the lattice).
 * Normals (p1 - p0) x (p2 - p0) point towards increasing phi.  tris [max_tris][3][3] (device,
 * may be NULL with max_tris 0) receives triangles in no fixed order; *n_tris (device int64)
 * the total number, which may exceed max_tris (then only max_tris are written: call again with
 * more room).  nx, ny, nz >= 2, step > 0. */
gs_status gs_extract_mesh(gs_ctx* ctx, const float* theta, const float* lo, float step, int32_t nx, int32_t ny,
                          int32_t nz, float iso, float* phi, float* tris, int64_t max_tris, int64_t* n_tris,
                          void* stream);

/* Camera-pose refinement (Sec. 3.4: the optimised parameters include the poses; Sec. 4: a
 * translation t in R^3 and nu in so(3) per frame).  Frame f's pose is its given
 * camera-to-world [R0 | t0] corrected by xi [F][6] = (dt, nu) (device floats):
 *   R = R0 Exp(nu) (Rodrigues' formula), t = t0 + dt.
 * gs_pose_apply writes the corrected c2w [F][3][4] (device) from c2w0 [F][3][4]; sample with
 * frames whose c2w points there.  The samples x = o + d r of a ray move with its frame's pose
 * (o = t, r = R d, d the pixel's direction with unit camera z); their depths and classes do
 * not.  gs_pose_backward adds to pose_grad [F][6] (device) the gradient of the per-ray losses
 * (rgb, depth, truncated SDF, free space) through the sample positions:
 *   dL/d dt = sum_s g_s,  dL/d nu = J_r(nu)^T [d]_x R^T sum_s d_s g_s,  g_s = sum_l (dz_l/dx)^T dL/dz_l,
 * over each frame's rays, with J_r the right Jacobian of Exp; dL/dz is batch->dz, which the
 * preceding gs_backward / gs_forward_backward of this batch wrote (batch->dz must be set
 * there and here).  frames: the corrected poses the batch was sampled with.  The smoothness
 * points are not differentiated with respect to the poses.  Accumulates with atomics.
 * GS_ARCH_PAPER: the colour grid moves with x too, g_s = sum_l (dz_l/dx)^T dL/dz_l +
 * (dW_beta/dx)^T dL/dW_beta, and the viewing direction r/|r| = R d/|d| turns with the pose:
 * dL/d nu = J_r(nu)^T [d]_x R^T (sum_s d_s g_s + sum_s dL/d(direction)_s / |d|). */
gs_status gs_pose_apply(gs_ctx* ctx, const float* c2w0, const float* xi, int32_t F, float* c2w, void* stream);
gs_status gs_pose_backward(gs_ctx* ctx, const float* theta, const gs_frames* frames, const float* xi,
                           const gs_batch* batch, float* pose_grad, void* stream);

/* Camera-pose gradient of the Eikonal term (Sec. 3.3 Eq. eikonal_loss; Sec. 3.4 puts the poses
 * among the optimised parameters): pose_grad [F][6] += dloss[0] dL_eik/d xi, L_eik the mean over
 * the batch's free-space samples (counts[2] of them) of (1 - |grad_x phi(x_s)|)^2, as
 * gs_eikonal.  The samples x_s = o + d_s r move with the pose (depths and classes fixed) and
 * grad_x phi moves with them through its x-Hessian H_s = sum_{l,k} (d phi/d z_{l,k}) Hess_x
 * z_{l,k}: the off-diagonal entries h12, h13, h23 of the trilinear interpolation (Supp.
 * Sec. 1), times 1/v_l^2, zero along clamped axes.  With a_s = dL/d(grad_x phi(x_s)), each
 * sample's position gradient H_s a_s reaches the pose as in gs_pose_backward.  xi [F][6], the
 * frames (their poses the refined ones the batch was sampled with) and the batch (pix, origin,
 * dir, t, cls, counts) as for gs_pose_backward; dloss a device float [1] or NULL (1).  Either
 * architecture.  Accumulates with atomics.  With batch->eik set, each free-space sample's
 * d phi / d z is read from the records that gs_eikonal wrote on this batch (that call must come
 * first) instead of being evaluated here. */
gs_status gs_eikonal_pose_backward(gs_ctx* ctx, const float* theta, const gs_frames* frames, const float* xi,
                                   const gs_batch* batch, const float* dloss, float* pose_grad, void* stream);

/* Cell lookup used by every gather: out [P][4] = flat base-vertex index of the cell holding
 * x (clamped to the grid box) at each level, decided in binary32. */
gs_status gs_voxel_index(gs_ctx* ctx, const float* x, int32_t P, int64_t* out, void* stream);

/* Allocation-free variant of gs_forward_backward (the paper has no counterpart).  For callers
 * that may not allocate device memory -- e.g. code inside a host framework that owns every
 * device allocation (a plugin or custom operator that must draw from the framework's pool),
 * or a latency-critical loop that cannot take cudaMalloc's implicit device synchronisation.
 * It takes the configuration instead of a context and allocates nothing: the kernels'
 * per-CTA partial rows live in a file-scope device array of 3.04 MB (rows for 448 CTAs),
 * which every GPU that loads the library holds until the process exits.  Devices with more
 * than 320 SMs are rejected with GS_ERR_UNSUPPORTED.  Every call resolves the array's device
 * address on the current device (cudaGetSymbolAddress, no allocation); the first call on a
 * device may also load the library's device code, so make that first call before any stream
 * capture.  All calls share the array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and give wrong results.  Each call starts by clearing the array's
 * status word and writing its default dloss on the stream (so nothing depends on an earlier
 * call) and ends by writing NaN into all six loss entries if a device-side check of this call
 * failed (a bounded wait of the render kernel that ran out): without a context there is no
 * gs_sync_status, so a caller checks the losses it reads back.  Configurations are checked by
 * the same rules as gs_create (same status codes); FP32 form and GS_ARCH_COMPACT only
 * (GS_ERR_UNSUPPORTED otherwise).  Arguments, outputs and errors as gs_forward_backward;
 * messages via gs_last_error(NULL). */
gs_status gs_forward_backward_noalloc(const gs_config* cfg, const float* theta, const gs_batch* batch,
                                      const float* dloss, float* loss, float* grad, void* stream);

/* Synchronises the context's last stream and reports device-side check failures: GS_ERR_DEVICE
 * when a kernel's bounded wait for its tensor-core products ran out in an earlier call (the
 * kernel then stopped early and that call's outputs are incomplete); gs_last_error names the
 * kernel(s).  The status word is not cleared: the context stays in error. */
gs_status gs_sync_status(gs_ctx* ctx);

/* Host: message of the last error raised through this context ("" if none). */
const char* gs_last_error(gs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GOSURF_H */
