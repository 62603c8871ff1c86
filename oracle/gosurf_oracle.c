/*
 * GO-Surf (arXiv 2206.14735) -- plain FP64 CPU oracle of one optimisation step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this file's library.  It shares no code, header or table with the
 * CUDA library; both read the same seeded inputs.
 *
 * What it computes, in the paper's order:
 *   ray batch sampling over all pixels of all frames ............ Sec. 3.4 (Optimization)
 *   ray generation x_i = o + d_i r ............................... Sec. 3.2, Eq. (volume rendering)
 *   per-ray samples (stratified + depth-guided, see below) ....... Sec. 3.2 (sampler reading)
 *   bound b = D - d, near-surface / free-space split at t ........ Sec. 3.3
 *   multi-level trilinear features, concatenated coarse->fine .... Sec. 3.1, Eq. (SDF_MLP); Supp. Sec. 1 Eq. (trilinear, coefficient vector)
 *   geometry decoder phi = f_w(z), colour decoder ................ Sec. 3.1
 *   NeuS opacity alpha_i, transmittance T_i, weights w_i ......... Sec. 3.2, Eq. (volume_rendering_alpha)
 *   rendered colour / depth ...................................... Sec. 3.2, Eq. (volume_rendering)
 *   l_rgb, l_d, l_sdf, l_fs and their batch normalisations ....... Sec. 3.2-3.4
 *   l_smooth on near-surface points, grad_x phi .................. Sec. 3.3 Eq. (smoothness_loss); Supp. Sec. 1 Eq. (sdf_first_grad, jacobian)
 *   gradients (hand reverse mode, incl. d/dtheta of grad_x phi) .. Supp. Sec. 1 Eq. (second_order_theta)
 *   l_eik on the free-space samples (separate entry) ............. Sec. 3.3 Eq. (eikonal_loss), Sec. 3.4
 *   hierarchical importance sampler (separate entry) ............. Sec. 3.2 (3 x 12 from N_c = 96), Sec. 4
 *   mesh extraction from phi on a lattice (separate entry) ....... Sec. 4 (marching cubes at 1 cm; tetrahedra here)
 *   camera-pose refinement gradient (separate entry) ............. Sec. 3.4, Sec. 4 (t, so(3))
 *   the paper's architecture: colour grid W_beta (h_c = 6) at the
 *     finest level, colour decoder fed W_beta(x) and the viewing
 *     direction, decoders with two hidden layers of 32 (separate
 *     entry oc_step_paper) ..................................... Sec. 3.1 Eq. (COLOR_MLP), Architecture Details
 *   Adam ......................................................... Sec. 4 (Implementation Details)
 *
 * Precision: every quantity that decides an integer (pixel index, sample depths and their
 * order, sample class, voxel cell, clamp flags, smoothness-point positions) is computed in
 * IEEE binary32 with round-to-nearest and no contraction, exactly as the CUDA path does,
 * so those results are comparable bit for bit.  Everything after the FP32 sample position
 * is FP64.  Build with -ffp-contract=off and without fast-math.
 *
 * Readings where the paper is silent or ambiguous (each also listed in the design notes):
 *   - l_rgb is the squared Euclidean norm, averaged over all rays; l_d is |D - d_hat|
 *     averaged over rays with D > 0; L_sdf / L_fs / L_smooth are means over all points of
 *     their set in the batch (an empty set contributes 0).
 *   - S_tr = {|D-d| <= t}, S_fs = {D-d > t} (free space in front of the surface only);
 *     rays with D = 0 supervise no sample.
 *   - alpha_N = 0 (the last sample has no successor); the denominator is max(Phi_i, 1e-6).
 *   - s = exp(kappa) with kappa learnable.
 *   - Sub-gradients: 0 at every tie (ReLU at 0, max(.,0) at 0, |.| at 0); the free-space
 *     max picks the first maximal entry of (0, exp term, linear term).
 *   - L_eik is normalised like L_fs (mean over all free-space samples of the batch); its
 *     sub-gradient at grad_x phi = 0 is 0.
 *   - Samples outside the grid box are clamped to it; the clamped axes get zero x-derivative.
 *   - Sampling: N_s stratified samples over [near, far] plus N_g samples stratified over
 *     [D - g, D + g] when D > 0 (all N_s + N_g stratified otherwise), merged by depth
 *     with ties resolved stratified-first.
 *   - Geometry decoder 16 -> 32 (ReLU) -> 16 linear outputs [phi, h_1..h_15]; colour decoder
 *     15 -> 32 (ReLU) -> 3 with a sigmoid, fed by h.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_LEVELS 4
#define OC_FEAT 4
#define OC_Z (OC_LEVELS * OC_FEAT) /* 16 */
#define OC_H1 32
#define OC_OUT 16
#define OC_HF 15
#define OC_H2 32
#define OC_RGB 3
#define OC_MLP 1684

enum { CLS_NONE = 0, CLS_TR = 1, CLS_FS = 2 };

typedef struct {
  int32_t dims[OC_LEVELS][3]; /* vertex counts (nx, ny, nz), level 0 = coarsest */
  float voxel[OC_LEVELS];     /* voxel edge length (m) */
  float origin[3];            /* position of vertex (0,0,0) */
  int32_t n_strat, n_guided;
  float near_m, far_m;
  float guide_half; /* g: half width of the depth-guided band */
  float trunc;      /* t: truncation distance of the SDF bound */
  float kappa_fs;   /* exponent scale of the free-space penalty (5) */
  float lam[5];     /* rgb, depth, sdf, fs, smooth */
  int32_t n_smooth;
  float delta_s;
  int32_t arch; /* 0: the workload's decoders (16-32-16, 15-32-3); 1: the paper's architecture (oc_step_paper) */
} oc_config;

typedef struct {
  int32_t F, H, W;
  const uint8_t* rgb;
  const float* depth;
  const float* c2w; /* [F][3][4] row-major */
  float fx, fy, cx, cy;
} oc_frames;

/* the paper's architecture (oc_config.arch = 1), defined at the end of this file */
static void pa_query_sdf(const oc_config* c, const double* theta, const float* x, int P, double* sdf, double* grad);
static void pa_query_sdf_backward(const oc_config* c, const double* theta, const float* x, int P, const double* dsdf,
                                  const double* dgrad, double* grad);
static double pa_phi_at(const oc_config* c, const double* theta, const float x[3]);
static double pa_kappa(const oc_config* c, const double* theta);

/* ------------------------------------------------------------------------------------ */
/* counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)            */
/* ------------------------------------------------------------------------------------ */
static uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
/* one SplitMix64 output: the generator seeded with x returns oc_sm64(x + (k-1) * golden gamma) as its k-th value */
uint64_t oc_sm64(uint64_t x) { return sm64(x); }
/* key chain (seed, stream, step, index, slot) -> 64 random bits */
uint64_t oc_draw(uint64_t seed, uint64_t stream, uint64_t step, uint64_t index, uint64_t slot) {
  uint64_t h = sm64(seed);
  h = sm64(h ^ stream);
  h = sm64(h ^ step);
  h = sm64(h ^ index);
  return sm64(h ^ slot);
}
/* uniform in [0,1): top 24 bits scaled by 2^-24 (exact in binary32) */
static float unif24(uint64_t h) { return (float)(h >> 40) * 0x1p-24f; }

/* ------------------------------------------------------------------------------------ */
/* ray sampling (binary32)                                                                */
/* ------------------------------------------------------------------------------------ */
/* pixel -> camera ray with unit camera-z direction, so the ray parameter is z-depth */
static void pixel_ray(const oc_frames* fr, int64_t pix, float o[3], float r[3], float rgb[3], float* D) {
  int64_t hw = (int64_t)fr->H * fr->W;
  int64_t f = pix / hw, rem = pix % hw;
  int v = (int)(rem / fr->W), u = (int)(rem % fr->W);
  float dx = (((float)u + 0.5f) - fr->cx) / fr->fx;
  float dy = (((float)v + 0.5f) - fr->cy) / fr->fy;
  const float* P = fr->c2w + 12 * f;
  for (int a = 0; a < 3; ++a) {
    float t0 = P[4 * a + 0] * dx;
    float t1 = P[4 * a + 1] * dy;
    r[a] = (t0 + t1) + P[4 * a + 2];
    o[a] = P[4 * a + 3];
  }
  for (int j = 0; j < 3; ++j) rgb[j] = (float)fr->rgb[3 * pix + j] / 255.0f;
  *D = fr->depth[pix];
}

static int sample_class(float D, float t, float trunc) {
  if (!(D > 0.0f)) return CLS_NONE;
  float b = D - t;
  if (fabsf(b) <= trunc) return CLS_TR;
  if (b > trunc) return CLS_FS;
  return CLS_NONE;
}

/*
 * Draw R rays uniformly (with replacement) over all F*H*W pixels, including pixels with
 * missing depth, and N = n_strat + n_guided sorted sample depths per ray.
 * Outputs: pix[R], o[R,3], r[R,3], rgb[R,3], D[R], t[R,N], cls[R,N], counts[4] =
 * (rays with D>0, |S_tr|, |S_fs|, 0).
 */
void oc_sample_rays(const oc_config* c, const oc_frames* fr, uint64_t seed, uint32_t step, int R, int64_t* pix,
                    float* o, float* r, float* rgb, float* D, float* t, uint8_t* cls, int64_t* counts) {
  const int Ns = c->n_strat, Ng = c->n_guided, N = Ns + Ng;
  const int64_t npix = (int64_t)fr->F * fr->H * fr->W;
  float* ts = (float*)malloc(sizeof(float) * N);
  float* tg = (float*)malloc(sizeof(float) * (Ng > 0 ? Ng : 1));
  int64_t nd = 0, ntr = 0, nfs = 0;
  for (int i = 0; i < R; ++i) {
    uint64_t h = oc_draw(seed, 0, step, (uint64_t)i, 0);
    int64_t p = (int64_t)(h % (uint64_t)npix);
    pix[i] = p;
    float Di;
    pixel_ray(fr, p, o + 3 * i, r + 3 * i, rgb + 3 * i, &Di);
    D[i] = Di;
    float* ti = t + (size_t)i * N;
    if (Di > 0.0f) {
      ++nd;
      float delta = (c->far_m - c->near_m) / (float)Ns;
      for (int k = 0; k < Ns; ++k) {
        float u = unif24(oc_draw(seed, 0, step, (uint64_t)i, 1 + (uint64_t)k));
        ts[k] = c->near_m + ((float)k + u) * delta;
      }
      float g = c->guide_half;
      float gstep = (2.0f * g) / (float)Ng;
      float g0 = Di - g;
      for (int k = 0; k < Ng; ++k) {
        float u = unif24(oc_draw(seed, 0, step, (uint64_t)i, 1 + (uint64_t)Ns + (uint64_t)k));
        tg[k] = g0 + ((float)k + u) * gstep;
      }
      /* merge two ascending lists; ties keep the stratified sample first */
      int a = 0, b = 0;
      for (int k = 0; k < N; ++k) {
        if (b >= Ng || (a < Ns && ts[a] <= tg[b])) ti[k] = ts[a++];
        else ti[k] = tg[b++];
      }
    } else {
      float delta = (c->far_m - c->near_m) / (float)N;
      for (int k = 0; k < N; ++k) {
        float u = unif24(oc_draw(seed, 0, step, (uint64_t)i, 1 + (uint64_t)k));
        ti[k] = c->near_m + ((float)k + u) * delta;
      }
    }
    for (int k = 0; k < N; ++k) {
      int cl = sample_class(Di, ti[k], c->trunc);
      cls[(size_t)i * N + k] = (uint8_t)cl;
      ntr += cl == CLS_TR;
      nfs += cl == CLS_FS;
    }
  }
  counts[0] = nd;
  counts[1] = ntr;
  counts[2] = nfs;
  counts[3] = 0;
  free(ts);
  free(tg);
}

/*
 * Near-surface points S_g for the smoothness term: back-projected observed depth of a
 * random valid pixel (up to 8 draws), jittered uniformly by +-t per axis; perturbation
 * eps of length delta_s with a direction drawn by rejection in [-1,1]^3 (up to 16 draws,
 * x axis otherwise).  valid[p] = 0 when no valid pixel was drawn.
 */
void oc_sample_smooth(const oc_config* c, const oc_frames* fr, uint64_t seed, uint32_t step, int P, float* xs,
                      float* eps, uint8_t* valid, int64_t* n_valid) {
  const int64_t npix = (int64_t)fr->F * fr->H * fr->W;
  int64_t nv = 0;
  for (int p = 0; p < P; ++p) {
    int64_t px = -1;
    for (int tr = 0; tr < 8; ++tr) {
      uint64_t h = oc_draw(seed, 1, step, (uint64_t)p, (uint64_t)tr);
      int64_t q = (int64_t)(h % (uint64_t)npix);
      if (fr->depth[q] > 0.0f) { px = q; break; }
    }
    if (px < 0) {
      valid[p] = 0;
      for (int a = 0; a < 3; ++a) xs[3 * p + a] = eps[3 * p + a] = 0.0f;
      continue;
    }
    valid[p] = 1;
    ++nv;
    float o[3], r[3], rgb[3], D;
    pixel_ray(fr, px, o, r, rgb, &D);
    for (int a = 0; a < 3; ++a) {
      float u = unif24(oc_draw(seed, 1, step, (uint64_t)p, 16 + (uint64_t)a));
      float base = o[a] + D * r[a];
      float jit = c->trunc * (2.0f * u - 1.0f);
      xs[3 * p + a] = base + jit;
    }
    float v[3] = {1.0f, 0.0f, 0.0f}, n2 = 1.0f;
    for (int tr = 0; tr < 16; ++tr) {
      float w[3];
      for (int a = 0; a < 3; ++a) w[a] = 2.0f * unif24(oc_draw(seed, 1, step, (uint64_t)p, 32 + 3 * (uint64_t)tr + a)) - 1.0f;
      float q = (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2];
      if (q >= 0.01f && q <= 1.0f) {
        v[0] = w[0]; v[1] = w[1]; v[2] = w[2];
        n2 = q;
        break;
      }
    }
    float sc = c->delta_s / sqrtf(n2);
    for (int a = 0; a < 3; ++a) eps[3 * p + a] = v[a] * sc;
  }
  *n_valid = nv;
}

/* ------------------------------------------------------------------------------------ */
/* multi-level trilinear interpolation (Sec. 3.1; Supp. Sec. 1)                           */
/* ------------------------------------------------------------------------------------ */
static int64_t level_offset(const oc_config* c, int l) {
  int64_t o = 0;
  for (int k = 0; k < l; ++k) o += (int64_t)c->dims[k][0] * c->dims[k][1] * c->dims[k][2] * OC_FEAT;
  return o;
}
static int64_t grid_size(const oc_config* c) { return level_offset(c, OC_LEVELS); }

typedef struct {
  int64_t corner[8];  /* flat float index of feature 0 of corner c = 4*bx + 2*by + bz */
  double w[8];        /* w_c(f), Supp. Eq. (coefficient vector) */
  double dw[8][3];    /* d w_c / d f_a (zero on clamped axes), Supp. Eq. (coeff_jacobian) */
  double inv_v;       /* 1 / v_l  (d f / d x) */
  double f[3];        /* in-cell coordinates */
  int clamped[3];     /* axis a clamped to the grid box (no x-derivative along it) */
} cell_t;

/* Cell and in-cell coordinates of x at level l.  The cell and the clamp flags are decided
 * in binary32; the fractional coordinate is then taken in FP64. */
static void locate(const oc_config* c, int l, const float x[3], cell_t* cl, int32_t base_out[3]) {
  double f[3];
  int idx[3], clamped[3];
  for (int a = 0; a < 3; ++a) {
    int n = c->dims[l][a];
    float u = (x[a] - c->origin[a]) / c->voxel[l];
    clamped[a] = 0;
    if (u < 0.0f) { u = 0.0f; clamped[a] = 1; }
    else if (u > (float)(n - 1)) { u = (float)(n - 1); clamped[a] = 1; }
    int i = (int)floorf(u);
    if (i > n - 2) i = n - 2;
    idx[a] = i;
    if (clamped[a]) f[a] = (double)u - (double)i;
    else f[a] = ((double)x[a] - (double)c->origin[a]) / (double)c->voxel[l] - (double)i;
    if (base_out) base_out[a] = i;
    cl->f[a] = f[a];
    cl->clamped[a] = clamped[a];
  }
  int nx = c->dims[l][0], ny = c->dims[l][1];
  int64_t off = level_offset(c, l);
  for (int cc = 0; cc < 8; ++cc) {
    int bx = (cc >> 2) & 1, by = (cc >> 1) & 1, bz = cc & 1;
    int64_t vtx = ((int64_t)(idx[2] + bz) * ny + (idx[1] + by)) * nx + (idx[0] + bx);
    cl->corner[cc] = off + vtx * OC_FEAT;
    double wx = bx ? f[0] : 1.0 - f[0], wy = by ? f[1] : 1.0 - f[1], wz = bz ? f[2] : 1.0 - f[2];
    double sx = bx ? 1.0 : -1.0, sy = by ? 1.0 : -1.0, sz = bz ? 1.0 : -1.0;
    cl->w[cc] = wx * wy * wz;
    cl->dw[cc][0] = clamped[0] ? 0.0 : sx * wy * wz;
    cl->dw[cc][1] = clamped[1] ? 0.0 : wx * sy * wz;
    cl->dw[cc][2] = clamped[2] ? 0.0 : wx * wy * sz;
  }
  cl->inv_v = 1.0 / (double)c->voxel[l];
}

/* z[16] = [V^0(x), V^1(x), V^2(x), V^3(x)]; optional dz/dx [16][3] */
static void features(const oc_config* c, const double* theta, const float x[3], cell_t cells[OC_LEVELS],
                     double z[OC_Z], double dzdx[OC_Z][3]) {
  for (int l = 0; l < OC_LEVELS; ++l) {
    locate(c, l, x, &cells[l], NULL);
    for (int k = 0; k < OC_FEAT; ++k) {
      double s = 0, g[3] = {0, 0, 0};
      for (int cc = 0; cc < 8; ++cc) {
        double th = theta[cells[l].corner[cc] + k];
        s += cells[l].w[cc] * th;
        for (int a = 0; a < 3; ++a) g[a] += cells[l].dw[cc][a] * th;
      }
      z[OC_FEAT * l + k] = s;
      if (dzdx)
        for (int a = 0; a < 3; ++a) dzdx[OC_FEAT * l + k][a] = g[a] * cells[l].inv_v;
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* decoders                                                                               */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4, *kappa;
} mlp_t;

static mlp_t mlp_view(const double* base) {
  mlp_t m;
  m.W1 = base;
  m.b1 = m.W1 + OC_H1 * OC_Z;
  m.W2 = m.b1 + OC_H1;
  m.b2 = m.W2 + OC_OUT * OC_H1;
  m.W3 = m.b2 + OC_OUT;
  m.b3 = m.W3 + OC_H2 * OC_HF;
  m.W4 = m.b3 + OC_H2;
  m.b4 = m.W4 + OC_RGB * OC_H2;
  m.kappa = m.b4 + OC_RGB;
  return m;
}

typedef struct {
  double z[OC_Z];
  double zmag[OC_Z]; /* sum_c w_c |theta_c| per feature (feature_mag; diagnostics only) */
  double y1[OC_H1], a1[OC_H1];
  double out[OC_OUT]; /* out[0] = phi, out[1..15] = h */
  double y2[OC_H2], a2[OC_H2];
  double pre[OC_RGB], c[OC_RGB];
} act_t;

static double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }

static void decode(const mlp_t* m, act_t* A) {
  for (int j = 0; j < OC_H1; ++j) {
    double s = m->b1[j];
    for (int k = 0; k < OC_Z; ++k) s += m->W1[j * OC_Z + k] * A->z[k];
    A->y1[j] = s;
    A->a1[j] = s > 0 ? s : 0;
  }
  for (int j = 0; j < OC_OUT; ++j) {
    double s = m->b2[j];
    for (int k = 0; k < OC_H1; ++k) s += m->W2[j * OC_H1 + k] * A->a1[k];
    A->out[j] = s;
  }
  for (int j = 0; j < OC_H2; ++j) {
    double s = m->b3[j];
    for (int k = 0; k < OC_HF; ++k) s += m->W3[j * OC_HF + k] * A->out[1 + k];
    A->y2[j] = s;
    A->a2[j] = s > 0 ? s : 0;
  }
  for (int j = 0; j < OC_RGB; ++j) {
    double s = m->b4[j];
    for (int k = 0; k < OC_H2; ++k) s += m->W4[j * OC_H2 + k] * A->a2[k];
    A->pre[j] = s;
    A->c[j] = sigm(s);
  }
}

/* Distance of a hidden unit from its ReLU kink relative to the scale of the rounding error of
 * a binary32 evaluation of it: |y| / mag(y), with mag propagated layer by layer as a
 * root-sum-square of independent rounding errors, mag(y_j) = sqrt(b_j^2 + sum_i (W_ji
 * mag(x_i))^2), starting from the features' corner magnitudes zmag_k = sum_c w_c |theta_c,k|
 * (where corner values of opposite sign cancel, |z_k| is much smaller than the scale of its
 * binary32 rounding).  An inactive unit's output is exactly 0 and carries no rounding.  A unit
 * closer to its kink than OC_KINK_REL (about 170 units in the last place of mag) may take the
 * other branch in binary32 (reading R9 puts the sub-gradient at the kink itself; this only
 * flags the neighbourhood where binary32 cannot tell the sides apart).  Diagnostic only: no
 * result depends on it. */
#define OC_KINK_REL 1e-5
/* a flip that moves a sample's gradient contribution by less than this is below every
 * gradient tolerance of the parity tests, so only larger ones are flagged (as for alpha) */
#define OC_KINK_IMPACT 1e-9
static double kink_rel(double y, double mag) { return mag > 0 ? fabs(y) / mag : INFINITY; }

/* mag(y) of one dense layer: out[j] = sqrt(b_j^2 + sum_i (W_ji xmag_i)^2) for W [n][k] */
static void layer_mag(const double* W, const double* b, const double* xmag, int n, int k, double* out) {
  for (int j = 0; j < n; ++j) {
    double s = b[j] * b[j];
    for (int i = 0; i < k; ++i) s += (W[j * k + i] * xmag[i]) * (W[j * k + i] * xmag[i]);
    out[j] = sqrt(s);
  }
}

/* corner magnitudes of the features at a sample: zmag_k = sum_c w_c |theta_c,k| */
static void feature_mag(const double* theta, const cell_t cells[OC_LEVELS], double zmag[OC_Z]) {
  for (int l = 0; l < OC_LEVELS; ++l)
    for (int k = 0; k < OC_FEAT; ++k) {
      double s = 0;
      for (int cc = 0; cc < 8; ++cc) s += cells[l].w[cc] * fabs(theta[cells[l].corner[cc] + k]);
      zmag[OC_FEAT * l + k] = s;
    }
}

/* mag of the hidden units of both decoders (geometry layer 1, colour layer 1 fed by
 * h = out[1..15]) from A->zmag */
static void decode_mags(const mlp_t* m, const act_t* A, double mag1[OC_H1], double mag2[OC_H2]) {
  double am[OC_H1], om[OC_OUT];
  layer_mag(m->W1, m->b1, A->zmag, OC_H1, OC_Z, mag1);
  for (int j = 0; j < OC_H1; ++j) am[j] = A->y1[j] > 0 ? mag1[j] : 0.0;
  layer_mag(m->W2, m->b2, am, OC_OUT, OC_H1, om);
  layer_mag(m->W3, m->b3, om + 1, OC_H2, OC_HF, mag2);
}

/* smallest relative kink distance over the hidden units of both decoders */
static double decode_kink(const mlp_t* m, const act_t* A) {
  double mag1[OC_H1], mag2[OC_H2], r = INFINITY, v;
  decode_mags(m, A, mag1, mag2);
  for (int j = 0; j < OC_H1; ++j)
    if ((v = kink_rel(A->y1[j], mag1[j])) < r) r = v;
  for (int j = 0; j < OC_H2; ++j)
    if ((v = kink_rel(A->y2[j], mag2[j])) < r) r = v;
  return r;
}

/* max(1, max_i |W_i|, max_i |x_i|): the scale of what a unit's mask multiplies */
static double unit_scale(const double* W, const double* x, int k) {
  double s = 1.0;
  for (int i = 0; i < k; ++i) {
    if (fabs(W[i]) > s) s = fabs(W[i]);
    if (fabs(x[i]) > s) s = fabs(x[i]);
  }
  return s;
}

/* reverse mode of decode(): given dphi and dc, accumulate parameter grads into gm (MLP
 * block) and return dz.  flip (may be NULL; diagnostic): over the hidden units within
 * OC_KINK_REL of their kink, the largest |dL/d(unit output)| times unit_scale, i.e. how much
 * this sample's gradient would move if binary32 arithmetic took the unit's other branch. */
static void decode_backward(const mlp_t* m, const act_t* A, double dphi, const double dc[OC_RGB], double* gm,
                            double dz[OC_Z], double* flip) {
  double* gW1 = gm;
  double* gb1 = gW1 + OC_H1 * OC_Z;
  double* gW2 = gb1 + OC_H1;
  double* gb2 = gW2 + OC_OUT * OC_H1;
  double* gW3 = gb2 + OC_OUT;
  double* gb3 = gW3 + OC_H2 * OC_HF;
  double* gW4 = gb3 + OC_H2;
  double* gb4 = gW4 + OC_RGB * OC_H2;
  double dpre[OC_RGB], da2[OC_H2], dy2[OC_H2], dout[OC_OUT], da1[OC_H1], dy1[OC_H1];
  for (int j = 0; j < OC_RGB; ++j) dpre[j] = dc[j] * A->c[j] * (1.0 - A->c[j]);
  for (int j = 0; j < OC_RGB; ++j) {
    gb4[j] += dpre[j];
    for (int k = 0; k < OC_H2; ++k) gW4[j * OC_H2 + k] += dpre[j] * A->a2[k];
  }
  for (int k = 0; k < OC_H2; ++k) {
    double s = 0;
    for (int j = 0; j < OC_RGB; ++j) s += m->W4[j * OC_H2 + k] * dpre[j];
    da2[k] = s;
    dy2[k] = A->y2[k] > 0 ? s : 0;
  }
  for (int j = 0; j < OC_H2; ++j) {
    gb3[j] += dy2[j];
    for (int k = 0; k < OC_HF; ++k) gW3[j * OC_HF + k] += dy2[j] * A->out[1 + k];
  }
  dout[0] = dphi;
  for (int k = 0; k < OC_HF; ++k) {
    double s = 0;
    for (int j = 0; j < OC_H2; ++j) s += m->W3[j * OC_HF + k] * dy2[j];
    dout[1 + k] = s;
  }
  for (int j = 0; j < OC_OUT; ++j) {
    gb2[j] += dout[j];
    for (int k = 0; k < OC_H1; ++k) gW2[j * OC_H1 + k] += dout[j] * A->a1[k];
  }
  for (int k = 0; k < OC_H1; ++k) {
    double s = 0;
    for (int j = 0; j < OC_OUT; ++j) s += m->W2[j * OC_H1 + k] * dout[j];
    da1[k] = s;
    dy1[k] = A->y1[k] > 0 ? s : 0;
  }
  for (int j = 0; j < OC_H1; ++j) {
    gb1[j] += dy1[j];
    for (int k = 0; k < OC_Z; ++k) gW1[j * OC_Z + k] += dy1[j] * A->z[k];
  }
  for (int k = 0; k < OC_Z; ++k) {
    double s = 0;
    for (int j = 0; j < OC_H1; ++j) s += m->W1[j * OC_Z + k] * dy1[j];
    dz[k] = s;
  }
  if (flip) {
    double f = 0, mag1[OC_H1], mag2[OC_H2];
    decode_mags(m, A, mag1, mag2);
    for (int j = 0; j < OC_H2; ++j)
      if (kink_rel(A->y2[j], mag2[j]) < OC_KINK_REL) {
        double v = fabs(da2[j]) * unit_scale(m->W3 + j * OC_HF, A->out + 1, OC_HF);
        if (v > f) f = v;
      }
    for (int j = 0; j < OC_H1; ++j)
      if (kink_rel(A->y1[j], mag1[j]) < OC_KINK_REL) {
        double v = fabs(da1[j]) * unit_scale(m->W1 + j * OC_Z, A->z, OC_Z);
        if (v > f) f = v;
      }
    *flip = f;
  }
}

/* p = d phi / d z = W1^T (m (.) W2[0,:]^T), m = 1[y1 > 0] (ReLU => piecewise linear) */
static void dphi_dz(const mlp_t* m, const act_t* A, double p[OC_Z], double mw2[OC_H1]) {
  for (int j = 0; j < OC_H1; ++j) mw2[j] = A->y1[j] > 0 ? m->W2[j] : 0.0; /* row 0 of W2 */
  for (int k = 0; k < OC_Z; ++k) {
    double s = 0;
    for (int j = 0; j < OC_H1; ++j) s += m->W1[j * OC_Z + k] * mw2[j];
    p[k] = s;
  }
}

/* ------------------------------------------------------------------------------------ */
/* query: phi(x) and grad_x phi(x) (Supp. Eq. sdf_first_grad)                            */
/* ------------------------------------------------------------------------------------ */
void oc_query_sdf(const oc_config* c, const double* theta, const float* x, int P, double* sdf, double* grad) {
  if (c->arch == 1) {
    pa_query_sdf(c, theta, x, P, sdf, grad);
    return;
  }
  mlp_t m = mlp_view(theta + grid_size(c));
#pragma omp parallel for schedule(static)
  for (int i = 0; i < P; ++i) {
    cell_t cells[OC_LEVELS];
    act_t A;
    double dzdx[OC_Z][3];
    features(c, theta, x + 3 * i, cells, A.z, dzdx);
    decode(&m, &A);
    sdf[i] = A.out[0];
    if (grad) {
      double p[OC_Z], mw2[OC_H1];
      dphi_dz(&m, &A, p, mw2);
      for (int a = 0; a < 3; ++a) {
        double s = 0;
        for (int k = 0; k < OC_Z; ++k) s += p[k] * dzdx[k][a];
        grad[3 * i + a] = s;
      }
    }
  }
}

/* Reverse mode of oc_query_sdf with respect to theta (grid and decoders):
 *   grad += sum_i dsdf_i d phi(x_i)/d theta + dgrad_i . d grad_x phi(x_i)/d theta.
 * The first term is the ordinary backward pass of the SDF decoder and the trilinear gather
 * (Sec. 3.1).  The second is the second-order path of Supp. Sec. 1: with p = d phi/d z and
 * a = dgrad_i, a . grad_x phi = sum_k p_k j_k where j_k = a . d z_k / d x, so
 *   d/d theta_{l,c,f} = p_{l,f} (1/v_l) (a . d w_c / d f)      (grid, through d z / d x),
 *   d/d W1[h][k] = m_h W2[0][h] j_k,   d/d W2[0][h] = m_h (W1 j)_h  (decoder, through p),
 * with m the layer-1 ReLU mask; p does not otherwise depend on theta (the decoder is
 * piecewise linear in z).  dsdf or dgrad may be NULL (zero).  x is not differentiated. */
void oc_query_sdf_backward(const oc_config* c, const double* theta, const float* x, int P, const double* dsdf,
                           const double* dgrad, double* grad) {
  if (c->arch == 1) {
    pa_query_sdf_backward(c, theta, x, P, dsdf, dgrad, grad);
    return;
  }
  const int64_t ng = grid_size(c);
  mlp_t m = mlp_view(theta + ng);
  double* gm = grad + ng;
  for (int i = 0; i < P; ++i) {
    cell_t cells[OC_LEVELS];
    act_t A;
    double dzdx[OC_Z][3];
    features(c, theta, x + 3 * i, cells, A.z, dzdx);
    decode(&m, &A);
    if (dsdf && dsdf[i] != 0.0) {
      const double dc[OC_RGB] = {0, 0, 0};
      double dz[OC_Z];
      decode_backward(&m, &A, dsdf[i], dc, gm, dz, NULL);
      for (int l = 0; l < OC_LEVELS; ++l)
        for (int cc = 0; cc < 8; ++cc)
          for (int f = 0; f < OC_FEAT; ++f) grad[cells[l].corner[cc] + f] += cells[l].w[cc] * dz[OC_FEAT * l + f];
    }
    if (dgrad) {
      const double* av = dgrad + 3 * i;
      double p[OC_Z], mw2[OC_H1], jv[OC_Z];
      dphi_dz(&m, &A, p, mw2);
      for (int k = 0; k < OC_Z; ++k) jv[k] = av[0] * dzdx[k][0] + av[1] * dzdx[k][1] + av[2] * dzdx[k][2];
      for (int l = 0; l < OC_LEVELS; ++l)
        for (int cc = 0; cc < 8; ++cc) {
          const double ad =
              (av[0] * cells[l].dw[cc][0] + av[1] * cells[l].dw[cc][1] + av[2] * cells[l].dw[cc][2]) * cells[l].inv_v;
          for (int f = 0; f < OC_FEAT; ++f) grad[cells[l].corner[cc] + f] += p[OC_FEAT * l + f] * ad;
        }
      double* gW1 = gm;
      double* gW2 = gm + OC_H1 * OC_Z + OC_H1; /* row 0 of W2 */
      for (int h = 0; h < OC_H1; ++h) {
        if (!(A.y1[h] > 0)) continue;
        double w1j = 0;
        for (int k = 0; k < OC_Z; ++k) {
          gW1[h * OC_Z + k] += m.W2[h] * jv[k];
          w1j += m.W1[h * OC_Z + k] * jv[k];
        }
        gW2[h] += w1j;
      }
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Eikonal term (Sec. 3.3 Eq. eikonal_loss; batch normalisation Sec. 3.4)                */
/* ------------------------------------------------------------------------------------ */
/* L_eik = mean over the free-space samples S_fs of the batch of (1 - |grad_x phi(x_s)|)^2,
 * the same set and the same normalisation as L_fs (0 when S_fs is empty).  The points are
 * the main samples x_s = o + d_s r, formed in binary32 exactly as in oc_step.
 * With grad != NULL: grad += dscale dL_eik/dtheta.  For one point, with g = grad_x phi,
 *   d l / d g = -2 (1 - |g|) g / |g|        (taken as 0 where |g| = 0),
 * and the rest is the reverse mode of grad_x phi with respect to theta (oc_query_sdf_backward
 * with that adjoint; x carries no gradient).  gnorm [R][N] (may be NULL) receives |g| at the
 * free-space samples and -1 elsewhere.  Returns |S_fs|, or -1 on a bad argument. */
int64_t oc_eikonal(const oc_config* c, const double* theta, int R, int N, const float* o, const float* r,
                   const float* t, const uint8_t* cls, double dscale, double* loss, double* grad, double* gnorm) {
  if (R < 0 || N < 1 || !loss) return -1;
  int64_t n_fs = 0;
  for (int64_t s = 0; s < (int64_t)R * N; ++s) n_fs += cls[s] == CLS_FS;
  *loss = 0.0;
  if (gnorm)
    for (int64_t s = 0; s < (int64_t)R * N; ++s) gnorm[s] = -1.0;
  if (n_fs == 0) return 0;
  float* x = (float*)malloc(sizeof(float) * 3 * (size_t)n_fs);
  int64_t* at = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_fs);
  double* sdf = (double*)malloc(sizeof(double) * (size_t)n_fs);
  double* g = (double*)malloc(sizeof(double) * 3 * (size_t)n_fs);
  int64_t q = 0;
  for (int i = 0; i < R; ++i)
    for (int k = 0; k < N; ++k) {
      const int64_t s = (int64_t)i * N + k;
      if (cls[s] != CLS_FS) continue;
      for (int a = 0; a < 3; ++a) {
        float step_ = t[s] * r[3 * i + a];
        x[3 * q + a] = o[3 * i + a] + step_;
      }
      at[q++] = s;
    }
  oc_query_sdf(c, theta, x, (int)n_fs, sdf, g);
  double sum = 0.0;
  for (int64_t p = 0; p < n_fs; ++p) {
    const double nrm = sqrt(g[3 * p] * g[3 * p] + g[3 * p + 1] * g[3 * p + 1] + g[3 * p + 2] * g[3 * p + 2]);
    sum += (1.0 - nrm) * (1.0 - nrm);
    if (gnorm) gnorm[at[p]] = nrm;
    /* the adjoint of g, kept in g */
    const double k = nrm > 0.0 ? dscale * (-2.0 / (double)n_fs) * (1.0 - nrm) / nrm : 0.0;
    for (int a = 0; a < 3; ++a) g[3 * p + a] *= k;
  }
  *loss = sum / (double)n_fs;
  if (grad) oc_query_sdf_backward(c, theta, x, (int)n_fs, NULL, g, grad);
  free(x);
  free(at);
  free(sdf);
  free(g);
  return n_fs;
}

/* ------------------------------------------------------------------------------------ */
/* mesh extraction (Sec. 4: the meshes are extracted from phi on a 1 cm lattice)          */
/* ------------------------------------------------------------------------------------ */
/* Lattice point (i, j, k) sits at lo + (i, j, k) * step (binary32, two roundings per axis);
 * phi there in FP64.  Each lattice cell is split into 6 tetrahedra around its diagonal from
 * corner 0 to corner 7 (corner c at offset (c & 1, (c >> 1) & 1, c >> 2)); a tetrahedron with
 * 1 or 3 corners below iso yields one triangle, with 2 below two, their vertices on the
 * tetrahedron's edges where the linear interpolation of phi equals iso.  An edge's point is
 * interpolated from its endpoint of lower lattice index, so that cells and tetrahedra that
 * share an edge produce the same point.  Triangles are oriented with their normal towards
 * the tetrahedron's corners above iso (increasing phi, out of the surface).
 * tris [max_tris][3][3] receives the first max_tris triangles, cells in x-fastest order;
 * phi_out [nz][ny][nx] (may be NULL) the lattice values.  Returns the number of triangles. */
static const int oc_tets[6][4] = {{0, 1, 3, 7}, {0, 3, 2, 7}, {0, 2, 6, 7}, {0, 6, 4, 7}, {0, 4, 5, 7}, {0, 5, 1, 7}};

static void mesh_edge(const double P[8][3], const double f[8], const int64_t id[8], int a, int b, double iso,
                      double out[3]) {
  if (id[b] < id[a]) { int t = a; a = b; b = t; }
  const double w = (iso - f[a]) / (f[b] - f[a]);
  for (int q = 0; q < 3; ++q) out[q] = P[a][q] + w * (P[b][q] - P[a][q]);
}

static int64_t mesh_emit(double* tris, int64_t max_tris, int64_t n, const double p0[3], const double p1[3],
                         const double p2[3], const double dir[3]) {
  double e1[3], e2[3], nrm[3];
  for (int q = 0; q < 3; ++q) { e1[q] = p1[q] - p0[q]; e2[q] = p2[q] - p0[q]; }
  nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
  nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
  nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const int flip = nrm[0] * dir[0] + nrm[1] * dir[1] + nrm[2] * dir[2] < 0.0;
  if (n < max_tris) {
    double* t = tris + 9 * n;
    for (int q = 0; q < 3; ++q) {
      t[q] = p0[q];
      t[3 + q] = flip ? p2[q] : p1[q];
      t[6 + q] = flip ? p1[q] : p2[q];
    }
  }
  return n + 1;
}

int64_t oc_extract_mesh(const oc_config* c, const double* theta, const float lo[3], float step, int nx, int ny, int nz,
                        double iso, double* tris, int64_t max_tris, double* phi_out) {
  if (nx < 2 || ny < 2 || nz < 2) return 0;
  const int64_t np = (int64_t)nx * ny * nz;
  float* x = (float*)malloc(sizeof(float) * 3 * (size_t)np);
  double* phi = phi_out ? phi_out : (double*)malloc(sizeof(double) * (size_t)np);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int64_t id = ((int64_t)k * ny + j) * nx + i;
        const int ijk[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          float d = (float)ijk[a] * step;
          x[3 * id + a] = lo[a] + d;
        }
      }
  /* phi by the pinned SDF query, in chunks (its P is an int) */
  for (int64_t s0 = 0; s0 < np; s0 += (1 << 24)) {
    const int64_t cnt = np - s0 < (1 << 24) ? np - s0 : (1 << 24);
    oc_query_sdf(c, theta, x + 3 * s0, (int)cnt, phi + s0, NULL);
  }
  int64_t n = 0;
  for (int k = 0; k + 1 < nz; ++k)
    for (int j = 0; j + 1 < ny; ++j)
      for (int i = 0; i + 1 < nx; ++i) {
        double P[8][3], f[8];
        int64_t id[8];
        for (int cc = 0; cc < 8; ++cc) {
          id[cc] = ((int64_t)(k + (cc >> 2)) * ny + (j + ((cc >> 1) & 1))) * nx + (i + (cc & 1));
          for (int a = 0; a < 3; ++a) P[cc][a] = (double)x[3 * id[cc] + a];
          f[cc] = phi[id[cc]];
        }
        for (int tt = 0; tt < 6; ++tt) {
          const int* v = oc_tets[tt];
          int in[4], out[4], ni = 0, no = 0;
          for (int q = 0; q < 4; ++q) {
            if (f[v[q]] < iso) in[ni++] = v[q];
            else out[no++] = v[q];
          }
          if (ni == 0 || no == 0) continue;
          double dir[3] = {0, 0, 0};
          for (int a = 0; a < 3; ++a) {
            for (int q = 0; q < no; ++q) dir[a] += P[out[q]][a] / no;
            for (int q = 0; q < ni; ++q) dir[a] -= P[in[q]][a] / ni;
          }
          double p0[3], p1[3], p2[3], p3[3];
          if (ni == 1 || no == 1) {
            const int apex = ni == 1 ? in[0] : out[0];
            const int* rest = ni == 1 ? out : in;
            mesh_edge(P, f, id, apex, rest[0], iso, p0);
            mesh_edge(P, f, id, apex, rest[1], iso, p1);
            mesh_edge(P, f, id, apex, rest[2], iso, p2);
            n = mesh_emit(tris, max_tris, n, p0, p1, p2, dir);
          } else { /* two below, two above: the quad in0-out0, in0-out1, in1-out1, in1-out0 */
            mesh_edge(P, f, id, in[0], out[0], iso, p0);
            mesh_edge(P, f, id, in[0], out[1], iso, p1);
            mesh_edge(P, f, id, in[1], out[1], iso, p2);
            mesh_edge(P, f, id, in[1], out[0], iso, p3);
            n = mesh_emit(tris, max_tris, n, p0, p1, p2, dir);
            n = mesh_emit(tris, max_tris, n, p0, p2, p3, dir);
          }
        }
      }
  free(x);
  if (!phi_out) free(phi);
  return n;
}

/* base vertex (cell) index per level, binary32 decision; out [P][4] flat vertex ids */
void oc_voxel_index(const oc_config* c, const float* x, int P, int64_t* out) {
  for (int i = 0; i < P; ++i)
    for (int l = 0; l < OC_LEVELS; ++l) {
      cell_t cl;
      int32_t b[3];
      locate(c, l, x + 3 * i, &cl, b);
      out[(size_t)OC_LEVELS * i + l] = ((int64_t)b[2] * c->dims[l][1] + b[1]) * c->dims[l][0] + b[0];
    }
}

/* trilinear pieces of one cell, for tests of Supp. Sec. 1: w[8], J[8][3] at f */
void oc_trilinear_coeffs(const double f[3], double w[8], double J[8][3]) {
  for (int cc = 0; cc < 8; ++cc) {
    int bx = (cc >> 2) & 1, by = (cc >> 1) & 1, bz = cc & 1;
    double wx = bx ? f[0] : 1 - f[0], wy = by ? f[1] : 1 - f[1], wz = bz ? f[2] : 1 - f[2];
    w[cc] = wx * wy * wz;
    J[cc][0] = (bx ? 1.0 : -1.0) * wy * wz;
    J[cc][1] = wx * (by ? 1.0 : -1.0) * wz;
    J[cc][2] = wx * wy * (bz ? 1.0 : -1.0);
  }
}

/* second x-derivatives of f = theta^T w(x) in cell coordinates: the off-diagonal entries
 * h12, h13, h23 (the diagonal is zero), obtained by differentiating each column of J
 * once more; used by the pose-refinement path and by tests */
void oc_trilinear_hessian(const double theta8[8], const double f[3], double h[3]) {
  double H[3][3] = {{0}};
  for (int cc = 0; cc < 8; ++cc) {
    int b[3] = {(cc >> 2) & 1, (cc >> 1) & 1, cc & 1};
    double lin[3], sgn[3];
    for (int a = 0; a < 3; ++a) {
      lin[a] = b[a] ? f[a] : 1 - f[a];
      sgn[a] = b[a] ? 1.0 : -1.0;
    }
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) {
        if (a == d) continue;
        int e = 3 - a - d;
        H[a][d] += theta8[cc] * sgn[a] * sgn[d] * lin[e];
      }
  }
  h[0] = H[0][1];
  h[1] = H[0][2];
  h[2] = H[1][2];
}

/* ------------------------------------------------------------------------------------ */
/* volume rendering along one ray (Sec. 3.2, Eq. volume_rendering / volume_rendering_alpha) */
/* ------------------------------------------------------------------------------------ */
/* Phi_i = sigma_s(phi_i) = 1/(1+exp(-s phi_i));
 * alpha_i = max((Phi_i - Phi_{i+1}) / max(Phi_i, 1e-6), 0) for i < N, alpha_N = 0;
 * T_i = prod_{j<i} (1 - alpha_j);  w_i = T_i alpha_i;
 * c_hat = sum_i w_i c_i;  d_hat = sum_i w_i d_i;  wsum = sum_i w_i. */
static void composite(int N, const double* phi, double s, const act_t* A, const float* d, double* Phi,
                      double* alpha, double* T, double* w, double ch[3], double* dh, double* ws) {
  for (int k = 0; k < N; ++k) Phi[k] = sigm(s * phi[k]);
  for (int k = 0; k < N; ++k) {
    if (k == N - 1) {
      alpha[k] = 0;
      continue;
    }
    double den = Phi[k] > 1e-6 ? Phi[k] : 1e-6;
    double q = (Phi[k] - Phi[k + 1]) / den;
    alpha[k] = q > 0 ? q : 0;
  }
  double Tk = 1.0;
  ch[0] = ch[1] = ch[2] = 0;
  *dh = 0;
  *ws = 0;
  for (int k = 0; k < N; ++k) {
    T[k] = Tk;
    w[k] = Tk * alpha[k];
    if (A)
      for (int j = 0; j < 3; ++j) ch[j] += w[k] * A[k].c[j];
    *dh += w[k] * (double)d[k];
    *ws += w[k];
    Tk *= 1.0 - alpha[k];
  }
}

/* test access to the renderer alone: phi[N], d[N] -> alpha[N], T[N], w[N], d_hat, wsum */
void oc_composite(int N, const double* phi, double s, const float* d, double* alpha, double* T, double* w,
                  double* d_hat, double* wsum) {
  double* Phi = (double*)malloc(sizeof(double) * N);
  double ch[3];
  composite(N, phi, s, NULL, d, Phi, alpha, T, w, ch, d_hat, wsum);
  free(Phi);
}

/* ------------------------------------------------------------------------------------ */
/* one optimisation step: losses (Sec. 3.2-3.4) and their gradients                     */
/* ------------------------------------------------------------------------------------ */
static double sgn(double v) { return v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0); }

/* margins[10]: distance of this evaluation from every branch point, for gradient tests:
 *  0 min |hidden pre-activation| (both decoders, main samples and smoothness points)
 *  1 min |Phi_i - Phi_{i+1}| / max(Phi_i,1e-6) over i < N (unsaturated, untied samples)
 *  2 min |Phi_i - 1e-6|
 *  3 min |phi - b| over S_tr
 *  4 min gap between the largest and second largest entry of the free-space max over S_fs
 *  5 min |d_hat - D| over rays with D > 0
 *  6 min |hidden pre-activation| at smoothness points (also folded into 0)
 *  7 signature of every branch decision taken (52-bit hash, as a double): two
 *    evaluations with equal signatures lie on the same smooth piece of the loss
 *  8 largest change of dL/dphi that flipping an ambiguous alpha > 0 decision would cause,
 *    over samples with |q| < 1e-6 (a binary32 evaluation may decide those either way)
 *  9 unused (0) */
typedef struct {
  double m[10];
  uint64_t sig;
} margins_t;
static void sigmix(uint64_t* sig, uint64_t id, uint64_t val) { *sig ^= sm64(id * 0x9E3779B97F4A7C15ULL + val); }
static uint64_t relu_mask(const double* y, int n) {
  uint64_t b = 0;
  for (int j = 0; j < n; ++j) b |= (uint64_t)(y[j] > 0) << j;
  return b;
}
static void mmin(double* a, double v) {
  v = fabs(v);
  if (v < *a) *a = v;
}

/*
 * Forward (and, if grad != NULL, backward) of one step on a given batch.
 * theta: flat parameters (grid levels 0..3 as [nz][ny][nx][4], then the 1684-entry
 * decoder block W1,b1,W2,b2,W3,b3,W4,b4,kappa).  Batch arrays as produced by the samplers.
 * dloss[6]: upstream derivative of each output (rgb, depth, sdf, fs, smooth, total); the
 * effective weight of term k is dloss[k] + lam[k] * dloss[5].  NULL means (0,..,0,1).
 * loss[6]: L_rgb, L_d, L_sdf, L_fs, L_smooth, total.  rgb_hat[R,3], d_hat[R], wsum[R] may be
 * NULL.  grad: same layout as theta, overwritten.  margins[10] may be NULL.
 * amb [R,N] (may be NULL) flags the samples whose branch decisions lie within binary32
 * rounding of a tie: bit 0 the alpha_k > 0 decision (|q_k| < 1e-5, unsaturated, untied),
 * bit 1 the sign of phi - b on S_tr (|phi - b| < 2e-5), bit 2 the free-space max (gap < 2e-5),
 * bit 3 a hidden unit of either decoder within OC_KINK_REL (relative) of its ReLU kink whose
 * flip would move the sample's gradient by more than OC_KINK_IMPACT (gradients requested),
 * bit 4 (on the ray's first sample) the sign of d_hat - D (|d_hat - D| < 1e-5 max(D, 1)).
 * Bit 0 is set only when gradients are requested and a flip would change dL/dphi by more
 * than 1e-7.  w_out [R,N] (may be NULL) receives the rendering weights w_i = T_i alpha_i.
 * Returns 0, or -1 on a bad argument.
 */
static int step_impl(const oc_config* c, const double* theta, int R, int N, const float* o, const float* r,
                     const float* rgb, const float* D, const float* t, const uint8_t* cls, int P, const float* xs,
                     const float* eps, const uint8_t* valid, const double* dloss, double* loss, double* rgb_hat,
                     double* d_hat, double* wsum, double* grad, double* margins, uint8_t* amb, double* w_out,
                     double* dz_out) {
  if (R < 0 || N < 2 || P < 0) return -1;
  const int64_t ng = grid_size(c);
  mlp_t m = mlp_view(theta + ng);
  const double s = exp(*m.kappa);

  /* set sizes for the batch normalisations */
  int64_t n_d = 0, n_tr = 0, n_fs = 0, n_g = 0;
  for (int i = 0; i < R; ++i) {
    n_d += D[i] > 0.0f;
    for (int k = 0; k < N; ++k) {
      n_tr += cls[(size_t)i * N + k] == CLS_TR;
      n_fs += cls[(size_t)i * N + k] == CLS_FS;
    }
  }
  for (int p = 0; p < P; ++p) n_g += valid[p] != 0;

  double wt[5];
  for (int k = 0; k < 5; ++k) wt[k] = dloss ? dloss[k] + (double)c->lam[k] * dloss[5] : (double)c->lam[k];
  if (amb) memset(amb, 0, (size_t)R * N);
  const int do_grad = grad != NULL;

  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  double* gm_all = (double*)calloc((size_t)nthreads * OC_MLP, sizeof(double));
  double* lsum_all = (double*)calloc((size_t)nthreads * 5, sizeof(double));
  margins_t* mg_all = (margins_t*)malloc(sizeof(margins_t) * nthreads);
  for (int th = 0; th < nthreads; ++th) {
    for (int k = 0; k < 10; ++k) mg_all[th].m[k] = INFINITY;
    mg_all[th].m[8] = 0.0;
    mg_all[th].m[9] = 0.0;
    mg_all[th].sig = 0;
  }
  /* per-sample dL/dz, scattered into the grid afterwards in sample order */
  double* dz_all = do_grad ? (double*)malloc(sizeof(double) * (size_t)R * N * OC_Z) : NULL;
  double* dzs_all = do_grad ? (double*)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1) * 2 * 8 * OC_LEVELS * OC_FEAT) : NULL;

#pragma omp parallel
  {
    int th = 0;
#ifdef _OPENMP
    th = omp_get_thread_num();
#endif
    double* gm = gm_all + (size_t)th * OC_MLP;
    double* lsum = lsum_all + (size_t)th * 5;
    margins_t* mg = mg_all + th;
    act_t* A = (act_t*)malloc(sizeof(act_t) * N);
    cell_t* cells = (cell_t*)malloc(sizeof(cell_t) * N * OC_LEVELS);
    double *phi = malloc(sizeof(double) * N), *Phi = malloc(sizeof(double) * N), *alpha = malloc(sizeof(double) * N),
           *T = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N), *U = malloc(sizeof(double) * N),
           *dPhi = malloc(sizeof(double) * N);

#pragma omp for schedule(static)
    for (int i = 0; i < R; ++i) {
      const float* ti = t + (size_t)i * N;
      /* samples x_i = o + d_i r (binary32), features, decoders */
      for (int k = 0; k < N; ++k) {
        float x[3];
        for (int a = 0; a < 3; ++a) {
          float step_ = ti[k] * r[3 * i + a];
          x[a] = o[3 * i + a] + step_;
        }
        features(c, theta, x, cells + (size_t)k * OC_LEVELS, A[k].z, NULL);
        feature_mag(theta, cells + (size_t)k * OC_LEVELS, A[k].zmag);
        decode(&m, &A[k]);
        phi[k] = A[k].out[0];
        for (int j = 0; j < OC_H1; ++j) mmin(&mg->m[0], A[k].y1[j]);
        for (int j = 0; j < OC_H2; ++j) mmin(&mg->m[0], A[k].y2[j]);
        uint64_t sid = ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8;
        sigmix(&mg->sig, sid + 0, relu_mask(A[k].y1, OC_H1));
        sigmix(&mg->sig, sid + 1, relu_mask(A[k].y2, OC_H2));
      }
      /* NeuS weights and expected colour / depth (Sec. 3.2) */
      double ch[3], dh, ws;
      composite(N, phi, s, A, ti, Phi, alpha, T, w, ch, &dh, &ws);
      for (int k = 0; k + 1 < N; ++k) {
        double den = Phi[k] > 1e-6 ? Phi[k] : 1e-6;
        /* a flip of the alpha > 0 branch changes dphi by about s (1 - Phi_k) |dL/dalpha|, so
         * saturated samples (1 - Phi_k < 1e-5) and exact ties (equal phi) are not counted */
        if (phi[k] != phi[k + 1] && 1.0 - Phi[k] > 1e-5) {
          double q = (Phi[k] - Phi[k + 1]) / den;
          mmin(&mg->m[1], q);

        }
        mmin(&mg->m[2], Phi[k] - 1e-6);
        uint64_t sid = ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8;
        sigmix(&mg->sig, sid + 2, (uint64_t)(alpha[k] > 0) | (uint64_t)(Phi[k] > 1e-6) << 1);
      }
      if (rgb_hat)
        for (int j = 0; j < 3; ++j) rgb_hat[3 * i + j] = ch[j];
      if (d_hat) d_hat[i] = dh;
      if (wsum) wsum[i] = ws;
      if (w_out)
        for (int k = 0; k < N; ++k) w_out[(size_t)i * N + k] = w[k];
      /* rendering losses */
      double lr = 0;
      for (int j = 0; j < 3; ++j) {
        double e = (double)rgb[3 * i + j] - ch[j];
        lr += e * e;
      }
      lsum[0] += lr;
      const double Di = (double)D[i];
      if (D[i] > 0.0f) {
        lsum[1] += fabs(Di - dh);
        mmin(&mg->m[5], dh - Di);
        /* the sign of d_hat - D decides the sign of every sample's depth gradient; a binary32
         * d_hat (a sum of N products w_k t_k) errs by up to about N ulps of D */
        if (amb && fabs(dh - Di) < 1e-5 * (Di > 1.0 ? Di : 1.0)) amb[(size_t)i * N] |= 16;
        sigmix(&mg->sig, ((uint64_t)i * (uint64_t)N) * 8 + 7, (uint64_t)(dh > Di));
      }
      /* approximate SDF supervision (Sec. 3.3) */
      for (int k = 0; k < N; ++k) {
        int cl = cls[(size_t)i * N + k];
        double b = Di - (double)ti[k];
        if (cl == CLS_TR) {
          lsum[2] += fabs(phi[k] - b);
          mmin(&mg->m[3], phi[k] - b);
          if (amb && fabs(phi[k] - b) < 2e-5) amb[(size_t)i * N + k] |= 2;
          sigmix(&mg->sig, ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8 + 3, (uint64_t)(phi[k] > b));
        } else if (cl == CLS_FS) {
          double e = exp(-(double)c->kappa_fs * phi[k]) - 1.0, lin = phi[k] - b;
          double v[3] = {0.0, e, lin};
          int arg = 0;
          for (int q = 1; q < 3; ++q)
            if (v[q] > v[arg]) arg = q;
          double top = v[arg], second = -INFINITY;
          for (int q = 0; q < 3; ++q)
            if (q != arg && v[q] > second) second = v[q];
          mmin(&mg->m[4], top - second);
          if (amb && top - second < 2e-5) amb[(size_t)i * N + k] |= 4;
          sigmix(&mg->sig, ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8 + 4, (uint64_t)arg);
          lsum[3] += top;
        }
      }
      if (!do_grad) continue;

      /* ---------------- backward ---------------- */
      double gc[3], gd = 0;
      for (int j = 0; j < 3; ++j) gc[j] = wt[0] / (double)R * 2.0 * (ch[j] - (double)rgb[3 * i + j]);
      if (D[i] > 0.0f && n_d > 0) gd = wt[1] / (double)n_d * sgn(dh - Di);
      /* dL/dalpha_k = T_k (e_k - U_k), U_{N-1} = 0, U_{k-1} = alpha_k e_k + (1 - alpha_k) U_k */
      U[N - 1] = 0;
      for (int k = N - 1; k >= 1; --k) {
        double ek = gc[0] * A[k].c[0] + gc[1] * A[k].c[1] + gc[2] * A[k].c[2] + gd * (double)ti[k];
        U[k - 1] = alpha[k] * ek + (1.0 - alpha[k]) * U[k];
      }
      for (int k = 0; k < N; ++k) dPhi[k] = 0;
      for (int k = 0; k < N - 1; ++k) {
        double ek = gc[0] * A[k].c[0] + gc[1] * A[k].c[1] + gc[2] * A[k].c[2] + gd * (double)ti[k];
        double dalpha = T[k] * (ek - U[k]);
        double den = Phi[k] > 1e-6 ? Phi[k] : 1e-6;
        double q = (Phi[k] - Phi[k + 1]) / den;
        if (fabs(q) < 1e-5 && phi[k] != phi[k + 1] && 1.0 - Phi[k] > 1e-5) {
          double self = fabs(dalpha) * s * Phi[k] * (1.0 - Phi[k]) / den;
          double next = fabs(dalpha) * s * Phi[k + 1] * (1.0 - Phi[k + 1]) / den;
          double imp = self > next ? self : next;
          if (fabs(q) < 1e-6 && imp > mg->m[8]) mg->m[8] = imp;
          /* binary32 decides sign(Phi_k - Phi_k+1) = sign(phi_k - phi_k+1) reliably once the
           * two SDF values differ by more than a few ulps */
          double dphi_rel = fabs(phi[k] - phi[k + 1]) / (fabs(phi[k]) > 1.0 ? fabs(phi[k]) : 1.0);
          if (amb && imp > 1e-7 && dphi_rel < 2e-6) amb[(size_t)i * N + k] |= 1;
        }
        if (q > 0) {
          dPhi[k + 1] += dalpha * (-1.0 / den);
          if (Phi[k] > 1e-6) dPhi[k] += dalpha * (Phi[k + 1] / (Phi[k] * Phi[k]));
          else dPhi[k] += dalpha * (1.0 / 1e-6);
        }
      }
      double* gkappa = gm + (OC_MLP - 1);
      for (int k = 0; k < N; ++k) {
        double dsig = Phi[k] * (1.0 - Phi[k]);
        double dphi = dPhi[k] * s * dsig;
        *gkappa += dPhi[k] * dsig * s * phi[k];
        int cl = cls[(size_t)i * N + k];
        double b = Di - (double)ti[k];
        if (cl == CLS_TR && n_tr > 0) dphi += wt[2] / (double)n_tr * sgn(phi[k] - b);
        if (cl == CLS_FS && n_fs > 0) {
          double e = exp(-(double)c->kappa_fs * phi[k]) - 1.0, lin = phi[k] - b;
          int arg = 0;
          double top = 0;
          if (e > top) { top = e; arg = 1; }
          if (lin > top) { arg = 2; }
          double dd = arg == 1 ? -(double)c->kappa_fs * (e + 1.0) : (arg == 2 ? 1.0 : 0.0);
          dphi += wt[3] / (double)n_fs * dd;
        }
        double dc[3];
        for (int j = 0; j < 3; ++j) dc[j] = w[k] * gc[j];
        double* dz = dz_all + ((size_t)i * N + k) * OC_Z;
        double flip = 0;
        decode_backward(&m, &A[k], dphi, dc, gm, dz, amb ? &flip : NULL);
        if (amb && flip > OC_KINK_IMPACT) amb[(size_t)i * N + k] |= 8;
      }
    }

    /* ------------- smoothness on S_g (Sec. 3.3, Supp. Sec. 1) ------------- */
#pragma omp for schedule(static)
    for (int p = 0; p < P; ++p) {
      if (!valid[p]) continue;
      float y[2][3];
      for (int a = 0; a < 3; ++a) {
        y[0][a] = xs[3 * p + a];
        y[1][a] = xs[3 * p + a] + eps[3 * p + a];
      }
      cell_t cl[2][OC_LEVELS];
      act_t Ay[2];
      double dzdx[2][OC_Z][3], pz[2][OC_Z], mw2[2][OC_H1], g[2][3];
      for (int e = 0; e < 2; ++e) {
        features(c, theta, y[e], cl[e], Ay[e].z, dzdx[e]);
        decode(&m, &Ay[e]);
        for (int j = 0; j < OC_H1; ++j) {
          mmin(&mg->m[6], Ay[e].y1[j]);
          mmin(&mg->m[0], Ay[e].y1[j]);
        }
        sigmix(&mg->sig, ((uint64_t)1 << 60) + (uint64_t)p * 2 + e, relu_mask(Ay[e].y1, OC_H1));
        dphi_dz(&m, &Ay[e], pz[e], mw2[e]);
        for (int a = 0; a < 3; ++a) {
          double sacc = 0;
          for (int k = 0; k < OC_Z; ++k) sacc += pz[e][k] * dzdx[e][k][a];
          g[e][a] = sacc;
        }
      }
      double dg[3], l2 = 0;
      for (int a = 0; a < 3; ++a) {
        dg[a] = g[0][a] - g[1][a];
        l2 += dg[a] * dg[a];
      }
      lsum[4] += l2;
      if (!do_grad || n_g == 0) continue;
      double* gW1 = gm;
      double* gW2 = gm + OC_H1 * OC_Z + OC_H1;
      for (int e = 0; e < 2; ++e) {
        /* adjoint of g at this point: a = dL/dg */
        double av[3];
        for (int a = 0; a < 3; ++a) av[a] = (e == 0 ? 1.0 : -1.0) * wt[4] / (double)n_g * 2.0 * dg[a];
        /* j_k = a . dz_k/dx ; direct theta term p_k (1/v) (a . dw_c/df) */
        double jv[OC_Z];
        for (int k = 0; k < OC_Z; ++k) jv[k] = av[0] * dzdx[e][k][0] + av[1] * dzdx[e][k][1] + av[2] * dzdx[e][k][2];
        double* dzs = dzs_all + ((size_t)p * 2 + e) * 8 * OC_LEVELS * OC_FEAT;
        for (int l = 0; l < OC_LEVELS; ++l)
          for (int cc = 0; cc < 8; ++cc) {
            double ad = (av[0] * cl[e][l].dw[cc][0] + av[1] * cl[e][l].dw[cc][1] + av[2] * cl[e][l].dw[cc][2]) *
                        cl[e][l].inv_v;
            for (int k = 0; k < OC_FEAT; ++k) dzs[(l * 8 + cc) * OC_FEAT + k] = pz[e][OC_FEAT * l + k] * ad;
          }
        /* decoder terms: a.g = w2^T (m (.) (W1 j)) */
        double W1j[OC_H1];
        for (int h = 0; h < OC_H1; ++h) {
          double sacc = 0;
          for (int k = 0; k < OC_Z; ++k) sacc += m.W1[h * OC_Z + k] * jv[k];
          W1j[h] = sacc;
        }
        for (int h = 0; h < OC_H1; ++h) {
          if (!(Ay[e].y1[h] > 0)) continue;
          for (int k = 0; k < OC_Z; ++k) gW1[h * OC_Z + k] += m.W2[h] * jv[k];
          gW2[h] += W1j[h];
        }
      }
    }
    free(A);
    free(cells);
    free(phi);
    free(Phi);
    free(alpha);
    free(T);
    free(w);
    free(U);
    free(dPhi);
  }

  double lsum[5] = {0, 0, 0, 0, 0};
  for (int th = 0; th < nthreads; ++th)
    for (int k = 0; k < 5; ++k) lsum[k] += lsum_all[(size_t)th * 5 + k];
  loss[0] = R > 0 ? lsum[0] / (double)R : 0.0;
  loss[1] = n_d > 0 ? lsum[1] / (double)n_d : 0.0;
  loss[2] = n_tr > 0 ? lsum[2] / (double)n_tr : 0.0;
  loss[3] = n_fs > 0 ? lsum[3] / (double)n_fs : 0.0;
  loss[4] = n_g > 0 ? lsum[4] / (double)n_g : 0.0;
  loss[5] = 0;
  for (int k = 0; k < 5; ++k) loss[5] += (double)c->lam[k] * loss[k];

  if (margins) {
    uint64_t sig = 0;
    for (int k = 0; k < 10; ++k) margins[k] = INFINITY;
    margins[8] = margins[9] = 0.0;
    for (int th = 0; th < nthreads; ++th) {
      for (int k = 0; k < 7; ++k)
        if (mg_all[th].m[k] < margins[k]) margins[k] = mg_all[th].m[k];
      if (mg_all[th].m[8] > margins[8]) margins[8] = mg_all[th].m[8];
      sig ^= mg_all[th].sig;
    }
    margins[7] = (double)(sig & ((1ULL << 52) - 1));
  }

  if (do_grad) {
    const int64_t ntot = ng + OC_MLP;
    memset(grad, 0, sizeof(double) * (size_t)ntot);
    for (int th = 0; th < nthreads; ++th)
      for (int k = 0; k < OC_MLP; ++k) grad[ng + k] += gm_all[(size_t)th * OC_MLP + k];
    /* scatter dL/dz of every main sample into the 8 corners of its cell at each level */
    for (int i = 0; i < R; ++i) {
      const float* ti = t + (size_t)i * N;
      for (int k = 0; k < N; ++k) {
        float x[3];
        for (int a = 0; a < 3; ++a) {
          float step_ = ti[k] * r[3 * i + a];
          x[a] = o[3 * i + a] + step_;
        }
        const double* dz = dz_all + ((size_t)i * N + k) * OC_Z;
        for (int l = 0; l < OC_LEVELS; ++l) {
          cell_t cl;
          locate(c, l, x, &cl, NULL);
          for (int cc = 0; cc < 8; ++cc)
            for (int f = 0; f < OC_FEAT; ++f) grad[cl.corner[cc] + f] += cl.w[cc] * dz[OC_FEAT * l + f];
        }
      }
    }
    /* smoothness: direct d/dtheta of grad_x phi */
    if (n_g > 0)
      for (int p = 0; p < P; ++p) {
        if (!valid[p]) continue;
        for (int e = 0; e < 2; ++e) {
          float y[3];
          for (int a = 0; a < 3; ++a) y[a] = e == 0 ? xs[3 * p + a] : xs[3 * p + a] + eps[3 * p + a];
          const double* dzs = dzs_all + ((size_t)p * 2 + e) * 8 * OC_LEVELS * OC_FEAT;
          for (int l = 0; l < OC_LEVELS; ++l) {
            cell_t cl;
            locate(c, l, y, &cl, NULL);
            for (int cc = 0; cc < 8; ++cc)
              for (int f = 0; f < OC_FEAT; ++f) grad[cl.corner[cc] + f] += dzs[(l * 8 + cc) * OC_FEAT + f];
          }
        }
      }
  }
  if (dz_out && do_grad) memcpy(dz_out, dz_all, sizeof(double) * (size_t)R * N * OC_Z);
  free(gm_all);
  free(lsum_all);
  free(mg_all);
  free(dz_all);
  free(dzs_all);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* hierarchical importance sampler (Sec. 3.2: 3 steps of 12 from N_c = 96, as in NeuS)     */
/* ------------------------------------------------------------------------------------ */
/* The rays are those of oc_sample_rays for the same (seed, step) (stream 0, slot 0 picks the
 * pixel).  Per ray, in the order the paper gives:
 *   1. N_c coarse depths stratified over [near, far]: t_k = near + (k + u_k)(far - near)/N_c,
 *      u_k from stream 3, slot 1 + k (binary32, as the plain sampler forms its strata);
 *   2. n_steps times: phi at every current sample (FP64), the NeuS weights of the current
 *      samples with the model's s = exp(kappa) (Sec. 3.2 Eq. volume_rendering_alpha: Phi =
 *      sigmoid(s phi), alpha_k = max((Phi_k - Phi_k+1) / max(Phi_k, 1e-6), 0), T_k the product
 *      of (1 - alpha_j) over j < k, w_k = T_k alpha_k) on the n - 1 intervals [t_k, t_k+1]; the
 *      interval masses p_k = (w_k + 1e-5) / sum (w + 1e-5); M new depths by stratified
 *      inverse-CDF draws u_j = (j + xi_j) / M (xi_j from stream 3, slot 1 + N_c + step_i M + j),
 *      each placed linearly inside its interval: t = t_k + (u - C_k) / p_k (t_k+1 - t_k) with
 *      C_k the mass left of interval k (FP64, rounded to binary32 at the end); the new
 *      depths are merged into the sorted list (an existing depth first on ties);
 *   3. classes by the bound b = D - t, as in oc_sample_rays.
 * Outputs as oc_sample_rays with N = N_c + n_steps M; phi_out [R][N] (may be NULL) receives
 * phi (FP64) at the final samples.  Returns 0, or -1 on a bad argument (M is at most 64). */
/* phi at depth tv of the ray (o, r): binary32 position as in oc_step, FP64 from there on */
static double phi_on_ray(const oc_config* c, const double* theta, const mlp_t* m, const float o[3], const float r[3],
                         float tv) {
  float x[3];
  for (int a = 0; a < 3; ++a) {
    float st = tv * r[a];
    x[a] = o[a] + st;
  }
  if (c->arch == 1) return pa_phi_at(c, theta, x);
  cell_t cl[OC_LEVELS];
  act_t A;
  features(c, theta, x, cl, A.z, NULL);
  decode(m, &A);
  return A.out[0];
}

int oc_sample_importance(const oc_config* c, const oc_frames* fr, const double* theta, uint64_t seed,
                         uint32_t step, int R, int Nc, int n_steps, int M, int64_t* pix, float* o, float* r,
                         float* rgb, float* D, float* t, uint8_t* cls, int64_t* counts, double* phi_out) {
  if (R < 0 || Nc < 2 || n_steps < 0 || M < 1 || M > 64) return -1;
  const int N = Nc + n_steps * M;
  const int64_t npix = (int64_t)fr->F * fr->H * fr->W;
  const mlp_t m = mlp_view(theta + grid_size(c)); /* not read for the paper's architecture */
  const double s = exp(c->arch == 1 ? pa_kappa(c, theta) : *m.kappa);
  int64_t nd = 0, ntr = 0, nfs = 0;
#pragma omp parallel for schedule(static) reduction(+ : nd, ntr, nfs)
  for (int i = 0; i < R; ++i) {
    float* ts = (float*)malloc(sizeof(float) * N);
    float* tn = (float*)malloc(sizeof(float) * N);
    double* ph = (double*)malloc(sizeof(double) * N);
    double* pn = (double*)malloc(sizeof(double) * N);
    double* C = (double*)malloc(sizeof(double) * N);
    double* Phi = (double*)malloc(sizeof(double) * N);
    double* al = (double*)malloc(sizeof(double) * N);
    double* Tr = (double*)malloc(sizeof(double) * N);
    double* wk = (double*)malloc(sizeof(double) * N);
    double ch3[3];
    float tnew[64];
    double phnew[64];
    uint64_t h = oc_draw(seed, 0, step, (uint64_t)i, 0);
    int64_t p = (int64_t)(h % (uint64_t)npix);
    pix[i] = p;
    float Di;
    pixel_ray(fr, p, o + 3 * i, r + 3 * i, rgb + 3 * i, &Di);
    D[i] = Di;
    nd += Di > 0.0f;
    const float* oi = o + 3 * i;
    const float* ri = r + 3 * i;
    const float delta = (c->far_m - c->near_m) / (float)Nc;
    for (int k = 0; k < Nc; ++k) {
      float u = unif24(oc_draw(seed, 3, step, (uint64_t)i, 1 + (uint64_t)k));
      ts[k] = c->near_m + ((float)k + u) * delta;
      ph[k] = phi_on_ray(c, theta, &m, oi, ri, ts[k]);
    }
    int n = Nc;
    for (int si = 0; si < n_steps; ++si) {
      /* NeuS weights of the current samples (the renderer's own compositing), interval
       * masses and their running sums */
      double dh, wsum, tot = 0.0;
      composite(n, ph, s, NULL, ts, Phi, al, Tr, wk, ch3, &dh, &wsum);
      for (int k = 0; k + 1 < n; ++k) {
        C[k] = wk[k] + 1e-5; /* unnormalised mass of interval k, for now */
        tot += C[k];
      }
      double run = 0.0;
      for (int k = 0; k + 1 < n; ++k) {
        const double pk = C[k] / tot;
        C[k] = run; /* mass left of interval k */
        run += pk;
      }
      for (int j = 0; j < M; ++j) {
        const double xi = (double)unif24(oc_draw(seed, 3, step, (uint64_t)i, 1 + (uint64_t)Nc + (uint64_t)si * M + j));
        const double u = ((double)j + xi) / (double)M;
        int k = 0;
        while (k + 2 < n && C[k + 1] <= u) ++k; /* last interval whose left mass is <= u */
        const double pk = (k + 2 < n ? C[k + 1] : 1.0) - C[k];
        double f = pk > 0.0 ? (u - C[k]) / pk : 0.0;
        if (f < 0.0) f = 0.0;
        if (f > 1.0) f = 1.0;
        tnew[j] = (float)((double)ts[k] + f * ((double)ts[k + 1] - (double)ts[k]));
        phnew[j] = phi_on_ray(c, theta, &m, oi, ri, tnew[j]);
      }
      /* merge (the new depths ascend with j): an existing depth first on ties */
      int a = 0, b = 0;
      for (int k = 0; k < n + M; ++k) {
        if (b >= M || (a < n && ts[a] <= tnew[b])) { tn[k] = ts[a]; pn[k] = ph[a]; ++a; }
        else { tn[k] = tnew[b]; pn[k] = phnew[b]; ++b; }
      }
      n += M;
      memcpy(ts, tn, sizeof(float) * n);
      memcpy(ph, pn, sizeof(double) * n);
    }
    for (int k = 0; k < N; ++k) {
      t[(size_t)i * N + k] = ts[k];
      if (phi_out) phi_out[(size_t)i * N + k] = ph[k];
      const int cl = sample_class(Di, ts[k], c->trunc);
      cls[(size_t)i * N + k] = (uint8_t)cl;
      ntr += cl == CLS_TR;
      nfs += cl == CLS_FS;
    }
    free(ts);
    free(tn);
    free(ph);
    free(pn);
    free(C);
    free(Phi);
    free(al);
    free(Tr);
    free(wk);
  }
  counts[0] = nd;
  counts[1] = ntr;
  counts[2] = nfs;
  counts[3] = 0;
  return 0;
}

int oc_step(const oc_config* c, const double* theta, int R, int N, const float* o, const float* r,
            const float* rgb, const float* D, const float* t, const uint8_t* cls, int P, const float* xs,
            const float* eps, const uint8_t* valid, const double* dloss, double* loss, double* rgb_hat,
            double* d_hat, double* wsum, double* grad, double* margins, uint8_t* amb, double* w_out) {
  return step_impl(c, theta, R, N, o, r, rgb, D, t, cls, P, xs, eps, valid, dloss, loss, rgb_hat, d_hat, wsum, grad,
                   margins, amb, w_out, NULL);
}
/* oc_step that also returns dL/dz of every main sample, dz_out [R][N][16] (needs grad) */
int oc_step_dz(const oc_config* c, const double* theta, int R, int N, const float* o, const float* r,
               const float* rgb, const float* D, const float* t, const uint8_t* cls, int P, const float* xs,
               const float* eps, const uint8_t* valid, const double* dloss, double* loss, double* grad,
               double* dz_out) {
  return step_impl(c, theta, R, N, o, r, rgb, D, t, cls, P, xs, eps, valid, dloss, loss, NULL, NULL, NULL, grad,
                   NULL, NULL, NULL, dz_out);
}

/* ------------------------------------------------------------------------------------ */
/* camera-pose refinement (Sec. 3.4: P includes the poses; Sec. 4: t in R^3, nu in so(3),  */
/* learning rate 5e-4)                                                                    */
/* ------------------------------------------------------------------------------------ */
/* Frame f's pose is the given camera-to-world [R0 | t0] corrected by xi_f = (dt, nu):
 *   R = R0 Exp(nu),  t = t0 + dt,  Exp by Rodrigues' formula.
 * A ray of pixel (u, v) has o = t and r = R d, d = ((u + 0.5 - cx)/fx, (v + 0.5 - cy)/fy, 1);
 * its samples x_s = o + d_s r move with the pose while their depths d_s and classes do not.
 * With g_s = dL/dx_s = sum_l (d z_l / d x)^T dL/dz_l (the step's own dL/dz):
 *   dL/d dt = sum over the frame's rays and samples of g_s,
 *   dL/d nu = J_r(nu)^T [d]_x R^T sum_s d_s g_s      (d(Exp(nu) d)/d nu = -Exp(nu) [d]_x J_r(nu)),
 * J_r(nu) = I - (1 - cos a)/a^2 [nu]_x + (a - sin a)/a^3 [nu]_x^2, a = |nu| (series near 0). */
static void skew(const double v[3], double K[3][3]) {
  K[0][0] = 0; K[0][1] = -v[2]; K[0][2] = v[1];
  K[1][0] = v[2]; K[1][1] = 0; K[1][2] = -v[0];
  K[2][0] = -v[1]; K[2][1] = v[0]; K[2][2] = 0;
}
static void so3_exp_jr(const double nu[3], double E[3][3], double J[3][3]) {
  const double a2 = nu[0] * nu[0] + nu[1] * nu[1] + nu[2] * nu[2], a = sqrt(a2);
  double K[3][3], K2[3][3];
  skew(nu, K);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      K2[i][j] = 0;
      for (int k = 0; k < 3; ++k) K2[i][j] += K[i][k] * K[k][j];
    }
  double s1, s2, j1, j2; /* E = I + s1 K + s2 K^2,  J = I - j1 K + j2 K^2 */
  if (a < 1e-4) {
    s1 = 1.0 - a2 / 6.0; s2 = 0.5 - a2 / 24.0; j1 = 0.5 - a2 / 24.0; j2 = 1.0 / 6.0 - a2 / 120.0;
  } else {
    s1 = sin(a) / a; s2 = (1.0 - cos(a)) / a2; j1 = (1.0 - cos(a)) / a2; j2 = (a - sin(a)) / (a2 * a);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double I = i == j ? 1.0 : 0.0;
      E[i][j] = I + s1 * K[i][j] + s2 * K2[i][j];
      J[i][j] = I - j1 * K[i][j] + j2 * K2[i][j];
    }
}

/* refined camera-to-world matrices c2w [F][3][4] (FP64) from the given ones and xi [F][6] */
void oc_pose_apply(const float* c2w0, const double* xi, int F, double* c2w) {
  for (int f = 0; f < F; ++f) {
    double E[3][3], J[3][3];
    so3_exp_jr(xi + 6 * f + 3, E, J);
    const float* P = c2w0 + 12 * f;
    double* Q = c2w + 12 * f;
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) {
        double sacc = 0;
        for (int k = 0; k < 3; ++k) sacc += (double)P[4 * i + k] * E[k][j];
        Q[4 * i + j] = sacc;
      }
      Q[4 * i + 3] = (double)P[4 * i + 3] + xi[6 * f + i];
    }
  }
}

/* o, r (binary32, as the sampler forms them) of the rays of pixels pix [R] */
void oc_rays_of_pixels(const oc_frames* fr, const int64_t* pix, int R, float* o, float* r) {
  for (int i = 0; i < R; ++i) {
    float rgb[3], D;
    pixel_ray(fr, pix[i], o + 3 * i, r + 3 * i, rgb, &D);
  }
}

/* dL/dxi [F][6] += the pose gradient of the rays pix [R] with sample depths t [R][N] and the
 * step's dL/dz [R][N][16], for frames whose refined poses are c2w [F][3][4] (FP64) with
 * corrections xi [F][6]; o, r [R][3] the rays the step used. */
void oc_pose_grad(const oc_config* c, const oc_frames* fr, const double* theta, const double* c2w, const double* xi,
                  int R, int N, const int64_t* pix, const float* o, const float* r, const float* t, const double* dz,
                  double* g) {
  const int64_t hw = (int64_t)fr->H * fr->W;
  for (int i = 0; i < R; ++i) {
    const int64_t f = pix[i] / hw, rem = pix[i] % hw;
    const int v = (int)(rem / fr->W), u = (int)(rem % fr->W);
    const double d[3] = {(((double)u + 0.5) - fr->cx) / fr->fx, (((double)v + 0.5) - fr->cy) / fr->fy, 1.0};
    double go[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
    for (int k = 0; k < N; ++k) {
      const float* ti = t + (size_t)i * N;
      float x[3];
      for (int a = 0; a < 3; ++a) {
        float st = ti[k] * r[3 * i + a];
        x[a] = o[3 * i + a] + st;
      }
      cell_t cells[OC_LEVELS];
      double z[OC_Z], dzdx[OC_Z][3];
      features(c, theta, x, cells, z, dzdx);
      const double* dzk = dz + ((size_t)i * N + k) * OC_Z;
      for (int a = 0; a < 3; ++a) {
        double gx = 0;
        for (int q = 0; q < OC_Z; ++q) gx += dzdx[q][a] * dzk[q];
        go[a] += gx;
        gr[a] += (double)ti[k] * gx;
      }
    }
    /* translation */
    for (int a = 0; a < 3; ++a) g[6 * f + a] += go[a];
    /* rotation: J_r^T [d]_x R^T gr */
    double E[3][3], J[3][3], Rt_gr[3], K[3][3], w[3];
    so3_exp_jr(xi + 6 * f + 3, E, J);
    const double* Q = c2w + 12 * f;
    for (int a = 0; a < 3; ++a) Rt_gr[a] = Q[a] * gr[0] + Q[4 + a] * gr[1] + Q[8 + a] * gr[2];
    skew(d, K);
    for (int a = 0; a < 3; ++a) w[a] = K[a][0] * Rt_gr[0] + K[a][1] * Rt_gr[1] + K[a][2] * Rt_gr[2];
    for (int a = 0; a < 3; ++a) g[6 * f + 3 + a] += J[0][a] * w[0] + J[1][a] * w[1] + J[2][a] * w[2];
  }
}

/* ------------------------------------------------------------------------------------ */
/* learned proposal sampler (not part of the paper: a sample-count reduction trained       */
/* online on the main model's rendering weights)                                         */
/* ------------------------------------------------------------------------------------ */
/* The interval [near, far] is cut into OC_PB equal bins.  For every bin centre x_b the
 * network reads the two coarsest grid levels' features z_0(x_b), z_1(x_b) and the unit ray
 * direction, u = [z_0, z_1, r/|r|] (11 values), and returns one logit:
 *   l_b = w3 . relu(W2 relu(W1 u + b1) + b2) + b3,    p = softmax_b(l).
 * Parameters (OC_PROP floats): W1[32][11], b1[32], W2[32][32], b2[32], w3[32], b3. */
#define OC_PB 32
#define OC_PIN 11
#define OC_PH 32
#define OC_PROP (OC_PH * OC_PIN + OC_PH + OC_PH * OC_PH + OC_PH + OC_PH + 1) /* 1473 */

typedef struct {
  double u[OC_PIN], y1[OC_PH], a1[OC_PH], y2[OC_PH], a2[OC_PH], logit;
} prop_act_t;

/* binary32 bin geometry: width and left edge of bin b */
static float prop_width(const oc_config* c) { return (c->far_m - c->near_m) / (float)OC_PB; }
static float prop_edge(const oc_config* c, int b) { return c->near_m + (float)b * prop_width(c); }

static void prop_eval(const oc_config* c, const double* theta, const double* q, const float o[3], const float r[3],
                      int b, prop_act_t* A) {
  const double *W1 = q, *b1 = W1 + OC_PH * OC_PIN, *W2 = b1 + OC_PH, *b2 = W2 + OC_PH * OC_PH, *w3 = b2 + OC_PH,
               *b3 = w3 + OC_PH;
  const float tc = c->near_m + ((float)b + 0.5f) * prop_width(c); /* bin centre (binary32) */
  float x[3];
  for (int a = 0; a < 3; ++a) {
    float step_ = tc * r[a];
    x[a] = o[a] + step_;
  }
  cell_t cells[OC_LEVELS];
  double z[OC_Z];
  features(c, theta, x, cells, z, NULL);
  for (int k = 0; k < 8; ++k) A->u[k] = z[k]; /* levels 0 and 1 */
  const double n = sqrt((double)r[0] * r[0] + (double)r[1] * r[1] + (double)r[2] * r[2]);
  for (int a = 0; a < 3; ++a) A->u[8 + a] = (double)r[a] / n;
  for (int j = 0; j < OC_PH; ++j) {
    double s = b1[j];
    for (int k = 0; k < OC_PIN; ++k) s += W1[j * OC_PIN + k] * A->u[k];
    A->y1[j] = s;
    A->a1[j] = s > 0 ? s : 0;
  }
  for (int j = 0; j < OC_PH; ++j) {
    double s = b2[j];
    for (int k = 0; k < OC_PH; ++k) s += W2[j * OC_PH + k] * A->a1[k];
    A->y2[j] = s;
    A->a2[j] = s > 0 ? s : 0;
  }
  double l = b3[0];
  for (int k = 0; k < OC_PH; ++k) l += w3[k] * A->a2[k];
  A->logit = l;
}

/* p [R][OC_PB]: the proposal distribution of every ray (FP64) */
void oc_prop_forward(const oc_config* c, const double* theta, const double* q, int R, const float* o, const float* r,
                     double* p) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < R; ++i) {
    prop_act_t A;
    double l[OC_PB], mx = -INFINITY, s = 0;
    for (int b = 0; b < OC_PB; ++b) {
      prop_eval(c, theta, q, o + 3 * i, r + 3 * i, b, &A);
      l[b] = A.logit;
      if (l[b] > mx) mx = l[b];
    }
    for (int b = 0; b < OC_PB; ++b) s += exp(l[b] - mx);
    for (int b = 0; b < OC_PB; ++b) p[(size_t)i * OC_PB + b] = exp(l[b] - mx) / s;
  }
}

/* bin of a sample depth (binary32 decision), clamped to [0, OC_PB) */
static int prop_bin(const oc_config* c, float t) {
  float f = (t - c->near_m) / prop_width(c);
  int b = (int)floorf(f);
  return b < 0 ? 0 : (b >= OC_PB ? OC_PB - 1 : b);
}

/*
 * Training loss of the proposal: for every ray, the main model's weights w [R][N] at its
 * samples t [R][N] are summed per bin, h_b = sum_{t_i in bin b} w_i, and normalised,
 * hh = h / sum(h); rays with sum(h) < 1e-3 are skipped.  The loss is the mean over the used
 * rays of the cross entropy -sum_b hh_b log p_b; the target is a constant (no gradient
 * reaches the main model or the grid).  Returns the loss; gq (+=, may be NULL) receives
 * its gradient with respect to the proposal parameters, d/d l_b = (p_b - hh_b) / n_used.
 */
double oc_prop_ce(const oc_config* c, const double* theta, const double* q, int R, int N, const float* o,
                  const float* r, const float* t, const double* w, double* gq, int64_t* n_used_out) {
  int64_t n_used = 0;
  double ce = 0;
  double* gtmp = (double*)calloc(OC_PROP, sizeof(double));
  const double *W2 = q + OC_PH * OC_PIN + OC_PH, *w3 = W2 + OC_PH * OC_PH + OC_PH;
  for (int i = 0; i < R; ++i) {
    double h[OC_PB] = {0}, S = 0;
    for (int k = 0; k < N; ++k) h[prop_bin(c, t[(size_t)i * N + k])] += w[(size_t)i * N + k];
    for (int b = 0; b < OC_PB; ++b) S += h[b];
    if (!(S >= 1e-3)) continue;
    ++n_used;
    prop_act_t A[OC_PB];
    double mx = -INFINITY, se = 0;
    for (int b = 0; b < OC_PB; ++b) {
      prop_eval(c, theta, q, o + 3 * i, r + 3 * i, b, &A[b]);
      if (A[b].logit > mx) mx = A[b].logit;
    }
    for (int b = 0; b < OC_PB; ++b) se += exp(A[b].logit - mx);
    const double lse = mx + log(se);
    for (int b = 0; b < OC_PB; ++b) {
      const double hh = h[b] / S, pb = exp(A[b].logit - lse);
      ce -= hh * (A[b].logit - lse);
      /* reverse mode through the bin's network, seed dl = p_b - hh_b (scaled later) */
      const double dl = pb - hh;
      double* gW1 = gtmp;
      double* gb1 = gW1 + OC_PH * OC_PIN;
      double* gW2 = gb1 + OC_PH;
      double* gb2 = gW2 + OC_PH * OC_PH;
      double* gw3 = gb2 + OC_PH;
      double* gb3 = gw3 + OC_PH;
      double dy2[OC_PH], dy1[OC_PH];
      gb3[0] += dl;
      for (int k = 0; k < OC_PH; ++k) {
        gw3[k] += dl * A[b].a2[k];
        dy2[k] = A[b].y2[k] > 0 ? dl * w3[k] : 0.0;
      }
      for (int j = 0; j < OC_PH; ++j) {
        gb2[j] += dy2[j];
        for (int k = 0; k < OC_PH; ++k) gW2[j * OC_PH + k] += dy2[j] * A[b].a1[k];
      }
      for (int k = 0; k < OC_PH; ++k) {
        double s = 0;
        for (int j = 0; j < OC_PH; ++j) s += W2[j * OC_PH + k] * dy2[j];
        dy1[k] = A[b].y1[k] > 0 ? s : 0.0;
      }
      for (int j = 0; j < OC_PH; ++j) {
        gb1[j] += dy1[j];
        for (int k = 0; k < OC_PIN; ++k) gW1[j * OC_PIN + k] += dy1[j] * A[b].u[k];
      }
    }
  }
  if (gq && n_used > 0)
    for (int k = 0; k < OC_PROP; ++k) gq[k] += gtmp[k] / (double)n_used;
  free(gtmp);
  if (n_used_out) *n_used_out = n_used;
  return n_used > 0 ? ce / (double)n_used : 0.0;
}

static int cmp_float(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return (x > y) - (x < y);
}

/*
 * Sample depths from the proposal (binary32, bit-exact given p): the mixture
 * pp = 0.95 p + 0.05 / OC_PB keeps every bin reachable; its running sums C_b (added in bin
 * order) form the inverse CDF.  K = N - n_guided stratified draws u_k = (k + xi_k) / K
 * (K = N when D <= 0: no depth to guide) land at target = u_k C_{last}; the bin is the
 * first with C_b > target and the depth is placed linearly inside it.  When D > 0 the
 * n_guided samples are stratified over [D - g, D + g] as in the plain sampler.  The N
 * depths are sorted ascending and classified like the plain sampler's.  Random numbers:
 * stream 2, slot 1 + k for draw k (the rays themselves are the plain sampler's).
 * p [R][OC_PB] binary32; t [R][N], cls [R][N]; counts[3] = (rays with D>0, |S_tr|, |S_fs|).
 */
void oc_prop_sample(const oc_config* c, int R, int N, int n_guided, const float* D, const float* p, uint64_t seed,
                    uint32_t step, float* t, uint8_t* cls, int64_t* counts) {
  const float width = prop_width(c);
  const float mixw = 0.05f / (float)OC_PB;
  int64_t nd = 0, ntr = 0, nfs = 0;
  for (int i = 0; i < R; ++i) {
    float pp[OC_PB], C[OC_PB], acc = 0.0f;
    for (int b = 0; b < OC_PB; ++b) {
      pp[b] = 0.95f * p[(size_t)i * OC_PB + b] + mixw;
      acc = acc + pp[b];
      C[b] = acc;
    }
    const float total = C[OC_PB - 1];
    const float Di = D[i];
    const int ng = (Di > 0.0f) ? n_guided : 0;
    const int K = N - ng;
    float* ti = t + (size_t)i * N;
    for (int k = 0; k < K; ++k) {
      float u = unif24(oc_draw(seed, 2, step, (uint64_t)i, 1 + (uint64_t)k));
      float target = (((float)k + u) / (float)K) * total;
      int b = 0;
      while (b < OC_PB && C[b] <= target) ++b;
      if (b > OC_PB - 1) b = OC_PB - 1;
      float lo = b > 0 ? C[b - 1] : 0.0f;
      float e0 = prop_edge(c, b), e1 = prop_edge(c, b + 1);
      float x = e0 + ((target - lo) / pp[b]) * width;
      ti[k] = x < e0 ? e0 : (x > e1 ? e1 : x);
    }
    if (ng > 0) {
      ++nd;
      float g = c->guide_half;
      float gstep = (2.0f * g) / (float)ng;
      float g0 = Di - g;
      for (int j = 0; j < ng; ++j) {
        float u = unif24(oc_draw(seed, 2, step, (uint64_t)i, 1 + (uint64_t)K + (uint64_t)j));
        ti[K + j] = g0 + ((float)j + u) * gstep;
      }
    } else if (Di > 0.0f) {
      ++nd;
    }
    qsort(ti, (size_t)N, sizeof(float), cmp_float);
    for (int k = 0; k < N; ++k) {
      int cl = sample_class(Di, ti[k], c->trunc);
      cls[(size_t)i * N + k] = (uint8_t)cl;
      ntr += cl == CLS_TR;
      nfs += cl == CLS_FS;
    }
  }
  counts[0] = nd;
  counts[1] = ntr;
  counts[2] = nfs;
}

/* ------------------------------------------------------------------------------------ */
/* Adam (Kingma & Ba 2015), per-group learning rates (Sec. 4 Implementation Details)     */
/* ------------------------------------------------------------------------------------ */
/* entries [0, n_grid) use lr_grid, the rest lr_mlp; t >= 1 is the step count; g is zeroed */
void oc_adam(double* p, double* g, double* mom, double* vel, int64_t n, int64_t n_grid, int t, double lr_grid,
             double lr_mlp, double b1, double b2, double eps) {
  double bc1 = 1.0 - pow(b1, (double)t), bc2 = 1.0 - pow(b2, (double)t);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double lr = i < n_grid ? lr_grid : lr_mlp;
    mom[i] = b1 * mom[i] + (1.0 - b1) * g[i];
    vel[i] = b2 * vel[i] + (1.0 - b2) * g[i] * g[i];
    double mh = mom[i] / bc1, vh = vel[i] / bc2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
    g[i] = 0.0;
  }
}

int oc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* the paper's architecture (Sec. 3.1 Eq. SDF_MLP, Eq. COLOR_MLP, "Architecture Details") */
/* ------------------------------------------------------------------------------------ */
/* Geometry: phi = f_omega(V_theta(x)) with f_omega a decoder of two hidden layers of 32
 * (ReLU) and one linear output.  Colour: c = g_gamma(W_beta(x), d), where W_beta(x) is the
 * trilinear interpolation of a separate grid of h_c = 6 colour features per vertex at the
 * finest level (same vertices as geometry level 3) and d the viewing direction, taken as
 * the unit ray direction r/|r|; g_gamma has two hidden layers of 32 (ReLU) and a sigmoid
 * on its 3 outputs.
 * Flat parameter vector: geometry levels 0..3 ([nz][ny][nx][4] each), the colour grid
 * [nz][ny][nx][6] of level 3 padded with zeros to a multiple of 4 floats, then PA_MLP
 * decoder floats: gW1[32][16], gb1[32], gW2[32][32], gb2[32], gw3[32], gb3,
 * cW1[32][9], cb1[32], cW2[32][32], cb2[32], cW3[3][32], cb3[3], kappa. */
#define PA_C 6            /* h_c */
#define PA_H 32           /* neurons per hidden layer */
#define PA_U (PA_C + 3)   /* colour decoder input [W_beta(x), d] */
#define PA_MLP (PA_H * OC_Z + PA_H + PA_H * PA_H + PA_H + PA_H + 1 + PA_H * PA_U + PA_H + PA_H * PA_H + PA_H + 3 * PA_H + 3 + 1)

static int64_t pa_colour_floats(const oc_config* c) {
  int64_t n = (int64_t)c->dims[3][0] * c->dims[3][1] * c->dims[3][2] * PA_C;
  return (n + 3) / 4 * 4;
}

/* number of floats of the flat vector; *n_grid (may be NULL) = geometry + colour grid floats */
int64_t oc_paper_param_count(const oc_config* c, int64_t* n_grid) {
  int64_t g = grid_size(c) + pa_colour_floats(c);
  if (n_grid) *n_grid = g;
  return g + PA_MLP;
}

typedef struct {
  const double *gW1, *gb1, *gW2, *gb2, *gw3, *gb3, *cW1, *cb1, *cW2, *cb2, *cW3, *cb3, *kappa;
} pa_mlp_t;

static pa_mlp_t pa_view(const double* b) {
  pa_mlp_t m;
  m.gW1 = b;
  m.gb1 = m.gW1 + PA_H * OC_Z;
  m.gW2 = m.gb1 + PA_H;
  m.gb2 = m.gW2 + PA_H * PA_H;
  m.gw3 = m.gb2 + PA_H;
  m.gb3 = m.gw3 + PA_H;
  m.cW1 = m.gb3 + 1;
  m.cb1 = m.cW1 + PA_H * PA_U;
  m.cW2 = m.cb1 + PA_H;
  m.cb2 = m.cW2 + PA_H * PA_H;
  m.cW3 = m.cb2 + PA_H;
  m.cb3 = m.cW3 + 3 * PA_H;
  m.kappa = m.cb3 + 3;
  return m;
}

typedef struct {
  double z[OC_Z], y1[PA_H], a1[PA_H], y2[PA_H], a2[PA_H], phi;  /* geometry decoder */
  double zmag[OC_Z], umag[PA_U]; /* input magnitudes for the kink diagnostics (see kink_rel) */
  double u[PA_U], q1[PA_H], r1[PA_H], q2[PA_H], r2[PA_H], pre[3], c[3]; /* colour decoder */
  int64_t cvtx[8];  /* flat colour-grid float index of feature 0 of each level-3 corner */
  double cw[8];     /* their trilinear weights */
} pa_act_t;

/* y = b + W x for W [n][k] row-major */
static void pa_affine(const double* W, const double* b, const double* x, int n, int k, double* y) {
  for (int j = 0; j < n; ++j) {
    double s = b[j];
    for (int i = 0; i < k; ++i) s += W[j * k + i] * x[i];
    y[j] = s;
  }
}

/* features and both decoders at the binary32 position x seen along unit direction d */
static void pa_eval(const oc_config* c, const double* theta, const pa_mlp_t* m, const float x[3], const double d[3],
                    cell_t cells[OC_LEVELS], double dzdx[OC_Z][3], pa_act_t* A) {
  features(c, theta, x, cells, A->z, dzdx);
  /* W_beta(x): the colour grid shares level 3's vertices, so it uses level 3's cell */
  const int64_t cbase = grid_size(c), off3 = level_offset(c, 3);
  for (int k = 0; k < PA_C; ++k) A->u[k] = A->umag[k] = 0.0;
  for (int cc = 0; cc < 8; ++cc) {
    const int64_t vtx = (cells[3].corner[cc] - off3) / OC_FEAT;
    A->cvtx[cc] = cbase + vtx * PA_C;
    A->cw[cc] = cells[3].w[cc];
    for (int k = 0; k < PA_C; ++k) {
      A->u[k] += cells[3].w[cc] * theta[A->cvtx[cc] + k];
      A->umag[k] += cells[3].w[cc] * fabs(theta[A->cvtx[cc] + k]);
    }
  }
  for (int a = 0; a < 3; ++a) A->u[PA_C + a] = d[a], A->umag[PA_C + a] = fabs(d[a]);
  feature_mag(theta, cells, A->zmag);
  pa_affine(m->gW1, m->gb1, A->z, PA_H, OC_Z, A->y1);
  for (int j = 0; j < PA_H; ++j) A->a1[j] = A->y1[j] > 0 ? A->y1[j] : 0;
  pa_affine(m->gW2, m->gb2, A->a1, PA_H, PA_H, A->y2);
  for (int j = 0; j < PA_H; ++j) A->a2[j] = A->y2[j] > 0 ? A->y2[j] : 0;
  pa_affine(m->gw3, m->gb3, A->a2, 1, PA_H, &A->phi);
  pa_affine(m->cW1, m->cb1, A->u, PA_H, PA_U, A->q1);
  for (int j = 0; j < PA_H; ++j) A->r1[j] = A->q1[j] > 0 ? A->q1[j] : 0;
  pa_affine(m->cW2, m->cb2, A->r1, PA_H, PA_H, A->q2);
  for (int j = 0; j < PA_H; ++j) A->r2[j] = A->q2[j] > 0 ? A->q2[j] : 0;
  pa_affine(m->cW3, m->cb3, A->r2, 3, PA_H, A->pre);
  for (int j = 0; j < 3; ++j) A->c[j] = sigm(A->pre[j]);
}

/* mag (see kink_rel) of the four hidden layers of the paper's decoders */
static void pa_mags(const pa_mlp_t* m, const pa_act_t* A, double g1[PA_H], double g2[PA_H], double c1[PA_H],
                    double c2[PA_H]) {
  double on[PA_H];
  layer_mag(m->gW1, m->gb1, A->zmag, PA_H, OC_Z, g1);
  for (int j = 0; j < PA_H; ++j) on[j] = A->y1[j] > 0 ? g1[j] : 0.0;
  layer_mag(m->gW2, m->gb2, on, PA_H, PA_H, g2);
  layer_mag(m->cW1, m->cb1, A->umag, PA_H, PA_U, c1);
  for (int j = 0; j < PA_H; ++j) on[j] = A->q1[j] > 0 ? c1[j] : 0.0;
  layer_mag(m->cW2, m->cb2, on, PA_H, PA_H, c2);
}

/* smallest relative kink distance (kink_rel) over the hidden units of the geometry decoder
 * and, when colour != 0, of the colour decoder */
static double pa_kink(const pa_mlp_t* m, const pa_act_t* A, int colour) {
  double g1[PA_H], g2[PA_H], c1[PA_H], c2[PA_H], r = INFINITY, v;
  pa_mags(m, A, g1, g2, c1, c2);
  for (int j = 0; j < PA_H; ++j) {
    if ((v = kink_rel(A->y1[j], g1[j])) < r) r = v;
    if ((v = kink_rel(A->y2[j], g2[j])) < r) r = v;
    if (!colour) continue;
    if ((v = kink_rel(A->q1[j], c1[j])) < r) r = v;
    if ((v = kink_rel(A->q2[j], c2[j])) < r) r = v;
  }
  return r;
}

/* one dense layer backwards: gW += dy x^T, gb += dy, and (dx != NULL) dx = W^T dy */
static void pa_affine_back(const double* W, const double* x, const double* dy, int n, int k, double* gW, double* gb,
                           double* dx) {
  for (int j = 0; j < n; ++j) {
    gb[j] += dy[j];
    for (int i = 0; i < k; ++i) gW[j * k + i] += dy[j] * x[i];
  }
  if (dx)
    for (int i = 0; i < k; ++i) {
      double s = 0;
      for (int j = 0; j < n; ++j) s += W[j * k + i] * dy[j];
      dx[i] = s;
    }
}

/* reverse mode of pa_eval's decoders for upstream dphi, dc: decoder gradients into gm (the
 * PA_MLP block), dL/dz [16] and dL/dW_beta(x) [6] returned */
/* flip diagnostic of one hidden layer (as decode_backward's): over its units within
 * OC_KINK_REL of their kink (mag: the layer's pa_mags), the largest |dL/d(unit output)| times
 * unit_scale */
static void pa_flip(const double* W, const double* x, int k, const double* y, const double* mag, const double* dy,
                    double* f) {
  for (int j = 0; j < PA_H; ++j)
    if (kink_rel(y[j], mag[j]) < OC_KINK_REL) {
      double v = fabs(dy[j]) * unit_scale(W + j * k, x, k);
      if (v > *f) *f = v;
    }
}

static void pa_backward(const pa_mlp_t* m, const pa_act_t* A, double dphi, const double dc[3], double* gm,
                        double dz[OC_Z], double dcf[PA_C], double ddir[3], double* flip) {
  pa_mlp_t g = pa_view(gm); /* same offsets in the gradient block */
  double d2[PA_H], d1[PA_H], du[PA_U], f = 0, g1m[PA_H], g2m[PA_H], c1m[PA_H], c2m[PA_H];
  if (flip) pa_mags(m, A, g1m, g2m, c1m, c2m);
  /* geometry: phi = gw3 . a2 + gb3 */
  pa_affine_back(m->gw3, A->a2, &dphi, 1, PA_H, (double*)g.gw3, (double*)g.gb3, d2);
  if (flip) pa_flip(m->gW2, A->a1, PA_H, A->y2, g2m, d2, &f);
  for (int j = 0; j < PA_H; ++j) d2[j] = A->y2[j] > 0 ? d2[j] : 0.0;
  pa_affine_back(m->gW2, A->a1, d2, PA_H, PA_H, (double*)g.gW2, (double*)g.gb2, d1);
  if (flip) pa_flip(m->gW1, A->z, OC_Z, A->y1, g1m, d1, &f);
  for (int j = 0; j < PA_H; ++j) d1[j] = A->y1[j] > 0 ? d1[j] : 0.0;
  pa_affine_back(m->gW1, A->z, d1, PA_H, OC_Z, (double*)g.gW1, (double*)g.gb1, dz);
  /* colour: c = sigmoid(cW3 r2 + cb3) */
  double dpre[3];
  for (int j = 0; j < 3; ++j) dpre[j] = dc[j] * A->c[j] * (1.0 - A->c[j]);
  pa_affine_back(m->cW3, A->r2, dpre, 3, PA_H, (double*)g.cW3, (double*)g.cb3, d2);
  if (flip) pa_flip(m->cW2, A->r1, PA_H, A->q2, c2m, d2, &f);
  for (int j = 0; j < PA_H; ++j) d2[j] = A->q2[j] > 0 ? d2[j] : 0.0;
  pa_affine_back(m->cW2, A->r1, d2, PA_H, PA_H, (double*)g.cW2, (double*)g.cb2, d1);
  if (flip) pa_flip(m->cW1, A->u, PA_U, A->q1, c1m, d1, &f);
  if (flip) *flip = f;
  for (int j = 0; j < PA_H; ++j) d1[j] = A->q1[j] > 0 ? d1[j] : 0.0;
  pa_affine_back(m->cW1, A->u, d1, PA_H, PA_U, (double*)g.cW1, (double*)g.cb1, du);
  for (int k = 0; k < PA_C; ++k) dcf[k] = du[k];
  if (ddir) /* the viewing direction is not a parameter; its gradient serves the pose refinement */
    for (int a = 0; a < 3; ++a) ddir[a] = du[PA_C + a];
}

/* d phi / d z of the two-hidden-layer geometry decoder (piecewise linear, masks fixed):
 * e = m2 (.) gw3, pm = m1 (.) (gW2^T e), p = gW1^T pm */
static void pa_dphi_dz(const pa_mlp_t* m, const pa_act_t* A, double p[OC_Z], double pm[PA_H], double e[PA_H]) {
  for (int j = 0; j < PA_H; ++j) e[j] = A->y2[j] > 0 ? m->gw3[j] : 0.0;
  for (int i = 0; i < PA_H; ++i) {
    double s = 0;
    for (int j = 0; j < PA_H; ++j) s += m->gW2[j * PA_H + i] * e[j];
    pm[i] = A->y1[i] > 0 ? s : 0.0;
  }
  for (int k = 0; k < OC_Z; ++k) {
    double s = 0;
    for (int i = 0; i < PA_H; ++i) s += m->gW1[i * OC_Z + k] * pm[i];
    p[k] = s;
  }
}

/*
 * One step of the paper's architecture: the losses of oc_step (rgb, depth, truncated SDF,
 * free space, smoothness, weighted total; same batch normalisations and readings) with
 * phi = f_omega(V_theta(x)) and c = g_gamma(W_beta(x), d), and (grad != NULL) their
 * gradient with respect to the flat vector laid out as oc_paper_param_count describes.
 * Arguments as oc_step.  margins: entry 0 = min |hidden pre-activation| of both decoders
 * (main samples and smoothness points), 5 = min |d_hat - D|, 7 = signature of the branch
 * decisions; the others are set to +inf (8 and 9 to 0).  amb flags as in oc_step.
 */
static int step_paper_impl(const oc_config* c, const double* theta, int R, int N, const float* o, const float* r,
                           const float* rgb, const float* D, const float* t, const uint8_t* cls, int P,
                           const float* xs, const float* eps, const uint8_t* valid, const double* dloss,
                           double* loss, double* rgb_hat, double* d_hat, double* wsum, double* grad, double* margins,
                           uint8_t* amb, double* w_out, double* dzc_out) {
  if (R < 0 || N < 2 || P < 0) return -1;
  int64_t ng = 0;
  const int64_t ntot = oc_paper_param_count(c, &ng);
  const pa_mlp_t m = pa_view(theta + ng);
  const double s = exp(*m.kappa);

  int64_t n_d = 0, n_tr = 0, n_fs = 0, n_g = 0;
  for (int i = 0; i < R; ++i) {
    n_d += D[i] > 0.0f;
    for (int k = 0; k < N; ++k) {
      n_tr += cls[(size_t)i * N + k] == CLS_TR;
      n_fs += cls[(size_t)i * N + k] == CLS_FS;
    }
  }
  for (int p = 0; p < P; ++p) n_g += valid[p] != 0;
  double wt[5];
  for (int k = 0; k < 5; ++k) wt[k] = dloss ? dloss[k] + (double)c->lam[k] * dloss[5] : (double)c->lam[k];
  if (amb) memset(amb, 0, (size_t)R * N);
  const int do_grad = grad != NULL;
  double lsum[5] = {0, 0, 0, 0, 0};
  double hid_margin = INFINITY, d_margin = INFINITY;
  uint64_t sig = 0;
  if (do_grad) memset(grad, 0, sizeof(double) * (size_t)ntot);
  double* gm = do_grad ? grad + ng : NULL;

  /* Rays one after another (plain and sequential: this form is checked on small batches). */
  pa_act_t* A = (pa_act_t*)malloc(sizeof(pa_act_t) * (size_t)N);
  cell_t* cells = (cell_t*)malloc(sizeof(cell_t) * (size_t)N * OC_LEVELS);
  double *phi = malloc(sizeof(double) * N), *Phi = malloc(sizeof(double) * N), *alpha = malloc(sizeof(double) * N),
         *T = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N), *U = malloc(sizeof(double) * N),
         *dPhi = malloc(sizeof(double) * N);
  for (int i = 0; i < R; ++i) {
    const float* ti = t + (size_t)i * N;
    double d[3], rn = 0;
    for (int a = 0; a < 3; ++a) rn += (double)r[3 * i + a] * (double)r[3 * i + a];
    rn = sqrt(rn);
    for (int a = 0; a < 3; ++a) d[a] = (double)r[3 * i + a] / rn;
    for (int k = 0; k < N; ++k) {
      float x[3];
      for (int a = 0; a < 3; ++a) {
        float step_ = ti[k] * r[3 * i + a];
        x[a] = o[3 * i + a] + step_;
      }
      pa_eval(c, theta, &m, x, d, cells + (size_t)k * OC_LEVELS, NULL, &A[k]);
      phi[k] = A[k].phi;
      const double* hid[4] = {A[k].y1, A[k].y2, A[k].q1, A[k].q2};
      for (int h = 0; h < 4; ++h) {
        for (int j = 0; j < PA_H; ++j) mmin(&hid_margin, hid[h][j]);
        sigmix(&sig, ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8 + (uint64_t)h, relu_mask(hid[h], PA_H));
      }
    }
    /* NeuS weights (Sec. 3.2); the colours are composited here with the same weights */
    double ch[3] = {0, 0, 0}, dh, ws;
    composite(N, phi, s, NULL, ti, Phi, alpha, T, w, ch, &dh, &ws);
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < 3; ++j) ch[j] += w[k] * A[k].c[j];
    for (int k = 0; k + 1 < N; ++k)
      sigmix(&sig, ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8 + 5,
             (uint64_t)(alpha[k] > 0) | (uint64_t)(Phi[k] > 1e-6) << 1);
    if (rgb_hat)
      for (int j = 0; j < 3; ++j) rgb_hat[3 * i + j] = ch[j];
    if (d_hat) d_hat[i] = dh;
    if (wsum) wsum[i] = ws;
    if (w_out)
      for (int k = 0; k < N; ++k) w_out[(size_t)i * N + k] = w[k];
    for (int j = 0; j < 3; ++j) {
      double e = (double)rgb[3 * i + j] - ch[j];
      lsum[0] += e * e;
    }
    const double Di = (double)D[i];
    if (D[i] > 0.0f) {
      lsum[1] += fabs(Di - dh);
      mmin(&d_margin, dh - Di);
      if (amb && fabs(dh - Di) < 1e-5 * (Di > 1.0 ? Di : 1.0)) amb[(size_t)i * N] |= 16;
      sigmix(&sig, ((uint64_t)i * (uint64_t)N) * 8 + 7, (uint64_t)(dh > Di));
    }
    for (int k = 0; k < N; ++k) {
      const int cl = cls[(size_t)i * N + k];
      const double b = Di - (double)ti[k];
      if (cl == CLS_TR) {
        lsum[2] += fabs(phi[k] - b);
        if (amb && fabs(phi[k] - b) < 2e-5) amb[(size_t)i * N + k] |= 2;
        sigmix(&sig, ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8 + 6, (uint64_t)(phi[k] > b));
      } else if (cl == CLS_FS) {
        double v[3] = {0.0, exp(-(double)c->kappa_fs * phi[k]) - 1.0, phi[k] - b};
        int arg = 0;
        for (int q = 1; q < 3; ++q)
          if (v[q] > v[arg]) arg = q;
        double second = -INFINITY;
        for (int q = 0; q < 3; ++q)
          if (q != arg && v[q] > second) second = v[q];
        if (amb && v[arg] - second < 2e-5) amb[(size_t)i * N + k] |= 4;
        sigmix(&sig, ((uint64_t)i * (uint64_t)N + (uint64_t)k) * 8 + 6, (uint64_t)arg + 2);
        lsum[3] += v[arg];
      }
    }
    if (!do_grad) continue;

    /* backward through the compositing (as in oc_step) */
    double gc[3], gd = 0;
    for (int j = 0; j < 3; ++j) gc[j] = wt[0] / (double)R * 2.0 * (ch[j] - (double)rgb[3 * i + j]);
    if (D[i] > 0.0f && n_d > 0) gd = wt[1] / (double)n_d * sgn(dh - Di);
    U[N - 1] = 0;
    for (int k = N - 1; k >= 1; --k) {
      double ek = gc[0] * A[k].c[0] + gc[1] * A[k].c[1] + gc[2] * A[k].c[2] + gd * (double)ti[k];
      U[k - 1] = alpha[k] * ek + (1.0 - alpha[k]) * U[k];
    }
    for (int k = 0; k < N; ++k) dPhi[k] = 0;
    for (int k = 0; k < N - 1; ++k) {
      double ek = gc[0] * A[k].c[0] + gc[1] * A[k].c[1] + gc[2] * A[k].c[2] + gd * (double)ti[k];
      double dalpha = T[k] * (ek - U[k]);
      double den = Phi[k] > 1e-6 ? Phi[k] : 1e-6;
      double q = (Phi[k] - Phi[k + 1]) / den;
      if (amb && fabs(q) < 1e-5 && phi[k] != phi[k + 1] && 1.0 - Phi[k] > 1e-5) {
        double self = fabs(dalpha) * s * Phi[k] * (1.0 - Phi[k]) / den;
        double next = fabs(dalpha) * s * Phi[k + 1] * (1.0 - Phi[k + 1]) / den;
        double dphi_rel = fabs(phi[k] - phi[k + 1]) / (fabs(phi[k]) > 1.0 ? fabs(phi[k]) : 1.0);
        if ((self > next ? self : next) > 1e-7 && dphi_rel < 2e-6) amb[(size_t)i * N + k] |= 1;
      }
      if (q > 0) {
        dPhi[k + 1] += dalpha * (-1.0 / den);
        if (Phi[k] > 1e-6) dPhi[k] += dalpha * (Phi[k + 1] / (Phi[k] * Phi[k]));
        else dPhi[k] += dalpha * (1.0 / 1e-6);
      }
    }
    for (int k = 0; k < N; ++k) {
      const double dsig = Phi[k] * (1.0 - Phi[k]);
      double dphi = dPhi[k] * s * dsig;
      gm[PA_MLP - 1] += dPhi[k] * dsig * s * phi[k];
      const int cl = cls[(size_t)i * N + k];
      const double b = Di - (double)ti[k];
      if (cl == CLS_TR && n_tr > 0) dphi += wt[2] / (double)n_tr * sgn(phi[k] - b);
      if (cl == CLS_FS && n_fs > 0) {
        double e = exp(-(double)c->kappa_fs * phi[k]) - 1.0, lin = phi[k] - b;
        int arg = 0;
        double top = 0;
        if (e > top) { top = e; arg = 1; }
        if (lin > top) { arg = 2; }
        dphi += wt[3] / (double)n_fs * (arg == 1 ? -(double)c->kappa_fs * (e + 1.0) : (arg == 2 ? 1.0 : 0.0));
      }
      double dc[3], dz[OC_Z], dcf[PA_C];
      for (int j = 0; j < 3; ++j) dc[j] = w[k] * gc[j];
      double ddir[3];
      double flip = 0;
      pa_backward(&m, &A[k], dphi, dc, gm, dz, dcf, ddir, amb ? &flip : NULL);
      if (amb && flip > OC_KINK_IMPACT) amb[(size_t)i * N + k] |= 8;
      if (dzc_out) { /* per sample: dL/dz, dL/dW_beta(x), dL/d(direction) */
        double* q = dzc_out + ((size_t)i * N + k) * 32;
        for (int f = 0; f < 32; ++f) q[f] = 0.0;
        for (int f = 0; f < OC_Z; ++f) q[f] = dz[f];
        for (int f = 0; f < PA_C; ++f) q[OC_Z + f] = dcf[f];
        for (int a = 0; a < 3; ++a) q[OC_Z + PA_C + a] = ddir[a];
      }
      /* adjoint of the trilinear gathers: geometry levels and the colour grid */
      for (int l = 0; l < OC_LEVELS; ++l) {
        const cell_t* cl_ = &cells[(size_t)k * OC_LEVELS + l];
        for (int cc = 0; cc < 8; ++cc)
          for (int f = 0; f < OC_FEAT; ++f) grad[cl_->corner[cc] + f] += cl_->w[cc] * dz[OC_FEAT * l + f];
      }
      for (int cc = 0; cc < 8; ++cc)
        for (int f = 0; f < PA_C; ++f) grad[A[k].cvtx[cc] + f] += A[k].cw[cc] * dcf[f];
    }
  }

  /* smoothness on S_g (Sec. 3.3) with the two-hidden-layer geometry decoder:
   * g(x) = grad_x phi = sum_k p_k dz_k/dx, p = d phi/dz (pa_dphi_dz) */
  for (int p = 0; p < P; ++p) {
    if (!valid[p]) continue;
    float y[2][3];
    for (int a = 0; a < 3; ++a) {
      y[0][a] = xs[3 * p + a];
      y[1][a] = xs[3 * p + a] + eps[3 * p + a];
    }
    const double dnone[3] = {0, 0, 1};
    cell_t cl[2][OC_LEVELS];
    pa_act_t Ay[2];
    double dzdx[2][OC_Z][3], pz[2][OC_Z], pm[2][PA_H], e[2][PA_H], g[2][3];
    for (int ev = 0; ev < 2; ++ev) {
      pa_eval(c, theta, &m, y[ev], dnone, cl[ev], dzdx[ev], &Ay[ev]);
      for (int j = 0; j < PA_H; ++j) {
        mmin(&hid_margin, Ay[ev].y1[j]);
        mmin(&hid_margin, Ay[ev].y2[j]);
      }
      sigmix(&sig, ((uint64_t)1 << 60) + (uint64_t)p * 4 + (uint64_t)ev * 2, relu_mask(Ay[ev].y1, PA_H));
      sigmix(&sig, ((uint64_t)1 << 60) + (uint64_t)p * 4 + (uint64_t)ev * 2 + 1, relu_mask(Ay[ev].y2, PA_H));
      pa_dphi_dz(&m, &Ay[ev], pz[ev], pm[ev], e[ev]);
      for (int a = 0; a < 3; ++a) {
        double acc = 0;
        for (int k = 0; k < OC_Z; ++k) acc += pz[ev][k] * dzdx[ev][k][a];
        g[ev][a] = acc;
      }
    }
    double dg[3], l2 = 0;
    for (int a = 0; a < 3; ++a) {
      dg[a] = g[0][a] - g[1][a];
      l2 += dg[a] * dg[a];
    }
    lsum[4] += l2;
    if (!do_grad || n_g == 0) continue;
    pa_mlp_t gg = pa_view(gm);
    for (int ev = 0; ev < 2; ++ev) {
      /* a = dL/dg at this evaluation; a . g = p . j with j_k = a . dz_k/dx */
      double av[3], jv[OC_Z], vj[PA_H];
      for (int a = 0; a < 3; ++a) av[a] = (ev == 0 ? 1.0 : -1.0) * wt[4] / (double)n_g * 2.0 * dg[a];
      for (int k = 0; k < OC_Z; ++k) jv[k] = av[0] * dzdx[ev][k][0] + av[1] * dzdx[ev][k][1] + av[2] * dzdx[ev][k][2];
      /* grid: d(a . g)/d theta_{l,c,f} = p_{l,f} (1/v_l) (a . d w_c / d f) */
      for (int l = 0; l < OC_LEVELS; ++l)
        for (int cc = 0; cc < 8; ++cc) {
          double ad = (av[0] * cl[ev][l].dw[cc][0] + av[1] * cl[ev][l].dw[cc][1] + av[2] * cl[ev][l].dw[cc][2]) *
                      cl[ev][l].inv_v;
          for (int f = 0; f < OC_FEAT; ++f) grad[cl[ev][l].corner[cc] + f] += pz[ev][OC_FEAT * l + f] * ad;
        }
      /* decoder: a . g = (gW2 (m1 (.) gW1 j)) . (m2 (.) gw3) */
      for (int i1 = 0; i1 < PA_H; ++i1) {
        double acc = 0;
        for (int k = 0; k < OC_Z; ++k) {
          ((double*)gg.gW1)[i1 * OC_Z + k] += pm[ev][i1] * jv[k];
          acc += m.gW1[i1 * OC_Z + k] * jv[k];
        }
        vj[i1] = Ay[ev].y1[i1] > 0 ? acc : 0.0;
      }
      for (int i2 = 0; i2 < PA_H; ++i2) {
        double acc = 0;
        for (int i1 = 0; i1 < PA_H; ++i1) {
          ((double*)gg.gW2)[i2 * PA_H + i1] += e[ev][i2] * vj[i1];
          acc += m.gW2[i2 * PA_H + i1] * vj[i1];
        }
        if (Ay[ev].y2[i2] > 0) ((double*)gg.gw3)[i2] += acc;
      }
    }
  }
  free(A);
  free(cells);
  free(phi);
  free(Phi);
  free(alpha);
  free(T);
  free(w);
  free(U);
  free(dPhi);

  loss[0] = R > 0 ? lsum[0] / (double)R : 0.0;
  loss[1] = n_d > 0 ? lsum[1] / (double)n_d : 0.0;
  loss[2] = n_tr > 0 ? lsum[2] / (double)n_tr : 0.0;
  loss[3] = n_fs > 0 ? lsum[3] / (double)n_fs : 0.0;
  loss[4] = n_g > 0 ? lsum[4] / (double)n_g : 0.0;
  loss[5] = 0;
  for (int k = 0; k < 5; ++k) loss[5] += (double)c->lam[k] * loss[k];
  if (margins) {
    for (int k = 0; k < 10; ++k) margins[k] = INFINITY;
    margins[0] = hid_margin;
    margins[5] = d_margin;
    margins[7] = (double)(sig & ((1ULL << 52) - 1));
    margins[8] = margins[9] = 0.0;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* the paper's architecture: SDF query, its reverse mode, phi and kappa for the samplers  */
/* ------------------------------------------------------------------------------------ */
static double pa_kappa(const oc_config* c, const double* theta) {
  int64_t ng = 0;
  oc_paper_param_count(c, &ng);
  return theta[ng + PA_MLP - 1];
}

static double pa_phi_at(const oc_config* c, const double* theta, const float x[3]) {
  int64_t ng = 0;
  oc_paper_param_count(c, &ng);
  const pa_mlp_t m = pa_view(theta + ng);
  const double d[3] = {0, 0, 1}; /* the colour decoder's input; phi does not read it */
  cell_t cells[OC_LEVELS];
  pa_act_t A;
  pa_eval(c, theta, &m, x, d, cells, NULL, &A);
  return A.phi;
}

/* phi(x) and grad_x phi(x) = sum_k p_k dz_k/dx with p = d phi/dz (Supp. Eq. sdf_first_grad) */
static void pa_query_sdf(const oc_config* c, const double* theta, const float* x, int P, double* sdf, double* grad) {
  int64_t ng = 0;
  oc_paper_param_count(c, &ng);
  const pa_mlp_t m = pa_view(theta + ng);
  const double d[3] = {0, 0, 1};
#pragma omp parallel for schedule(static)
  for (int i = 0; i < P; ++i) {
    cell_t cells[OC_LEVELS];
    pa_act_t A;
    double dzdx[OC_Z][3];
    pa_eval(c, theta, &m, x + 3 * i, d, cells, dzdx, &A);
    sdf[i] = A.phi;
    if (grad) {
      double p[OC_Z], pm[PA_H], e[PA_H];
      pa_dphi_dz(&m, &A, p, pm, e);
      for (int a = 0; a < 3; ++a) {
        double acc = 0;
        for (int k = 0; k < OC_Z; ++k) acc += p[k] * dzdx[k][a];
        grad[3 * i + a] = acc;
      }
    }
  }
}

/* grad += sum_i dsdf_i d phi(x_i)/d theta + dgrad_i . d grad_x phi(x_i)/d theta for the
 * paper's architecture: the first term is the geometry decoder's backward pass and the
 * adjoint of the gathers; the second the second-order path of Supp. Sec. 1 through the
 * two-hidden-layer decoder (as in the smoothness term of oc_step_paper).  The colour grid
 * and the colour decoder get nothing.  dsdf or dgrad may be NULL; x carries no gradient. */
static void pa_query_sdf_backward(const oc_config* c, const double* theta, const float* x, int P, const double* dsdf,
                                  const double* dgrad, double* grad) {
  int64_t ng = 0;
  oc_paper_param_count(c, &ng);
  const pa_mlp_t m = pa_view(theta + ng);
  double* gm = grad + ng;
  pa_mlp_t gg = pa_view(gm);
  const double d[3] = {0, 0, 1};
  for (int i = 0; i < P; ++i) {
    cell_t cells[OC_LEVELS];
    pa_act_t A;
    double dzdx[OC_Z][3];
    pa_eval(c, theta, &m, x + 3 * i, d, cells, dzdx, &A);
    if (dsdf && dsdf[i] != 0.0) {
      const double dc[3] = {0, 0, 0};
      double dz[OC_Z], dcf[PA_C];
      pa_backward(&m, &A, dsdf[i], dc, gm, dz, dcf, NULL, NULL);
      for (int l = 0; l < OC_LEVELS; ++l)
        for (int cc = 0; cc < 8; ++cc)
          for (int f = 0; f < OC_FEAT; ++f) grad[cells[l].corner[cc] + f] += cells[l].w[cc] * dz[OC_FEAT * l + f];
    }
    if (dgrad) {
      const double* av = dgrad + 3 * i;
      double p[OC_Z], pm[PA_H], e[PA_H], jv[OC_Z], vj[PA_H];
      pa_dphi_dz(&m, &A, p, pm, e);
      for (int k = 0; k < OC_Z; ++k) jv[k] = av[0] * dzdx[k][0] + av[1] * dzdx[k][1] + av[2] * dzdx[k][2];
      for (int l = 0; l < OC_LEVELS; ++l)
        for (int cc = 0; cc < 8; ++cc) {
          const double ad =
              (av[0] * cells[l].dw[cc][0] + av[1] * cells[l].dw[cc][1] + av[2] * cells[l].dw[cc][2]) * cells[l].inv_v;
          for (int f = 0; f < OC_FEAT; ++f) grad[cells[l].corner[cc] + f] += p[OC_FEAT * l + f] * ad;
        }
      for (int i1 = 0; i1 < PA_H; ++i1) {
        double acc = 0;
        for (int k = 0; k < OC_Z; ++k) {
          ((double*)gg.gW1)[i1 * OC_Z + k] += pm[i1] * jv[k];
          acc += m.gW1[i1 * OC_Z + k] * jv[k];
        }
        vj[i1] = A.y1[i1] > 0 ? acc : 0.0;
      }
      for (int i2 = 0; i2 < PA_H; ++i2) {
        double acc = 0;
        for (int i1 = 0; i1 < PA_H; ++i1) {
          ((double*)gg.gW2)[i2 * PA_H + i1] += e[i2] * vj[i1];
          acc += m.gW2[i2 * PA_H + i1] * vj[i1];
        }
        if (A.y2[i2] > 0) ((double*)gg.gw3)[i2] += acc;
      }
    }
  }
}

/* Hidden pre-activations at points, for tests that must know which ReLU branches the points
 * take (diagnostic; no step result depends on it).  kink[P]: smallest relative distance of
 * any evaluated hidden unit from its kink (kink_rel).  Workload decoders: h1 [P][32] the
 * geometry decoder's layer 1, h2 [P][32] the colour decoder's layer 1 (h3, h4, d unused).
 * Paper architecture (c->arch == 1): h1, h2 the geometry decoder's two hidden layers; with
 * unit viewing directions d [P][3] also the colour decoder's, h3 and h4 (d NULL: the colour
 * decoder is not evaluated).  h1..h4 may be NULL. */
void oc_hidden_at(const oc_config* c, const double* theta, const float* x, const double* d, int P, double* kink,
                  double* h1, double* h2, double* h3, double* h4) {
  if (c->arch == 1) {
    int64_t ng = 0;
    oc_paper_param_count(c, &ng);
    pa_mlp_t m = pa_view(theta + ng);
    const double dnone[3] = {0, 0, 1};
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P; ++i) {
      cell_t cells[OC_LEVELS];
      pa_act_t A;
      pa_eval(c, theta, &m, x + 3 * i, d ? d + 3 * i : dnone, cells, NULL, &A);
      kink[i] = pa_kink(&m, &A, d != NULL);
      for (int j = 0; j < PA_H; ++j) {
        if (h1) h1[(size_t)i * PA_H + j] = A.y1[j];
        if (h2) h2[(size_t)i * PA_H + j] = A.y2[j];
        if (h3 && d) h3[(size_t)i * PA_H + j] = A.q1[j];
        if (h4 && d) h4[(size_t)i * PA_H + j] = A.q2[j];
      }
    }
    return;
  }
  mlp_t m = mlp_view(theta + grid_size(c));
#pragma omp parallel for schedule(static)
  for (int i = 0; i < P; ++i) {
    cell_t cells[OC_LEVELS];
    act_t A;
    features(c, theta, x + 3 * i, cells, A.z, NULL);
    feature_mag(theta, cells, A.zmag);
    decode(&m, &A);
    kink[i] = decode_kink(&m, &A);
    for (int j = 0; j < OC_H1; ++j)
      if (h1) h1[(size_t)i * OC_H1 + j] = A.y1[j];
    for (int j = 0; j < OC_H2; ++j)
      if (h2) h2[(size_t)i * OC_H2 + j] = A.y2[j];
  }
}

int oc_step_paper(const oc_config* c, const double* theta, int R, int N, const float* o, const float* r,
                  const float* rgb, const float* D, const float* t, const uint8_t* cls, int P, const float* xs,
                  const float* eps, const uint8_t* valid, const double* dloss, double* loss, double* rgb_hat,
                  double* d_hat, double* wsum, double* grad, double* margins, uint8_t* amb, double* w_out) {
  return step_paper_impl(c, theta, R, N, o, r, rgb, D, t, cls, P, xs, eps, valid, dloss, loss, rgb_hat, d_hat, wsum,
                         grad, margins, amb, w_out, NULL);
}

/* oc_step_paper that also returns, per main sample, dzc_out [R][N][32]: dL/dz (16), dL/dW_beta(x)
 * (6) and dL/d(viewing direction) (3), zeros after (needs grad) */
int oc_step_paper_dz(const oc_config* c, const double* theta, int R, int N, const float* o, const float* r,
                     const float* rgb, const float* D, const float* t, const uint8_t* cls, int P, const float* xs,
                     const float* eps, const uint8_t* valid, const double* dloss, double* loss, double* grad,
                     double* dzc_out) {
  return step_paper_impl(c, theta, R, N, o, r, rgb, D, t, cls, P, xs, eps, valid, dloss, loss, NULL, NULL, NULL, grad,
                         NULL, NULL, NULL, dzc_out);
}

/* Camera-pose gradient with the paper's architecture (Sec. 3.4): as oc_pose_grad, where the
 * per-ray losses reach the pose through the sample positions x_s = o + d_s r (geometry grid
 * and colour grid: g_s = (dz/dx)^T dL/dz + (dW_beta/dx)^T dL/dW_beta) and through the viewing
 * direction r/|r| = R d/|d| (d the pixel's camera direction):
 *   dL/d dt = sum_s g_s,   dL/d nu = J_r(nu)^T [d]_x R^T (sum_s d_s g_s + dL/d(dir) / |d|),
 * with dL/d(dir) = sum_s of the per-sample direction gradients in dzc [R][N][32]. */
void oc_pose_grad_paper(const oc_config* c, const oc_frames* fr, const double* theta, const double* c2w,
                        const double* xi, int R, int N, const int64_t* pix, const float* o, const float* r,
                        const float* t, const double* dzc, double* g) {
  const int64_t hw = (int64_t)fr->H * fr->W;
  const int64_t cbase = grid_size(c), off3 = level_offset(c, 3);
  for (int i = 0; i < R; ++i) {
    const int64_t f = pix[i] / hw, rem = pix[i] % hw;
    const int v = (int)(rem / fr->W), u = (int)(rem % fr->W);
    const double d[3] = {(((double)u + 0.5) - fr->cx) / fr->fx, (((double)v + 0.5) - fr->cy) / fr->fy, 1.0};
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double go[3] = {0, 0, 0}, gr[3] = {0, 0, 0}, gd[3] = {0, 0, 0};
    for (int k = 0; k < N; ++k) {
      const float* ti = t + (size_t)i * N;
      float x[3];
      for (int a = 0; a < 3; ++a) {
        float st = ti[k] * r[3 * i + a];
        x[a] = o[3 * i + a] + st;
      }
      cell_t cells[OC_LEVELS];
      double z[OC_Z], dzdx[OC_Z][3];
      features(c, theta, x, cells, z, dzdx);
      const double* q = dzc + ((size_t)i * N + k) * 32;
      for (int a = 0; a < 3; ++a) {
        double gx = 0;
        for (int e = 0; e < OC_Z; ++e) gx += dzdx[e][a] * q[e];
        /* colour features: d W_beta_f / d x_a = (1/v_3) sum_c beta_{c,f} d w_c / d f_a */
        for (int cc = 0; cc < 8; ++cc) {
          const int64_t cv = cbase + (cells[3].corner[cc] - off3) / OC_FEAT * PA_C;
          double sf = 0;
          for (int e = 0; e < PA_C; ++e) sf += theta[cv + e] * q[OC_Z + e];
          gx += sf * cells[3].dw[cc][a] * cells[3].inv_v;
        }
        go[a] += gx;
        gr[a] += (double)ti[k] * gx;
        gd[a] += q[OC_Z + PA_C + a];
      }
    }
    for (int a = 0; a < 3; ++a) g[6 * f + a] += go[a];
    double E[3][3], J[3][3], Rt_gr[3], K[3][3], w[3];
    so3_exp_jr(xi + 6 * f + 3, E, J);
    const double* Q = c2w + 12 * f;
    for (int a = 0; a < 3; ++a) gr[a] += gd[a] / dn;
    for (int a = 0; a < 3; ++a) Rt_gr[a] = Q[a] * gr[0] + Q[4 + a] * gr[1] + Q[8 + a] * gr[2];
    skew(d, K);
    for (int a = 0; a < 3; ++a) w[a] = K[a][0] * Rt_gr[0] + K[a][1] * Rt_gr[1] + K[a][2] * Rt_gr[2];
    for (int a = 0; a < 3; ++a) g[6 * f + 3 + a] += J[0][a] * w[0] + J[1][a] * w[1] + J[2][a] * w[2];
  }
}

/* ------------------------------------------------------------------------------------ */
/* camera-pose gradient of the Eikonal term (Sec. 3.3 Eq. eikonal_loss; Sec. 3.4)         */
/* ------------------------------------------------------------------------------------ */
/* grad_x phi and its x-Hessian at x, for either architecture.  phi = f(z(x)) with f
 * piecewise linear in z (ReLU decoders), so within a ReLU region grad_x phi = sum_l J_l^T p_l
 * with p = d phi / d z constant and H = sum_{l,k} p_{l,k} Hess_x z_{l,k}: the Hessian of a
 * trilinear interpolation has a zero diagonal and the off-diagonal entries h12, h13, h23 of
 * Supp. Sec. 1 in cell coordinates (times 1 / v_l^2 in metres, reading R22), zero along a
 * clamped axis (reading R15). */
static void sdf_grad_hessian(const oc_config* c, const double* theta, const float x[3], double gx[3], double H[3][3]) {
  cell_t cells[OC_LEVELS];
  double z[OC_Z], dzdx[OC_Z][3], p[OC_Z];
  if (c->arch == 1) {
    int64_t ng = 0;
    oc_paper_param_count(c, &ng);
    pa_mlp_t m = pa_view(theta + ng);
    pa_act_t A;
    const double dnone[3] = {0, 0, 1};
    pa_eval(c, theta, &m, x, dnone, cells, dzdx, &A);
    double pm[PA_H], e[PA_H];
    pa_dphi_dz(&m, &A, p, pm, e);
    (void)z;
  } else {
    mlp_t m = mlp_view(theta + grid_size(c));
    act_t A;
    features(c, theta, x, cells, A.z, dzdx);
    decode(&m, &A);
    double mw2[OC_H1];
    dphi_dz(&m, &A, p, mw2);
  }
  for (int a = 0; a < 3; ++a) {
    gx[a] = 0.0;
    for (int k = 0; k < OC_Z; ++k) gx[a] += p[k] * dzdx[k][a];
    for (int b = 0; b < 3; ++b) H[a][b] = 0.0;
  }
  for (int l = 0; l < OC_LEVELS; ++l) {
    const double iv2 = cells[l].inv_v * cells[l].inv_v;
    for (int k = 0; k < OC_FEAT; ++k) {
      double th8[8], h[3];
      for (int cc = 0; cc < 8; ++cc) th8[cc] = theta[cells[l].corner[cc] + k];
      oc_trilinear_hessian(th8, cells[l].f, h);
      const int* cl = cells[l].clamped;
      const double s = p[OC_FEAT * l + k] * iv2;
      const double h01 = (cl[0] || cl[1]) ? 0.0 : h[0], h02 = (cl[0] || cl[2]) ? 0.0 : h[1],
                   h12 = (cl[1] || cl[2]) ? 0.0 : h[2];
      H[0][1] += s * h01;
      H[1][0] += s * h01;
      H[0][2] += s * h02;
      H[2][0] += s * h02;
      H[1][2] += s * h12;
      H[2][1] += s * h12;
    }
  }
}

/* Pose gradient of dscale * L_eik, L_eik = mean over the batch's free-space samples of
 * (1 - |g_s|)^2, g_s = grad_x phi(x_s).  The samples x_s = o + d_s r move with the pose (the
 * depths d_s and the classes stay fixed, reading R36), g_s with them: d g_s / d x_s = H_s.
 * With a_s = dL/d g_s = dscale (-2 (1 - |g_s|) g_s / (|g_s| |S_fs|)) (0 where g_s = 0), the
 * sample's position gradient is H_s a_s (H_s symmetric), and it reaches the frame's pose as
 * the per-ray terms' do (oc_pose_grad):
 *   dL/d dt += sum_s H_s a_s,   dL/d nu += J_r(nu)^T [d]_x R^T sum_s d_s H_s a_s.
 * Either architecture (c->arch).  g [F][6] (+=). */
void oc_eikonal_pose_grad(const oc_config* c, const oc_frames* fr, const double* theta, const double* c2w,
                          const double* xi, int R, int N, const int64_t* pix, const float* o, const float* r,
                          const float* t, const uint8_t* cls, double dscale, double* g) {
  int64_t n_fs = 0;
  for (int64_t s = 0; s < (int64_t)R * N; ++s) n_fs += cls[s] == CLS_FS;
  if (n_fs == 0) return;
  const int64_t hw = (int64_t)fr->H * fr->W;
  for (int i = 0; i < R; ++i) {
    double go[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
    for (int k = 0; k < N; ++k) {
      const int64_t s = (int64_t)i * N + k;
      if (cls[s] != CLS_FS) continue;
      float x[3];
      for (int a = 0; a < 3; ++a) {
        float st = t[s] * r[3 * i + a];
        x[a] = o[3 * i + a] + st;
      }
      double gx[3], H[3][3];
      sdf_grad_hessian(c, theta, x, gx, H);
      const double nrm = sqrt(gx[0] * gx[0] + gx[1] * gx[1] + gx[2] * gx[2]);
      if (!(nrm > 0.0)) continue;
      const double kk = dscale * (-2.0 / (double)n_fs) * (1.0 - nrm) / nrm;
      for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        for (int b = 0; b < 3; ++b) v += H[a][b] * kk * gx[b];
        go[a] += v;
        gr[a] += (double)t[s] * v;
      }
    }
    const int64_t f = pix[i] / hw, rem = pix[i] % hw;
    const int v = (int)(rem / fr->W), u = (int)(rem % fr->W);
    const double d[3] = {(((double)u + 0.5) - fr->cx) / fr->fx, (((double)v + 0.5) - fr->cy) / fr->fy, 1.0};
    for (int a = 0; a < 3; ++a) g[6 * f + a] += go[a];
    double E[3][3], J[3][3], Rt_gr[3], K[3][3], w[3];
    so3_exp_jr(xi + 6 * f + 3, E, J);
    const double* Q = c2w + 12 * f;
    for (int a = 0; a < 3; ++a) Rt_gr[a] = Q[a] * gr[0] + Q[4 + a] * gr[1] + Q[8 + a] * gr[2];
    skew(d, K);
    for (int a = 0; a < 3; ++a) w[a] = K[a][0] * Rt_gr[0] + K[a][1] * Rt_gr[1] + K[a][2] * Rt_gr[2];
    for (int a = 0; a < 3; ++a) g[6 * f + 3 + a] += J[0][a] * w[0] + J[1][a] * w[1] + J[2][a] * w[2];
  }
}
