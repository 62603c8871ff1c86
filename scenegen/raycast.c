/*
 * Seeded synthetic RGB-D frame generator (input synthesis only).
 *
 * Renders posed pinhole RGB-D frames of scenes built from analytic primitives
 * (room interior box, solid boxes, spheres, capsules).  Depth is the exact
 * first-hit z-depth along each pixel ray (the value sphere tracing of the
 * scene SDF converges to), with optional Gaussian noise sigma = k * z^2,
 * i.i.d. pixel dropout and contiguous disc-shaped dropout blobs.
 *
 * This file holds no step of the reconstruction method: it only makes the
 * seeded inputs that both the CUDA path and the CPU oracle consume.
 *
 * Conventions: OpenCV camera (x right, y down, z forward), c2w poses stored
 * row-major [3][4]; ray direction R * ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1) so the
 * ray parameter equals z-depth; misses get depth 0 and colour 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { SG_ROOM = 0, SG_BOX = 1, SG_SPHERE = 2, SG_CAPSULE = 3 };

typedef struct {
  int32_t kind;
  int32_t pad;
  double a[3];   /* room/box: centre; sphere: centre; capsule: end point A */
  double b[3];   /* room/box: half extents; capsule: end point B */
  double r;      /* sphere/capsule radius */
  double col[3]; /* base colour in [0,1] */
} sg_prim;

/* SplitMix64 finaliser step (Steele, Lea & Flood 2014); generator-private. */
static inline uint64_t sg_mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
static inline double sg_unif(uint64_t h) { return (double)(h >> 11) * 0x1p-53; }

static const double SG_TMIN = 1e-4;

static double hit_sphere(const double o[3], const double d[3], const double c[3], double r) {
  double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
  double A = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double B = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
  double C = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - r * r;
  double disc = B * B - A * C;
  if (disc < 0) return INFINITY;
  double s = sqrt(disc);
  double t0 = (-B - s) / A, t1 = (-B + s) / A;
  if (C > 0) return t0 > SG_TMIN ? t0 : INFINITY; /* origin outside */
  (void)t1;
  return INFINITY; /* origin inside a solid: not visible from inside */
}

/* slab test; inside=1 returns the exit distance (room interior) */
static double hit_box(const double o[3], const double d[3], const double c[3], const double h[3], int inside) {
  double tn = -INFINITY, tf = INFINITY;
  for (int a = 0; a < 3; ++a) {
    double lo = c[a] - h[a], hi = c[a] + h[a];
    if (d[a] == 0.0) {
      if (o[a] < lo || o[a] > hi) return INFINITY;
      continue;
    }
    double t1 = (lo - o[a]) / d[a], t2 = (hi - o[a]) / d[a];
    if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; }
    if (t1 > tn) tn = t1;
    if (t2 < tf) tf = t2;
  }
  if (tn > tf) return INFINITY;
  if (inside) return tf > SG_TMIN ? tf : INFINITY;
  return tn > SG_TMIN ? tn : INFINITY;
}

static double hit_capsule(const double o[3], const double d[3], const double pa[3], const double pb[3], double r) {
  double best = INFINITY;
  double ax[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
  double L = sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
  if (L > 0) {
    double u[3] = {ax[0] / L, ax[1] / L, ax[2] / L};
    double oa[3] = {o[0] - pa[0], o[1] - pa[1], o[2] - pa[2]};
    double dd = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
    double od = oa[0] * u[0] + oa[1] * u[1] + oa[2] * u[2];
    double dp[3] = {d[0] - dd * u[0], d[1] - dd * u[1], d[2] - dd * u[2]};
    double op[3] = {oa[0] - od * u[0], oa[1] - od * u[1], oa[2] - od * u[2]};
    double A = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
    double B = dp[0] * op[0] + dp[1] * op[1] + dp[2] * op[2];
    double C = op[0] * op[0] + op[1] * op[1] + op[2] * op[2] - r * r;
    double disc = B * B - A * C;
    if (A > 0 && disc >= 0 && C > 0) {
      double t = (-B - sqrt(disc)) / A;
      double s = od + t * dd;
      if (t > SG_TMIN && s >= 0 && s <= L) best = t;
    }
  }
  double t1 = hit_sphere(o, d, pa, r), t2 = hit_sphere(o, d, pb, r);
  if (t1 < best) best = t1;
  if (t2 < best) best = t2;
  return best;
}

static void shade(int mode, const sg_prim* p, const double x[3], double out[3]) {
  if (mode == 0) {
    /* c_j = 0.5 + 0.5 sin(k_j x_j + phase_j), k = (3,5,7) 1/m, phase = (0,1,2) */
    out[0] = 0.5 + 0.5 * sin(3.0 * x[0] + 0.0);
    out[1] = 0.5 + 0.5 * sin(5.0 * x[1] + 1.0);
    out[2] = 0.5 + 0.5 * sin(7.0 * x[2] + 2.0);
  } else {
    double tex = 0.75 + 0.25 * sin(3.0 * x[0] + 5.0 * x[1] + 7.0 * x[2]);
    for (int j = 0; j < 3; ++j) out[j] = p->col[j] * tex;
  }
}

/*
 * Render F frames.  poses: [F][3][4] float64 c2w.  Outputs: rgb u8 [F][H][W][3],
 * depth f32 [F][H][W] (noisy, with dropout), gt f32 [F][H][W] (noise-free, may be NULL).
 * noise_k: sigma = noise_k * z^2 (0 disables); drop_p: i.i.d. dropout probability;
 * blob_frac: per frame, zero discs until this fraction of pixels is dropped (0 disables).
 */
void sg_render(const sg_prim* prims, int n_prims, int shade_mode, const double* poses, int F, int H, int W,
               double fx, double fy, double cx, double cy, double noise_k, double drop_p, double blob_frac,
               uint64_t seed, uint8_t* rgb, float* depth, float* gt) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int f = 0; f < F; ++f) {
    const double* P = poses + 12 * (size_t)f;
    for (int v = 0; v < H; ++v) {
      for (int u = 0; u < W; ++u) {
        double cd[3] = {(u + 0.5 - cx) / fx, (v + 0.5 - cy) / fy, 1.0};
        double o[3] = {P[3], P[7], P[11]};
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = P[4 * a] * cd[0] + P[4 * a + 1] * cd[1] + P[4 * a + 2] * cd[2];
        double best = INFINITY;
        int bi = -1;
        for (int k = 0; k < n_prims; ++k) {
          const sg_prim* p = prims + k;
          double t = INFINITY;
          if (p->kind == SG_ROOM) t = hit_box(o, d, p->a, p->b, 1);
          else if (p->kind == SG_BOX) t = hit_box(o, d, p->a, p->b, 0);
          else if (p->kind == SG_SPHERE) t = hit_sphere(o, d, p->a, p->r);
          else if (p->kind == SG_CAPSULE) t = hit_capsule(o, d, p->a, p->b, p->r);
          if (t < best) { best = t; bi = k; }
        }
        size_t idx = ((size_t)f * H + v) * W + u;
        if (bi < 0) {
          rgb[3 * idx] = rgb[3 * idx + 1] = rgb[3 * idx + 2] = 0;
          depth[idx] = 0.0f;
          if (gt) gt[idx] = 0.0f;
          continue;
        }
        double x[3] = {o[0] + best * d[0], o[1] + best * d[1], o[2] + best * d[2]};
        double c[3];
        shade(shade_mode, prims + bi, x, c);
        for (int j = 0; j < 3; ++j) {
          double q = floor(c[j] * 255.0 + 0.5);
          rgb[3 * idx + j] = (uint8_t)(q < 0 ? 0 : (q > 255 ? 255 : q));
        }
        double z = best;
        if (gt) gt[idx] = (float)z;
        uint64_t h0 = sg_mix(sg_mix(seed ^ 0xD1B54A32D192ED03ULL) ^ (uint64_t)idx);
        if (noise_k > 0) {
          uint64_t h1 = sg_mix(h0), h2 = sg_mix(h1);
          double u1 = sg_unif(h1), u2 = sg_unif(h2);
          if (u1 < 1e-300) u1 = 1e-300;
          double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
          z += noise_k * best * best * g;
          if (z < 0) z = 0;
        }
        if (drop_p > 0 && sg_unif(sg_mix(h0 ^ 0x5851F42D4C957F2DULL)) < drop_p) z = 0.0;
        depth[idx] = (float)z;
      }
    }
    if (blob_frac > 0) {
      /* contiguous dropout: seeded discs until blob_frac of the frame's pixels are zeroed */
      size_t npx = (size_t)H * W, zeroed = 0;
      uint8_t* mask = (uint8_t*)calloc(npx, 1);
      uint64_t hb = sg_mix(seed ^ 0xA24BAED4963EE407ULL ^ ((uint64_t)f << 20));
      int guard = 0;
      while ((double)zeroed < blob_frac * (double)npx && guard++ < 10000) {
        hb = sg_mix(hb);
        double bx = sg_unif(hb) * W;
        hb = sg_mix(hb);
        double by = sg_unif(hb) * H;
        hb = sg_mix(hb);
        double br = (0.03 + 0.09 * sg_unif(hb)) * (H < W ? H : W);
        int y0 = (int)(by - br), y1 = (int)(by + br) + 1, x0 = (int)(bx - br), x1 = (int)(bx + br) + 1;
        if (y0 < 0) y0 = 0;
        if (x0 < 0) x0 = 0;
        if (y1 > H) y1 = H;
        if (x1 > W) x1 = W;
        for (int yy = y0; yy < y1; ++yy)
          for (int xx = x0; xx < x1; ++xx) {
            double ddx = xx + 0.5 - bx, ddy = yy + 0.5 - by;
            if (ddx * ddx + ddy * ddy <= br * br && !mask[(size_t)yy * W + xx]) {
              mask[(size_t)yy * W + xx] = 1;
              ++zeroed;
            }
          }
      }
      for (size_t i = 0; i < npx; ++i)
        if (mask[i]) depth[(size_t)f * npx + i] = 0.0f;
      free(mask);
    }
  }
}

/* Exact scene SDF (negative inside solids, positive in free space) for tests. */
double sg_sdf(const sg_prim* prims, int n_prims, const double x[3]) {
  double best = INFINITY;
  for (int k = 0; k < n_prims; ++k) {
    const sg_prim* p = prims + k;
    double s;
    if (p->kind == SG_SPHERE) {
      double dx = x[0] - p->a[0], dy = x[1] - p->a[1], dz = x[2] - p->a[2];
      s = sqrt(dx * dx + dy * dy + dz * dz) - p->r;
    } else if (p->kind == SG_BOX || p->kind == SG_ROOM) {
      double q[3], out = 0, mx = -INFINITY;
      for (int a = 0; a < 3; ++a) {
        q[a] = fabs(x[a] - p->a[a]) - p->b[a];
        if (q[a] > 0) out += q[a] * q[a];
        if (q[a] > mx) mx = q[a];
      }
      s = sqrt(out) + (mx < 0 ? mx : 0);
      if (p->kind == SG_ROOM) s = -s;
    } else {
      double ba[3] = {p->b[0] - p->a[0], p->b[1] - p->a[1], p->b[2] - p->a[2]};
      double pa[3] = {x[0] - p->a[0], x[1] - p->a[1], x[2] - p->a[2]};
      double bb = ba[0] * ba[0] + ba[1] * ba[1] + ba[2] * ba[2];
      double hh = bb > 0 ? (pa[0] * ba[0] + pa[1] * ba[1] + pa[2] * ba[2]) / bb : 0;
      if (hh < 0) hh = 0;
      if (hh > 1) hh = 1;
      double e[3] = {pa[0] - hh * ba[0], pa[1] - hh * ba[1], pa[2] - hh * ba[2]};
      s = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) - p->r;
    }
    if (s < best) best = s;
  }
  return best;
}

/* Scene SDF at P points x [P][3] (OpenMP). */
void sg_sdf_batch(const sg_prim* prims, int n_prims, const double* x, long long P, double* out) {
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < P; ++i) out[i] = sg_sdf(prims, n_prims, x + 3 * i);
}
