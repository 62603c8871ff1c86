// Mesh extraction: the isosurface phi = iso of the learned SDF on a lattice (Sec. 4: the
// meshes are extracted by marching cubes at 1 cm; here each lattice cell is split into 6
// tetrahedra around its corner-0-to-corner-7 diagonal, which needs no case table and gives a
// closed surface wherever the lattice values do).
//
// lattice_sdf_kernel: phi at lo + (i, j, k) * step (binary32 positions, FP32 SDF).
// mesh_kernel: one thread per cell; a tetrahedron with 1 or 3 corners below iso gives one
// triangle, with 2 below two; each vertex is interpolated along its tetrahedron edge from the
// endpoint of lower lattice index (cells sharing an edge produce the same point), and each
// triangle is oriented with its normal towards the corners above iso.  A cell's triangles
// take their slots with one atomic on a 64-bit counter; slots at or past max_tris are counted
// but not written.
#include <algorithm>

#include "gs_internal.h"
#include "gs_paper.cuh"

namespace gs {

struct LatticeArgs {
  GridDesc g;
  const float* theta;
  float lo[3];
  float step;
  int nx, ny, nz;
  float* phi;
};

// kPaper: phi from the paper's two-hidden-layer geometry decoder (GS_ARCH_PAPER)
template <bool kPaper>
__global__ void __launch_bounds__(128) lattice_sdf_kernel(LatticeArgs a) {
  __shared__ __align__(16) float sm[kPaper ? paper::kGeoPad : sb2 + 4];
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
  const long long np = (long long)a.nx * a.ny * a.nz;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < np; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % a.nx), j = (int)((id / a.nx) % a.ny), k = (int)(id / ((long long)a.nx * a.ny));
    const float x[3] = {__fadd_rn(a.lo[0], __fmul_rn((float)i, a.step)), __fadd_rn(a.lo[1], __fmul_rn((float)j, a.step)),
                        __fadd_rn(a.lo[2], __fmul_rn((float)k, a.step))};
    a.phi[id] = kPaper ? paper::phi_at(a.g, a.theta, sm, x) : sdf_at(a.g, a.theta, sm, x);
  }
}

struct MeshArgs {
  float lo[3];
  float step;
  int nx, ny, nz;
  float iso;
  const float* phi;
  float* tris;  // [max_tris][3][3]
  long long max_tris;
  unsigned long long* n_tris;
};

__constant__ int kTets[6][4] = {{0, 1, 3, 7}, {0, 3, 2, 7}, {0, 2, 6, 7}, {0, 6, 4, 7}, {0, 4, 5, 7}, {0, 5, 1, 7}};

__device__ __forceinline__ void mesh_edge(const float P[8][3], const float f[8], const long long id[8], int a, int b,
                                          float iso, float out[3]) {
  if (id[b] < id[a]) {
    const int t = a;
    a = b;
    b = t;
  }
  const float w = (iso - f[a]) / (f[b] - f[a]);
#pragma unroll
  for (int q = 0; q < 3; ++q) out[q] = P[a][q] + w * (P[b][q] - P[a][q]);
}

__device__ __forceinline__ void mesh_put(float* dst, const float p0[3], const float p1[3], const float p2[3],
                                         const float dir[3]) {
  const float e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
  const float e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
  const float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const bool flip = n[0] * dir[0] + n[1] * dir[1] + n[2] * dir[2] < 0.f;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    dst[q] = p0[q];
    dst[3 + q] = flip ? p2[q] : p1[q];
    dst[6 + q] = flip ? p1[q] : p2[q];
  }
}

__global__ void __launch_bounds__(128) mesh_kernel(MeshArgs a) {
  const long long cx = a.nx - 1, cy = a.ny - 1, ncell = cx * cy * (a.nz - 1);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % cx), j = (int)((c / cx) % cy), k = (int)(c / (cx * cy));
    float P[8][3], f[8];
    long long id[8];
    bool below = false, above = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int ii = i + (q & 1), jj = j + ((q >> 1) & 1), kk = k + (q >> 2);
      id[q] = ((long long)kk * a.ny + jj) * a.nx + ii;
      f[q] = a.phi[id[q]];
      P[q][0] = __fadd_rn(a.lo[0], __fmul_rn((float)ii, a.step));
      P[q][1] = __fadd_rn(a.lo[1], __fmul_rn((float)jj, a.step));
      P[q][2] = __fadd_rn(a.lo[2], __fmul_rn((float)kk, a.step));
      below |= f[q] < a.iso;
      above |= !(f[q] < a.iso);
    }
    if (!(below && above)) continue;
    // triangles of this cell: count first, then one slot reservation
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      int ni = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) ni += f[kTets[t][q]] < a.iso;
      cnt += (ni == 0 || ni == 4) ? 0 : (ni == 2 ? 2 : 1);
    }
    unsigned long long slot = atomicAdd(a.n_tris, (unsigned long long)cnt);
#pragma unroll 1
    for (int t = 0; t < 6; ++t) {
      int in[4], out[4], ni = 0, no = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int v = kTets[t][q];
        if (f[v] < a.iso) in[ni++] = v;
        else out[no++] = v;
      }
      if (ni == 0 || no == 0) continue;
      float dir[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float so = 0.f, si = 0.f;
        for (int q = 0; q < no; ++q) so += P[out[q]][d];
        for (int q = 0; q < ni; ++q) si += P[in[q]][d];
        dir[d] = so / (float)no - si / (float)ni;
      }
      float p0[3], p1[3], p2[3], p3[3];
      if (ni == 1 || no == 1) {
        const int apex = ni == 1 ? in[0] : out[0];
        const int* rest = ni == 1 ? out : in;
        mesh_edge(P, f, id, apex, rest[0], a.iso, p0);
        mesh_edge(P, f, id, apex, rest[1], a.iso, p1);
        mesh_edge(P, f, id, apex, rest[2], a.iso, p2);
        if ((long long)slot < a.max_tris) mesh_put(a.tris + 9 * slot, p0, p1, p2, dir);
        ++slot;
      } else {
        mesh_edge(P, f, id, in[0], out[0], a.iso, p0);
        mesh_edge(P, f, id, in[0], out[1], a.iso, p1);
        mesh_edge(P, f, id, in[1], out[1], a.iso, p2);
        mesh_edge(P, f, id, in[1], out[0], a.iso, p3);
        if ((long long)slot < a.max_tris) mesh_put(a.tris + 9 * slot, p0, p1, p2, dir);
        ++slot;
        if ((long long)slot < a.max_tris) mesh_put(a.tris + 9 * slot, p0, p2, p3, dir);
        ++slot;
      }
    }
  }
}

}  // namespace gs

using namespace gs;

gs_status gs_launch_mesh(const gs_ctx* ctx, const float* theta, const float lo[3], float step, int nx, int ny, int nz,
                         float iso, float* phi, float* tris, long long max_tris, unsigned long long* n_tris,
                         cudaStream_t st) {
  if (cudaMemsetAsync(n_tris, 0, sizeof(unsigned long long), st) != cudaSuccess) return GS_ERR_CUDA;
  LatticeArgs la;
  la.g = ctx->grid;
  la.theta = theta;
  for (int q = 0; q < 3; ++q) la.lo[q] = lo[q];
  la.step = step;
  la.nx = nx;
  la.ny = ny;
  la.nz = nz;
  la.phi = phi;
  const long long np = (long long)nx * ny * nz;
  const int blocks = (int)std::min<long long>((np + 127) / 128, 64LL * ctx->num_sms);
  if (ctx->cfg.arch == GS_ARCH_PAPER) lattice_sdf_kernel<true><<<blocks, 128, 0, st>>>(la);
  else lattice_sdf_kernel<false><<<blocks, 128, 0, st>>>(la);
  MeshArgs ma;
  for (int q = 0; q < 3; ++q) ma.lo[q] = lo[q];
  ma.step = step;
  ma.nx = nx;
  ma.ny = ny;
  ma.nz = nz;
  ma.iso = iso;
  ma.phi = phi;
  ma.tris = tris;
  ma.max_tris = tris ? max_tris : 0;
  ma.n_tris = n_tris;
  const long long ncell = (long long)(nx - 1) * (ny - 1) * (nz - 1);
  const int mblocks = (int)std::min<long long>((ncell + 127) / 128, 64LL * ctx->num_sms);
  mesh_kernel<<<mblocks, 128, 0, st>>>(ma);
  return cudaPeekAtLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
