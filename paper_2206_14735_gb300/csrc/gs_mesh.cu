// Mesh extraction: the isosurface phi = iso of the learned SDF on a lattice (Sec. 4: the
// meshes are extracted by marching cubes at 1 cm; here each lattice cell is split into 6
// tetrahedra around its corner-0-to-corner-7 diagonal, which needs no case table and gives a
// closed surface wherever the lattice values do).
//
// lattice_sdf_pair_kernel / lattice_sdf_paper_kernel: phi at lo + (i, j, k) * step (binary32
// positions, FP32 SDF) with the workload's decoder (two points per thread, packed FMAs) or the
// paper's.
// mesh_kernel: one thread per cell; a tetrahedron with 1 or 3 corners below iso gives one
// triangle, with 2 below two; each vertex is interpolated along its tetrahedron edge from the
// endpoint of lower lattice index (cells sharing an edge produce the same point), and each
// triangle is oriented with its normal towards the corners above iso.  A warp's 32 cells take
// their slots with one atomic on a 64-bit counter (an exclusive warp scan of the per-cell
// counts places each cell's run; a floor or a wall parallel to x puts a surface cell in every
// lane); slots at or past max_tris are counted but not written.
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

// (i, j, k) of the flat index id = (k ny + j) nx + i; 32-bit division when every index of
// the lattice fits in 32 bits (a 64-bit division costs several times as many instructions)
__device__ __forceinline__ void lattice_ijk(long long id, int nx, int ny, bool narrow, int& i, int& j, int& k) {
  if (narrow) {
    const unsigned u = (unsigned)id, q = u / (unsigned)nx;
    i = (int)(u - q * (unsigned)nx);
    j = (int)(q % (unsigned)ny);
    k = (int)(q / (unsigned)ny);
  } else {
    const long long q = id / nx;
    i = (int)(id - q * nx);
    j = (int)(q % ny);
    k = (int)(q / ny);
  }
}

// lattice point id's position lo + (i, j, k) step
__device__ __forceinline__ void lattice_x(const LatticeArgs& a, long long id, bool narrow, float x[3]) {
  int i, j, k;
  lattice_ijk(id, a.nx, a.ny, narrow, i, j, k);
  x[0] = __fadd_rn(a.lo[0], __fmul_rn((float)i, a.step));
  x[1] = __fadd_rn(a.lo[1], __fmul_rn((float)j, a.step));
  x[2] = __fadd_rn(a.lo[2], __fmul_rn((float)k, a.step));
}

// The paper's decoder: one lattice point per thread, phi from its two hidden layers.
__global__ void __launch_bounds__(128) lattice_sdf_paper_kernel(LatticeArgs a) {
  __shared__ __align__(16) float sm[paper::kGeoPad];
  paper::load_geometry_decoder(a.theta + a.g.n_grid, sm);
  __syncthreads();
  const long long np = (long long)a.nx * a.ny * a.nz;
  const bool narrow = np <= 0xffffffffLL;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < np; id += (long long)gridDim.x * blockDim.x) {
    float x[3];
    lattice_x(a, id, narrow, x);
    a.phi[id] = paper::phi_at(a.g, a.theta, sm, x);
  }
}

// packed pair of FP32 values: element 0 in the low half
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
// both halves: d = a * b + c, each an IEEE fma rounded to nearest, as fmaf
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// The workload's decoder: two neighbouring lattice points per thread, their features side by
// side in packed pairs; every weight is kept twice in shared memory so that one 128-bit
// broadcast read gives two packed weight pairs and one packed FMA advances both points.  Per
// point the operations and their order are sdf_at's, so phi is the same to the bit.
struct LatticePairDecoder {
  unsigned long long W1[kH1][kZ];  // (W1[j][k], W1[j][k])
  unsigned long long bw[kH1][2];   // (b1[j], b1[j]), (W2[0][j], W2[0][j])
  unsigned long long b2;           // (b2[0], b2[0])
};

__global__ void __launch_bounds__(128) lattice_sdf_pair_kernel(LatticeArgs a) {
  __shared__ __align__(16) LatticePairDecoder d;
  const float* mlp = a.theta + a.g.n_grid;
  for (int i = threadIdx.x; i < kH1 * kZ; i += blockDim.x) {
    const float v = mlp[oW1 + i];
    d.W1[i / kZ][i % kZ] = pk2(v, v);
  }
  for (int j = threadIdx.x; j < kH1; j += blockDim.x) {
    d.bw[j][0] = pk2(mlp[ob1 + j], mlp[ob1 + j]);
    d.bw[j][1] = pk2(mlp[oW2 + j], mlp[oW2 + j]);
  }
  if (threadIdx.x == 0) d.b2 = pk2(mlp[ob2], mlp[ob2]);
  __syncthreads();
  const long long np = (long long)a.nx * a.ny * a.nz, npair = (np + 1) / 2;
  const bool narrow = np <= 0xffffffffLL;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npair; p += (long long)gridDim.x * blockDim.x) {
    const long long id0 = 2 * p, id1 = id0 + 1 < np ? id0 + 1 : id0;  // an odd count repeats the last point
    unsigned long long zz[kZ];
    {
      float x[3], z0[kZ], z1[kZ];
      lattice_x(a, id0, narrow, x);
      grid_z(a.g, a.theta, x, z0);
      lattice_x(a, id1, narrow, x);
      grid_z(a.g, a.theta, x, z1);
#pragma unroll
      for (int k = 0; k < kZ; ++k) zz[k] = pk2(z0[k], z1[k]);
    }
    unsigned long long phi = d.b2;
#pragma unroll 4
    for (int j = 0; j < kH1; ++j) {
      unsigned long long s = d.bw[j][0];
#pragma unroll
      for (int k = 0; k < kZ; ++k) s = ffma2(d.W1[j][k], zz[k], s);
      float s0, s1;
      upk2(s, s0, s1);
      phi = ffma2(d.bw[j][1], pk2(fmaxf(s0, 0.f), fmaxf(s1, 0.f)), phi);
    }
    float phi0, phi1;
    upk2(phi, phi0, phi1);
    a.phi[id0] = phi0;
    if (id1 != id0) a.phi[id1] = phi1;
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

// corner q (bit 0: +x, bit 1: +y, bit 2: +z) of the cell with lower corner (i, j, k)
__device__ __forceinline__ void mesh_corner(const MeshArgs& a, int i, int j, int k, int q, float out[3]) {
  out[0] = __fadd_rn(a.lo[0], __fmul_rn((float)(i + (q & 1)), a.step));
  out[1] = __fadd_rn(a.lo[1], __fmul_rn((float)(j + ((q >> 1) & 1)), a.step));
  out[2] = __fadd_rn(a.lo[2], __fmul_rn((float)(k + (q >> 2)), a.step));
}

// the point of phi = iso on the edge between corners qa and qb, interpolated from the endpoint
// of lower lattice index: with nx, ny >= 2 the lattice index of corner q grows with q
__device__ __forceinline__ void mesh_edge(const MeshArgs& a, int i, int j, int k, const float f[8], int qa, int qb,
                                          float out[3]) {
  if (qb < qa) {
    const int t = qa;
    qa = qb;
    qb = t;
  }
  const float w = (a.iso - f[qa]) / (f[qb] - f[qa]);
  float A[3], B[3];
  mesh_corner(a, i, j, k, qa, A);
  mesh_corner(a, i, j, k, qb, B);
#pragma unroll
  for (int q = 0; q < 3; ++q) out[q] = A[q] + w * (B[q] - A[q]);
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
  const int lane = threadIdx.x & 31;
  const bool narrow = ncell + 32LL * gridDim.x * blockDim.x <= 0xffffffffLL;
  // the loop runs warp-uniformly (c0 is the same for all lanes) so that the slot scan below
  // always has the whole warp; lanes past the last cell take part with a count of 0
  for (long long c0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < ncell;
       c0 += (long long)gridDim.x * blockDim.x) {
    const long long c = c0 + lane;
    const bool live = c < ncell;
    const long long cc = live ? c : 0;
    int i, j, k;
    lattice_ijk(cc, (int)cx, (int)cy, narrow, i, j, k);
    // the eight values stay in registers (static indices) for the test every cell takes
    float f[8];
    unsigned m = 0;  // bit q: corner q below iso
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      f[q] = a.phi[((long long)(k + (q >> 2)) * a.ny + j + ((q >> 1) & 1)) * a.nx + i + (q & 1)];
      m |= (f[q] < a.iso ? 1u : 0u) << q;
    }
    // triangles of this cell: the corners of tetrahedron t below iso are m & kTetMask[t]
    int cnt = 0;
    if (live && m != 0u && m != 0xffu) {
      constexpr unsigned kTetMask[6] = {0x8Bu, 0x8Du, 0xC5u, 0xD1u, 0xB1u, 0xA3u};
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const int ni = __popc(m & kTetMask[t]);
        cnt += (ni == 0 || ni == 4) ? 0 : (ni == 2 ? 2 : 1);
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    unsigned long long base = 0;
    if (lane == 31 && incl > 0) base = atomicAdd(a.n_tris, (unsigned long long)incl);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (cnt == 0) continue;
    unsigned long long slot = base + (unsigned long long)(incl - cnt);
    // surface cells only: a copy that the tetrahedra below index by corner number
    float fs[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) fs[q] = f[q];
#pragma unroll 1
    for (int t = 0; t < 6; ++t) {
      int in[4], out[4], ni = 0, no = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int v = kTets[t][q];
        if (fs[v] < a.iso) in[ni++] = v;
        else out[no++] = v;
      }
      if (ni == 0 || no == 0) continue;
      float dir[3], so[3] = {0.f, 0.f, 0.f}, si[3] = {0.f, 0.f, 0.f}, Pq[3];
      for (int q = 0; q < no; ++q) {
        mesh_corner(a, i, j, k, out[q], Pq);
#pragma unroll
        for (int d = 0; d < 3; ++d) so[d] += Pq[d];
      }
      for (int q = 0; q < ni; ++q) {
        mesh_corner(a, i, j, k, in[q], Pq);
#pragma unroll
        for (int d = 0; d < 3; ++d) si[d] += Pq[d];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) dir[d] = so[d] / (float)no - si[d] / (float)ni;
      float p0[3], p1[3], p2[3], p3[3];
      if (ni == 1 || no == 1) {
        const int apex = ni == 1 ? in[0] : out[0];
        const int* rest = ni == 1 ? out : in;
        mesh_edge(a, i, j, k, fs, apex, rest[0], p0);
        mesh_edge(a, i, j, k, fs, apex, rest[1], p1);
        mesh_edge(a, i, j, k, fs, apex, rest[2], p2);
        if ((long long)slot < a.max_tris) mesh_put(a.tris + 9 * slot, p0, p1, p2, dir);
        ++slot;
      } else {
        mesh_edge(a, i, j, k, fs, in[0], out[0], p0);
        mesh_edge(a, i, j, k, fs, in[0], out[1], p1);
        mesh_edge(a, i, j, k, fs, in[1], out[1], p2);
        mesh_edge(a, i, j, k, fs, in[1], out[0], p3);
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
  if (ctx->cfg.arch == GS_ARCH_PAPER) {
    const int blocks = (int)std::min<long long>((np + 127) / 128, 64LL * ctx->num_sms);
    lattice_sdf_paper_kernel<<<blocks, 128, 0, st>>>(la);
  } else {
    const int blocks = (int)std::min<long long>(((np + 1) / 2 + 127) / 128, 64LL * ctx->num_sms);
    lattice_sdf_pair_kernel<<<blocks, 128, 0, st>>>(la);
  }
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
