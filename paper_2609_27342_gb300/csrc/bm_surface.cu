// Reference-grid surface reconstruction (Sec. III-F) as CUDA kernels over a
// scene's sub-cell particle lattice: links disconnected where the side codes
// conflict, local regions per lattice cell, one dual-contouring vertex per
// region with Hermite data, quads around every Hermite link, and the one-way
// side-aware trilinear embedding in the logical grids' motion fields.  It is
// visual only: nothing here feeds back into the substep.
//
// Every output index is fixed by the lattice order (cells x-fastest, then
// regions by lowest corner; links by lower end, then axis; lower end's quad
// first), through count / exclusive-scan / write passes without atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bm_internal.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kQefCut = 0.1f;  // eigenvalues of sum n n^T below this count as zero (unit normals)
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int lat_at(const SurfParams &sp, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= sp.n[0] || y >= sp.n[1] || z >= sp.n[2]) return -1;
  return sp.lat[((long long)z * sp.n[1] + y) * sp.n[0] + x];
}

__device__ __forceinline__ uint32_t conflict_bits(uint32_t a1, uint32_t a2, uint32_t b1, uint32_t b2) {
  return (a1 & b2) | (a2 & b1);
}

__device__ __forceinline__ void cell_of(const SurfParams &sp, long long i, int j[3]) {
  j[0] = (int)(i % sp.nc[0]) - 1;
  j[1] = (int)((i / sp.nc[0]) % sp.nc[1]) - 1;
  j[2] = (int)(i / ((long long)sp.nc[0] * sp.nc[1])) - 1;
}

__device__ __forceinline__ long long cell_index(const SurfParams &sp, const int j[3]) {
  return ((long long)(j[2] + 1) * sp.nc[1] + (j[1] + 1)) * sp.nc[0] + (j[0] + 1);
}

// Corners (q = qx + 2 qy + 4 qz) of the cell with lower corner j: particle
// (scene-relative, -1 empty), code, and region by union-find over the
// connected links; regions are numbered by their lowest corner.
struct CellInfo {
  int part[8];
  uint32_t c1[8], c2[8];
  int reg[8];
  int nreg;
};

__device__ void cell_info(const World &w, const SurfParams &sp, const int j[3], CellInfo &ci) {
  int parent[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int p = lat_at(sp, j[0] + (q & 1), j[1] + ((q >> 1) & 1), j[2] + ((q >> 2) & 1));
    ci.part[q] = p;
    ci.c1[q] = p >= 0 ? w.P.s1[sp.p_begin + p] : 0u;
    ci.c2[q] = p >= 0 ? w.P.s2[sp.p_begin + p] : 0u;
    parent[q] = q;
  }
  for (int q = 0; q < 8; ++q)
    for (int a = 0; a < 3; ++a) {
      if ((q >> a) & 1) continue;
      const int r = q | (1 << a);
      if (ci.part[q] < 0 || ci.part[r] < 0) continue;
      if (conflict_bits(ci.c1[q], ci.c2[q], ci.c1[r], ci.c2[r])) continue;
      int x = q, y = r;
      while (parent[x] != x) x = parent[x];
      while (parent[y] != y) y = parent[y];
      if (x != y) parent[max(x, y)] = min(x, y);  // roots stay the lowest corners
    }
  ci.nreg = 0;
  for (int q = 0; q < 8; ++q) {
    if (ci.part[q] < 0) {
      ci.reg[q] = -1;
      continue;
    }
    int x = q;
    while (parent[x] != x) x = parent[x];
    ci.reg[q] = (x == q) ? ci.nreg++ : ci.reg[x];
  }
}

// Hermite data of the cell edge qa -> qb (axis a) seen from corner qa, in
// coordinates relative to the cell's lower corner jl: false when qa is empty
// or the link is connected.
__device__ bool hermite(const SurfParams &sp, const DevScene &sc, const CellInfo &ci, const int jl[3],
                        int qa, int qb, int a, float p[3], float nrm[3]) {
  const int pa = ci.part[qa], pb = ci.part[qb];
  if (pa < 0) return false;
  const float sgn = qb > qa ? 1.f : -1.f;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    p[t] = (float)(((qa >> t) & 1) * sp.h[t]);
    nrm[t] = 0.f;
  }
  if (pb >= 0) {
    const uint32_t c = conflict_bits(ci.c1[qa], ci.c2[qa], ci.c1[qb], ci.c2[qb]);
    if (!c) return false;
    const int k = __ffs(c) - 1;  // lowest conflicting cut
    if ((sc.cutpl_set >> k) & 1u) {
      // crossing of the cut's plane n . X = off with the link, clamped
      const double da = sgn * sp.h[a];
      const double den = sc.cutpl[k][a] * da;
      double t = 0.5;
      if (fabs(den) > 1e-6 * sp.h[a]) {
        double nx = 0.0;
        for (int u = 0; u < 3; ++u) nx += sc.cutpl[k][u] * (sp.Xmin[u] + (jl[u] + ((qa >> u) & 1)) * sp.h[u]);
        t = fmin(fmax((sc.cutpl[k][3] - nx) / den, 0.0), 1.0);
      }
      p[a] += (float)(t * da);
      const float s = ((ci.c1[qa] >> k) & 1u) ? 1.f : -1.f;  // digit 1 lies on the -n side
#pragma unroll
      for (int u = 0; u < 3; ++u) nrm[u] = s * (float)sc.cutpl[k][u];
      return true;
    }
  }
  // boundary link (voxel face), or a cut without a recorded plane: midpoint
  p[a] += 0.5f * sgn * (float)sp.h[a];
  nrm[a] = sgn;
  return true;
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations:
// on return A is diagonal (the eigenvalues) and the columns of V the vectors.
__device__ void jacobi3(float A[3][3], float V[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.f : 0.f;
  for (int sweep = 0; sweep < 10; ++sweep) {
    const float off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const float dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-14f * dia || off < 1e-30f) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const float apq = A[p][q];
      if (fabsf(apq) < 1e-30f) continue;
      // rotation angle with tan t that zeroes A[p][q]
      const float theta = (A[q][q] - A[p][p]) / (2.f * apq);
      const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      const float c = 1.f / sqrtf(t * t + 1.f), s = t * c;
      const int r = 3 - p - q;
      const float arp = A[r][p], arq = A[r][q];
      A[p][p] -= t * apq;
      A[q][q] += t * apq;
      A[p][q] = A[q][p] = 0.f;
      A[r][p] = A[p][r] = c * arp - s * arq;
      A[r][q] = A[q][r] = s * arp + c * arq;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
}

// --------------------------------------------------------------------------
// lattice map: lattice point -> particle, and the reference positions
// --------------------------------------------------------------------------
__global__ void k_sf_map(World w, SurfParams sp, int n, const int *jlin, const float *Xc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // scene-relative pool index
  if (i >= n) return;
  const int c = w.P.perm[sp.p_begin + i];                // caller index
  sp.lat[jlin[c]] = i;
#pragma unroll
  for (int a = 0; a < 3; ++a) sp.Xr[a][i] = Xc[3 * c + a];
}

// --------------------------------------------------------------------------
// regions: per cell the active regions (a disconnected or boundary link at
// one of their corners) and each corner's vertex ordinal
// --------------------------------------------------------------------------
__global__ void k_sf_cells(World w, SurfParams sp) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= sp.n_cells) return;
  int j[3];
  cell_of(sp, i, j);
  CellInfo ci;
  cell_info(w, sp, j, ci);
  unsigned active = 0;
  for (int q = 0; q < 8; ++q)
    for (int a = 0; a < 3; ++a) {
      if ((q >> a) & 1) continue;
      const int r = q | (1 << a);
      const bool m0 = ci.part[q] >= 0, m1 = ci.part[r] >= 0;
      if (m0 && !m1) active |= 1u << ci.reg[q];
      else if (!m0 && m1) active |= 1u << ci.reg[r];
      else if (m0 && m1 && conflict_bits(ci.c1[q], ci.c2[q], ci.c1[r], ci.c2[r]))
        active |= (1u << ci.reg[q]) | (1u << ci.reg[r]);
    }
  int ord[8], cnt = 0;
  for (int r = 0; r < ci.nreg; ++r) ord[r] = ((active >> r) & 1u) ? cnt++ : 15;
  uint32_t packed = 0;
  for (int q = 0; q < 8; ++q) packed |= (uint32_t)(ci.part[q] >= 0 ? ord[ci.reg[q]] : 15) << (4 * q);
  sp.cell_cnt[i] = cnt;
  sp.cell_reg[i] = packed;
}

// one vertex per active region: local dual contouring on the region's
// Hermite data, relative to the mass point, pseudo-inverse, clamped to the cell
__global__ void k_sf_vertices(World w, SurfParams sp) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= sp.n_cells) return;
  const int cnt = sp.cell_cnt[i];
  if (cnt == 0) return;
  int j[3];
  cell_of(sp, i, j);
  CellInfo ci;
  cell_info(w, sp, j, ci);
  const DevScene &sc = w.scenes[sp.slot];
  const uint32_t packed = sp.cell_reg[i];
  const int base = sp.cell_off[i];
  for (int o = 0; o < cnt; ++o) {
    float m[3] = {0.f, 0.f, 0.f};
    int k = 0, anchor = -1;
    for (int q = 7; q >= 0; --q)
      if (((packed >> (4 * q)) & 15u) == (uint32_t)o) anchor = q;
    // pass 1: mass point of the region's Hermite points
    for (int q = 0; q < 8; ++q)
      for (int a = 0; a < 3; ++a) {
        if ((q >> a) & 1) continue;
        const int r = q | (1 << a);
        for (int side = 0; side < 2; ++side) {
          const int qa = side ? r : q, qb = side ? q : r;
          if (((packed >> (4 * qa)) & 15u) != (uint32_t)o) continue;
          float p[3], nn[3];
          if (!hermite(sp, sc, ci, j, qa, qb, a, p, nn)) continue;
          m[0] += p[0];
          m[1] += p[1];
          m[2] += p[2];
          ++k;
        }
      }
    const float ik = 1.f / (float)k;
    m[0] *= ik;
    m[1] *= ik;
    m[2] *= ik;
    // pass 2: sum n n^T and sum n (n . (p - m))
    float A[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, rr[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < 8; ++q)
      for (int a = 0; a < 3; ++a) {
        if ((q >> a) & 1) continue;
        const int r = q | (1 << a);
        for (int side = 0; side < 2; ++side) {
          const int qa = side ? r : q, qb = side ? q : r;
          if (((packed >> (4 * qa)) & 15u) != (uint32_t)o) continue;
          float p[3], nn[3];
          if (!hermite(sp, sc, ci, j, qa, qb, a, p, nn)) continue;
          const float d = nn[0] * (p[0] - m[0]) + nn[1] * (p[1] - m[1]) + nn[2] * (p[2] - m[2]);
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            rr[u] += nn[u] * d;
#pragma unroll
            for (int v = 0; v < 3; ++v) A[u][v] += nn[u] * nn[v];
          }
        }
      }
    float V[3][3];
    jacobi3(A, V);
    float c[3] = {m[0], m[1], m[2]};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const float lam = A[e][e];
      if (lam < kQefCut) continue;
      const float g = (V[0][e] * rr[0] + V[1][e] * rr[1] + V[2][e] * rr[2]) / lam;
#pragma unroll
      for (int u = 0; u < 3; ++u) c[u] += g * V[u][e];
    }
    const int v = base + o;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const float cl = fminf(fmaxf(c[u], 0.f), (float)sp.h[u]);
      sp.ref[u][v] = (float)(sp.Xmin[u] + j[u] * sp.h[u] + (double)cl);
    }
    sp.anchor[v] = ci.part[anchor];
  }
}

// --------------------------------------------------------------------------
// faces: for every link with Hermite data (lower end j, axis a) and each of
// its material ends, the quad over that end's vertices in the 4 cells around
// the link, wound counter-clockwise about the outward direction
// --------------------------------------------------------------------------
template <bool WRITE>
__global__ void k_sf_tris(World w, SurfParams sp) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= sp.n_cells) return;
  if (sp.cell_cnt[i] == 0) {  // the link's own cell (lower corner j) carries a vertex
    if (!WRITE) sp.pt_cnt[i] = 0;
    return;
  }
  int j[3];
  cell_of(sp, i, j);
  int cnt = 0;
  const int out0 = WRITE ? sp.pt_off[i] : 0;
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    if (j[b] < 0 || j[b] >= sp.n[b] || j[c] < 0 || j[c] >= sp.n[c]) continue;
    int j1[3] = {j[0], j[1], j[2]};
    j1[a] += 1;
    const int pa = lat_at(sp, j[0], j[1], j[2]), pb = lat_at(sp, j1[0], j1[1], j1[2]);
    bool ha, hb;
    if (pa >= 0 && pb >= 0) {
      const uint32_t cf = conflict_bits(w.P.s1[sp.p_begin + pa], w.P.s2[sp.p_begin + pa],
                                        w.P.s1[sp.p_begin + pb], w.P.s2[sp.p_begin + pb]);
      ha = hb = cf != 0u;
    } else {
      ha = pa >= 0;
      hb = pb >= 0;
    }
    for (int side = 0; side < 2; ++side) {
      if (!(side ? hb : ha)) continue;
      const int *je = side ? j1 : j;
      int rs[4];
      bool ok = true;
      for (int k = 0; k < 4; ++k) {
        // (s_b, s_c): (0,0) (1,0) (1,1) (0,1) about +a; reversed for the upper end
        const int kk = side ? (4 - k) & 3 : k;
        const int sb = (kk == 1 || kk == 2) ? 1 : 0, sc = (kk >= 2) ? 1 : 0;
        int L[3] = {j[0], j[1], j[2]};
        L[b] -= sb;
        L[c] -= sc;
        const long long lin = cell_index(sp, L);
        const int q = ((je[0] - L[0]) << 0) | ((je[1] - L[1]) << 1) | ((je[2] - L[2]) << 2);
        const uint32_t nib = (sp.cell_reg[lin] >> (4 * q)) & 15u;
        ok &= nib != 15u;
        rs[k] = sp.cell_off[lin] + (int)nib;
      }
      if (!ok) continue;
      const int t0[3] = {rs[0], rs[1], rs[2]}, t1[3] = {rs[0], rs[2], rs[3]};
      if (t0[0] != t0[1] && t0[1] != t0[2] && t0[0] != t0[2]) {
        if (WRITE) {
          int *o = sp.tri + 3 * (size_t)(out0 + cnt);
          o[0] = t0[0];
          o[1] = t0[1];
          o[2] = t0[2];
        }
        ++cnt;
      }
      if (t1[0] != t1[1] && t1[1] != t1[2] && t1[0] != t1[2]) {
        if (WRITE) {
          int *o = sp.tri + 3 * (size_t)(out0 + cnt);
          o[0] = t1[0];
          o[1] = t1[1];
          o[2] = t1[2];
        }
        ++cnt;
      }
    }
  }
  if (!WRITE) sp.pt_cnt[i] = cnt;
}

// --------------------------------------------------------------------------
// side-aware embedding: 8 lanes per vertex share the lattice points around
// its 8 trilinear nodes (the union of the nodes' B-spline supports, split by
// z slice); each lane sums, for every node, the weights and weighted
// displacements of the particles with the anchor's exact code, then the
// group adds the lanes' sums (xor butterfly) and lane 0 combines the nodes
// in node order
// --------------------------------------------------------------------------
__device__ __forceinline__ int jfirst(const SurfParams &sp, int a, int B) {
  if (B <= sp.bmin[a]) return 0;
  if (B > sp.bmax[a]) return sp.n[a];
  return sp.jstart[a][B - sp.bmin[a]];
}

// quadratic B-spline weight of node base + o for fractional offset f in
// [0.5, 1.5); zero outside the stencil (o not in 0..2)
__device__ __forceinline__ float bsw(int o, float f) {
  if (o == 0) {
    const float t = 1.5f - f;
    return 0.5f * t * t;
  }
  if (o == 1) {
    const float t = f - 1.f;
    return 0.75f - t * t;
  }
  if (o == 2) {
    const float t = f - 0.5f;
    return 0.5f * t * t;
  }
  return 0.f;
}

__global__ void k_sf_embed(World w, SurfParams sp, int nv) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int v = (int)(t >> 3), lane8 = (int)(t & 7);
  const bool valid = v < nv;
  float acc[8][4];  // per trilinear node: sum N, sum N (x - X)
#pragma unroll
  for (int d = 0; d < 8; ++d) acc[d][0] = acc[d][1] = acc[d][2] = acc[d][3] = 0.f;
  float c[3] = {0.f, 0.f, 0.f}, tw[3] = {0.f, 0.f, 0.f};
  int g0 = 0;
  uint32_t a1 = 0u, a2 = 0u;
  if (valid) {
    g0 = sp.p_begin + sp.anchor[v];
    a1 = w.P.s1[g0];
    a2 = w.P.s2[g0];
    int n0[3], jlo[3], jhi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      c[a] = sp.ref[a][v];
      const double f = ((double)c[a] - sp.origin[a]) / sp.dx;
      const double fb = floor(f);
      tw[a] = (float)(f - fb);
      n0[a] = (int)fb;
      // particles whose stencil holds node n0 or n0 + 1: base cells n0 - 2 .. n0 + 1
      jlo[a] = jfirst(sp, a, n0[a] - 2);
      jhi[a] = jfirst(sp, a, n0[a] + 2);
    }
    for (int z = jlo[2] + lane8; z < jhi[2]; z += 8)
      for (int y = jlo[1]; y < jhi[1]; ++y)
        for (int x = jlo[0]; x < jhi[0]; ++x) {
          const int p = sp.lat[((long long)z * sp.n[1] + y) * sp.n[0] + x];
          if (p < 0) continue;
          const int g = sp.p_begin + p;
          if (w.P.s1[g] != a1 || w.P.s2[g] != a2) continue;
          const uint32_t bb = w.P.base[g];
          const int ox = n0[0] - ((int)(bb & 1023u) + sp.lo[0]);
          const int oy = n0[1] - ((int)((bb >> 10) & 1023u) + sp.lo[1]);
          const int oz = n0[2] - ((int)((bb >> 20) & 1023u) + sp.lo[2]);
          const float fx = w.P.fx[0][g], fy = w.P.fx[1][g], fz = w.P.fx[2][g];
          const float wx[2] = {bsw(ox, fx), bsw(ox + 1, fx)};
          const float wy[2] = {bsw(oy, fy), bsw(oy + 1, fy)};
          const float wz[2] = {bsw(oz, fz), bsw(oz + 1, fz)};
          const float u0 = w.P.x[0][g] - sp.Xr[0][p], u1 = w.P.x[1][g] - sp.Xr[1][p],
                      u2 = w.P.x[2][g] - sp.Xr[2][p];
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            const float N = wx[d & 1] * wy[(d >> 1) & 1] * wz[d >> 2];
            acc[d][0] += N;
            acc[d][1] += N * u0;
            acc[d][2] += N * u1;
            acc[d][3] += N * u2;
          }
        }
  }
  // sums over the group's 8 lanes (the xor partners stay inside the group)
#pragma unroll
  for (int m = 1; m < 8; m <<= 1)
#pragma unroll
    for (int d = 0; d < 8; ++d)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[d][e] += __shfl_xor_sync(kFull, acc[d][e], m);
  if (valid && lane8 == 0) {
    float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      if (!(acc[d][0] > 0.f)) continue;  // no particle of this code around the node
      const float wt = ((d & 1) ? tw[0] : 1.f - tw[0]) * (((d >> 1) & 1) ? tw[1] : 1.f - tw[1]) *
                       ((d >> 2) ? tw[2] : 1.f - tw[2]);
      const float s = wt / acc[d][0];
      num[0] += s * acc[d][1];
      num[1] += s * acc[d][2];
      num[2] += s * acc[d][3];
      den += wt;
    }
    const int p0 = sp.anchor[v];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float u = den > 0.f ? num[a] / den : w.P.x[a][g0] - sp.Xr[a][p0];
      sp.cur[a][v] = c[a] + u;
    }
    sp.vmask[0][v] = a1;
    sp.vmask[1][v] = a2;
  }
}

// --------------------------------------------------------------------------
// exclusive scan of n ints into out[0..n] (out[n] = total)
// --------------------------------------------------------------------------
__device__ int block_scan_excl(int v, int *sm, int &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sm[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < nw; ++k) {
      const int s = sm[k];
      sm[k] = acc;
      acc += s;
    }
    sm[nw] = acc;
  }
  __syncthreads();
  total = sm[nw];
  const int r = x - v + sm[wid];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanBlock) k_sf_scan_block(const int *in, int *out, int *bsum, long long n) {
  __shared__ int sm[kScanBlock / 32 + 1];
  const long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
  int total;
  const int ex = block_scan_excl(i < n ? in[i] : 0, sm, total);
  if (i < n) out[i] = ex;
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_sf_scan_top(int *bsum, int nb, int *total_out) {
  __shared__ int sm[kScanBlock / 32 + 1];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanBlock) {
    const int k = b0 + (int)threadIdx.x;
    int total;
    const int ex = block_scan_excl(k < nb ? bsum[k] : 0, sm, total);
    if (k < nb) bsum[k] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_sf_scan_add(int *out, const int *bsum, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] += bsum[i / kScanBlock];
}

cudaError_t scan_excl(const int *in, int *out, int *tmp, long long n, cudaStream_t st) {
  const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
  if (nb > 0) k_sf_scan_block<<<nb, kScanBlock, 0, st>>>(in, out, tmp, n);
  k_sf_scan_top<<<1, kScanBlock, 0, st>>>(tmp, nb, out + n);
  if (nb > 0) k_sf_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, tmp, n);
  return cudaGetLastError();
}

inline unsigned grid_of(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t bm_launch_surface_map(const World &w, const SurfParams &sp, int n, const int *jlin,
                                  const float *Xc, cudaStream_t st) {
  if (n > 0) k_sf_map<<<grid_of(n, 256), 256, 0, st>>>(w, sp, n, jlin, Xc);
  return cudaGetLastError();
}

cudaError_t bm_launch_surface_cells(const World &w, const SurfParams &sp, cudaStream_t st) {
  k_sf_cells<<<grid_of(sp.n_cells, 128), 128, 0, st>>>(w, sp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return scan_excl(sp.cell_cnt, sp.cell_off, sp.scan_tmp, sp.n_cells, st);
}

cudaError_t bm_launch_surface_vertices(const World &w, const SurfParams &sp, cudaStream_t st) {
  k_sf_vertices<<<grid_of(sp.n_cells, 128), 128, 0, st>>>(w, sp);
  return cudaGetLastError();
}

cudaError_t bm_launch_surface_tri_count(const World &w, const SurfParams &sp, cudaStream_t st) {
  k_sf_tris<false><<<grid_of(sp.n_cells, 128), 128, 0, st>>>(w, sp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return scan_excl(sp.pt_cnt, sp.pt_off, sp.scan_tmp, sp.n_cells, st);
}

cudaError_t bm_launch_surface_tris(const World &w, const SurfParams &sp, cudaStream_t st) {
  k_sf_tris<true><<<grid_of(sp.n_cells, 128), 128, 0, st>>>(w, sp);
  return cudaGetLastError();
}

cudaError_t bm_launch_surface_embed(const World &w, const SurfParams &sp, int n_vertices, cudaStream_t st) {
  if (n_vertices > 0) k_sf_embed<<<grid_of(8LL * n_vertices, 256), 256, 0, st>>>(w, sp, n_vertices);
  return cudaGetLastError();
}
