// Adjoint (reverse mode) of one TLMPM cutting substep on sm_103a, for
// calibration of the material (E, nu) and the blade velocity from reaction-
// force trajectories (Eq. 16).
//
// The substep is differentiated with every discrete decision of the forward
// substep held fixed: the codes (side labels, Eq. 6-7), the contact active
// sets (Eq. 14-15), the sign test of the normal velocity in phi_hat, stick
// or slip (Eq. 12), the front band and the D release (Eq. 5), and the face
// or clamp pattern of the blade-box closest point.  Given the codes, the
// logical-grid masses and the coupling of Eq. 8 are constants, so everything
// from P2G to the F update is a fixed linear map whose transpose is applied
// here by per-node gathers (no atomics; every sum in a fixed order).  The
// decisions are re-taken from the restored state of the substep with the
// forward kernels' float32 expressions.
//
// Kernels of one adjoint substep (scene-local launches):
//   k_adj_musl    per node (a warp each): slot masses; adjoint of v* from the F update;
//                 through v* = C p* / m (transpose of Eq. 8)
//   k_adj_v1      per particle: adjoint of the G2P velocity v^{n+1} (MUSL)
//   k_adj_g2p     per node (a warp each): adjoints of the coupled momentum and momentum
//                 change (Eq. 17 and x update), through Eq. 8 transposed
//   k_adj_part    per particle: P2G (Eq. 2) transposed, stress, blade and
//                 floor contact; block partials of the parameter adjoints
//   k_adj_reduce  one block: partials summed in block order (float64), tool
//                 position and segment velocity adjoints updated
// Scope: kinematic blade translating without rotation, rigid interval 1, no
// material-material contact (checked on the host).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bm_internal.cuh"

namespace {

constexpr int kAdjBlock = 128;
constexpr int kParts = 8;  // mu, lambda, tool position (3), tool velocity (3)

// quadratic B-spline weight and d/dxl of node offset o at fractional offset f
__device__ __forceinline__ void wgt(int o, float f, float &w, float &dw) {
  if (o == 0) {
    const float t = 1.5f - f;
    w = 0.5f * t * t;
    dw = -t;
  } else if (o == 1) {
    const float t = f - 1.0f;
    w = 0.75f - t * t;
    dw = -2.0f * t;
  } else {
    const float t = f - 0.5f;
    w = 0.5f * t * t;
    dw = t;
  }
}

__device__ __forceinline__ bool incompatible(uint2 a, uint2 b) {
  return ((a.x & b.y) | (a.y & b.x)) != 0u;
}

// brick-major index of a scene-local base cell (bricks of 4 x 4 x 4 cells)
__device__ __forceinline__ int cell_at(const DevScene &sc, int bx, int by, int bz) {
  const int b = ((bz >> 2) * sc.nbr[1] + (by >> 2)) * sc.nbr[0] + (bx >> 2);
  return b * 64 + (((bz & 3) * 4 + (by & 3)) * 4 + (bx & 3));
}

__device__ __forceinline__ int node_at(const DevScene &sc, int ix, int iy, int iz) {
  return (iz * sc.nn[1] + iy) * sc.nn[0] + ix;
}

// slot (pool index) holding code c at scene-local node li, or -1
__device__ __forceinline__ int find_slot(const World &w, const DevScene &sc, int li, uint2 c) {
  const int node = sc.node_begin + li;
  const int off = w.N.slot_off[node], cnt = w.N.slot_cnt[node];
  for (int a = 0; a < cnt; ++a) {
    const uint2 k = w.S.code[off + a];
    if (k.x == c.x && k.y == c.y) return off + a;
  }
  return -1;
}

struct AdjWork {
  float *xb[3], *vb[3], *Fb[9], *ub[3];  // state adjoints, scene-relative pool order
  float *v1b[3];                          // adjoint of the G2P velocity
  float *sm;                              // slot mass (scene-relative slot index)
  float *s3[3];                           // per slot: adjoint of the MUSL momentum
  float *s6[6];                           // per slot: adjoints of momentum, momentum change
  double *part;                           // [block][kParts]
  double *acc;                            // mu, lambda, tool position (3), segments (3 each)
  int slot;                               // scene slot in the world
  double fbar[3];                         // dL/dF_B of this substep
};

// Transpose of Eq. 8 at one node (masses and codes fixed):
// (C^T S)^b = S^b + 1/M sum_{a != b, compatible} m^a (S^a - S^b)
template <int NC>
__device__ __forceinline__ void couple_T(int ns, const uint2 *codes, const float *m, float (*S)[NC]) {
  float M = 0.f;
  for (int a = 0; a < ns; ++a) M += m[a];
  if (!(M > 0.f)) return;
  const float iM = 1.0f / M;
  float out[BM_MAXS][NC];
  for (int b = 0; b < ns; ++b)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float acc = 0.f;
      for (int a = 0; a < ns; ++a) {
        if (a == b || incompatible(codes[a], codes[b])) continue;
        acc += m[a] * (S[a][c] - S[b][c]);
      }
      out[b][c] = S[b][c] + acc * iM;
    }
  for (int b = 0; b < ns; ++b)
#pragma unroll
    for (int c = 0; c < NC; ++c) S[b][c] = out[b][c];
}

// Visit the (particle, weight, gradient) pairs of scene-local node li whose
// particle lies in stencil cell l (< 27: ox = l % 3, oy = l / 3 % 3,
// oz = l / 9, the base cell li - (ox, oy, oz)), in pool order.
template <class Fn>
__device__ __forceinline__ void for_cell_particles(const World &w, const DevScene &sc, int li, int l, Fn fn) {
  const int ix = li % sc.nn[0], iy = (li / sc.nn[0]) % sc.nn[1], iz = li / (sc.nn[0] * sc.nn[1]);
  const int ox = l % 3, oy = (l / 3) % 3, oz = l / 9;
  const int bx = ix - ox, by = iy - oy, bz = iz - oz;
  if (bx < 0 || by < 0 || bz < 0 || bx >= sc.nb[0] || by >= sc.nb[1] || bz >= sc.nb[2]) return;
  const int *cs = w.N.cell_start + sc.cell_begin;
  const int c = cell_at(sc, bx, by, bz);
  for (int p = cs[c]; p < cs[c + 1]; ++p) {
    float wx, wy, wz, dx, dy, dz;
    wgt(ox, w.P.fx[0][p], wx, dx);
    wgt(oy, w.P.fx[1][p], wy, dy);
    wgt(oz, w.P.fx[2][p], wz, dz);
    const float N = wx * wy * wz;
    const float gN[3] = {dx * wy * wz * sc.inv_dx, wx * dy * wz * sc.inv_dx, wx * wy * dz * sc.inv_dx};
    fn(p, N, gN);
  }
}

// sum over the warp's lanes in a fixed butterfly order (every lane gets it)
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The per-node adjoint kernels run one warp per node: lane l < 27 walks the
// node's particles in stencil cell l, the lanes' sums are combined by
// warp_sum, one pass per logical grid of the node (codes fixed), and lane 0
// applies the transposed coupling to the node's slot sums.
constexpr int kAdjNodesPerBlock = kAdjBlock / 32;

// per node: slot masses, adjoint of v* from F' = F + dt sum v* (x) grad N,
// then through v* = C p* / m
__global__ void __launch_bounds__(kAdjBlock) k_adj_musl(World w, AdjWork aw) {
  __shared__ float red[kAdjNodesPerBlock][BM_MAXS][4];
  const DevScene &sc = w.scenes[aw.slot];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int li = blockIdx.x * kAdjNodesPerBlock + wid;
  if (li >= sc.n_node) return;
  const int node = sc.node_begin + li;
  const int off = w.N.slot_off[node], ns = w.N.slot_cnt[node];
  if (ns == 0) return;
  const int pb = sc.p_begin;
  const float dt = sc.dt, mp = sc.mp;
  for (int a = 0; a < ns; ++a) {
    const uint2 ca = w.S.code[off + a];
    float m = 0.f, S0 = 0.f, S1 = 0.f, S2 = 0.f;
    if (lane < 27)
      for_cell_particles(w, sc, li, lane, [&](int p, float N, const float *gN) {
        if (w.P.s1[p] != ca.x || w.P.s2[p] != ca.y) return;
        m += N * mp;
        const int i = p - pb;
        S0 += dt * (aw.Fb[0][i] * gN[0] + aw.Fb[1][i] * gN[1] + aw.Fb[2][i] * gN[2]);
        S1 += dt * (aw.Fb[3][i] * gN[0] + aw.Fb[4][i] * gN[1] + aw.Fb[5][i] * gN[2]);
        S2 += dt * (aw.Fb[6][i] * gN[0] + aw.Fb[7][i] * gN[1] + aw.Fb[8][i] * gN[2]);
      });
    m = warp_sum(m);
    S0 = warp_sum(S0);
    S1 = warp_sum(S1);
    S2 = warp_sum(S2);
    if (lane == 0) {
      red[wid][a][0] = m;
      red[wid][a][1] = S0;
      red[wid][a][2] = S1;
      red[wid][a][3] = S2;
    }
  }
  if (lane != 0) return;
  uint2 codes[BM_MAXS];
  float m[BM_MAXS], S[BM_MAXS][3];
  for (int a = 0; a < ns; ++a) {
    codes[a] = w.S.code[off + a];
    m[a] = red[wid][a][0];
    const float im = m[a] > 0.f ? 1.0f / m[a] : 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) S[a][r] = red[wid][a][1 + r] * im;
  }
  couple_T<3>(ns, codes, m, S);
  const int rel = off - sc.slot_begin;
  for (int a = 0; a < ns; ++a) {
    aw.sm[rel + a] = m[a];
#pragma unroll
    for (int r = 0; r < 3; ++r) aw.s3[r][rel + a] = S[a][r];
  }
}

// per particle: adjoint of v^{n+1} = incoming adjoint + MUSL re-scatter term
__global__ void __launch_bounds__(kAdjBlock) k_adj_v1(World w, AdjWork aw) {
  const DevScene &sc = w.scenes[aw.slot];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.n_p) return;
  const int p = sc.p_begin + i;
  const uint32_t b = w.P.base[p];
  const int bx = (int)(b & 1023u), by = (int)((b >> 10) & 1023u), bz = (int)((b >> 20) & 1023u);
  const uint2 c = make_uint2(w.P.s1[p], w.P.s2[p]);
  float acc[3] = {aw.vb[0][i], aw.vb[1][i], aw.vb[2][i]};
  const float mp = sc.mp;
  for (int oz = 0; oz < 3; ++oz)
    for (int oy = 0; oy < 3; ++oy)
      for (int ox = 0; ox < 3; ++ox) {
        float wx, wy, wz, d0, d1, d2;
        wgt(ox, w.P.fx[0][p], wx, d0);
        wgt(oy, w.P.fx[1][p], wy, d1);
        wgt(oz, w.P.fx[2][p], wz, d2);
        const int s = find_slot(w, sc, node_at(sc, bx + ox, by + oy, bz + oz), c);
        if (s < 0) continue;
        const float N = wx * wy * wz;
        const int rel = s - sc.slot_begin;
#pragma unroll
        for (int r = 0; r < 3; ++r) acc[r] += N * mp * aw.s3[r][rel];
      }
#pragma unroll
  for (int r = 0; r < 3; ++r) aw.v1b[r][i] = acc[r];
}

// per node: adjoints of the coupled momentum and momentum change per slot
// from v^{n+1} = beta v + sum N/m ((1-beta) p + dp) and x^{n+1} = x + dt sum
// N (p + dp)/m, then through Eq. 8 transposed
__global__ void __launch_bounds__(kAdjBlock) k_adj_g2p(World w, AdjWork aw) {
  __shared__ float red[kAdjNodesPerBlock][BM_MAXS][6];
  const DevScene &sc = w.scenes[aw.slot];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int li = blockIdx.x * kAdjNodesPerBlock + wid;
  if (li >= sc.n_node) return;
  const int node = sc.node_begin + li;
  const int off = w.N.slot_off[node], ns = w.N.slot_cnt[node];
  if (ns == 0) return;
  const int rel = off - sc.slot_begin;
  const int pb = sc.p_begin;
  const float dt = sc.dt, beta = sc.beta;
  for (int a = 0; a < ns; ++a) {
    const uint2 ca = w.S.code[off + a];
    const float ma = aw.sm[rel + a];
    float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (lane < 27 && ma > 0.f)
      for_cell_particles(w, sc, li, lane, [&](int p, float N, const float *) {
        if (w.P.s1[p] != ca.x || w.P.s2[p] != ca.y) return;
        const float q = N / ma;
        const int i = p - pb;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float v1 = aw.v1b[r][i], xx = dt * aw.xb[r][i];
          S[r] += q * ((1.0f - beta) * v1 + xx);
          S[3 + r] += q * (v1 + xx);
        }
      });
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      const float t = warp_sum(S[r]);
      if (lane == 0) red[wid][a][r] = t;
    }
  }
  if (lane != 0) return;
  uint2 codes[BM_MAXS];
  float m[BM_MAXS], S[BM_MAXS][6];
  for (int a = 0; a < ns; ++a) {
    codes[a] = w.S.code[off + a];
    m[a] = aw.sm[rel + a];
#pragma unroll
    for (int r = 0; r < 6; ++r) S[a][r] = red[wid][a][r];
  }
  couple_T<6>(ns, codes, m, S);
  for (int a = 0; a < ns; ++a)
#pragma unroll
    for (int r = 0; r < 6; ++r) aw.s6[r][rel + a] = S[a][r];
}

__device__ __forceinline__ float dot3f(const float *a, const float *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// VJP of the neo-Hookean stress P = mu F + (lam ln J - mu) F^-T
__device__ void piola_vjp(const float F[9], float mu, float lam, const float Pb[9], float Fb[9],
                          float &mub, float &lamb) {
  float c[9];
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
  float J = F[0] * c[0] + F[1] * c[1] + F[2] * c[2];
  if (!(J > 1e-6f)) J = 1e-6f;
  const float iJ = 1.0f / J, lj = logf(J);
  float G[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) G[k] = c[k] * iJ;
  float PG = 0.f, PF = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    PG += Pb[k] * G[k];
    PF += Pb[k] * F[k];
  }
  // (G Pb^T G)_lk = sum_ij G_lj Pb_ij G_ik
  float T[9];  // T_jk = sum_i Pb_ij G_ik = (Pb^T G)_jk
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) T[3 * j + k] = Pb[j] * G[k] + Pb[3 + j] * G[3 + k] + Pb[6 + j] * G[6 + k];
  const float cG = lam * lj - mu;
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float GPtG = G[3 * l] * T[k] + G[3 * l + 1] * T[3 + k] + G[3 * l + 2] * T[6 + k];
      Fb[3 * l + k] += mu * Pb[3 * l + k] - cG * GPtG + lam * PG * G[3 * l + k];
    }
  mub += PF - PG;
  lamb += lj * PG;
}

// per particle: P2G transposed, stress, blade contact (with friction and the
// D release) and floor contact; block partials of the parameter adjoints
__global__ void __launch_bounds__(kAdjBlock) k_adj_part(World w, AdjWork aw) {
  __shared__ double red[kParts][kAdjBlock / 32];
  const DevScene &sc = w.scenes[aw.slot];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float th[kParts] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (i < sc.n_p) {
    const int p = sc.p_begin + i;
    const uint32_t b = w.P.base[p];
    const int bx = (int)(b & 1023u), by = (int)((b >> 10) & 1023u), bz = (int)((b >> 20) & 1023u);
    const uint2 code = make_uint2(w.P.s1[p], w.P.s2[p]);
    const float dt = sc.dt, mp = sc.mp, beta = sc.beta;
    float vb[3], Jb[3] = {0.f, 0.f, 0.f}, Pb[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) vb[r] = beta * aw.v1b[r][i];
#pragma unroll
    for (int k = 0; k < 9; ++k) Pb[k] = 0.f;
    const float cA = -dt * sc.V0;
    for (int oz = 0; oz < 3; ++oz)
      for (int oy = 0; oy < 3; ++oy)
        for (int ox = 0; ox < 3; ++ox) {
          float wx, wy, wz, d0, d1, d2;
          wgt(ox, w.P.fx[0][p], wx, d0);
          wgt(oy, w.P.fx[1][p], wy, d1);
          wgt(oz, w.P.fx[2][p], wz, d2);
          const int s = find_slot(w, sc, node_at(sc, bx + ox, by + oy, bz + oz), code);
          if (s < 0) continue;
          const int rel = s - sc.slot_begin;
          const float N = wx * wy * wz;
          const float gN[3] = {d0 * wy * wz * sc.inv_dx, wx * d1 * wz * sc.inv_dx, wx * wy * d2 * sc.inv_dx};
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const float pbar = aw.s6[r][rel], dpbar = aw.s6[3 + r][rel];
            vb[r] += N * mp * pbar;
            Jb[r] += N * dpbar;
            Pb[3 * r] += cA * dpbar * gN[0];
            Pb[3 * r + 1] += cA * dpbar * gN[1];
            Pb[3 * r + 2] += cA * dpbar * gN[2];
          }
        }
    // stress
    float F[9], Fb[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      F[k] = w.P.F[k][p];
      Fb[k] = aw.Fb[k][i];
    }
    piola_vjp(F, sc.mu, sc.lam, Pb, Fb, th[0], th[1]);
#pragma unroll
    for (int k = 0; k < 9; ++k) aw.Fb[k][i] = Fb[k];
    // contact (state of this substep)
    const float x[3] = {w.P.x[0][p], w.P.x[1][p], w.P.x[2][p]};
    const float v[3] = {w.P.v[0][p], w.P.v[1][p], w.P.v[2][p]};
    float xb[3] = {aw.xb[0][i], aw.xb[1][i], aw.xb[2][i]};
    const float ubn[3] = {aw.ub[0][i], aw.ub[1][i], aw.ub[2][i]};
    float ubo[3] = {0.f, 0.f, 0.f};
    if (sc.has_blade && sc.tool_contact_on) {
      const float *ax[3] = {sc.fn, sc.fe, sc.fd};
      const float y[3] = {x[0] - sc.fc[0], x[1] - sc.fc[1], x[2] - sc.fc[2]};
      float q[3];
      bool outside = false, cl[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        q[a] = y[0] * ax[a][0] + y[1] * ax[a][1] + y[2] * ax[a][2];
        cl[a] = fabsf(q[a]) > sc.fhext[a];
        outside |= cl[a];
      }
      float nB[3], phi, nl[3] = {0.f, 0.f, 0.f}, dist = 1.f, sg = 1.f;
      int best = 0;
      if (outside) {
        float diff[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) diff[a] = q[a] - fminf(fmaxf(q[a], -sc.fhext[a]), sc.fhext[a]);
        dist = sqrtf(diff[0] * diff[0] + diff[1] * diff[1] + diff[2] * diff[2]);
        const float id = 1.0f / dist;
#pragma unroll
        for (int a = 0; a < 3; ++a) nl[a] = diff[a] * id;
        phi = dist - sc.Rp;
      } else {
        float bd = sc.fhext[0] - fabsf(q[0]);
#pragma unroll
        for (int a = 1; a < 3; ++a) {
          const float dd = sc.fhext[a] - fabsf(q[a]);
          if (dd < bd) {
            bd = dd;
            best = a;
          }
        }
        sg = q[best] < 0.0f ? -1.0f : 1.0f;
        nl[best] = sg;
        phi = -bd - sc.Rp;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) nB[r] = nl[0] * ax[0][r] + nl[1] * ax[1][r] + nl[2] * ax[2][r];
      const float vrel[3] = {v[0] - sc.fvB[0], v[1] - sc.fvB[1], v[2] - sc.fvB[2]};
      const float vn = vrel[0] * nB[0] + vrel[1] * nB[1] + vrel[2] * nB[2];
      const bool neg = vn < 0.0f;
      const float phihat = phi + dt * fminf(vn, 0.0f);
      const float meff = 1.0f / (1.0f / mp + 0.0f);
      const float kn = sc.s_n * meff / dt;
      const float Jn = kn * fmaxf(-phihat, 0.0f);
      if (Jn > 0.0f) {
        const float uh[3] = {w.P.ut[0][p], w.P.ut[1][p], w.P.ut[2][p]};
        const float fn = Jn / dt;
        const float udn = dot3f(uh, nB);
        const float ul = sqrtf(dot3f(uh, uh));
        const float tu[3] = {uh[0] - udn * nB[0], uh[1] - udn * nB[1], uh[2] - udn * nB[2]};
        const float tl = sqrtf(dot3f(tu, tu));
        const float scl = tl > 0.0f ? ul / tl : 0.0f;
        const float ut[3] = {tu[0] * scl, tu[1] * scl, tu[2] * scl};
        const float vnn = vn;
        const float vt[3] = {vrel[0] - vnn * nB[0], vrel[1] - vnn * nB[1], vrel[2] - vnn * nB[2]};
        const float kt = sc.gamma_k * meff / (dt * dt);
        const float ct = 2.0f * sc.gamma_c * sqrtf(meff * kt);
        const float ftr[3] = {-kt * ut[0] - ct * vt[0], -kt * ut[1] - ct * vt[1], -kt * ut[2] - ct * vt[2]};
        const float fl = sqrtf(dot3f(ftr, ftr));
        const bool stick = fl <= sc.fmu_s * fn;
        float JB[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) JB[r] = Jn * nB[r] + dt * (stick ? ftr[r] : sc.fmu_d * fn / fl * ftr[r]);
        bool rel = false;
        if (sc.cut >= 0) {
          const float r0[3] = {x[0] - sc.fxe[0], x[1] - sc.fxe[1], x[2] - sc.fxe[2]};
          const float sp = dot3f(r0, sc.fn), lp = dot3f(r0, sc.fe), fp = dot3f(r0, sc.fd);
          const float uc = (sc.fve[0] - v[0]) * sc.fd[0] + (sc.fve[1] - v[1]) * sc.fd[1] +
                           (sc.fve[2] - v[2]) * sc.fd[2];
          const bool front = fabsf(sp) <= sc.h && fabsf(lp) <= sc.fL && fp >= 0.0f && fp <= sc.b_lead &&
                             uc > sc.u_min;
          const float D = sc.reset_D ? 0.0f : w.P.D[p];
          rel = front && !(D < 1.0f) && dot3f(JB, sc.fd) > 0.0f;
        }
        // reverse; the loss enters through F_B = -sum J_pB / dt
        const float idt = 1.0f / dt;
        float Jbb[3] = {Jb[0] - (float)aw.fbar[0] * idt, Jb[1] - (float)aw.fbar[1] * idt,
                        Jb[2] - (float)aw.fbar[2] * idt};
        if (rel) {
          const float t = dot3f(Jbb, sc.fd);
#pragma unroll
          for (int r = 0; r < 3; ++r) Jbb[r] -= t * sc.fd[r];
        }
        float Jnb = dot3f(Jbb, nB);
        float nBb[3] = {Jn * Jbb[0], Jn * Jbb[1], Jn * Jbb[2]};
        float utb[3] = {0.f, 0.f, 0.f}, vtb[3] = {0.f, 0.f, 0.f}, ftrb[3];
        float fnb = 0.f;
        if (stick) {
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            ftrb[r] = dt * Jbb[r];
            utb[r] = ubn[r];
            vtb[r] = dt * ubn[r];
          }
        } else {
          const float ikt = 1.0f / kt, ifl = 1.0f / fl;
          float g[3], hh[3], hb[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            g[r] = dt * Jbb[r] - ubn[r] * ikt;
            vtb[r] = -ct * ubn[r] * ikt;
            hh[r] = ftr[r] * ifl;
          }
          fnb = sc.fmu_d * dot3f(g, hh);
#pragma unroll
          for (int r = 0; r < 3; ++r) hb[r] = sc.fmu_d * fn * g[r];
          const float t = dot3f(hb, hh);
#pragma unroll
          for (int r = 0; r < 3; ++r) ftrb[r] = (hb[r] - t * hh[r]) * ifl;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          utb[r] += -kt * ftrb[r];
          vtb[r] += -ct * ftrb[r];
        }
        float vrelb[3];
        {
          const float t = dot3f(vtb, nB);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            vrelb[r] = vtb[r] - t * nB[r];
            nBb[r] += -vnn * vtb[r] - t * vrel[r];
          }
        }
        if (tl > 0.0f) {
          const float scb = dot3f(utb, tu);
          const float ulb = scb / tl, tlb = -scb * ul / (tl * tl);
          float tub[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) tub[r] = scl * utb[r] + tlb * tu[r] / tl;
          const float t = dot3f(tub, nB);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            ubo[r] = ulb * uh[r] / ul + tub[r] - t * nB[r];
            nBb[r] += -udn * tub[r] - t * uh[r];
          }
        }
        Jnb += fnb * idt;
        const float phihatb = -kn * Jnb;
        const float vnb = neg ? dt * phihatb : 0.0f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          vrelb[r] += vnb * nB[r];
          nBb[r] += vnb * vrel[r];
          vb[r] += vrelb[r];
          th[5 + r] -= vrelb[r];
        }
        float qb[3] = {0.f, 0.f, 0.f};
        if (outside) {
          float nlb[3], t = 0.f;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            nlb[a] = dot3f(nBb, ax[a]);
            t += nlb[a] * nl[a];
          }
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (cl[a]) qb[a] = (nlb[a] - t * nl[a]) / dist + phihatb * nl[a];
        } else {
          qb[best] = sg * phihatb;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float yb = qb[0] * ax[0][r] + qb[1] * ax[1][r] + qb[2] * ax[2][r];
          xb[r] += yb;
          th[2 + r] -= yb;
        }
      }
    }
    if (sc.floor_on) {
      const float phi = x[2] - sc.floor_z - sc.Rp;
      const float phihat = phi + dt * fminf(v[2], 0.0f);
      const float kn = sc.s_n * mp / dt;
      if (kn * fmaxf(-phihat, 0.0f) > 0.0f) {
        const float phihatb = -kn * Jb[2];
        xb[2] += phihatb;
        if (v[2] < 0.0f) vb[2] += dt * phihatb;
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      aw.xb[r][i] = xb[r];
      aw.vb[r][i] = vb[r];
      aw.ub[r][i] = ubo[r];
    }
  }
  // block partials: float64 shuffle tree, warps in order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kParts; ++k) {
    double v = th[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < kParts) {
    double s = 0.0;
    for (int q = 0; q < kAdjBlock / 32; ++q) s += red[threadIdx.x][q];
    aw.part[(size_t)blockIdx.x * kParts + threadIdx.x] = s;
  }
}

// one block: partials summed in block order; x_B^{n+1} = x_B^n + dt v_B^n
// with v_B^n the velocity of the segment active at this substep
__global__ void k_adj_reduce(World w, AdjWork aw, int nblocks) {
  __shared__ double tot[kParts];
  const DevScene &sc = w.scenes[aw.slot];
  if (threadIdx.x < kParts) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += aw.part[(size_t)b * kParts + threadIdx.x];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  aw.acc[0] += tot[0];
  aw.acc[1] += tot[1];
  int seg = -1;
  long long a = 0;
  for (int k = 0; k < sc.nseg; ++k) {
    a += sc.seg[k].n_steps;
    if (sc.step < a) {
      seg = k;
      break;
    }
  }
  if (seg < 0) seg = sc.nseg - 1;  // program ended: the last twist holds
  for (int r = 0; r < 3; ++r) {
    const double vtot = tot[5 + r] + sc.dt_d * aw.acc[2 + r];
    aw.acc[2 + r] += tot[2 + r];
    if (seg >= 0) aw.acc[5 + 3 * seg + r] += vtot;
  }
}

// state adjoints <-> caller order (perm maps pool index -> caller index)
__global__ void k_adj_io(World w, AdjWork aw, int field, float *buf, int to_work) {
  const DevScene &sc = w.scenes[aw.slot];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.n_p) return;
  const int q = w.P.perm[sc.p_begin + i];
  float *const *src = field == 0 ? aw.xb : field == 1 ? aw.vb : field == 2 ? aw.Fb : aw.ub;
  const int nc = field == 2 ? 9 : 3;
  for (int k = 0; k < nc; ++k) {
    if (to_work) src[k][i] = buf[(size_t)q * nc + k];
    else buf[(size_t)q * nc + k] = src[k][i];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers (called by the runtime)
// ---------------------------------------------------------------------------
// carve one allocation into the work arrays (256-byte aligned pieces)
void *bm_adj_carve(void *base, int64_t n_p, int64_t slot_cap, int scene_slot, void *out_work) {
  AdjWork &aw = *reinterpret_cast<AdjWork *>(out_work);
  char *c = (char *)base;
  auto take = [&](size_t bytes) {
    char *r = c;
    c += (bytes + 255) & ~size_t(255);
    return (void *)r;
  };
  for (int k = 0; k < 3; ++k) aw.xb[k] = (float *)take(sizeof(float) * n_p);
  for (int k = 0; k < 3; ++k) aw.vb[k] = (float *)take(sizeof(float) * n_p);
  for (int k = 0; k < 9; ++k) aw.Fb[k] = (float *)take(sizeof(float) * n_p);
  for (int k = 0; k < 3; ++k) aw.ub[k] = (float *)take(sizeof(float) * n_p);
  for (int k = 0; k < 3; ++k) aw.v1b[k] = (float *)take(sizeof(float) * n_p);
  aw.sm = (float *)take(sizeof(float) * slot_cap);
  for (int k = 0; k < 3; ++k) aw.s3[k] = (float *)take(sizeof(float) * slot_cap);
  for (int k = 0; k < 6; ++k) aw.s6[k] = (float *)take(sizeof(float) * slot_cap);
  const int64_t nb = (n_p + kAdjBlock - 1) / kAdjBlock;
  aw.part = (double *)take(sizeof(double) * nb * kParts);
  aw.acc = (double *)take(sizeof(double) * (5 + 3 * BM_MAX_SEGMENTS));
  aw.slot = scene_slot;
  return c;
}

size_t bm_adj_work_struct_size() { return sizeof(AdjWork); }

size_t bm_adj_work_alloc_bytes(int64_t n_p, int64_t slot_cap) {
  // exact size of what bm_adj_carve takes
  size_t t = 0;
  auto add = [&](size_t b) { t += (b + 255) & ~size_t(255); };
  for (int k = 0; k < 21; ++k) add(sizeof(float) * n_p);
  for (int k = 0; k < 10; ++k) add(sizeof(float) * slot_cap);
  add(sizeof(double) * ((n_p + kAdjBlock - 1) / kAdjBlock) * kParts);
  add(sizeof(double) * (5 + 3 * BM_MAX_SEGMENTS));
  return t;
}

void bm_adj_set_slot(void *work, int scene_slot) { reinterpret_cast<AdjWork *>(work)->slot = scene_slot; }

double *bm_adj_acc(void *work) { return reinterpret_cast<AdjWork *>(work)->acc; }

cudaError_t bm_launch_adjoint_substep(const World &w, const void *work, const double fbar[3], int n_p,
                                      int n_node, cudaStream_t st) {
  AdjWork aw = *reinterpret_cast<const AdjWork *>(work);
  aw.fbar[0] = fbar[0];
  aw.fbar[1] = fbar[1];
  aw.fbar[2] = fbar[2];
  if (n_p == 0) return cudaSuccess;
  // per-node kernels: a warp per node; per-particle kernels: a thread per particle
  const int gn = (n_node + kAdjNodesPerBlock - 1) / kAdjNodesPerBlock, gp = (n_p + kAdjBlock - 1) / kAdjBlock;
  k_adj_musl<<<gn, kAdjBlock, 0, st>>>(w, aw);
  k_adj_v1<<<gp, kAdjBlock, 0, st>>>(w, aw);
  k_adj_g2p<<<gn, kAdjBlock, 0, st>>>(w, aw);
  k_adj_part<<<gp, kAdjBlock, 0, st>>>(w, aw);
  k_adj_reduce<<<1, 32, 0, st>>>(w, aw, gp);
  return cudaGetLastError();
}

cudaError_t bm_launch_adjoint_io(const World &w, const void *work, int field, float *buf, int to_work,
                                 int n_p, cudaStream_t st) {
  if (n_p == 0) return cudaSuccess;
  const AdjWork aw = *reinterpret_cast<const AdjWork *>(work);
  k_adj_io<<<(n_p + 255) / 256, 256, 0, st>>>(w, aw, field, buf, to_work);
  return cudaGetLastError();
}
