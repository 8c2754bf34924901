// sm_103a kernels of one TLMPM cutting substep (arXiv 2609.27342, Sec. III).
//
//   k_pre      per particle: tool + floor contact (Eq. 14-15, friction Eq. 12),
//              cutting progress D and release (Eq. 5), reaction wrench (Eq. 16,
//              deterministic block tree), side labels for the next substep
//              (Eq. 3, 4, 6), neo-Hookean stress -> A = -dt V0 P(F)
//   k_p2g      per node: atomic-free gather over the node's fixed reference
//              neighbourhood (Eq. 1-2), per logical grid; coupling (Eq. 8) and
//              grid update (Eq. 9) in registers
//   k_g2p      per particle: PIC/FLIP velocity (Eq. 17) and x update
//   k_musl     per node: re-scatter m v^{n+1} per logical grid + coupling
//   k_fupd     per particle: F += dt sum v* (x) grad0 N
//   k_tool     per scene: commit labels, reduce the wrench, rigid tool step,
//              frame of the next substep
//   k_slot_*   per node: compact logical-grid slots (Sec. III-G), only in
//              substeps after a label changed
//
// All arithmetic is float32 except the tool state and the near-threshold
// fallback of the side-label predicate, which is float64 with explicitly
// rounded operations so it reproduces a plain double-precision evaluation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bm_internal.cuh"

#define FULL 0xffffffffu

namespace {

// --------------------------------------------------------------------------
// quadratic B-spline of Eq. 1: weight and d/dxl of node base+o, o in {0,1,2},
// for a particle at fractional offset f = xl - base in [0.5, 1.5)
// --------------------------------------------------------------------------
template <int O>
__device__ __forceinline__ void bs(float f, float &w, float &dw) {
  if (O == 0) {
    float t = 1.5f - f;
    w = 0.5f * t * t;
    dw = -t;
  } else if (O == 1) {
    float t = f - 1.0f;
    w = 0.75f - t * t;
    dw = -2.0f * t;
  } else {
    float t = f - 0.5f;
    w = 0.5f * t * t;
    dw = t;
  }
}

__device__ __forceinline__ void bs_rt(int o, float f, float &w, float &dw) {
  if (o == 0) bs<0>(f, w, dw);
  else if (o == 1) bs<1>(f, w, dw);
  else bs<2>(f, w, dw);
}

__device__ __forceinline__ bool conflict(uint32_t a1, uint32_t a2, uint32_t b1, uint32_t b2) {
  return ((a1 & b2) | (a2 & b1)) != 0u;
}

// --------------------------------------------------------------------------
// neo-Hookean first Piola-Kirchhoff stress, P = mu (F - F^-T) + lam ln J F^-T
// --------------------------------------------------------------------------
__device__ __forceinline__ bool piola(const float F[9], float mu, float lam, float P[9]) {
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
  bool clamped = false;
  if (!(J > 1e-6f)) {
    J = 1e-6f;
    clamped = true;
  }
  float iJ = 1.0f / J;
  float lj = logf(J);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float FinvT = c[k] * iJ;
    P[k] = mu * (F[k] - FinvT) + lam * lj * FinvT;
  }
  return clamped;
}

// --------------------------------------------------------------------------
// Eq. 12: spring-history Coulomb friction (float32)
// --------------------------------------------------------------------------
__device__ __forceinline__ void friction(const float uh[3], const float n[3], const float vrel[3],
                                         float fn, float meff, float dt, float gk, float gc,
                                         float mus, float mud, float ft[3], float un[3]) {
  float udn = uh[0] * n[0] + uh[1] * n[1] + uh[2] * n[2];
  float ul = sqrtf(uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2]);
  float tu[3] = {uh[0] - udn * n[0], uh[1] - udn * n[1], uh[2] - udn * n[2]};
  float tl = sqrtf(tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2]);
  float sc = tl > 0.0f ? ul / tl : 0.0f;
  float ut[3] = {tu[0] * sc, tu[1] * sc, tu[2] * sc};
  float vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
  float vt[3] = {vrel[0] - vn * n[0], vrel[1] - vn * n[1], vrel[2] - vn * n[2]};
  float kt = gk * meff / (dt * dt);
  float ct = 2.0f * gc * sqrtf(meff * kt);
  float ftr[3] = {-kt * ut[0] - ct * vt[0], -kt * ut[1] - ct * vt[1], -kt * ut[2] - ct * vt[2]};
  float fl = sqrtf(ftr[0] * ftr[0] + ftr[1] * ftr[1] + ftr[2] * ftr[2]);
  if (fl <= mus * fn) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ft[i] = ftr[i];
      un[i] = ut[i] + dt * vt[i];
    }
  } else {
    float s = mud * fn / fl;
    float ikt = 1.0f / kt;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ft[i] = s * ftr[i];
      un[i] = -(ft[i] + ct * vt[i]) * ikt;
    }
  }
}

// --------------------------------------------------------------------------
// blade box: closest point, outward normal, sphere gap (float32)
// --------------------------------------------------------------------------
__device__ __forceinline__ void box_closest(const DevScene &sc, const float x[3], float R,
                                            float xc[3], float nB[3], float &phi) {
  const float *ax[3] = {sc.fn, sc.fe, sc.fd};
  float r[3] = {x[0] - sc.fc[0], x[1] - sc.fc[1], x[2] - sc.fc[2]};
  float q[3], qc[3], nl[3] = {0.f, 0.f, 0.f};
  bool outside = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    q[a] = r[0] * ax[a][0] + r[1] * ax[a][1] + r[2] * ax[a][2];
    outside |= fabsf(q[a]) > sc.fhext[a];
  }
  if (outside) {
    float diff[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      qc[a] = fminf(fmaxf(q[a], -sc.fhext[a]), sc.fhext[a]);
      diff[a] = q[a] - qc[a];
    }
    float dist = sqrtf(diff[0] * diff[0] + diff[1] * diff[1] + diff[2] * diff[2]);
    float id = 1.0f / dist;
#pragma unroll
    for (int a = 0; a < 3; ++a) nl[a] = diff[a] * id;
    phi = dist - R;
  } else {
    int best = 0;
    float bd = sc.fhext[0] - fabsf(q[0]);
#pragma unroll
    for (int a = 1; a < 3; ++a) {
      float dd = sc.fhext[a] - fabsf(q[a]);
      if (dd < bd) {
        bd = dd;
        best = a;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) qc[a] = q[a];
    float sg = q[best] < 0.0f ? -1.0f : 1.0f;
    qc[best] = sg * sc.fhext[best];
    nl[best] = sg;
    phi = -bd - R;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    xc[i] = sc.fc[i] + qc[0] * ax[0][i] + qc[1] * ax[1][i] + qc[2] * ax[2][i];
    nB[i] = nl[0] * ax[0][i] + nl[1] * ax[1][i] + nl[2] * ax[2][i];
  }
}

// --------------------------------------------------------------------------
// Eq. 3, 4, 6 side label.  float32 filter with a forward-error bound; within
// the bound of any threshold the decision is re-taken in float64 with every
// operation rounded separately, in the order of a plain double evaluation:
// r = x - x_e; s = (r0 n0 + r1 n1) + r2 n2; (same for l, f);
// u_c = ((ve0-v0) d0 + (ve1-v1) d1) + (ve2-v2) d2; lowb = -b_back - max(u_c dt, 0).
// --------------------------------------------------------------------------
__device__ __noinline__ int side_label_exact(const DevScene &sc, const float xf[3],
                                             const float vf[3]) {
  double x0 = xf[0], x1 = xf[1], x2 = xf[2];
  double r0 = __dsub_rn(x0, sc.dxe[0]), r1 = __dsub_rn(x1, sc.dxe[1]), r2 = __dsub_rn(x2, sc.dxe[2]);
  double s = __dadd_rn(__dadd_rn(__dmul_rn(r0, sc.dn[0]), __dmul_rn(r1, sc.dn[1])), __dmul_rn(r2, sc.dn[2]));
  double l = __dadd_rn(__dadd_rn(__dmul_rn(r0, sc.de[0]), __dmul_rn(r1, sc.de[1])), __dmul_rn(r2, sc.de[2]));
  double f = __dadd_rn(__dadd_rn(__dmul_rn(r0, sc.dd[0]), __dmul_rn(r1, sc.dd[1])), __dmul_rn(r2, sc.dd[2]));
  double u0 = __dsub_rn(sc.dve[0], (double)vf[0]);
  double u1 = __dsub_rn(sc.dve[1], (double)vf[1]);
  double u2 = __dsub_rn(sc.dve[2], (double)vf[2]);
  double uc = __dadd_rn(__dadd_rn(__dmul_rn(u0, sc.dd[0]), __dmul_rn(u1, sc.dd[1])), __dmul_rn(u2, sc.dd[2]));
  double ucdt = __dmul_rn(uc, sc.dt_d);
  double lowb = __dsub_rn(-sc.b_back_d, ucdt > 0.0 ? ucdt : 0.0);
  bool band = fabs(s) <= sc.h_d && fabs(l) <= sc.L_d && lowb <= f && f <= sc.b_lead_d;
  if (!band || !(f <= 0.0)) return 0;
  return s < 0.0 ? 1 : 2;
}

__device__ __forceinline__ int side_label(const DevScene &sc, const float x[3], const float v[3]) {
  const float r0 = x[0] - sc.fxe[0], r1 = x[1] - sc.fxe[1], r2 = x[2] - sc.fxe[2];
  const float s = r0 * sc.fn[0] + r1 * sc.fn[1] + r2 * sc.fn[2];
  const float l = r0 * sc.fe[0] + r1 * sc.fe[1] + r2 * sc.fe[2];
  const float f = r0 * sc.fd[0] + r1 * sc.fd[1] + r2 * sc.fd[2];
  const float uc = (sc.fve[0] - v[0]) * sc.fd[0] + (sc.fve[1] - v[1]) * sc.fd[1] +
                   (sc.fve[2] - v[2]) * sc.fd[2];
  const float ucdt = uc * sc.dt;
  const float lowb = -sc.b_back - fmaxf(ucdt, 0.0f);
  // forward-error bounds (2^-20 = 16 u, generous over the ~5 u analysis)
  const float k = 9.5367431640625e-07f;
  const float mag = fabsf(x[0]) + fabsf(x[1]) + fabsf(x[2]) +
                    2.0f * (fabsf(sc.fxe[0]) + fabsf(sc.fxe[1]) + fabsf(sc.fxe[2]));
  const float E = k * mag + 1e-30f;
  const float Eu = k * ((fabsf(sc.fve[0]) + fabsf(sc.fve[1]) + fabsf(sc.fve[2]) + fabsf(v[0]) +
                         fabsf(v[1]) + fabsf(v[2])) * sc.dt + sc.b_back + fabsf(ucdt));
  const float as = fabsf(s), al = fabsf(l);
  const bool near = as <= E || fabsf(as - sc.h) <= E + k * sc.h || fabsf(al - sc.fL) <= E + k * sc.fL ||
                    fabsf(f) <= E || fabsf(f - sc.b_lead) <= E + k * sc.b_lead ||
                    fabsf(f - lowb) <= E + Eu;
  if (near) return side_label_exact(sc, x, v);
  const bool band = as <= sc.h && al <= sc.fL && lowb <= f && f <= sc.b_lead;
  if (!band || !(f <= 0.0f)) return 0;
  return s < 0.0f ? 1 : 2;
}

// deterministic block sum of a double (fixed shuffle tree, warps in order)
__device__ __forceinline__ double block_sum(double v, double *sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  __syncthreads();
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += sm[i];
  return t;  // valid in thread 0
}

// --------------------------------------------------------------------------
// k_pre
// --------------------------------------------------------------------------
__global__ void k_pre(World w, LaunchSet ls) {
  const int4 t = ls.ptiles[blockIdx.x];
  const DevScene &sc = w.scenes[t.x];
  const PPool &P = w.P;
  const int i = threadIdx.x;
  const bool act = i < t.z;
  const int p = t.y + i;
  double wr[6] = {0, 0, 0, 0, 0, 0};
  int want = 0;
  int entry = 0;
  if (act) {
    float x[3] = {P.x[0][p], P.x[1][p], P.x[2][p]};
    float v[3] = {P.v[0][p], P.v[1][p], P.v[2][p]};
    float J[3] = {0.f, 0.f, 0.f};
    const float dt = sc.dt, mp = sc.mp;
    const int cut = sc.cut;
    float D = sc.reset_D ? 0.0f : P.D[p];
    float uh[3] = {P.ut[0][p], P.ut[1][p], P.ut[2][p]};
    if (sc.has_blade && sc.tool_contact_on) {
      float xc[3], nB[3], phi;
      box_closest(sc, x, sc.Rp, xc, nB, phi);
      float rc[3] = {xc[0] - sc.fxB[0], xc[1] - sc.fxB[1], xc[2] - sc.fxB[2]};
      float wr3[3] = {sc.fwB[1] * rc[2] - sc.fwB[2] * rc[1], sc.fwB[2] * rc[0] - sc.fwB[0] * rc[2],
                      sc.fwB[0] * rc[1] - sc.fwB[1] * rc[0]};
      float vrel[3] = {v[0] - (sc.fvB[0] + wr3[0]), v[1] - (sc.fvB[1] + wr3[1]),
                       v[2] - (sc.fvB[2] + wr3[2])};
      float vn = vrel[0] * nB[0] + vrel[1] * nB[1] + vrel[2] * nB[2];
      float phihat = phi + dt * fminf(vn, 0.0f);
      float wB = 0.0f;
      if (sc.finv_mass > 0.0f) {
        float rn[3] = {rc[1] * nB[2] - rc[2] * nB[1], rc[2] * nB[0] - rc[0] * nB[2],
                       rc[0] * nB[1] - rc[1] * nB[0]};
        float q0 = sc.fIinv[0] * rn[0] + sc.fIinv[1] * rn[1] + sc.fIinv[2] * rn[2];
        float q1 = sc.fIinv[3] * rn[0] + sc.fIinv[4] * rn[1] + sc.fIinv[5] * rn[2];
        float q2 = sc.fIinv[6] * rn[0] + sc.fIinv[7] * rn[1] + sc.fIinv[8] * rn[2];
        wB = sc.finv_mass + rn[0] * q0 + rn[1] * q1 + rn[2] * q2;
      }
      float meff = 1.0f / (1.0f / mp + wB);
      float Jn = sc.s_n * meff / dt * fmaxf(-phihat, 0.0f);
      float JB[3] = {0.f, 0.f, 0.f};
      if (Jn > 0.0f) {
        float ft[3], un[3];
        friction(uh, nB, vrel, Jn / dt, meff, dt, sc.gamma_k, sc.gamma_c, sc.fmu_s, sc.fmu_d, ft, un);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          JB[a] = Jn * nB[a] + dt * ft[a];
          uh[a] = un[a];
        }
        if (cut >= 0) {  // Eq. 5: front band, advancing cut
          float r[3] = {x[0] - sc.fxe[0], x[1] - sc.fxe[1], x[2] - sc.fxe[2]};
          float sp = r[0] * sc.fn[0] + r[1] * sc.fn[1] + r[2] * sc.fn[2];
          float lp = r[0] * sc.fe[0] + r[1] * sc.fe[1] + r[2] * sc.fe[2];
          float fp = r[0] * sc.fd[0] + r[1] * sc.fd[1] + r[2] * sc.fd[2];
          float uc = (sc.fve[0] - v[0]) * sc.fd[0] + (sc.fve[1] - v[1]) * sc.fd[1] +
                     (sc.fve[2] - v[2]) * sc.fd[2];
          bool front = fabsf(sp) <= sc.h && fabsf(lp) <= sc.fL && fp >= 0.0f && fp <= sc.b_lead &&
                       uc > sc.u_min;
          if (front) {
            float Jc = fmaxf(JB[0] * sc.fd[0] + JB[1] * sc.fd[1] + JB[2] * sc.fd[2], 0.0f);
            if (D < 1.0f) {
              D = fminf(D + Jc * uc / sc.Wth, 1.0f);
            } else {
#pragma unroll
              for (int a = 0; a < 3; ++a) JB[a] -= Jc * sc.fd[a];
            }
          }
        }
      } else {
        uh[0] = uh[1] = uh[2] = 0.0f;
      }
      // Eq. 16: reaction on the tool
      float idt = 1.0f / dt;
      float FB[3] = {-JB[0] * idt, -JB[1] * idt, -JB[2] * idt};
      wr[0] = FB[0];
      wr[1] = FB[1];
      wr[2] = FB[2];
      wr[3] = rc[1] * FB[2] - rc[2] * FB[1];
      wr[4] = rc[2] * FB[0] - rc[0] * FB[2];
      wr[5] = rc[0] * FB[1] - rc[1] * FB[0];
      J[0] += JB[0];
      J[1] += JB[1];
      J[2] += JB[2];
    }
    if (sc.floor_on) {
      float phi = x[2] - sc.floor_z - sc.Rp;
      float phihat = phi + dt * fminf(v[2], 0.0f);
      J[2] += sc.s_n * mp / dt * fmaxf(-phihat, 0.0f);
    }
    // body force folded into the impulse scattered by P2G
#pragma unroll
    for (int a = 0; a < 3; ++a) J[a] += mp * sc.g[a] * dt;
    // side labels for the next substep
    if (cut >= 0) {
      const uint32_t bit = 1u << cut;
      if (((P.s1[p] | P.s2[p]) & bit) == 0u) {
        int d = side_label(sc, x, v);
        if (d) {
          want = 1;
          entry = ((p - sc.p_begin) << 1) | (d - 1);
        }
      }
    }
    // stress
    float F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = P.F[k][p];
    float Pk[9];
    bool clamped = piola(F, sc.mu, sc.lam, Pk);
    const float c = -dt * sc.V0;
#pragma unroll
    for (int k = 0; k < 9; ++k) P.A[k][p] = c * Pk[k];
    P.J[0][p] = J[0];
    P.J[1][p] = J[1];
    P.J[2][p] = J[2];
    P.D[p] = D;
    P.ut[0][p] = uh[0];
    P.ut[1][p] = uh[1];
    P.ut[2][p] = uh[2];
    if (clamped) atomicOr(&w.scenes[t.x].err, BM_ERRBIT_INVERTED);
  }
  // warp-aggregated append of new labels (order is irrelevant: each entry is
  // a distinct particle and the commit is an OR of one bit)
  const unsigned m = __ballot_sync(FULL, want);
  if (m) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int basei = 0;
    if (lane == leader) basei = atomicAdd(&w.scenes[t.x].list_count, __popc(m));
    basei = __shfl_sync(FULL, basei, leader);
    if (want) {
      const int rank = __popc(m & ((1u << lane) - 1u));
      P.list[sc.p_begin + basei + rank] = entry;
    }
  }
  // wrench partials of this tile
  if (sc.has_blade) {
    __shared__ double sm[32];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double s = block_sum(wr[k], sm);
      if (threadIdx.x == 0) w.wpart[(size_t)t.w * 6 + k] = s;
    }
  }
}

// --------------------------------------------------------------------------
// P2G gather + coupling + grid update (one thread per node)
// --------------------------------------------------------------------------
struct Acc {
  float m, mv[3], dp[3];
};

template <int OX, int OY, int OZ>
__device__ __forceinline__ void p2g_cell(const PPool &P, int p0, int p1, float inv_dx, Acc &a) {
  for (int p = p0; p < p1; ++p) {
    float wx, dwx, wy, dwy, wz, dwz;
    bs<OX>(P.fx[0][p], wx, dwx);
    bs<OY>(P.fx[1][p], wy, dwy);
    bs<OZ>(P.fx[2][p], wz, dwz);
    const float N = wx * wy * wz;
    const float g0 = dwx * wy * wz * inv_dx, g1 = wx * dwy * wz * inv_dx, g2 = wx * wy * dwz * inv_dx;
    const float v0 = P.v[0][p], v1 = P.v[1][p], v2 = P.v[2][p];
    a.m += N;
    a.mv[0] += N * v0;
    a.mv[1] += N * v1;
    a.mv[2] += N * v2;
    a.dp[0] += P.A[0][p] * g0 + P.A[1][p] * g1 + P.A[2][p] * g2 + N * P.J[0][p];
    a.dp[1] += P.A[3][p] * g0 + P.A[4][p] * g1 + P.A[5][p] * g2 + N * P.J[1][p];
    a.dp[2] += P.A[6][p] * g0 + P.A[7][p] * g1 + P.A[8][p] * g2 + N * P.J[2][p];
  }
}

// multi-slot version: particles go to the slot holding their exact code
__device__ __forceinline__ void p2g_cell_ms(const PPool &P, int p0, int p1, int ox, int oy, int oz,
                                            float inv_dx, int ns, const uint2 *codes, Acc *acc) {
  for (int p = p0; p < p1; ++p) {
    const uint32_t c1 = P.s1[p], c2 = P.s2[p];
    int a = 0;
    for (; a < ns; ++a)
      if (codes[a].x == c1 && codes[a].y == c2) break;
    if (a == ns) continue;
    float wx, dwx, wy, dwy, wz, dwz;
    bs_rt(ox, P.fx[0][p], wx, dwx);
    bs_rt(oy, P.fx[1][p], wy, dwy);
    bs_rt(oz, P.fx[2][p], wz, dwz);
    const float N = wx * wy * wz;
    const float g0 = dwx * wy * wz * inv_dx, g1 = wx * dwy * wz * inv_dx, g2 = wx * wy * dwz * inv_dx;
    Acc &A = acc[a];
    A.m += N;
    A.mv[0] += N * P.v[0][p];
    A.mv[1] += N * P.v[1][p];
    A.mv[2] += N * P.v[2][p];
    A.dp[0] += P.A[0][p] * g0 + P.A[1][p] * g1 + P.A[2][p] * g2 + N * P.J[0][p];
    A.dp[1] += P.A[3][p] * g0 + P.A[4][p] * g1 + P.A[5][p] * g2 + N * P.J[1][p];
    A.dp[2] += P.A[6][p] * g0 + P.A[7][p] * g1 + P.A[8][p] * g2 + N * P.J[2][p];
  }
}

__device__ __forceinline__ void node_coords(const DevScene &sc, int li, int &ix, int &iy, int &iz) {
  ix = li % sc.nn[0];
  int r = li / sc.nn[0];
  iy = r % sc.nn[1];
  iz = r / sc.nn[1];
}

__device__ __forceinline__ int cell_index(const DevScene &sc, int bx, int by, int bz) {
  return (bz * sc.nb[1] + by) * sc.nb[0] + bx;
}

#define BM_FOR_27(BODY)                                               \
  BODY(0, 0, 0) BODY(1, 0, 0) BODY(2, 0, 0) BODY(0, 1, 0) BODY(1, 1, 0) \
  BODY(2, 1, 0) BODY(0, 2, 0) BODY(1, 2, 0) BODY(2, 2, 0)               \
  BODY(0, 0, 1) BODY(1, 0, 1) BODY(2, 0, 1) BODY(0, 1, 1) BODY(1, 1, 1) \
  BODY(2, 1, 1) BODY(0, 2, 1) BODY(1, 2, 1) BODY(2, 2, 1)               \
  BODY(0, 0, 2) BODY(1, 0, 2) BODY(2, 0, 2) BODY(0, 1, 2) BODY(1, 1, 2) \
  BODY(2, 1, 2) BODY(0, 2, 2) BODY(1, 2, 2) BODY(2, 2, 2)

// Eq. 8 on ns logical grids with masses m and states S[a][nc]
template <int NC>
__device__ __forceinline__ void couple(int ns, const uint2 *codes, const float *m, float (*S)[NC]) {
  float M = 0.f;
  for (int a = 0; a < ns; ++a) M += m[a];
  if (!(M > 0.f)) return;
  const float iM = 1.0f / M;
  float out[BM_MAXS][NC];
  for (int a = 0; a < ns; ++a) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float acc = 0.f;
      for (int b = 0; b < ns; ++b) {
        if (b == a || conflict(codes[a].x, codes[a].y, codes[b].x, codes[b].y)) continue;
        acc += m[a] * S[b][c] - m[b] * S[a][c];
      }
      out[a][c] = S[a][c] + acc * iM;
    }
  }
  for (int a = 0; a < ns; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) S[a][c] = out[a][c];
}

__global__ void k_p2g(World w, LaunchSet ls) {
  const int4 t = ls.ntiles[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= t.z) return;
  const DevScene &sc = w.scenes[t.x];
  const PPool &P = w.P;
  const int node = t.y + i;
  const int ns = w.N.slot_cnt[node];
  if (ns == 0) return;
  const int off = w.N.slot_off[node];
  int ix, iy, iz;
  node_coords(sc, node - sc.node_begin, ix, iy, iz);
  const int *cs = w.N.cell_start + sc.cell_begin;
  const float inv_dx = sc.inv_dx;
  if (ns == 1) {
    Acc a = {0.f, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#define P2G_BODY(OX, OY, OZ)                                                      \
  {                                                                               \
    const int bx = ix - OX, by = iy - OY, bz = iz - OZ;                           \
    if (bx >= 0 && by >= 0 && bz >= 0 && bx < sc.nb[0] && by < sc.nb[1] && bz < sc.nb[2]) { \
      const int c = cell_index(sc, bx, by, bz);                                   \
      p2g_cell<OX, OY, OZ>(P, cs[c], cs[c + 1], inv_dx, a);                        \
    }                                                                             \
  }
    BM_FOR_27(P2G_BODY)
#undef P2G_BODY
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f), nw = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.m > 0.f) {
      const float im = 1.0f / a.m, imm = 1.0f / (sc.mp * a.m);
      o = make_float4(a.mv[0] * im, a.mv[1] * im, a.mv[2] * im, sc.mp * a.m);
      nw = make_float4(o.x + a.dp[0] * imm, o.y + a.dp[1] * imm, o.z + a.dp[2] * imm, 0.f);
    }
    w.S.vold[off] = o;
    w.S.vnew[off] = nw;
    return;
  }
  // several logical grids at this node
  uint2 codes[BM_MAXS];
  Acc acc[BM_MAXS];
  for (int a = 0; a < ns; ++a) {
    codes[a] = w.S.code[off + a];
    acc[a] = Acc{0.f, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  }
  for (int oz = 0; oz < 3; ++oz)
    for (int oy = 0; oy < 3; ++oy)
      for (int ox = 0; ox < 3; ++ox) {
        const int bx = ix - ox, by = iy - oy, bz = iz - oz;
        if (bx < 0 || by < 0 || bz < 0 || bx >= sc.nb[0] || by >= sc.nb[1] || bz >= sc.nb[2]) continue;
        const int c = cell_index(sc, bx, by, bz);
        p2g_cell_ms(P, cs[c], cs[c + 1], ox, oy, oz, inv_dx, ns, codes, acc);
      }
  float m[BM_MAXS];
  float S[BM_MAXS][6];
  for (int a = 0; a < ns; ++a) {
    m[a] = sc.mp * acc[a].m;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S[a][c] = sc.mp * acc[a].mv[c];
      S[a][3 + c] = acc[a].dp[c];
    }
  }
  couple<6>(ns, codes, m, S);
  for (int a = 0; a < ns; ++a) {
    float4 o = make_float4(0.f, 0.f, 0.f, m[a]), nw = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m[a] > 0.f) {
      const float im = 1.0f / m[a];
      o = make_float4(S[a][0] * im, S[a][1] * im, S[a][2] * im, m[a]);
      nw = make_float4((S[a][0] + S[a][3]) * im, (S[a][1] + S[a][4]) * im, (S[a][2] + S[a][5]) * im, 0.f);
    }
    w.S.vold[off + a] = o;
    w.S.vnew[off + a] = nw;
  }
}

// slot of a particle's code at a node (-1: none)
__device__ __forceinline__ int find_slot(const World &w, int node, uint32_t s1, uint32_t s2) {
  const int ns = w.N.slot_cnt[node];
  const int off = w.N.slot_off[node];
  if (ns == 1) return off;
  for (int a = 0; a < ns; ++a) {
    const uint2 c = w.S.code[off + a];
    if (c.x == s1 && c.y == s2) return off + a;
  }
  return -1;
}

__device__ __forceinline__ void particle_base(const DevScene &sc, uint32_t b, int &bx, int &by, int &bz) {
  bx = (int)(b & 1023u);
  by = (int)((b >> 10) & 1023u);
  bz = (int)((b >> 20) & 1023u);
}

// --------------------------------------------------------------------------
// G2P: Eq. 17 and the position update
// --------------------------------------------------------------------------
__global__ void k_g2p(World w, LaunchSet ls) {
  const int4 t = ls.ptiles[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= t.z) return;
  const DevScene &sc = w.scenes[t.x];
  const PPool &P = w.P;
  const int p = t.y + i;
  int bx, by, bz;
  particle_base(sc, P.base[p], bx, by, bz);
  const uint32_t s1 = P.s1[p], s2 = P.s2[p];
  float wx[3], wy[3], wz[3], d;
  const float f0 = P.fx[0][p], f1 = P.fx[1][p], f2 = P.fx[2][p];
  bs<0>(f0, wx[0], d); bs<1>(f0, wx[1], d); bs<2>(f0, wx[2], d);
  bs<0>(f1, wy[0], d); bs<1>(f1, wy[1], d); bs<2>(f1, wy[2], d);
  bs<0>(f2, wz[0], d); bs<1>(f2, wz[1], d); bs<2>(f2, wz[2], d);
  float sn[3] = {0.f, 0.f, 0.f}, so[3] = {0.f, 0.f, 0.f};
  const int nb0 = sc.node_begin;
#pragma unroll
  for (int oz = 0; oz < 3; ++oz)
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) {
        const int node = nb0 + ((bz + oz) * sc.nn[1] + (by + oy)) * sc.nn[0] + (bx + ox);
        const int a = find_slot(w, node, s1, s2);
        if (a < 0) continue;
        const float4 vo = w.S.vold[a];
        if (!(vo.w > 0.f)) continue;
        const float4 vn = w.S.vnew[a];
        const float N = wx[ox] * wy[oy] * wz[oz];
        sn[0] += N * vn.x;
        sn[1] += N * vn.y;
        sn[2] += N * vn.z;
        so[0] += N * vo.x;
        so[1] += N * vo.y;
        so[2] += N * vo.z;
      }
  const float beta = sc.beta, dt = sc.dt;
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float vv = beta * (P.v[a][p] - so[a]) + sn[a];
    const float xx = P.x[a][p] + dt * sn[a];
    P.v[a][p] = vv;
    P.x[a][p] = xx;
    bad |= !isfinite(vv) || !isfinite(xx);
  }
  if (bad) atomicOr(&w.scenes[t.x].err, BM_ERRBIT_NONFINITE);
}

// --------------------------------------------------------------------------
// MUSL re-scatter with coupling -> v*
// --------------------------------------------------------------------------
template <int OX, int OY, int OZ>
__device__ __forceinline__ void musl_cell(const PPool &P, int p0, int p1, float &m, float mv[3]) {
  for (int p = p0; p < p1; ++p) {
    float wx, wy, wz, d;
    bs<OX>(P.fx[0][p], wx, d);
    bs<OY>(P.fx[1][p], wy, d);
    bs<OZ>(P.fx[2][p], wz, d);
    const float N = wx * wy * wz;
    m += N;
    mv[0] += N * P.v[0][p];
    mv[1] += N * P.v[1][p];
    mv[2] += N * P.v[2][p];
  }
}

__global__ void k_musl(World w, LaunchSet ls) {
  const int4 t = ls.ntiles[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= t.z) return;
  const DevScene &sc = w.scenes[t.x];
  const PPool &P = w.P;
  const int node = t.y + i;
  const int ns = w.N.slot_cnt[node];
  if (ns == 0) return;
  const int off = w.N.slot_off[node];
  int ix, iy, iz;
  node_coords(sc, node - sc.node_begin, ix, iy, iz);
  const int *cs = w.N.cell_start + sc.cell_begin;
  if (ns == 1) {
    float m = 0.f, mv[3] = {0.f, 0.f, 0.f};
#define MUSL_BODY(OX, OY, OZ)                                                     \
  {                                                                               \
    const int bx = ix - OX, by = iy - OY, bz = iz - OZ;                           \
    if (bx >= 0 && by >= 0 && bz >= 0 && bx < sc.nb[0] && by < sc.nb[1] && bz < sc.nb[2]) { \
      const int c = cell_index(sc, bx, by, bz);                                   \
      musl_cell<OX, OY, OZ>(P, cs[c], cs[c + 1], m, mv);                           \
    }                                                                             \
  }
    BM_FOR_27(MUSL_BODY)
#undef MUSL_BODY
    float4 vs = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m > 0.f) {
      const float im = 1.0f / m;
      vs = make_float4(mv[0] * im, mv[1] * im, mv[2] * im, 0.f);
    }
    w.S.vstar[off] = vs;
    return;
  }
  uint2 codes[BM_MAXS];
  float mass[BM_MAXS];
  float S[BM_MAXS][3];
  for (int a = 0; a < ns; ++a) {
    codes[a] = w.S.code[off + a];
    mass[a] = w.S.vold[off + a].w;
    S[a][0] = S[a][1] = S[a][2] = 0.f;
  }
  for (int oz = 0; oz < 3; ++oz)
    for (int oy = 0; oy < 3; ++oy)
      for (int ox = 0; ox < 3; ++ox) {
        const int bx = ix - ox, by = iy - oy, bz = iz - oz;
        if (bx < 0 || by < 0 || bz < 0 || bx >= sc.nb[0] || by >= sc.nb[1] || bz >= sc.nb[2]) continue;
        const int c = cell_index(sc, bx, by, bz);
        for (int p = cs[c]; p < cs[c + 1]; ++p) {
          const uint32_t c1 = P.s1[p], c2 = P.s2[p];
          int a = 0;
          for (; a < ns; ++a)
            if (codes[a].x == c1 && codes[a].y == c2) break;
          if (a == ns) continue;
          float wx, wy, wz, d;
          bs_rt(ox, P.fx[0][p], wx, d);
          bs_rt(oy, P.fx[1][p], wy, d);
          bs_rt(oz, P.fx[2][p], wz, d);
          const float N = wx * wy * wz * sc.mp;
          S[a][0] += N * P.v[0][p];
          S[a][1] += N * P.v[1][p];
          S[a][2] += N * P.v[2][p];
        }
      }
  couple<3>(ns, codes, mass, S);
  for (int a = 0; a < ns; ++a) {
    float4 vs = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mass[a] > 0.f) {
      const float im = 1.0f / mass[a];
      vs = make_float4(S[a][0] * im, S[a][1] * im, S[a][2] * im, 0.f);
    }
    w.S.vstar[off + a] = vs;
  }
}

// --------------------------------------------------------------------------
// deformation gradient update
// --------------------------------------------------------------------------
__global__ void k_fupd(World w, LaunchSet ls) {
  const int4 t = ls.ptiles[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= t.z) return;
  const DevScene &sc = w.scenes[t.x];
  const PPool &P = w.P;
  const int p = t.y + i;
  int bx, by, bz;
  particle_base(sc, P.base[p], bx, by, bz);
  const uint32_t s1 = P.s1[p], s2 = P.s2[p];
  float wx[3], wy[3], wz[3], gx[3], gy[3], gz[3];
  const float f0 = P.fx[0][p], f1 = P.fx[1][p], f2 = P.fx[2][p];
  bs<0>(f0, wx[0], gx[0]); bs<1>(f0, wx[1], gx[1]); bs<2>(f0, wx[2], gx[2]);
  bs<0>(f1, wy[0], gy[0]); bs<1>(f1, wy[1], gy[1]); bs<2>(f1, wy[2], gy[2]);
  bs<0>(f2, wz[0], gz[0]); bs<1>(f2, wz[1], gz[1]); bs<2>(f2, wz[2], gz[2]);
  float G[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int nb0 = sc.node_begin;
#pragma unroll
  for (int oz = 0; oz < 3; ++oz)
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) {
        const int node = nb0 + ((bz + oz) * sc.nn[1] + (by + oy)) * sc.nn[0] + (bx + ox);
        const int a = find_slot(w, node, s1, s2);
        if (a < 0) continue;
        const float4 vs = w.S.vstar[a];
        const float g0 = gx[ox] * wy[oy] * wz[oz], g1 = wx[ox] * gy[oy] * wz[oz],
                    g2 = wx[ox] * wy[oy] * gz[oz];
        G[0] += vs.x * g0; G[1] += vs.x * g1; G[2] += vs.x * g2;
        G[3] += vs.y * g0; G[4] += vs.y * g1; G[5] += vs.y * g2;
        G[6] += vs.z * g0; G[7] += vs.z * g1; G[8] += vs.z * g2;
      }
  const float c = sc.dt * sc.inv_dx;
#pragma unroll
  for (int k = 0; k < 9; ++k) P.F[k][p] += c * G[k];
}

// --------------------------------------------------------------------------
// tool: rigid interval, frame of the next substep (float64, one thread)
// --------------------------------------------------------------------------
__device__ void matvec_rn(const double M[9], const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i)
    y[i] = __dadd_rn(__dadd_rn(__dmul_rn(M[3 * i], x[0]), __dmul_rn(M[3 * i + 1], x[1])),
                     __dmul_rn(M[3 * i + 2], x[2]));
}

__device__ void matmul_d(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

__device__ void world_inv_inertia(const DevScene &sc, double Iw[9]) {
  double RT[9], tmp[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) RT[3 * i + j] = sc.R[3 * j + i];
  matmul_d(sc.R, sc.Ib_inv, tmp);
  matmul_d(tmp, RT, Iw);
}

__device__ const DevSeg *seg_at(const DevScene &sc, long long step) {
  long long acc = 0;
  for (int i = 0; i < sc.nseg; ++i) {
    acc += sc.seg[i].n_steps;
    if (step < acc) return &sc.seg[i];
  }
  return nullptr;
}

// Sets up substep sc.step: prescribed twist, cut, D reset, blade frame.
__device__ void prepare_substep(DevScene &sc) {
  if (!sc.has_blade) {
    sc.cut = -1;
    sc.reset_D = 0;
    return;
  }
  const DevSeg *sg = seg_at(sc, sc.step);
  const int cut = sg ? sg->cut_id : -1;
  const bool dynamic = sc.mass > 0.0;
  if (!dynamic && sg)
    for (int i = 0; i < 3; ++i) {
      sc.vB[i] = sg->v[i];
      sc.wB[i] = sg->w[i];
    }
  sc.cut = cut;
  sc.reset_D = (cut >= 0 && cut != sc.cur_cut) ? 1 : 0;
  double t[3];
  matvec_rn(sc.R, sc.edgeT, t);
  for (int i = 0; i < 3; ++i) sc.dxe[i] = __dadd_rn(sc.xB[i], t[i]);
  matvec_rn(sc.R, sc.nT, sc.dn);
  matvec_rn(sc.R, sc.eT, sc.de);
  matvec_rn(sc.R, sc.dT, sc.dd);
  double r[3] = {__dsub_rn(sc.dxe[0], sc.xB[0]), __dsub_rn(sc.dxe[1], sc.xB[1]),
                 __dsub_rn(sc.dxe[2], sc.xB[2])};
  double wr[3] = {__dsub_rn(__dmul_rn(sc.wB[1], r[2]), __dmul_rn(sc.wB[2], r[1])),
                  __dsub_rn(__dmul_rn(sc.wB[2], r[0]), __dmul_rn(sc.wB[0], r[2])),
                  __dsub_rn(__dmul_rn(sc.wB[0], r[1]), __dmul_rn(sc.wB[1], r[0]))};
  for (int i = 0; i < 3; ++i) sc.dve[i] = __dadd_rn(sc.vB[i], wr[i]);
  for (int i = 0; i < 3; ++i) {
    sc.fxe[i] = (float)sc.dxe[i];
    sc.fn[i] = (float)sc.dn[i];
    sc.fe[i] = (float)sc.de[i];
    sc.fd[i] = (float)sc.dd[i];
    sc.fve[i] = (float)sc.dve[i];
    sc.fc[i] = (float)(sc.dxe[i] - sc.half_height * sc.dd[i]);
    sc.fxB[i] = (float)sc.xB[i];
    sc.fvB[i] = (float)sc.vB[i];
    sc.fwB[i] = (float)sc.wB[i];
  }
  sc.fhext[0] = (float)sc.half_thick;
  sc.fhext[1] = (float)sc.half_len;
  sc.fhext[2] = (float)sc.half_height;
  sc.fL = (float)sc.L_d;
  sc.fmu_s = (float)sc.mu_s;
  sc.fmu_d = (float)sc.mu_d;
  if (dynamic) {
    double Iw[9];
    world_inv_inertia(sc, Iw);
    for (int k = 0; k < 9; ++k) sc.fIinv[k] = (float)Iw[k];
    sc.finv_mass = (float)(1.0 / sc.mass);
  } else {
    for (int k = 0; k < 9; ++k) sc.fIinv[k] = 0.f;
    sc.finv_mass = 0.f;
  }
}

__device__ void rot_exp(const double th[3], double Rm[9]) {
  double a = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
  for (int k = 0; k < 9; ++k) Rm[k] = (k % 4 == 0) ? 1.0 : 0.0;
  if (!(a > 0)) return;
  double k0 = th[0] / a, k1 = th[1] / a, k2 = th[2] / a;
  double K[9] = {0, -k2, k1, k2, 0, -k0, -k1, k0, 0};
  double K2[9];
  matmul_d(K, K, K2);
  double sa = sin(a), ca = 1.0 - cos(a);
  for (int k = 0; k < 9; ++k) Rm[k] += sa * K[k] + ca * K2[k];
}

__global__ void k_prepare(World w, LaunchSet ls) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ls.n_scenes) return;
  prepare_substep(w.scenes[ls.scene_ids[idx]]);
}

// tool states {x_B, R, v_B, omega_B} of several scenes, then their frames
__global__ void k_set_tools(World w, const int *ids, int n, const double *states) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  DevScene &sc = w.scenes[ids[idx]];
  const double *q = states + (size_t)idx * 18;
  for (int k = 0; k < 3; ++k) sc.xB[k] = q[k];
  for (int k = 0; k < 9; ++k) sc.R[k] = q[3 + k];
  for (int k = 0; k < 3; ++k) {
    sc.vB[k] = q[12 + k];
    sc.wB[k] = q[15 + k];
  }
  prepare_substep(sc);
}

__global__ void k_get_wrenches(World w, const int *ids, int n, double *out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const DevScene &sc = w.scenes[ids[idx]];
  for (int k = 0; k < 6; ++k) out[(size_t)idx * 6 + k] = sc.lastW[k];
}

__global__ void k_tool(World w, LaunchSet ls) {
  const int sid = ls.scene_ids[blockIdx.x];
  DevScene &sc = w.scenes[sid];
  __shared__ double sm[32];
  // 1. commit the side labels assigned this substep
  const int cnt = sc.list_count;
  const int cut = sc.cut;
  if (cut >= 0) {
    const uint32_t bit = 1u << cut;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int e = w.P.list[sc.p_begin + i];
      const int p = sc.p_begin + (e >> 1);
      if (e & 1) w.P.s2[p] |= bit;
      else w.P.s1[p] |= bit;
    }
  }
  // 2. reduce this substep's wrench partials (fixed order)
  double W[6];
  for (int k = 0; k < 6; ++k) {
    double acc = 0.0;
    if (sc.has_blade)
      for (int j = threadIdx.x; j < sc.n_ptile; j += blockDim.x)
        acc += w.wpart[(size_t)(sc.ptile_begin + j) * 6 + k];
    W[k] = block_sum(acc, sm);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  sc.need_rebuild = cnt > 0 ? 1 : 0;
  sc.list_count = 0;
  if (sc.has_blade) {
    const long long st = sc.step;
    if (st < sc.hist_cap)
      for (int k = 0; k < 6; ++k) w.whist[(size_t)(sc.hist_begin + st) * 6 + k] = W[k];
    for (int k = 0; k < 3; ++k) {
      sc.accF[k] += W[k];
      sc.accT[k] += W[3 + k];
    }
    sc.acc_cnt++;
    if (sc.acc_cnt >= sc.rigid_interval) {
      const double H = sc.dt_d * sc.acc_cnt;
      double Fa[3], Ta[3];
      for (int k = 0; k < 3; ++k) {
        Fa[k] = sc.accF[k] / sc.acc_cnt;
        Ta[k] = sc.accT[k] / sc.acc_cnt;
      }
      if (sc.mass > 0.0) {
        const DevSeg *tg = seg_at(sc, st);
        double vt[3] = {0, 0, 0}, wt[3] = {0, 0, 0};
        if (tg)
          for (int k = 0; k < 3; ++k) {
            vt[k] = tg->v[k];
            wt[k] = tg->w[k];
          }
        double Iw[9], dw[3];
        world_inv_inertia(sc, Iw);
        for (int k = 0; k < 3; ++k) dw[k] = Iw[3 * k] * Ta[0] + Iw[3 * k + 1] * Ta[1] + Iw[3 * k + 2] * Ta[2];
        for (int k = 0; k < 3; ++k) {
          sc.vB[k] += H * (sc.kv * (vt[k] - sc.vB[k]) + Fa[k] / sc.mass);
          sc.wB[k] += H * (sc.kv * (wt[k] - sc.wB[k]) + dw[k]);
        }
      }
      double th[3] = {H * sc.wB[0], H * sc.wB[1], H * sc.wB[2]};
      double Rinc[9], Rn[9];
      rot_exp(th, Rinc);
      matmul_d(Rinc, sc.R, Rn);
      for (int k = 0; k < 9; ++k) sc.R[k] = Rn[k];
      for (int k = 0; k < 3; ++k) sc.xB[k] += H * sc.vB[k];
      for (int k = 0; k < 3; ++k) {
        sc.lastW[k] = Fa[k];
        sc.lastW[3 + k] = Ta[k];
        sc.accF[k] = sc.accT[k] = 0.0;
      }
      sc.acc_cnt = 0;
    }
    if (sc.cut >= 0) sc.cur_cut = sc.cut;
  }
  sc.step++;
  prepare_substep(sc);
}

// --------------------------------------------------------------------------
// logical-grid slot table (rebuilt after label changes)
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ckey(uint2 c) {
  return ((unsigned long long)c.y << 32) | c.x;
}

__device__ __forceinline__ int block_excl_scan(int v, int *sm, int &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sm[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < nw; ++i) {
      int t = sm[i];
      sm[i] = acc;
      acc += t;
    }
    sm[nw] = acc;
  }
  __syncthreads();
  total = sm[nw];
  return x - v + sm[wid];
}

__global__ void k_slot_count(World w, LaunchSet ls, int force) {
  const int4 t = ls.ntiles[blockIdx.x];
  DevScene &sc = w.scenes[t.x];
  if (!force && !sc.need_rebuild) return;
  __shared__ int sm[33];
  const int i = threadIdx.x;
  int cnt = 0;
  if (i < t.z) {
    const int node = t.y + i;
    int ix, iy, iz;
    node_coords(sc, node - sc.node_begin, ix, iy, iz);
    const int *cs = w.N.cell_start + sc.cell_begin;
    unsigned long long keys[BM_MAXS];
    bool over = false;
    for (int oz = 0; oz < 3; ++oz)
      for (int oy = 0; oy < 3; ++oy)
        for (int ox = 0; ox < 3; ++ox) {
          const int bx = ix - ox, by = iy - oy, bz = iz - oz;
          if (bx < 0 || by < 0 || bz < 0 || bx >= sc.nb[0] || by >= sc.nb[1] || bz >= sc.nb[2]) continue;
          const int c = cell_index(sc, bx, by, bz);
          for (int p = cs[c]; p < cs[c + 1]; ++p) {
            const unsigned long long k = ((unsigned long long)w.P.s2[p] << 32) | w.P.s1[p];
            int j = 0;
            while (j < cnt && keys[j] < k) ++j;
            if (j < cnt && keys[j] == k) continue;
            if (cnt == BM_MAXS) {
              over = true;
              continue;
            }
            for (int q = cnt; q > j; --q) keys[q] = keys[q - 1];
            keys[j] = k;
            ++cnt;
          }
        }
    if (over) atomicOr(&sc.err, BM_ERRBIT_SLOT_OVERFLOW);
    w.N.slot_cnt[node] = (uint8_t)cnt;
    for (int a = 0; a < cnt; ++a)
      w.N.tmp_codes[(size_t)node * BM_MAXS + a] = make_uint2((uint32_t)keys[a], (uint32_t)(keys[a] >> 32));
  }
  int total;
  block_excl_scan(cnt, sm, total);
  if (threadIdx.x == 0) w.N.tile_sum[t.w] = total;
}

__global__ void k_slot_scan(World w, LaunchSet ls, int force) {
  DevScene &sc = w.scenes[ls.scene_ids[blockIdx.x]];
  if (!force && !sc.need_rebuild) return;
  __shared__ int sm[33];
  int carry = 0;
  for (int base = 0; base < sc.n_ntile; base += blockDim.x) {
    const int j = base + threadIdx.x;
    const int v = j < sc.n_ntile ? w.N.tile_sum[sc.ntile_begin + j] : 0;
    int total;
    const int ex = block_excl_scan(v, sm, total);
    if (j < sc.n_ntile) w.N.tile_sum[sc.ntile_begin + j] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sc.n_slots = carry;
    if (carry > sc.slot_cap) atomicOr(&sc.err, BM_ERRBIT_SLOT_OVERFLOW);
  }
}

__global__ void k_slot_fill(World w, LaunchSet ls, int force) {
  const int4 t = ls.ntiles[blockIdx.x];
  DevScene &sc = w.scenes[t.x];
  if (!force && !sc.need_rebuild) return;
  __shared__ int sm[33];
  const int i = threadIdx.x;
  const int node = t.y + i;
  const int cnt = i < t.z ? (int)w.N.slot_cnt[node] : 0;
  int total;
  const int ex = block_excl_scan(cnt, sm, total);
  if (i < t.z) {
    const int off = w.N.tile_sum[t.w] + ex;
    if (off + cnt > sc.slot_cap) {
      w.N.slot_cnt[node] = 0;
      w.N.slot_off[node] = sc.slot_begin;
      return;
    }
    w.N.slot_off[node] = sc.slot_begin + off;
    for (int a = 0; a < cnt; ++a)
      w.S.code[sc.slot_begin + off + a] = w.N.tmp_codes[(size_t)node * BM_MAXS + a];
  }
}

// --------------------------------------------------------------------------
// state I/O between pool order and the caller's order
// --------------------------------------------------------------------------
__global__ void k_io(World w, int p_begin, int n, int field, void *buf, int to_pool) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = p_begin + i;
  const int o = w.P.perm[p];
  const PPool &P = w.P;
  float *fb = (float *)buf;
  uint32_t *ub = (uint32_t *)buf;
  switch (field) {
    case 0:  // X (from fx and base cannot reproduce X exactly: kept separately)
      break;
    case 1:
      for (int a = 0; a < 3; ++a) {
        if (to_pool) P.x[a][p] = fb[3 * o + a];
        else fb[3 * o + a] = P.x[a][p];
      }
      break;
    case 2:
      for (int a = 0; a < 3; ++a) {
        if (to_pool) P.v[a][p] = fb[3 * o + a];
        else fb[3 * o + a] = P.v[a][p];
      }
      break;
    case 3:
      for (int a = 0; a < 9; ++a) {
        if (to_pool) P.F[a][p] = fb[9 * o + a];
        else fb[9 * o + a] = P.F[a][p];
      }
      break;
    case 4:
      if (to_pool) P.D[p] = fb[o];
      else fb[o] = P.D[p];
      break;
    case 5:
      for (int a = 0; a < 3; ++a) {
        if (to_pool) P.ut[a][p] = fb[3 * o + a];
        else fb[3 * o + a] = P.ut[a][p];
      }
      break;
    case 7:
      if (to_pool) P.s1[p] = ub[o];
      else ub[o] = P.s1[p];
      break;
    case 8:
      if (to_pool) P.s2[p] = ub[o];
      else ub[o] = P.s2[p];
      break;
  }
}

__global__ void k_code(World w, int p_begin, int n, int64_t *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = p_begin + i;
  const uint32_t a = w.P.s1[p], b = w.P.s2[p];
  int64_t c = 0, pw = 1;
  for (int k = 0; k < BM_MAX_CUTS; ++k) {
    const int d = ((a >> k) & 1u) ? 1 : (((b >> k) & 1u) ? 2 : 0);
    c += d * pw;
    pw *= 3;
  }
  out[w.P.perm[p]] = c;
}

}  // namespace

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
cudaError_t bm_launch_prepare(const World &w, const LaunchSet &ls, cudaStream_t st) {
  if (ls.n_scenes == 0) return cudaSuccess;
  k_prepare<<<(ls.n_scenes + 63) / 64, 64, 0, st>>>(w, ls);
  return cudaGetLastError();
}

const char *const bm_kernel_names[BM_NUM_KERNELS] = {
    "k_pre", "k_p2g", "k_g2p", "k_musl", "k_fupd", "k_tool", "k_slot_count", "k_slot_scan", "k_slot_fill"};

// ev (optional): 2 * BM_NUM_KERNELS events recorded around each launch
static inline void rec(cudaEvent_t *ev, int k, int after, cudaStream_t st) {
  if (ev) cudaEventRecord(ev[2 * k + after], st);
}

static cudaError_t launch_rebuild(const World &w, const LaunchSet &ls, cudaStream_t st, int force,
                                  cudaEvent_t *ev) {
  if (ls.n_ntiles == 0) return cudaSuccess;
  rec(ev, 6, 0, st);
  k_slot_count<<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls, force);
  rec(ev, 6, 1, st);
  rec(ev, 7, 0, st);
  k_slot_scan<<<ls.n_scenes, 256, 0, st>>>(w, ls, force);
  rec(ev, 7, 1, st);
  rec(ev, 8, 0, st);
  k_slot_fill<<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls, force);
  rec(ev, 8, 1, st);
  return cudaGetLastError();
}

cudaError_t bm_launch_rebuild(const World &w, const LaunchSet &ls, cudaStream_t st, int force) {
  return launch_rebuild(w, ls, st, force, nullptr);
}

cudaError_t bm_launch_substep_ev(const World &w, const LaunchSet &ls, cudaStream_t st, cudaEvent_t *ev) {
  if (ls.n_ptiles == 0) return cudaSuccess;
  rec(ev, 0, 0, st);
  k_pre<<<ls.n_ptiles, ls.ptile_size, 0, st>>>(w, ls);
  rec(ev, 0, 1, st);
  rec(ev, 1, 0, st);
  k_p2g<<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls);
  rec(ev, 1, 1, st);
  rec(ev, 2, 0, st);
  k_g2p<<<ls.n_ptiles, ls.ptile_size, 0, st>>>(w, ls);
  rec(ev, 2, 1, st);
  rec(ev, 3, 0, st);
  k_musl<<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls);
  rec(ev, 3, 1, st);
  rec(ev, 4, 0, st);
  k_fupd<<<ls.n_ptiles, ls.ptile_size, 0, st>>>(w, ls);
  rec(ev, 4, 1, st);
  rec(ev, 5, 0, st);
  k_tool<<<ls.n_scenes, 256, 0, st>>>(w, ls);
  rec(ev, 5, 1, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_rebuild(w, ls, st, 0, ev);
}

cudaError_t bm_launch_substep(const World &w, const LaunchSet &ls, cudaStream_t st) {
  return bm_launch_substep_ev(w, ls, st, nullptr);
}

cudaError_t bm_launch_io(const World &w, int scene_slot, int p_begin, int n, int field, void *buf,
                         int to_pool, cudaStream_t st) {
  (void)scene_slot;
  if (n == 0) return cudaSuccess;
  k_io<<<(n + 255) / 256, 256, 0, st>>>(w, p_begin, n, field, buf, to_pool);
  return cudaGetLastError();
}

cudaError_t bm_launch_set_tools(const World &w, const int *scene_ids, int n, const double *states,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_set_tools<<<(n + 63) / 64, 64, 0, st>>>(w, scene_ids, n, states);
  return cudaGetLastError();
}

cudaError_t bm_launch_get_wrenches(const World &w, const int *scene_ids, int n, double *out,
                                   cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_get_wrenches<<<(n + 63) / 64, 64, 0, st>>>(w, scene_ids, n, out);
  return cudaGetLastError();
}

cudaError_t bm_launch_code(const World &w, int p_begin, int n, int64_t *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_code<<<(n + 255) / 256, 256, 0, st>>>(w, p_begin, n, out);
  return cudaGetLastError();
}
