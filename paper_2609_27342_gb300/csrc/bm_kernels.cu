// sm_103a kernels of one TLMPM cutting substep (arXiv 2609.27342, Sec. III).
//
// Particles are sorted brick-major (4x4x4 reference base cells per brick) and
// every particle-side kernel runs one CTA per brick:
//   k_p2g_brick  contact (Eq. 12, 14-16), cutting progress (Eq. 5), side
//                labels for the next substep (Eq. 3, 4, 6), neo-Hookean
//                stress, and the brick's share of the per-code P2G sums
//                (Eq. 2) in its 6x6x6 node tile, in shared memory
//   k_p2g_node   per node: the <= 8 overlapping brick tiles summed in brick
//                order, coupling (Eq. 8), grid update (Eq. 9)
//   k_g2p_musl   G2P (Eq. 17), x update, the brick's share of the MUSL
//                re-scatter
//   k_musl_node  per node: MUSL sums, coupling, v*
//   k_fupd       F update, commit of the new side labels
//   k_tool       per scene: wrench, rigid tool step, next frame
//   k_slot_*     compact logical-grid slots (Sec. III-G) after label changes
//   k_pair_*     material-material contact (Eq. 10-13): the rebuild test,
//                spatial hash and candidate lists, and the pair impulses,
//                ahead of P2G
// No atomics touch floating-point sums: every sum is taken in a fixed order,
// so a scene gives bit-identical results alone or inside any batch.
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
// fixed-corotated stress, P = 2 mu (F - R) + lam (J - 1) J F^-T, with the
// rotation R of the polar decomposition F = R S from Newton's iteration
// R <- (g R + R^-T / g) / 2 (g = (|R^-1| / |R|)^(1/2), Frobenius norms),
// which converges quadratically to R for det F > 0.
// --------------------------------------------------------------------------
__device__ __forceinline__ void cof3(const float F[9], float c[9]) {
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
}

__device__ bool piola_fcr(const float F[9], float mu, float lam, float P[9]) {
  float c[9];
  cof3(F, c);
  const float J = F[0] * c[0] + F[1] * c[1] + F[2] * c[2];
  const bool clamped = !(J > 1e-6f);
  float R[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = F[k];
  for (int it = 0; it < 16; ++it) {
    float q[9];
    cof3(R, q);
    const float d = R[0] * q[0] + R[1] * q[1] + R[2] * q[2];  // R^-T = cof(R) / det R
    if (d == 0.0f) break;
    const float id = 1.0f / d;
    float nr = 0.f, ni = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      q[k] *= id;
      nr += R[k] * R[k];
      ni += q[k] * q[k];
    }
    const float g = sqrtf(sqrtf(ni / nr));
    const float ig = 1.0f / g;
    float dif = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float r = 0.5f * (g * R[k] + ig * q[k]);
      dif += (r - R[k]) * (r - R[k]);
      R[k] = r;
    }
    if (dif <= 1e-13f) break;
  }
  const float jl = lam * (J - 1.0f);
#pragma unroll
  for (int k = 0; k < 9; ++k) P[k] = 2.0f * mu * (F[k] - R[k]) + jl * c[k];
  return clamped;
}

__device__ __forceinline__ void mat3mul(const float A[9], const float B[9], float C[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// symmetric 3x3 eigen-decomposition A = V diag(w) V^T by cyclic Jacobi
// rotations (float32, at most 10 sweeps)
__device__ void sym_eig3(const float Ain[9], float V[9], float w[3]) {
  float A[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    A[k] = Ain[k];
    V[k] = (k % 4 == 0) ? 1.0f : 0.0f;
  }
  for (int sweep = 0; sweep < 10; ++sweep) {
    const float off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    const float dg = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (!(off > 1e-14f * dg)) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
      const float apq = A[3 * p + q];
      if (apq == 0.0f) continue;
      const float th = (A[3 * q + q] - A[3 * p + p]) / (2.0f * apq);
      const float t = copysignf(1.0f, th) / (fabsf(th) + sqrtf(th * th + 1.0f));
      const float c = 1.0f / sqrtf(t * t + 1.0f), sn = t * c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - sn * akq;
        A[3 * k + q] = sn * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - sn * aqk;
        A[3 * q + k] = sn * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - sn * vkq;
        V[3 * k + q] = sn * vkp + c * vkq;
      }
    }
  }
  w[0] = A[0];
  w[1] = A[4];
  w[2] = A[8];
}

// von Mises plasticity: radial return of the deviatoric principal Hencky
// strains e of Fe onto sqrt(3/2) |2 mu e| = sigma_y (isochoric).  Returns
// whether Fe was projected.
__device__ bool vonmises(float Fe[9], float mu, float sy) {
  float C[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = Fe[i] * Fe[j] + Fe[3 + i] * Fe[3 + j] + Fe[6 + i] * Fe[6 + j];
  float V[9], w[3];
  sym_eig3(C, V, w);
  if (!(w[0] > 0.f) || !(w[1] > 0.f) || !(w[2] > 0.f)) return false;
  float sg[3], e[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sg[k] = sqrtf(w[k]);
    e[k] = logf(sg[k]);
  }
  const float mean = (e[0] + e[1] + e[2]) * (1.0f / 3.0f);
#pragma unroll
  for (int k = 0; k < 3; ++k) e[k] -= mean;
  const float q = 2.4494897f * mu * sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);  // sqrt(6) mu |e|
  if (!(q > sy)) return false;
  const float sc = sy / q;
  float rt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) rt[k] = expf(mean + sc * e[k]) / sg[k];
  float M[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      M[3 * i + j] = V[3 * i] * rt[0] * V[3 * j] + V[3 * i + 1] * rt[1] * V[3 * j + 1] +
                     V[3 * i + 2] * rt[2] * V[3 * j + 2];
  float out[9];
  mat3mul(Fe, M, out);
#pragma unroll
  for (int k = 0; k < 9; ++k) Fe[k] = out[k];
  return true;
}

// Stress of a particle of a scene with plasticity or viscosity (kept out of
// line so that the elastic path keeps its registers): plastic projection of
// Fe = F Fp^-1 with Fp^-1 = F^-1 Fe stored back, P = P(Fe) Fp^-T, and the
// viscous part J eta (L + L^T) F^-T with L = dF/dt F^-1 of the last substep.
__device__ __noinline__ bool inelastic_stress(const DevScene &sc, const PPool &P, int p, const float F[9],
                                              float Pk[9]) {
  bool clamped = false;
  if (sc.yield_stress > 0.0f) {
    // Fe = F Fp^-1, projected; Fp^-1 = F^-1 Fe; P = P(Fe) Fp^-T
    float Fpi[9], Fe[9], Pe[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fpi[k] = P.Fpi[k][p];
    mat3mul(F, Fpi, Fe);
    if (vonmises(Fe, sc.mu, sc.yield_stress)) {
      float c[9];
      cof3(F, c);
      const float d = F[0] * c[0] + F[1] * c[1] + F[2] * c[2];
      if (d != 0.0f) {
        const float id = 1.0f / d;
        float Fi[9] = {c[0] * id, c[3] * id, c[6] * id, c[1] * id, c[4] * id,
                       c[7] * id, c[2] * id, c[5] * id, c[8] * id};  // F^-1 = cof(F)^T / det F
        mat3mul(Fi, Fe, Fpi);
#pragma unroll
        for (int k = 0; k < 9; ++k) P.Fpi[k][p] = Fpi[k];
      }
    }
    clamped |= sc.model == BM_MODEL_FIXED_COROTATED ? piola_fcr(Fe, sc.mu, sc.lam, Pe)
                                                    : piola(Fe, sc.mu, sc.lam, Pe);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Pk[3 * i + j] = Pe[3 * i] * Fpi[3 * j] + Pe[3 * i + 1] * Fpi[3 * j + 1] + Pe[3 * i + 2] * Fpi[3 * j + 2];
  } else {
    clamped |= sc.model == BM_MODEL_FIXED_COROTATED ? piola_fcr(F, sc.mu, sc.lam, Pk)
                                                    : piola(F, sc.mu, sc.lam, Pk);
  }
  if (sc.viscosity > 0.0f) {
    // Cauchy eta (L + L^T), L = dF/dt F^-1 (last substep), as J sigma F^-T = sigma cof(F)
    float c[9], Fd[9], L[9];
    cof3(F, c);
    const float d = F[0] * c[0] + F[1] * c[1] + F[2] * c[2];
    if (d != 0.0f) {
      const float id = 1.0f / d;
      const float Fi[9] = {c[0] * id, c[3] * id, c[6] * id, c[1] * id, c[4] * id,
                           c[7] * id, c[2] * id, c[5] * id, c[8] * id};
#pragma unroll
      for (int k = 0; k < 9; ++k) Fd[k] = P.Fdot[k][p];
      mat3mul(Fd, Fi, L);
      float sv[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) sv[3 * i + j] = sc.viscosity * (L[3 * i + j] + L[3 * j + i]);
      float add[9];
      mat3mul(sv, c, add);
#pragma unroll
      for (int k = 0; k < 9; ++k) Pk[k] += add[k];
    }
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
  // forward-error bounds (2^-20 = 16 u, generous over the ~5 u analysis)
  const float k = 9.5367431640625e-07f;
  const float mag = fabsf(x[0]) + fabsf(x[1]) + fabsf(x[2]) +
                    2.0f * (fabsf(sc.fxe[0]) + fabsf(sc.fxe[1]) + fabsf(sc.fxe[2]));
  const float E = k * mag + 1e-30f;
  const float as = fabsf(s);
  // beyond the band's half-width by more than the bound: outside the band
  // in float64 too (the decision below and the exact path both give 0)
  if (as > sc.h + (E + k * sc.h)) return 0;
  const float l = r0 * sc.fe[0] + r1 * sc.fe[1] + r2 * sc.fe[2];
  const float f = r0 * sc.fd[0] + r1 * sc.fd[1] + r2 * sc.fd[2];
  const float uc = (sc.fve[0] - v[0]) * sc.fd[0] + (sc.fve[1] - v[1]) * sc.fd[1] +
                   (sc.fve[2] - v[2]) * sc.fd[2];
  const float ucdt = uc * sc.dt;
  const float lowb = -sc.b_back - fmaxf(ucdt, 0.0f);
  const float Eu = k * ((fabsf(sc.fve[0]) + fabsf(sc.fve[1]) + fabsf(sc.fve[2]) + fabsf(v[0]) +
                         fabsf(v[1]) + fabsf(v[2])) * sc.dt + sc.b_back + fabsf(ucdt));
  const float al = fabsf(l);
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

// exclusive block scan of one int per thread (fixed order); total in all threads
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

// --------------------------------------------------------------------------
// Brick geometry.  Particles are stored brick-major: bricks of 4x4x4 base
// cells, cells x-fastest inside a brick, so a brick's particles form one
// contiguous range.  A brick's particles touch the 6x6x6 node tile starting
// at its first cell (quadratic stencil: nodes base..base+2).
// --------------------------------------------------------------------------
#define BR 4
#define BR3 64
#define TE 6
#define TN 216
#define TSCAP BM_TILE_SLOTS

// Index of particle j of cell c in a brick's [particle-in-cell][cell]
// staging in shared memory.  The cell column is XOR-swizzled by the particle
// index, so that both the staging stores (consecutive particles of a few
// cells) and the per-cell reads (consecutive cells, one particle index) fall
// on distinct banks.
__device__ __forceinline__ int pic(int j, int c) { return j * BR3 + (c ^ ((j & 7) << 2)); }

#define BT 192  // threads per brick CTA: 64 cells x 3 z-offsets

__device__ __forceinline__ void node_coords(const DevScene &sc, int li, int &ix, int &iy, int &iz) {
  ix = li % sc.nn[0];
  int r = li / sc.nn[0];
  iy = r % sc.nn[1];
  iz = r / sc.nn[1];
}

// brick-major index of base cell (bx, by, bz), scene-local coordinates
__device__ __forceinline__ int cell_index(const DevScene &sc, int bx, int by, int bz) {
  const int b = ((bz >> 2) * sc.nbr[1] + (by >> 2)) * sc.nbr[0] + (bx >> 2);
  return b * BR3 + (((bz & 3) * BR + (by & 3)) * BR + (bx & 3));
}

// The cell (0..63) of the brick's particle i: particles are sorted by cell,
// so it is the last cell whose range (cs: the brick's 65 cell starts,
// relative to its first particle) starts at or before i.
__device__ __forceinline__ int cell_of(const int *cs, int i) {
  int c = 0;
#pragma unroll
  for (int step = 32; step > 0; step >>= 1)
    if (cs[c + step] <= i) c += step;
  return c;
}

__device__ __forceinline__ void particle_base(uint32_t b, int &bx, int &by, int &bz) {
  bx = (int)(b & 1023u);
  by = (int)((b >> 10) & 1023u);
  bz = (int)((b >> 20) & 1023u);
}

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

// The node tile of one brick: for each of its 6x6x6 nodes the first tile
// slot (the node's logical grids laid out node by node in each node's own
// slot order), the slot count and the node's first pool slot.  A tile holds
// at most 216 x BM_MAXS slots; shared-memory working sets cover windows of
// TSCAP slots at a time.
struct Tile {
  uint16_t lo[TN];
  uint8_t cnt[TN];
  int goff[TN];
  int total;
};

__device__ __forceinline__ void brick_coords(const DevScene &sc, int lb, int &c0x, int &c0y, int &c0z) {
  c0x = (lb % sc.nbr[0]) * BR;
  c0y = ((lb / sc.nbr[0]) % sc.nbr[1]) * BR;
  c0z = (lb / (sc.nbr[0] * sc.nbr[1])) * BR;
}

// Cooperative load of a brick's tile (all threads; ends with a barrier).  The
// per-node slot counts and first tile slots come from the descriptor the
// slot rebuild wrote for this brick; the nodes' first pool slots from the
// slot table.  Returns (in every thread) whether every tile node holds at
// most one logical grid; the kernels then keep the tile's values by node
// (entry t for tile node t) instead of by tile slot.
__device__ bool tile_load(const World &w, const DevScene &sc, int brick, int c0x, int c0y, int c0z,
                          Tile &T) {
  bool single = true;
  for (int t = threadIdx.x; t < TN; t += blockDim.x) {
    const int d = w.B.tdesc[(size_t)brick * TN + t];
    const int cnt = d >> 16;
    const int off = w.B.tgoff[(size_t)brick * TN + t];  // valid where cnt > 0
    T.lo[t] = (uint16_t)(d & 0xffff);
    T.cnt[t] = (uint8_t)cnt;
    T.goff[t] = off;
    single &= cnt <= 1;
  }
  if (threadIdx.x == 0) T.total = w.B.ptot[brick];
  return __syncthreads_and(single) != 0;
}

// tile slot holding code (s1, s2) at tile node t, or -1.  Nodes with several
// logical grids compare against the tile's codes in shared memory when the
// tile fits the window (codes != nullptr), else against the pool's codes.
__device__ __forceinline__ int tile_slot(const World &w, const Tile &T, const uint2 *codes, int t,
                                         uint32_t s1, uint32_t s2) {
  const int n = T.cnt[t];
  const int lo = T.lo[t];
  if (n == 1) return lo;
  if (codes) {
    for (int a = 0; a < n; ++a) {
      const uint2 c = codes[lo + a];
      if (c.x == s1 && c.y == s2) return lo + a;
    }
    return -1;
  }
  const int off = T.goff[t];
  for (int a = 0; a < n; ++a) {
    const uint2 c = w.S.code[off + a];
    if (c.x == s1 && c.y == s2) return lo + a;
  }
  return -1;
}

// --------------------------------------------------------------------------
// Per-particle work ahead of P2G (one thread per particle, inside the P2G
// brick kernel): tool and floor contact (Eq. 14-15 with friction Eq. 12),
// cutting progress D and release (Eq. 5), reaction wrench (Eq. 16), side
// label for the next substep (Eq. 3, 4, 6), and the P2G inputs
// A = -dt V0 P(F) / dx and the particle's total impulse J.
// --------------------------------------------------------------------------
// Whether the blade box is farther from the particle than one substep of
// relative motion can close: d > R_p + 2 dt (|v| + |v_B| + |w_B| r_max) (1-norms
// bound the speeds; r_max bounds the reach of the box from the blade's
// reference point), so that the predicted gap phi_hat = phi + dt min(v_n, 0)
// of the contact test is positive with a margin far above rounding.
__device__ __forceinline__ bool blade_out_of_reach(const DevScene &sc, const float x[3], const float v[3]) {
  const float *ax[3] = {sc.fn, sc.fe, sc.fd};
  const float r[3] = {x[0] - sc.fc[0], x[1] - sc.fc[1], x[2] - sc.fc[2]};
  float d2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float q = r[0] * ax[a][0] + r[1] * ax[a][1] + r[2] * ax[a][2];
    const float e = fmaxf(fabsf(q) - sc.fhext[a], 0.0f);
    d2 += e * e;
  }
  const float rmax = fabsf(sc.fc[0] - sc.fxB[0]) + fabsf(sc.fc[1] - sc.fxB[1]) + fabsf(sc.fc[2] - sc.fxB[2]) +
                     sc.fhext[0] + sc.fhext[1] + sc.fhext[2];
  const float vb = fabsf(v[0]) + fabsf(v[1]) + fabsf(v[2]) + fabsf(sc.fvB[0]) + fabsf(sc.fvB[1]) +
                   fabsf(sc.fvB[2]) + (fabsf(sc.fwB[0]) + fabsf(sc.fwB[1]) + fabsf(sc.fwB[2])) * rmax;
  const float reach = sc.Rp * 1.0001f + 2.0f * sc.dt * vb;
  return d2 > reach * reach;
}

// INELASTIC: the launch set holds a scene with plasticity or viscosity (the
// elastic instantiation carries no trace of those paths)
template <bool INELASTIC>
__device__ __forceinline__ void pre_particle(const DevScene &sc, const PPool &P, int p, uint8_t tf, const float x[3],
                                             const float v[3], uint32_t s1, uint32_t s2, float A[9], float J[3],
                                             float wr[6], bool &clamped, bool &anyc) {
  const float dt = sc.dt, mp = sc.mp;
  const int cut = sc.cut;
  J[0] = J[1] = J[2] = 0.f;
  // most particles never touch the blade: D and u_t are read only where the
  // flag says they may be nonzero (both are exactly zero where it is clear)
  const float D0 = tf ? P.D[p] : 0.0f;
  float D = sc.reset_D ? 0.0f : D0;
  const float u00 = tf ? P.ut[0][p] : 0.0f, u01 = tf ? P.ut[1][p] : 0.0f, u02 = tf ? P.ut[2][p] : 0.0f;
  float uh[3] = {u00, u01, u02};
  if (sc.has_blade && sc.tool_contact_on && blade_out_of_reach(sc, x, v)) {
    uh[0] = uh[1] = uh[2] = 0.0f;  // as on the no-contact branch below
  } else if (sc.has_blade && sc.tool_contact_on) {
    float xc[3], nB[3], phi;
    box_closest(sc, x, sc.Rp, xc, nB, phi);
    float rc[3] = {xc[0] - sc.fxB[0], xc[1] - sc.fxB[1], xc[2] - sc.fxB[2]};
    float wr3[3] = {sc.fwB[1] * rc[2] - sc.fwB[2] * rc[1], sc.fwB[2] * rc[0] - sc.fwB[0] * rc[2],
                    sc.fwB[0] * rc[1] - sc.fwB[1] * rc[0]};
    float vrel[3] = {v[0] - (sc.fvB[0] + wr3[0]), v[1] - (sc.fvB[1] + wr3[1]), v[2] - (sc.fvB[2] + wr3[2])};
    float vn = vrel[0] * nB[0] + vrel[1] * nB[1] + vrel[2] * nB[2];
    float phihat = phi + dt * fminf(vn, 0.0f);
    // no predicted overlap: J_n = 0 below, and the impulse, reaction and
    // friction history come out as on the no-contact branch
    if (!(phihat < 0.0f)) {
      uh[0] = uh[1] = uh[2] = 0.0f;
      goto contact_done;
    }
    {
    float wB = 0.0f;
    if (sc.finv_mass > 0.0f) {
      float rn[3] = {rc[1] * nB[2] - rc[2] * nB[1], rc[2] * nB[0] - rc[0] * nB[2], rc[0] * nB[1] - rc[1] * nB[0]};
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
        float uc = (sc.fve[0] - v[0]) * sc.fd[0] + (sc.fve[1] - v[1]) * sc.fd[1] + (sc.fve[2] - v[2]) * sc.fd[2];
        bool front = fabsf(sp) <= sc.h && fabsf(lp) <= sc.fL && fp >= 0.0f && fp <= sc.b_lead && uc > sc.u_min;
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
    const float idt = 1.0f / dt;
    const float FB[3] = {-JB[0] * idt, -JB[1] * idt, -JB[2] * idt};
    anyc |= Jn > 0.0f;
    wr[0] += FB[0];
    wr[1] += FB[1];
    wr[2] += FB[2];
    wr[3] += rc[1] * FB[2] - rc[2] * FB[1];
    wr[4] += rc[2] * FB[0] - rc[0] * FB[2];
    wr[5] += rc[0] * FB[1] - rc[1] * FB[0];
    J[0] += JB[0];
    J[1] += JB[1];
    J[2] += JB[2];
    }
  contact_done:;
  }
  if (sc.floor_on) {
    const float phi = x[2] - sc.floor_z - sc.Rp;
    const float phihat = phi + dt * fminf(v[2], 0.0f);
    J[2] += sc.s_n * mp / dt * fmaxf(-phihat, 0.0f);
  }
  if (sc.pair_on) {
    J[0] += P.J[0][p];
    J[1] += P.J[1][p];
    J[2] += P.J[2][p];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) J[a] += mp * sc.g[a] * dt;
  uint8_t pend = 0;
  if (cut >= 0 && ((s1 | s2) & (1u << cut)) == 0u) pend = (uint8_t)side_label(sc, x, v);
  float F[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) F[k] = P.F[k][p];
  float Pk[9];
  if (INELASTIC && (sc.yield_stress > 0.0f || sc.viscosity > 0.0f))
    clamped |= inelastic_stress(sc, P, p, F, Pk);
  else
    clamped |= sc.model == BM_MODEL_FIXED_COROTATED ? piola_fcr(F, sc.mu, sc.lam, Pk) : piola(F, sc.mu, sc.lam, Pk);
  const float cA = -dt * sc.V0 * sc.inv_dx;  // grad N is applied per axis in units of 1/dx
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = cA * Pk[k];
  // cutting progress and friction history are written back only when they
  // change (most particles touch no tool in a substep)
  if (!(D == D0)) P.D[p] = D;
  if (!(uh[0] == u00 && uh[1] == u01 && uh[2] == u02)) {
    P.ut[0][p] = uh[0];
    P.ut[1][p] = uh[1];
    P.ut[2][p] = uh[2];
  }
  // cleared only when the values in memory are zero: a value equal to zero
  // (either sign) was either written above or already held as zero
  const uint8_t nf = (D != 0.0f || uh[0] != 0.0f || uh[1] != 0.0f || uh[2] != 0.0f) ? 1 : 0;
  if (nf != tf) P.tflag[p] = nf;
  P.pend[p] = pend;
}

// Per-brick wrench partial of this substep: float32 sums inside the brick
// (fixed shuffle tree, warps in order), one double per component; bricks
// without tool contact write zeros.  All threads of the CTA call it.
__device__ __forceinline__ void brick_wrench(const World &w, int brick, const float wr[6], bool anyc,
                                             float (*red)[BT / 32]) {
  const int tid = threadIdx.x;
  if (__syncthreads_or(anyc)) {
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float v = wr[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
      if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (tid < 6) {
      double s = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += (double)red[tid][q];
      w.wpart[(size_t)brick * 6 + tid] = s;
    }
  } else if (tid < 6) {
    w.wpart[(size_t)brick * 6 + tid] = 0.0;
  }
}

// --------------------------------------------------------------------------
// k_p2g_brick: the brick's share of P2G (Eq. 2) into its node tile, per
// logical grid, from the particles' A, J, v staged in shared memory.
// --------------------------------------------------------------------------
// Reduction of per-(cell, z-offset) sums to per-node sums inside a warp.
// Cells are x-fastest in a brick and a warp holds 32 consecutive cells of one
// z-offset, so the 4 cells of an x-row are adjacent lanes and the 4 rows of a
// z-layer are 4 lanes apart.  On entry a[i][j][k] is value k of the thread's
// own cell for node (cx + j, cy + i, cz + oz).  The x pass adds, for node
// cx, the contributions of cells cx - 1 and cx - 2 (shuffles); the lane at
// the row's end also keeps the row's sums for the two node columns beyond it
// (nodes 4 and 5 of the tile's 6).  The y pass does the same along y.  On
// exit lane (cx, cy) holds, for its z-layer, the sums over the layer's cells
// of nodes (tx, ty) = (cx + j, cy + i), with j > 0 only at cx = 3 and i > 0
// only at cy = 3 (zeros elsewhere).  Each sum is taken in a fixed order (own
// cell, then the one before, then the one before that).
template <int NV>
__device__ __forceinline__ void xy_reduce(float (&a)[3][3][NV], int cx, int cy) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float t1 = __shfl_up_sync(FULL, a[i][1][k], 1);
      const float t2 = __shfl_up_sync(FULL, a[i][2][k], 2);
      const float t3 = __shfl_up_sync(FULL, a[i][2][k], 1);
      float sum = a[i][0][k];
      if (cx >= 1) sum += t1;
      if (cx >= 2) sum += t2;
      a[i][0][k] = sum;
      a[i][1][k] = cx == 3 ? a[i][1][k] + t3 : 0.f;
      a[i][2][k] = cx == 3 ? a[i][2][k] : 0.f;
    }
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float t1 = __shfl_up_sync(FULL, a[1][j][k], 4);
      const float t2 = __shfl_up_sync(FULL, a[2][j][k], 8);
      const float t3 = __shfl_up_sync(FULL, a[2][j][k], 4);
      float sum = a[0][j][k];
      if (cy >= 1) sum += t1;
      if (cy >= 2) sum += t2;
      a[0][j][k] = sum;
      a[1][j][k] = cy == 3 ? a[1][j][k] + t3 : 0.f;
      a[2][j][k] = cy == 3 ? a[2][j][k] : 0.f;
    }
}

// The layer sums of xy_reduce into the z stage, value k of tile node (tx,
// ty, cz + oz) from the cells of z-layer cz: with ZN = TN at sz[k][oz][t] (t
// the tile node), with ZN = TZ at sz[k][oz][(cz * TE + ty) * TE + tx] (a
// z-offset reaches 4 of the tile's 6 node layers, so each offset keeps
// 4 x 36 entries; the compact stage lets P2G run 4 CTAs per SM).  Each (node,
// oz) entry that the tile gather reads has exactly one writer.
#define TZ (BR * TE * TE)
template <int NV, int ZN>
__device__ __forceinline__ void stage_layer(float (*sz)[3][ZN], const float (&a)[3][3][NV], int cx, int cy,
                                            int cz, int oz) {
  const int lz = ZN == TN ? cz + oz : cz;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if ((i > 0 && cy != 3) || (j > 0 && cx != 3)) continue;
      const int e = (lz * TE + cy + i) * TE + cx + j;
#pragma unroll
      for (int k = 0; k < NV; ++k) sz[k][oz][e] = a[i][j][k];
    }
}

// Sums of tile node t over the z-offsets of the z stage (<= 3 terms, in
// ascending offset order); in the compact stage offset o holds node t at
// entry t - o * 36.
template <int NV, int ZN>
__device__ __forceinline__ void gather_z(const float (*sz)[3][ZN], int t, float (&acc)[NV]) {
  const int tz = t / (TE * TE);
  const int o0 = max(0, tz - (BR - 1)), o1 = min(2, tz);
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.f;
  for (int o = o0; o <= o1; ++o)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += sz[k][o][ZN == TN ? t : t - o * TE * TE];
}

#define BM_BRICK_CODES 64  // distinct codes kept per brick (more raise the slot-overflow flag)

// Distinct codes of the brick's particles (one warp, lane L holding cells 2L
// and 2L + 1): the next code not yet listed is taken from the lowest lane
// that has one, so the list is in first-occurrence order over the cells.
template <int PPC>
__device__ void brick_codes(const uint32_t *ps1, const uint32_t *ps2, const uint8_t (*ccode)[PPC],
                            const uint8_t *ncode, uint2 *bcode, int *nbcode, unsigned int *err) {
  const int lane = threadIdx.x & 31;
  const int c0 = 2 * lane;
  const int tot = ncode[c0] + ncode[c0 + 1];
  int cur = 0, n = 0;
  auto code_of = [&](int q, uint32_t &a, uint32_t &b) {
    const int c = q < ncode[c0] ? c0 : c0 + 1;
    const int j = ccode[c][q < ncode[c0] ? q : q - ncode[c0]];
    const int k = pic(j, c);
    a = ps1[k];
    b = ps2[k];
  };
  for (;;) {
    // advance past candidates already listed
    uint32_t a = 0, b = 0;
    while (cur < tot) {
      code_of(cur, a, b);
      bool seen = false;
      for (int q = 0; q < n; ++q)
        if (bcode[q].x == a && bcode[q].y == b) {
          seen = true;
          break;
        }
      if (!seen) break;
      ++cur;
    }
    const unsigned pend = __ballot_sync(FULL, cur < tot);
    if (!pend) break;
    const int src = __ffs(pend) - 1;
    const uint32_t ka = __shfl_sync(FULL, a, src), kb = __shfl_sync(FULL, b, src);
    if (n < BM_BRICK_CODES) {
      if (lane == 0) bcode[n] = make_uint2(ka, kb);
      __syncwarp();
    } else if (lane == 0) {
      atomicOr(err, BM_ERRBIT_SLOT_OVERFLOW);
    }
    ++n;
    if (n > BM_BRICK_CODES) break;
  }
  if (lane == 0) *nbcode = min(n, BM_BRICK_CODES);
}

template <int PPC>
struct K2S {
  Tile T;
  float part[18][PPC * BR3];   // the brick's particles (fx, v, A, J), [particle-in-cell][cell]
  float sz[7][3][TZ];          // one pass's (node, z-offset) sums
  uint32_t ps1[PPC * BR3], ps2[PPC * BR3];
  uint2 bcode[BM_BRICK_CODES]; // distinct codes of the brick's particles
  float red[6][BT / 32];       // wrench partials of the warps
  uint8_t ccode[BR3][PPC];  // distinct codes of each cell: particle-in-cell index of the
                            // first particle with each code (first-occurrence order)
  uint8_t ncode[BR3];
  int cs[BR3 + 1];
  int maxcodes;
  int nbcode;
};

// The brick's particles into shared memory, transposed to
// [particle-in-cell][cell] so that the (cell, z-offset) threads read
// consecutive words: the fractional offset, v, and the P2G inputs A and J
// that pre_particle computes from x, v, F, D, u_t and the codes.  The caller
// provides the barrier that publishes it.
template <int PPC, bool INELASTIC>
__device__ void stage_particles(const World &w, const DevScene &sc, const int4 &bt, int c0x, int c0y, int c0z,
                                K2S<PPC> &S, float wr[6], bool &clamped, bool &anyc) {
  const PPool &P = w.P;
  // each thread fetches its next particle's flag one iteration ahead, so the
  // loads of D and u_t it gates do not wait on it
  uint8_t tf_next = (int)threadIdx.x < bt.w ? P.tflag[bt.z + threadIdx.x] : 0;
  for (int i = threadIdx.x; i < bt.w; i += blockDim.x) {
    const int p = bt.z + i;
    const uint8_t tf = tf_next;
    if (i + (int)blockDim.x < bt.w) tf_next = P.tflag[p + blockDim.x];
    const float x[3] = {P.x[0][p], P.x[1][p], P.x[2][p]};
    const float v[3] = {P.v[0][p], P.v[1][p], P.v[2][p]};
    const uint32_t s1 = P.s1[p], s2 = P.s2[p];
    const float f0 = P.fx[0][p], f1 = P.fx[1][p], f2 = P.fx[2][p];
    float A[9], J[3];
    pre_particle<INELASTIC>(sc, P, p, tf, x, v, s1, s2, A, J, wr, clamped, anyc);
    const int c = cell_of(S.cs, i);
    const int si = pic(i - S.cs[c], c);
    S.part[0][si] = f0;
    S.part[1][si] = f1;
    S.part[2][si] = f2;
    S.part[3][si] = v[0];
    S.part[4][si] = v[1];
    S.part[5][si] = v[2];
#pragma unroll
    for (int k = 0; k < 9; ++k) S.part[6 + k][si] = A[k];
    S.part[15][si] = J[0];
    S.part[16][si] = J[1];
    S.part[17][si] = J[2];
    S.ps1[si] = s1;
    S.ps2[si] = s2;
  }
}

// distinct codes of each cell, once per cell (threads of z-offset 0), from
// the [particle-in-cell][cell] staging of the codes: each code is kept as the
// particle-in-cell index of its first particle.
template <int PPC>
__device__ __forceinline__ void cell_codes(const uint32_t *s1, const uint32_t *s2, const int *cs,
                                           uint8_t (*ccode)[PPC], uint8_t *ncode, int *maxcodes) {
  const int c = threadIdx.x;
  if (c >= BR3) return;
  const int n = cs[c + 1] - cs[c];
  int cnt = 0;
  for (int j = 0; j < n; ++j) {
    const int k = pic(j, c);
    const uint32_t a = s1[k], b = s2[k];
    bool seen = false;
    for (int q = 0; q < cnt; ++q) {
      const int kq = pic(ccode[c][q], c);
      if (s1[kq] == a && s2[kq] == b) {
        seen = true;
        break;
      }
    }
    if (!seen) ccode[c][cnt++] = (uint8_t)j;
  }
  ncode[c] = (uint8_t)cnt;
  atomicMax(maxcodes, cnt);
}

// Whether cell c holds particles with code (k1, k2), and whether they are
// all of the cell's particles.
template <int PPC>
__device__ __forceinline__ bool cell_has_code(const uint32_t *ps1, const uint32_t *ps2,
                                              const uint8_t (*ccode)[PPC], const uint8_t *ncode, int c,
                                              uint32_t k1, uint32_t k2) {
  for (int q = 0; q < ncode[c]; ++q) {
    const int k = pic(ccode[c][q], c);
    if (ps1[k] == k1 && ps2[k] == k2) return true;
  }
  return false;
}

// Tile slot of node t holding code (k1, k2) as an index into the node's
// slots, or -1; `uniform`: one code in the brick and one slot per node.
// tcodes: the tile's slot codes in shared memory (by tile slot), or null to
// read them from the slot pool.
__device__ __forceinline__ uint2 tile_code(const World &w, const Tile &T, const uint2 *tcodes, int t, int a) {
  return tcodes ? tcodes[T.lo[t] + a] : w.S.code[T.goff[t] + a];
}

__device__ __forceinline__ int node_slot_of(const World &w, const Tile &T, const uint2 *tcodes, int t,
                                            bool uniform, uint32_t k1, uint32_t k2) {
  const int n = T.cnt[t];
  if (uniform) return n > 0 ? 0 : -1;
  for (int a = 0; a < n; ++a) {
    const uint2 c = tile_code(w, T, tcodes, t, a);
    if (c.x == k1 && c.y == k2) return a;
  }
  return -1;
}

// In the first pass over a multi-code brick, the tile slots whose code no
// particle of the brick carries get zero partial sums (every other slot is
// written by the pass of its code).
__device__ __forceinline__ bool code_listed(const uint2 *bcode, int n, uint2 c) {
  for (int q = 0; q < n; ++q)
    if (bcode[q].x == c.x && bcode[q].y == c.y) return true;
  return false;
}

template <int PPC, int MB, bool INELASTIC>
__global__ void __launch_bounds__(BT, MB) k_p2g_brick(World w, LaunchSet ls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  K2S<PPC> &S = *reinterpret_cast<K2S<PPC> *>(smraw);
  const int4 bt = ls.btiles[blockIdx.x];  // scene, pool brick, first particle, count
  DevScene &scm = w.scenes[bt.x];
  const DevScene &sc = scm;
  if (sc.frozen) return;
  const int tid = threadIdx.x;
  const int lb = bt.y - sc.brick_begin;
  int c0x, c0y, c0z;
  brick_coords(sc, lb, c0x, c0y, c0z);
  const int *csg = w.N.cell_start + sc.cell_begin + lb * BR3;
  for (int i = tid; i <= BR3; i += BT) S.cs[i] = csg[i] - bt.z;
  if (tid == 0) S.maxcodes = 0;
  __syncthreads();
  // the particles (with contact, labels and stress) and the tile descriptors
  // load together
  float wr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  bool clamped = false, anyc = false;
  stage_particles<PPC, INELASTIC>(w, sc, bt, c0x, c0y, c0z, S, wr, clamped, anyc);
  if (clamped) atomicOr(&scm.err, BM_ERRBIT_INVERTED);
  const bool single = tile_load(w, sc, bt.y, c0x, c0y, c0z, S.T);
  if (sc.has_blade) brick_wrench(w, bt.y, wr, anyc, S.red);  // (its barriers publish the copy too)
  cell_codes<PPC>(S.ps1, S.ps2, S.cs, S.ccode, S.ncode, &S.maxcodes);
  __syncthreads();
  // every tile node holds one logical grid (so all the brick's particles
  // share one code): one pass, no code tests
  const bool uniform = single && S.maxcodes <= 1;
  if (!uniform) {
    if (tid < 32) brick_codes<PPC>(S.ps1, S.ps2, S.ccode, S.ncode, S.bcode, &S.nbcode, &scm.err);
    __syncthreads();
  }
  // a brick without particles still runs one pass: it writes zeros to its tile
  const int nbc = uniform ? 1 : S.nbcode;
  const int npass = max(nbc, 1);

  // ---- one pass per code of the brick ----
  // Each thread sums, for its cell and one z-offset, m N, m v N and
  // A grad N + N J over the cell's particles with the pass's code; the warp
  // reduces the sums along x and y (xy_reduce), the z stage collects the
  // layers, and each tile node adds its <= 3 layer sums and writes the slot
  // of the pass's code.  Every float sum has one owner: no atomics, and each
  // partial-sum entry is written exactly once.
  const int c = tid % BR3, oz = tid / BR3;
  const int cx = c & 3, cy = (c >> 2) & 3, cz = c >> 4;
  const int n_c = S.cs[c + 1] - S.cs[c];
  const int pbase = w.B.poff[bt.y];  // this brick's partial-sum range (negative: pool overflow)
  for (int b = 0; b < npass; ++b) {
    const bool coded = b < nbc;  // false only in the single pass of a brick without particles
    const uint32_t k1 = (uniform || !coded) ? 0u : S.bcode[b].x, k2 = (uniform || !coded) ? 0u : S.bcode[b].y;
    const bool has = coded && n_c > 0 &&
                     (uniform || cell_has_code<PPC>(S.ps1, S.ps2, S.ccode, S.ncode, c, k1, k2));
    const bool filt = !uniform && S.ncode[c] > 1;
    // two walks over the cell's particles, each reducing its own values, so
    // that fewer sums are live at once: (m N, m v N), then A grad N + N J
    {
      float a[3][3][4];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int f = 0; f < 4; ++f) a[i][j][f] = 0.f;
      if (has) {
        for (int j = 0; j < n_c; ++j) {
          const int si = pic(j, c);
          if (filt && (S.ps1[si] != k1 || S.ps2[si] != k2)) continue;
          float wx[3], wy[3], wz, d;
          const float f0 = S.part[0][si], f1 = S.part[1][si], f2 = S.part[2][si];
          bs<0>(f0, wx[0], d); bs<1>(f0, wx[1], d); bs<2>(f0, wx[2], d);
          bs<0>(f1, wy[0], d); bs<1>(f1, wy[1], d); bs<2>(f1, wy[2], d);
          bs_rt(oz, f2, wz, d);
          const float v0 = S.part[3][si], v1 = S.part[4][si], v2 = S.part[5][si];
#pragma unroll
          for (int oy = 0; oy < 3; ++oy) {
            const float wyz = wy[oy] * wz;
            const float M0 = v0 * wyz, M1 = v1 * wyz, M2 = v2 * wyz;
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
              float *q = a[oy][ox];
              const float wxx = wx[ox];
              q[0] += wxx * wyz;
              q[1] += wxx * M0;
              q[2] += wxx * M1;
              q[3] += wxx * M2;
            }
          }
        }
      }
      xy_reduce<4>(a, cx, cy);
      stage_layer<4, TZ>(S.sz, a, cx, cy, cz, oz);
    }
    {
      float a[3][3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int f = 0; f < 3; ++f) a[i][j][f] = 0.f;
      if (has) {
        for (int j = 0; j < n_c; ++j) {
          const int si = pic(j, c);
          if (filt && (S.ps1[si] != k1 || S.ps2[si] != k2)) continue;
          float wx[3], dwx[3], wy[3], dwy[3], wz, dwz;
          const float f0 = S.part[0][si], f1 = S.part[1][si], f2 = S.part[2][si];
          bs<0>(f0, wx[0], dwx[0]); bs<1>(f0, wx[1], dwx[1]); bs<2>(f0, wx[2], dwx[2]);
          bs<0>(f1, wy[0], dwy[0]); bs<1>(f1, wy[1], dwy[1]); bs<2>(f1, wy[2], dwy[2]);
          bs_rt(oz, f2, wz, dwz);
          float A[9];
#pragma unroll
          for (int k = 0; k < 9; ++k) A[k] = S.part[6 + k][si];
          const float J0 = S.part[15][si], J1 = S.part[16][si], J2 = S.part[17][si];
#pragma unroll
          for (int oy = 0; oy < 3; ++oy) {
            // with N = wx wyz and grad N = (dwx wyz, wx dyz, wx wyd):
            // A grad N + N J = wx (A_:1 dyz + A_:2 wyd + J wyz) + dwx (A_:0 wyz)
            const float wyz = wy[oy] * wz, dyz = dwy[oy] * wz, wyd = wy[oy] * dwz;
            const float U0 = A[1] * dyz + A[2] * wyd + J0 * wyz;
            const float U1 = A[4] * dyz + A[5] * wyd + J1 * wyz;
            const float U2 = A[7] * dyz + A[8] * wyd + J2 * wyz;
            const float V0 = A[0] * wyz, V1 = A[3] * wyz, V2 = A[6] * wyz;
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
              float *q = a[oy][ox];
              const float wxx = wx[ox], dxx = dwx[ox];
              q[0] += wxx * U0 + dxx * V0;
              q[1] += wxx * U1 + dxx * V1;
              q[2] += wxx * U2 + dxx * V2;
            }
          }
        }
      }
      xy_reduce<3>(a, cx, cy);
      stage_layer<3, TZ>(S.sz + 4, a, cx, cy, cz, oz);
    }
    __syncthreads();
    if (pbase >= 0) {
      for (int t = tid; t < TN; t += BT) {
        const int n = S.T.cnt[t];
        if (n == 0) continue;
        const size_t e0 = (size_t)pbase + S.T.lo[t];
        if (b == 0 && !uniform)
          for (int q = 0; q < n; ++q)
            if (!code_listed(S.bcode, S.nbcode, tile_code(w, S.T, nullptr, t, q))) {
              w.B.pm[e0 + q] = make_float4(0.f, 0.f, 0.f, 0.f);
              w.B.pd[e0 + q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        const int sl = coded ? node_slot_of(w, S.T, nullptr, t, uniform, k1, k2) : -1;
        if (sl < 0) continue;
        float acc[7];
        gather_z<7, TZ>(S.sz, t, acc);
        w.B.pm[e0 + sl] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        w.B.pd[e0 + sl] = make_float4(acc[4], acc[5], acc[6], 0.f);
      }
    }
    if (b + 1 < npass) __syncthreads();  // the next pass overwrites the z stage
  }
}

// bricks whose tiles hold node coordinate i along one axis: [first, last]
__device__ __forceinline__ void covering(int i, int nbr, int &first, int &last) {
  last = min(i >> 2, nbr - 1);
  first = max((i - (TE - 1) + (BR - 1)) >> 2, 0);
  if (i - (TE - 1) < 0) first = 0;
}

// First partial-sum entry of a node in each of the (up to 8) brick tiles that
// cover it, in brick order (k = dz*4 + dy*2 + dx over the covering bricks'
// offsets); -1 where no brick or where the brick's partials overflowed.  All
// loads of the eight candidates are issued together.
__device__ __forceinline__ void covering_entries(const World &w, const DevScene &sc, int ix, int iy, int iz,
                                                 long long e[8]) {
  int x0, x1, y0, y1, z0, z1;
  covering(ix, sc.nbr[0], x0, x1);
  covering(iy, sc.nbr[1], y0, y1);
  covering(iz, sc.nbr[2], z0, z1);
  int b[8], tt[8], pb[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int Bx = x0 + (k & 1), By = y0 + ((k >> 1) & 1), Bz = z0 + (k >> 2);
    const bool ok = Bx <= x1 && By <= y1 && Bz <= z1;
    b[k] = ok ? sc.brick_begin + (Bz * sc.nbr[1] + By) * sc.nbr[0] + Bx : -1;
    tt[k] = ((iz - Bz * BR) * TE + (iy - By * BR)) * TE + (ix - Bx * BR);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) pb[k] = b[k] >= 0 ? w.B.poff[b[k]] : -1;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    e[k] = pb[k] >= 0 ? (long long)pb[k] + (w.B.tdesc[(size_t)b[k] * TN + tt[k]] & 0xffff) : -1;
}

// --------------------------------------------------------------------------
// k_p2g_node: per node, sum the tile partials of the bricks covering it (in
// brick order), couple compatible logical grids (Eq. 8), grid update (Eq. 9)
// --------------------------------------------------------------------------
__global__ void k_p2g_node(World w, LaunchSet ls) {
  const int4 t = ls.ntiles[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= t.z) return;
  const DevScene &sc = w.scenes[t.x];
  if (sc.frozen) return;
  const int node = t.y + i;
  const int ns = w.N.slot_cnt[node];
  if (ns == 0) return;
  const int off = w.N.slot_off[node];
  int ix, iy, iz;
  node_coords(sc, node - sc.node_begin, ix, iy, iz);
  long long ent[8];
  covering_entries(w, sc, ix, iy, iz, ent);
  if (ns == 1) {
    float4 sm = make_float4(0.f, 0.f, 0.f, 0.f), sd = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a[k] = ent[k] >= 0 ? w.B.pm[ent[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
      d[k] = ent[k] >= 0 ? w.B.pd[ent[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (ent[k] < 0) continue;
      sm.x += a[k].x; sm.y += a[k].y; sm.z += a[k].z; sm.w += a[k].w;
      sd.x += d[k].x; sd.y += d[k].y; sd.z += d[k].z;
    }
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f), nw = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sm.x > 0.f) {
      const float im = 1.0f / sm.x, imm = 1.0f / (sc.mp * sm.x);
      o = make_float4(sm.y * im, sm.z * im, sm.w * im, sc.mp * sm.x);
      nw = make_float4(o.x + sd.x * imm, o.y + sd.y * imm, o.z + sd.z * imm, 0.f);
    }
    w.S.vold[off] = o;
    w.S.vnew[off] = nw;
    return;
  }
  uint2 codes[BM_MAXS];
  float m[BM_MAXS];
  float S[BM_MAXS][6];
  for (int a = 0; a < ns; ++a) {
    codes[a] = w.S.code[off + a];
    m[a] = 0.f;
    for (int c = 0; c < 6; ++c) S[a][c] = 0.f;
  }
  for (int k = 0; k < 8; ++k) {
    if (ent[k] < 0) continue;
    const size_t e = (size_t)ent[k];
    for (int a = 0; a < ns; ++a) {
      const float4 q = w.B.pm[e + a];
      const float4 d = w.B.pd[e + a];
      m[a] += q.x;
      S[a][0] += q.y; S[a][1] += q.z; S[a][2] += q.w;
      S[a][3] += d.x; S[a][4] += d.y; S[a][5] += d.z;
    }
  }
  for (int a = 0; a < ns; ++a) {
    m[a] *= sc.mp;
    for (int c = 0; c < 3; ++c) S[a][c] *= sc.mp;
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

// --------------------------------------------------------------------------
// k_g2p_musl: per particle G2P (Eq. 17) and x update from the brick's tile of
// grid velocities, then the brick's share of the MUSL re-scatter sum m v^{n+1}
// N per logical grid, committed in the same fixed phase order as P2G.
// --------------------------------------------------------------------------
template <int PPC>
struct K4S {
  Tile T;
  uint2 codes[TSCAP];
  union {
    struct {
      float4 tvo[TSCAP];      // v_old xyz, m of the tile slots (G2P)
      float4 tvn[TSCAP];      // v_new xyz
    };
    float sz[3][3][TN];       // then: one MUSL pass's (node, z-offset) sums
  };
  float pf[3][PPC * BR3];
  float pv[3][PPC * BR3];
  uint32_t ps1[PPC * BR3], ps2[PPC * BR3];
  uint2 bcode[BM_BRICK_CODES];  // as in K2S
  uint8_t ccode[BR3][PPC];
  uint8_t ncode[BR3];
  int cs[BR3 + 1];
  int maxcodes;
  int nbcode;
};

template <int PPC, int MB>
__global__ void __launch_bounds__(BT, MB) k_g2p_musl(World w, LaunchSet ls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  K4S<PPC> &S = *reinterpret_cast<K4S<PPC> *>(smraw);
  const int4 bt = ls.btiles[blockIdx.x];
  DevScene &scm = w.scenes[bt.x];
  const DevScene &sc = scm;
  if (sc.frozen) return;
  const PPool &P = w.P;
  const int tid = threadIdx.x;
  const int lb = bt.y - sc.brick_begin;
  int c0x, c0y, c0z;
  brick_coords(sc, lb, c0x, c0y, c0z);
  const int *csg = w.N.cell_start + sc.cell_begin + lb * BR3;
  for (int i = tid; i <= BR3; i += BT) S.cs[i] = csg[i] - bt.z;
  if (tid == 0) S.maxcodes = 0;
  const bool single = tile_load(w, sc, bt.y, c0x, c0y, c0z, S.T);
  const int total = S.T.total;
  const bool in_smem = total <= TSCAP;  // otherwise G2P reads the pool slots directly
  const uint2 *tcodes = in_smem ? S.codes : nullptr;
  if (single) {  // by node: a particle's node t holds its (only) logical grid
    for (int t = tid; t < TN; t += BT) {
      const bool has = S.T.cnt[t] != 0;
      const int g = S.T.goff[t];
      S.tvo[t] = has ? w.S.vold[g] : make_float4(0.f, 0.f, 0.f, 0.f);
      S.tvn[t] = has ? w.S.vnew[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else if (in_smem) {
    for (int t = tid; t < TN; t += BT) {
      const int n = S.T.cnt[t], lo = S.T.lo[t], g = S.T.goff[t];
      for (int a = 0; a < n; ++a) {
        S.codes[lo + a] = w.S.code[g + a];  // every slot: the MUSL passes look codes up by slot
        S.tvo[lo + a] = w.S.vold[g + a];
        S.tvn[lo + a] = w.S.vnew[g + a];
      }
    }
  }
  __syncthreads();
  // ---- phase 0: G2P ----
  const float beta = sc.beta, dt = sc.dt;
  bool bad = false;
  for (int i = tid; i < bt.w; i += BT) {
    const int p = bt.z + i;
    const int c = cell_of(S.cs, i);
    const int lx = c & 3, ly = (c >> 2) & 3, lz = c >> 4;
    const int si = pic(i - S.cs[c], c);
    const uint32_t s1 = P.s1[p], s2 = P.s2[p];
    const float f0 = P.fx[0][p], f1 = P.fx[1][p], f2 = P.fx[2][p];
    float wx[3], wy[3], wz[3], d;
    bs<0>(f0, wx[0], d); bs<1>(f0, wx[1], d); bs<2>(f0, wx[2], d);
    bs<0>(f1, wy[0], d); bs<1>(f1, wy[1], d); bs<2>(f1, wy[2], d);
    bs<0>(f2, wz[0], d); bs<1>(f2, wz[1], d); bs<2>(f2, wz[2], d);
    float sn[3] = {0.f, 0.f, 0.f}, so[3] = {0.f, 0.f, 0.f};
    if (single) {
      // one logical grid per node, values by node; a node without mass holds
      // zero velocities, so it needs no test
      const int t0 = (lz * TE + ly) * TE + lx;
#pragma unroll
      for (int oz = 0; oz < 3; ++oz)
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
          const float wyz = wy[oy] * wz[oz];
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) {
            const int t = t0 + (oz * TE + oy) * TE + ox;
            const float4 vo = S.tvo[t], vn = S.tvn[t];
            const float N = wx[ox] * wyz;
            sn[0] += N * vn.x;
            sn[1] += N * vn.y;
            sn[2] += N * vn.z;
            so[0] += N * vo.x;
            so[1] += N * vo.y;
            so[2] += N * vo.z;
          }
        }
    } else if (in_smem) {
      // tile slots in shared memory: branch-free over the stencil (a missing
      // or massless logical grid contributes zero)
      const int t0 = (lz * TE + ly) * TE + lx;
#pragma unroll
      for (int oz = 0; oz < 3; ++oz)
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
          const float wyz = wy[oy] * wz[oz];
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) {
            const int s = tile_slot(w, S.T, tcodes, t0 + (oz * TE + oy) * TE + ox, s1, s2);
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 vo = s >= 0 ? S.tvo[s] : zero, vn = s >= 0 ? S.tvn[s] : zero;
            const float N = vo.w > 0.f ? wx[ox] * wyz : 0.f;
            sn[0] += N * vn.x;
            sn[1] += N * vn.y;
            sn[2] += N * vn.z;
            so[0] += N * vo.x;
            so[1] += N * vo.y;
            so[2] += N * vo.z;
          }
        }
    } else
#pragma unroll
    for (int oz = 0; oz < 3; ++oz)
#pragma unroll
      for (int oy = 0; oy < 3; ++oy)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
          const int t = ((lz + oz) * TE + (ly + oy)) * TE + (lx + ox);
          const int s = tile_slot(w, S.T, tcodes, t, s1, s2);
          if (s < 0) continue;
          float4 vo, vn;
          {
            const int g = S.T.goff[t] + s - S.T.lo[t];
            vo = w.S.vold[g];
            vn = w.S.vnew[g];
          }
          if (!(vo.w > 0.f)) continue;
          const float N = wx[ox] * wy[oy] * wz[oz];
          sn[0] += N * vn.x;
          sn[1] += N * vn.y;
          sn[2] += N * vn.z;
          so[0] += N * vo.x;
          so[1] += N * vo.y;
          so[2] += N * vo.z;
        }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float vv = beta * (P.v[a][p] - so[a]) + sn[a];
      const float xx = P.x[a][p] + dt * sn[a];
      P.v[a][p] = vv;
      P.x[a][p] = xx;
      S.pv[a][si] = vv;
      bad |= !isfinite(vv) || !isfinite(xx);
    }
    S.pf[0][si] = f0;
    S.pf[1][si] = f1;
    S.pf[2][si] = f2;
    S.ps1[si] = s1;
    S.ps2[si] = s2;
  }
  if (bad) atomicOr(&scm.err, BM_ERRBIT_NONFINITE);
  // ---- phase 1: MUSL sums m v^{n+1} N, one pass per code of the brick,
  // reduced as in k_p2g_brick (xy_reduce, z stage, <= 3 layer sums per node) ----
  const int c = tid % BR3, oz = tid / BR3;
  const int cx = c & 3, cy = (c >> 2) & 3, cz = c >> 4;
  const int n_c = S.cs[c + 1] - S.cs[c];
  __syncthreads();  // G2P reads of the tile velocities are done: the z stage may reuse them
  cell_codes<PPC>(S.ps1, S.ps2, S.cs, S.ccode, S.ncode, &S.maxcodes);
  __syncthreads();
  const bool uniform = single && S.maxcodes <= 1;
  if (!uniform) {
    if (tid < 32) brick_codes<PPC>(S.ps1, S.ps2, S.ccode, S.ncode, S.bcode, &S.nbcode, &scm.err);
    __syncthreads();
  }
  const int nbc = uniform ? 1 : S.nbcode;
  const int npass = max(nbc, 1);  // a brick without particles writes zeros in one pass
  const int pbase = w.B.poff[bt.y];
  for (int b = 0; b < npass; ++b) {
    const bool coded = b < nbc;
    const uint32_t k1 = (uniform || !coded) ? 0u : S.bcode[b].x, k2 = (uniform || !coded) ? 0u : S.bcode[b].y;
    const bool has = coded && n_c > 0 &&
                     (uniform || cell_has_code<PPC>(S.ps1, S.ps2, S.ccode, S.ncode, c, k1, k2));
    const bool filt = !uniform && S.ncode[c] > 1;
    float a[3][3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) a[i][j][0] = a[i][j][1] = a[i][j][2] = 0.f;
    if (has) {
      for (int j = 0; j < n_c; ++j) {
        const int si = pic(j, c);
        if (filt && (S.ps1[si] != k1 || S.ps2[si] != k2)) continue;
        float wx[3], wy[3], wz, d;
        const float f0 = S.pf[0][si], f1 = S.pf[1][si], f2 = S.pf[2][si];
        bs<0>(f0, wx[0], d); bs<1>(f0, wx[1], d); bs<2>(f0, wx[2], d);
        bs<0>(f1, wy[0], d); bs<1>(f1, wy[1], d); bs<2>(f1, wy[2], d);
        bs_rt(oz, f2, wz, d);
        const float v0 = S.pv[0][si], v1 = S.pv[1][si], v2 = S.pv[2][si];
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
          const float wyz = wy[oy] * wz;
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) {
            const float N = wx[ox] * wyz;
            a[oy][ox][0] += N * v0;
            a[oy][ox][1] += N * v1;
            a[oy][ox][2] += N * v2;
          }
        }
      }
    }
    xy_reduce<3>(a, cx, cy);
    stage_layer<3, TN>(S.sz, a, cx, cy, cz, oz);
    __syncthreads();
    if (pbase >= 0) {
      for (int t = tid; t < TN; t += BT) {
        const int n = S.T.cnt[t];
        if (n == 0) continue;
        const size_t e0 = (size_t)pbase + S.T.lo[t];
        if (b == 0 && !uniform)
          for (int q = 0; q < n; ++q)
            if (!code_listed(S.bcode, S.nbcode, tile_code(w, S.T, tcodes, t, q)))
              w.B.pm[e0 + q] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int sl = coded ? node_slot_of(w, S.T, tcodes, t, uniform, k1, k2) : -1;
        if (sl < 0) continue;
        float acc[3];
        gather_z<3, TN>(S.sz, t, acc);
        w.B.pm[e0 + sl] = make_float4(acc[0], acc[1], acc[2], 0.f);
      }
    }
    if (b + 1 < npass) __syncthreads();  // the next pass overwrites the z stage
  }
}

// --------------------------------------------------------------------------
// k_musl_node: per node, MUSL sums of the covering bricks, coupling, v*
// --------------------------------------------------------------------------
__global__ void k_musl_node(World w, LaunchSet ls) {
  const int4 t = ls.ntiles[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= t.z) return;
  const DevScene &sc = w.scenes[t.x];
  if (sc.frozen) return;
  const int node = t.y + i;
  const int ns = w.N.slot_cnt[node];
  if (ns == 0) return;
  const int off = w.N.slot_off[node];
  int ix, iy, iz;
  node_coords(sc, node - sc.node_begin, ix, iy, iz);
  int x0, x1, y0, y1, z0, z1;
  covering(ix, sc.nbr[0], x0, x1);
  covering(iy, sc.nbr[1], y0, y1);
  covering(iz, sc.nbr[2], z0, z1);
  float S[BM_MAXS][3];
  for (int a = 0; a < ns; ++a) S[a][0] = S[a][1] = S[a][2] = 0.f;
  for (int Bz = z0; Bz <= z1; ++Bz)
    for (int By = y0; By <= y1; ++By)
      for (int Bx = x0; Bx <= x1; ++Bx) {
        const int b = sc.brick_begin + (Bz * sc.nbr[1] + By) * sc.nbr[0] + Bx;
        const int tt = ((iz - Bz * BR) * TE + (iy - By * BR)) * TE + (ix - Bx * BR);
        const int pb = w.B.poff[b];
        if (pb < 0) continue;
        const size_t e = (size_t)pb + (w.B.tdesc[(size_t)b * TN + tt] & 0xffff);
        for (int a = 0; a < ns; ++a) {
          const float4 q = w.B.pm[e + a];
          S[a][0] += q.x;
          S[a][1] += q.y;
          S[a][2] += q.z;
        }
      }
  if (ns == 1) {
    const float m = w.S.vold[off].w;
    float4 vs = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m > 0.f) {
      const float im = sc.mp / m;
      vs = make_float4(S[0][0] * im, S[0][1] * im, S[0][2] * im, 0.f);
    }
    w.S.vstar[off] = vs;
    return;
  }
  uint2 codes[BM_MAXS];
  float mass[BM_MAXS];
  for (int a = 0; a < ns; ++a) {
    codes[a] = w.S.code[off + a];
    mass[a] = w.S.vold[off + a].w;
    for (int c = 0; c < 3; ++c) S[a][c] *= sc.mp;
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
// k_fupd: F += dt sum_i v*_i (x) grad0 N_ip from the brick's tile of v*, and
// commit the side labels assigned this substep (they act from the next one)
// --------------------------------------------------------------------------
struct K1S {
  Tile T;
  uint2 codes[TSCAP];
  float4 tvs[TSCAP];
  int any;
};

template <int MB, bool INELASTIC>
__global__ void __launch_bounds__(BT, MB) k_fupd(World w, LaunchSet ls) {
  __shared__ K1S S;
  const int4 bt = ls.btiles[blockIdx.x];
  DevScene &scm = w.scenes[bt.x];
  const DevScene &sc = scm;
  if (sc.frozen) return;
  const PPool &P = w.P;
  const int tid = threadIdx.x;
  const int lb = bt.y - sc.brick_begin;
  int c0x, c0y, c0z;
  brick_coords(sc, lb, c0x, c0y, c0z);
  if (tid == 0) S.any = 0;
  const bool single = tile_load(w, sc, bt.y, c0x, c0y, c0z, S.T);
  const bool in_smem = S.T.total <= TSCAP;
  const uint2 *tcodes = in_smem ? S.codes : nullptr;
  if (single) {  // by node
    for (int t = tid; t < TN; t += BT)
      S.tvs[t] = S.T.cnt[t] ? w.S.vstar[S.T.goff[t]] : make_float4(0.f, 0.f, 0.f, 0.f);
  } else if (in_smem) {
    for (int t = tid; t < TN; t += BT) {
      const int n = S.T.cnt[t], lo = S.T.lo[t], g = S.T.goff[t];
      for (int a = 0; a < n; ++a) {
        if (n > 1) S.codes[lo + a] = w.S.code[g + a];
        S.tvs[lo + a] = w.S.vstar[g + a];
      }
    }
  }
  __syncthreads();
  const float c = sc.dt * sc.inv_dx;
  const int cut = sc.cut;
  bool any = false;
  for (int i = tid; i < bt.w; i += BT) {
    const int p = bt.z + i;
    int bx, by, bz;
    particle_base(P.base[p], bx, by, bz);
    const int lx = bx - c0x, ly = by - c0y, lz = bz - c0z;
    const uint32_t s1 = P.s1[p], s2 = P.s2[p];
    const float f0 = P.fx[0][p], f1 = P.fx[1][p], f2 = P.fx[2][p];
    float wx[3], wy[3], wz[3], gx[3], gy[3], gz[3];
    bs<0>(f0, wx[0], gx[0]); bs<1>(f0, wx[1], gx[1]); bs<2>(f0, wx[2], gx[2]);
    bs<0>(f1, wy[0], gy[0]); bs<1>(f1, wy[1], gy[1]); bs<2>(f1, wy[2], gy[2]);
    bs<0>(f2, wz[0], gz[0]); bs<1>(f2, wz[1], gz[1]); bs<2>(f2, wz[2], gz[2]);
    float G[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int t0 = (lz * TE + ly) * TE + lx;
#pragma unroll
    for (int oz = 0; oz < 3; ++oz)
#pragma unroll
      for (int oy = 0; oy < 3; ++oy) {
        // grad N = (gx wyz, wx gyz, wx wgz): sum v* gx and v* wx along the
        // row of three nodes first, then scale by the row's y-z factors
        const float wyz = wy[oy] * wz[oz], gyz = gy[oy] * wz[oz], wgz = wy[oy] * gz[oz];
        float sx[3] = {0.f, 0.f, 0.f}, sw[3] = {0.f, 0.f, 0.f};
        if (single) {  // by node; nodes without mass hold v* = 0
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) {
            const float4 v = S.tvs[t0 + (oz * TE + oy) * TE + ox];
            sx[0] += v.x * gx[ox]; sx[1] += v.y * gx[ox]; sx[2] += v.z * gx[ox];
            sw[0] += v.x * wx[ox]; sw[1] += v.y * wx[ox]; sw[2] += v.z * wx[ox];
          }
        } else {
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) {
            const int t = t0 + (oz * TE + oy) * TE + ox;
            const int s = tile_slot(w, S.T, tcodes, t, s1, s2);
            if (s < 0) continue;
            const float4 v = in_smem ? S.tvs[s] : w.S.vstar[S.T.goff[t] + s - S.T.lo[t]];
            sx[0] += v.x * gx[ox]; sx[1] += v.y * gx[ox]; sx[2] += v.z * gx[ox];
            sw[0] += v.x * wx[ox]; sw[1] += v.y * wx[ox]; sw[2] += v.z * wx[ox];
          }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          G[3 * a] += sx[a] * wyz;
          G[3 * a + 1] += sw[a] * gyz;
          G[3 * a + 2] += sw[a] * wgz;
        }
      }
#pragma unroll
    for (int k = 0; k < 9; ++k) P.F[k][p] += c * G[k];
    if (INELASTIC && sc.viscosity > 0.0f)
#pragma unroll
      for (int k = 0; k < 9; ++k) P.Fdot[k][p] = sc.inv_dx * G[k];
    const uint8_t pend = P.pend[p];
    if (pend && cut >= 0) {
      if (pend == 1) P.s1[p] = s1 | (1u << cut);
      else P.s2[p] = s2 | (1u << cut);
      any = true;
      // the nodes of this particle's stencil need their codes recounted
      for (int oz = 0; oz < 3; ++oz)
        for (int oy = 0; oy < 3; ++oy)
          for (int ox = 0; ox < 3; ++ox)
            w.N.dirty[sc.node_begin + ((bz + oz) * sc.nn[1] + (by + oy)) * sc.nn[0] + (bx + ox)] = 1;
    }
  }
  if (any) S.any = 1;
  __syncthreads();
  if (tid == 0 && S.any) atomicOr(&scm.label_pending, 1);
}

// --------------------------------------------------------------------------
// Material-material contact (Eq. 10-13) with per-particle candidate lists.
// Every particle keeps the particles of its scene that were within
// r_l = 2 R_p + skin (skin = 1.5 R_p) at the lists' last build.  A pair in
// contact this substep satisfies dist < 2 R_p + dt (|v_p| + |v_q|) (Eq. 10),
// and a pair missing from the lists was farther than r_l at the build, so
// its distance is at least r_l - d_p - d_q (d: displacement since the
// build).  Hence the lists hold every pair that can touch while every
// particle keeps d_p + dt |v_p| <= skin / 2; they are rebuilt (spatial hash
// of the current configuration, cell = r_l) when one does not, or when the
// state was written from outside.  A list is in (neighbour cell, pool index)
// order, the same alone and in any batch.  A pair is always evaluated in
// canonical (lower, higher) pool-index order by both of its particles, so
// the two impulses are exact negatives; the lower index owns the pair's
// tangential history (double-buffered by substep parity).
// --------------------------------------------------------------------------
__device__ __forceinline__ int hash_cell(int scene, int cx, int cy, int cz, int nb) {
  const unsigned h = ((unsigned)cx * 73856093u) ^ ((unsigned)cy * 19349663u) ^
                     ((unsigned)cz * 83492791u) ^ ((unsigned)scene * 2654435761u);
  return (int)(h & (unsigned)(nb - 1));
}

// scene and hash-cell coordinates in one word (16 bits each, coordinates
// wrapped): equal for the entries of one cell; two cells with equal words
// are at least 65,536 cells apart
__device__ __forceinline__ unsigned long long cell_key(int scene, int cx, int cy, int cz) {
  return ((unsigned long long)(scene & 0xffff) << 48) | ((unsigned long long)(cx & 0xffff) << 32) |
         ((unsigned long long)(cy & 0xffff) << 16) | (unsigned long long)(cz & 0xffff);
}

// per-substep reset of the scenes' reductions and of the world's build flag
__global__ void k_pair_reset(World w, LaunchSet ls) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *w.H.build = 0;
  if (i < ls.n_scenes) {
    DevScene &sc = w.scenes[ls.scene_ids[i]];
    sc.pair_vmax_bits = 0;
    sc.pair_disp_bits = 0;
  }
}

// per scene: largest particle speed, and largest displacement since the
// candidate lists were built (non-negative floats order like their bits)
__global__ void k_pair_vmax(World w, LaunchSet ls) {
  const int4 bt = ls.btiles[blockIdx.x];
  DevScene &sc = w.scenes[bt.x];
  if (!sc.pair_on || sc.frozen) return;
  float m = 0.f, dm = 0.f;
  const bool valid = sc.pair_valid != 0;
  for (int i = threadIdx.x; i < bt.w; i += blockDim.x) {
    const int p = bt.z + i;
    const float a = w.P.v[0][p], b = w.P.v[1][p], c = w.P.v[2][p];
    const float sp = sqrtf(a * a + b * b + c * c);
    m = fmaxf(m, sp);
    if (valid) {
      const float d0 = w.P.x[0][p] - w.P.xb[0][p], d1 = w.P.x[1][p] - w.P.xb[1][p],
                  d2 = w.P.x[2][p] - w.P.xb[2][p];
      dm = fmaxf(dm, sqrtf(d0 * d0 + d1 * d1 + d2 * d2) + sc.dt * sp);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_down_sync(FULL, m, o));
    dm = fmaxf(dm, __shfl_down_sync(FULL, dm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (m > 0.f) atomicMax(&sc.pair_vmax_bits, __float_as_int(m));
    if (dm > 0.f) atomicMax(&sc.pair_disp_bits, __float_as_int(dm));
  }
}

// per scene: whether the candidate lists are rebuilt this substep
__global__ void k_pair_decide(World w, LaunchSet ls) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ls.n_scenes) return;
  DevScene &sc = w.scenes[ls.scene_ids[i]];
  if (!sc.pair_on || sc.frozen) {
    sc.pair_build = 0;
    return;
  }
  const float reach = __int_as_float(sc.pair_disp_bits);  // max of d_p + dt |v_p|
  const float skin = 1.5f * sc.Rp;
  // 10% margin against rounding in the distances
  const bool build = !sc.pair_valid || !(reach <= 0.45f * skin);
  sc.pair_build = build ? 1 : 0;
  if (build) {
    sc.pair_h = 1.001f * (2.0f * sc.Rp + skin);
    sc.pair_inv_h = 1.0f / sc.pair_h;
    sc.pair_valid = 1;
    sc.pair_builds++;
    atomicOr(w.H.build, 1);
  }
}

__global__ void k_pair_hash(World w, LaunchSet ls) {
  const int4 bt = ls.btiles[blockIdx.x];
  const DevScene &sc = w.scenes[bt.x];
  if (!sc.pair_on || !sc.pair_build) return;
  const PPool &P = w.P;
  const float ih = sc.pair_inv_h;
  for (int i = threadIdx.x; i < bt.w; i += blockDim.x) {
    const int p = bt.z + i;
    const int cx = (int)floorf(P.x[0][p] * ih);
    const int cy = (int)floorf(P.x[1][p] * ih);
    const int cz = (int)floorf(P.x[2][p] * ih);
    const int b = hash_cell(bt.x, cx, cy, cz, w.H.n_buckets);
    P.hkey[p] = b;
    P.hcell[p] = cell_key(bt.x, cx, cy, cz);
    atomicAdd(&w.H.bucket_start[b], 1);
  }
}

__global__ void k_scan_local(World w) {
  if (!*w.H.build) return;
  __shared__ int sm[33];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = i < w.H.n_buckets ? w.H.bucket_start[i] : 0;
  int total;
  const int ex = block_excl_scan(v, sm, total);
  if (i < w.H.n_buckets) w.H.bucket_start[i] = ex;
  if (threadIdx.x == 0) w.H.block_sum[blockIdx.x] = total;
}

__global__ void k_scan_top(World w, int nblocks) {
  if (!*w.H.build) return;
  __shared__ int sm[33];
  int carry = 0;
  for (int base = 0; base < nblocks; base += blockDim.x) {
    const int j = base + threadIdx.x;
    const int v = j < nblocks ? w.H.block_sum[j] : 0;
    int total;
    const int ex = block_excl_scan(v, sm, total);
    if (j < nblocks) w.H.block_sum[j] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) w.H.bucket_start[w.H.n_buckets] = carry;
}

__global__ void k_scan_add(World w) {
  if (!*w.H.build) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < w.H.n_buckets) w.H.bucket_start[i] += w.H.block_sum[blockIdx.x];
}

__global__ void k_pair_fill(World w, LaunchSet ls) {
  const int4 bt = ls.btiles[blockIdx.x];
  const DevScene &sc = w.scenes[bt.x];
  if (!sc.pair_on || !sc.pair_build) return;
  for (int i = threadIdx.x; i < bt.w; i += blockDim.x) {
    const int p = bt.z + i;
    const int b = w.P.hkey[p];
    w.P.horder[w.H.bucket_start[b] + atomicAdd(&w.H.bucket_fill[b], 1)] = p;
  }
}

// order each bucket by pool index (buckets are short), then lay out its
// entries (position, pool index, base cell, cell key) for the list build
__global__ void k_pair_sort(World w) {
  if (!*w.H.build) return;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < w.H.n_buckets; b += gridDim.x * blockDim.x) {
    const int s0 = w.H.bucket_start[b], s1 = w.H.bucket_start[b + 1];
    for (int i = s0 + 1; i < s1; ++i) {
      const int key = w.P.horder[i];
      int j = i - 1;
      while (j >= s0 && w.P.horder[j] > key) {
        w.P.horder[j + 1] = w.P.horder[j];
        --j;
      }
      w.P.horder[j + 1] = key;
    }
    for (int i = s0; i < s1; ++i) {
      const int q = w.P.horder[i];
      w.P.hent[i] = make_float4(w.P.x[0][q], w.P.x[1][q], w.P.x[2][q], __int_as_float(q));
      w.P.hbase[i] = w.P.base[q];
      w.P.hentk[i] = w.P.hcell[q];
    }
  }
}

// Whether two particles' reference stencils overlap (base cells at most two
// cells apart on every axis): such a pair interacts through the grid, and is
// a contact pair only once a cut separates it (self-contact exclusion).
__device__ __forceinline__ bool share_stencil(uint32_t bp, uint32_t bq) {
  int px, py, pz, qx, qy, qz;
  particle_base(bp, px, py, pz);
  particle_base(bq, qx, qy, qz);
  return abs(px - qx) <= 2 && abs(py - qy) <= 2 && abs(pz - qz) <= 2;
}

// Candidate lists of the particles in entries [c0, c1) of one bucket (at most
// 32, lane i holding entry c0 + i), by one warp.  The particles are taken in
// groups of one cell (and scene); a group shares its 27 neighbour cells
// (dz, dy, dx in -1..1, x fastest), whose bucket entries are laid end to end
// and tested 32 at a time, one per lane, against each member in turn: an
// entry counts when it belongs to the neighbour cell (its key; a bucket's
// hash may be shared), is another particle and lies within r_l = 2 R_p +
// skin.  A ballot gives each accepted entry its place, so every list is in
// (cell, pool index) order, as a walk of the cells in order would give;
// bit 31 of an entry marks a pair whose reference stencils overlap.
__device__ __forceinline__ void bucket_lists(const World &w, int c0, int c1, int lane) {
  const PPool &P = w.P;
  const bool mine = lane < c1 - c0;
  const float4 me = mine ? P.hent[c0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  const unsigned long long mkey = mine ? P.hentk[c0 + lane] : ~0ull;
  const uint32_t mbase = mine ? P.hbase[c0 + lane] : 0u;
  const int mscene = (int)(mkey >> 48);
  int mx = 0, my = 0, mz = 0;
  if (mine) {
    const float ih = w.scenes[mscene].pair_inv_h;
    mx = (int)floorf(me.x * ih);
    my = (int)floorf(me.y * ih);
    mz = (int)floorf(me.z * ih);
  }
  int cnt = 0;
  unsigned todo = __ballot_sync(FULL, mine);
  while (todo) {
    const int lead = __ffs(todo) - 1;
    const unsigned long long K = __shfl_sync(FULL, mkey, lead);
    const int cx0 = __shfl_sync(FULL, mx, lead), cy0 = __shfl_sync(FULL, my, lead),
              cz0 = __shfl_sync(FULL, mz, lead);
    const unsigned grp = __ballot_sync(FULL, mine && mkey == K && mx == cx0 && my == cy0 && mz == cz0) & todo;
    todo &= ~grp;
    const int scene = (int)(K >> 48);
    const DevScene &sc = w.scenes[scene];
    const float rl = 2.0f * sc.Rp + 1.5f * sc.Rp, rl2 = rl * rl;
    int a0 = 0, sz = 0;
    unsigned long long nk = 0;
    if (lane < 27) {
      const int cx = cx0 + lane % 3 - 1, cy = cy0 + (lane / 3) % 3 - 1, cz = cz0 + lane / 9 - 1;
      const int hb = hash_cell(scene, cx, cy, cz, w.H.n_buckets);
      a0 = w.H.bucket_start[hb];
      sz = w.H.bucket_start[hb + 1] - a0;
      nk = cell_key(scene, cx, cy, cz);
    }
    int incl = sz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    const int T = __shfl_sync(FULL, incl, 31);
    const int excl = incl - sz;
    for (int base = 0; base < T; base += 32) {
      const int j = base + lane;
      // neighbour cell of candidate j: the last cell whose entries start at or before j
      int L = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int t = L + step;
        const int ex = __shfl_sync(FULL, excl, t < 27 ? t : 26);
        if (t < 27 && ex <= j) L = t;
      }
      const int aL = __shfl_sync(FULL, a0, L), exL = __shfl_sync(FULL, excl, L);
      const unsigned long long kL = __shfl_sync(FULL, nk, L);
      const bool inr = j < T;
      const int k = aL + (j - exL);
      const float4 e = inr ? P.hent[k] : make_float4(0.f, 0.f, 0.f, 0.f);
      const unsigned long long ek = inr ? P.hentk[k] : 0ull;
      const uint32_t eb = inr ? P.hbase[k] : 0u;
      const bool valid = inr && ek == kL;
      const int q = __float_as_int(e.w);
      unsigned g = grp;
      while (g) {
        const int m = __ffs(g) - 1;
        g &= g - 1;
        const float px = __shfl_sync(FULL, me.x, m), py = __shfl_sync(FULL, me.y, m),
                    pz = __shfl_sync(FULL, me.z, m);
        const int p = __float_as_int(__shfl_sync(FULL, me.w, m));
        const uint32_t bp = __shfl_sync(FULL, mbase, m);
        const float d0 = px - e.x, d1 = py - e.y, d2 = pz - e.z;
        const bool acc = valid && q != p && d0 * d0 + d1 * d1 + d2 * d2 <= rl2;
        const unsigned am = __ballot_sync(FULL, acc);
        const int c = __shfl_sync(FULL, cnt, m);
        if (acc) {
          const int pos = c + __popc(am & ((1u << lane) - 1u));
          if (pos < BM_NBR)
            P.nbr[(size_t)p * BM_NBR + pos] = share_stencil(bp, eb) ? (int)((uint32_t)q | 0x80000000u) : q;
        }
        if (lane == m) cnt += __popc(am);
      }
    }
  }
  if (mine) {
    const int p = __float_as_int(me.w);
    P.nbr_n[p] = (uint8_t)min(cnt, BM_NBR);
    P.xb[0][p] = me.x;
    P.xb[1][p] = me.y;
    P.xb[2][p] = me.z;
    if (cnt > BM_NBR) atomicOr(&w.scenes[mscene].err, BM_ERRBIT_CONTACT_OVERFLOW);
  }
}

// candidate lists of every particle of the scenes that rebuild them: each
// warp takes groups of 32 buckets (grid-stride) and builds the lists of the
// particles of each non-empty one, 32 entries at a time.  The positions of
// the build are kept.
__global__ void __launch_bounds__(256) k_pair_list(World w) {
  if (!*w.H.build) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nb = w.H.n_buckets;
  for (int b0 = warp * 32; b0 < nb; b0 += nwarps * 32) {
    const int b = b0 + lane;
    const int e0 = b < nb ? w.H.bucket_start[b] : 0, e1 = b < nb ? w.H.bucket_start[b + 1] : 0;
    unsigned todo = __ballot_sync(FULL, e1 > e0);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int k0 = __shfl_sync(FULL, e0, src), k1 = __shfl_sync(FULL, e1, src);
      for (int c = k0; c < k1; c += 32) bucket_lists(w, c, min(k1, c + 32), lane);
    }
  }
}

// Pair impulses (Eq. 10-13), one thread per particle walking its list
// (gridDim.y CTAs per brick).  A candidate sharing p's reference stencil is
// skipped unless the two are on opposite sides of a cut, before its state
// is read.
__global__ void k_pair(World w, LaunchSet ls) {
  const int4 bt = ls.btiles[blockIdx.x];
  DevScene &scm = w.scenes[bt.x];
  const DevScene &sc = scm;
  if (!sc.pair_on || sc.frozen) return;
  const PPool &P = w.P;
  const int rb = (int)(sc.step & 1), wb = rb ^ 1;
  const float dt = sc.dt, R2 = 2.0f * sc.Rp;
  const float meff = sc.mp * sc.mp / (sc.mp + sc.mp);
  bool over = false;
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < bt.w; i += blockDim.x * gridDim.y) {
    const int p = bt.z + i;
    const float xp[3] = {P.x[0][p], P.x[1][p], P.x[2][p]};
    const float vp[3] = {P.v[0][p], P.v[1][p], P.v[2][p]};
    const uint32_t a1 = P.s1[p], a2 = P.s2[p];
    float J[3] = {0.f, 0.f, 0.f};
    int cnt = 0;
    const int n = P.nbr_n[p];
    const int *lst = P.nbr + (size_t)p * BM_NBR;
    for (int k = 0; k < n; ++k) {
      const int ent = lst[k];
      const int q = ent & 0x7fffffff;
      if (ent < 0 && !conflict(a1, a2, P.s1[q], P.s2[q])) continue;  // self-contact exclusion
      const float xq[3] = {P.x[0][q], P.x[1][q], P.x[2][q]};
      const float vq[3] = {P.v[0][q], P.v[1][q], P.v[2][q]};
      const bool plo = p < q;
      const int lo = plo ? p : q, hi = plo ? q : p;
      const float *xl = plo ? xp : xq, *xh = plo ? xq : xp;
      const float *vl = plo ? vp : vq, *vh = plo ? vq : vp;
      const float d[3] = {xl[0] - xh[0], xl[1] - xh[1], xl[2] - xh[2]};
      const float dist = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (!(dist > 0.f)) continue;
      const float id = 1.0f / dist;
      const float nn[3] = {d[0] * id, d[1] * id, d[2] * id};
      const float vr[3] = {vl[0] - vh[0], vl[1] - vh[1], vl[2] - vh[2]};
      const float vn = vr[0] * nn[0] + vr[1] * nn[1] + vr[2] * nn[2];
      const float dhat = R2 - (dist + fminf(dt * vn, 0.0f));  // Eq. 10
      if (!(dhat > 0.f)) continue;
      const float fn = sc.s_n * meff / (dt * dt) * dhat;  // Eq. 11
      float uh[3] = {0.f, 0.f, 0.f};
      for (int h = 0; h < BM_HIST; ++h) {
        const int pt = P.hist_partner[rb][(size_t)lo * BM_HIST + h];
        if (pt < 0) break;
        if (pt == hi) {
          const float *u = P.hist_u[rb] + ((size_t)lo * BM_HIST + h) * 3;
          uh[0] = u[0];
          uh[1] = u[1];
          uh[2] = u[2];
          break;
        }
      }
      float ft[3], un[3];
      friction(uh, nn, vr, fn, meff, dt, sc.gamma_k, sc.gamma_c, sc.pair_mu_s, sc.pair_mu_d, ft, un);
      const float Jv[3] = {dt * (fn * nn[0] + ft[0]), dt * (fn * nn[1] + ft[1]), dt * (fn * nn[2] + ft[2])};
      if (plo) {  // Eq. 13: +J on the lower index, -J on the higher
        J[0] += Jv[0];
        J[1] += Jv[1];
        J[2] += Jv[2];
        if (cnt < BM_HIST) {
          P.hist_partner[wb][(size_t)p * BM_HIST + cnt] = hi;
          float *u = P.hist_u[wb] + ((size_t)p * BM_HIST + cnt) * 3;
          u[0] = un[0];
          u[1] = un[1];
          u[2] = un[2];
          ++cnt;
        } else {
          over = true;
        }
      } else {
        J[0] -= Jv[0];
        J[1] -= Jv[1];
        J[2] -= Jv[2];
      }
    }
    if (cnt < BM_HIST) P.hist_partner[wb][(size_t)p * BM_HIST + cnt] = -1;
    P.J[0][p] = J[0];
    P.J[1][p] = J[1];
    P.J[2][p] = J[2];
  }
  if (over) atomicOr(&scm.err, BM_ERRBIT_CONTACT_OVERFLOW);
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
  if (sc.reset_D) {  // a new cut begins: keep its plane for the cut faces
    for (int i = 0; i < 3; ++i) sc.cutpl[cut][i] = sc.dn[i];
    sc.cutpl[cut][3] = __dadd_rn(__dadd_rn(__dmul_rn(sc.dn[0], sc.dxe[0]), __dmul_rn(sc.dn[1], sc.dxe[1])),
                                 __dmul_rn(sc.dn[2], sc.dxe[2]));
    sc.cutpl_set |= 1u << cut;
  }
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

// the serial part of k_tool (one thread): wrench history, interval-averaged
// rigid tool step, and the frame of the next substep
__device__ __forceinline__ void tool_step(const World &w, DevScene &sc, const double W[6]) {
  // labels committed by k_fupd this substep -> rebuild the slot table
  sc.need_rebuild = sc.label_pending ? 1 : 0;
  sc.label_pending = 0;
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
  if (sc.stop_at >= 0 && sc.step >= sc.stop_at) sc.frozen = 1;
  prepare_substep(sc);
}


__global__ void k_tool(World w, LaunchSet ls) {
  const int sid = ls.scene_ids[blockIdx.x];
  DevScene &g = w.scenes[sid];
  if (g.frozen) {  // a scene that has taken its substeps: nothing moves, nothing to rebuild
    if (threadIdx.x == 0) g.need_rebuild = 0;
    return;
  }
  __shared__ double sm[32];
  // the scene record into shared memory (coalesced), so that the serial tool
  // step and frame below read and write it at shared-memory latency
  __shared__ DevScene sc;
  static_assert(sizeof(DevScene) % sizeof(double) == 0, "the scene record copies as doubles");
  constexpr int kWords = (int)(sizeof(DevScene) / sizeof(double));
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    reinterpret_cast<double *>(&sc)[i] = reinterpret_cast<const double *>(&g)[i];
  __syncthreads();
  // reduce this substep's per-brick wrench partials in brick order
  double W[6];
  for (int k = 0; k < 6; ++k) {
    double acc = 0.0;
    if (sc.has_blade)
      for (int j = threadIdx.x; j < sc.n_brick; j += blockDim.x)
        acc += w.wpart[(size_t)(sc.brick_begin + j) * 6 + k];
    W[k] = block_sum(acc, sm);
  }
  __syncthreads();
  if (threadIdx.x == 0) tool_step(w, sc, W);
  __syncthreads();
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    reinterpret_cast<double *>(&g)[i] = reinterpret_cast<const double *>(&sc)[i];
}

// --------------------------------------------------------------------------
// logical-grid slot table (rebuilt after label changes)
// --------------------------------------------------------------------------


// Distinct codes at every node of a node tile.  Nodes next to a newly
// labelled particle (dirty) are recounted, the others keep their distinct
// codes from the last rebuild.  A recount takes one warp per node: lane l <
// 27 holds base cell (i - l % 3, j - l / 3 % 3, k - l / 9) of the node's
// stencil, and the node's codes are found in ascending order of the key
// (mask2 << 32 | mask1) as repeated warp-wide minima over the lanes' particles
// of the keys above the last one found.
// KR: particles per cell whose label keys a lane keeps in registers across
// the passes (8 or 16, the launch set's largest cell)
template <int KR>
__global__ void k_slot_count(World w, LaunchSet ls, int force) {
  const int4 t = ls.ntiles[blockIdx.x];
  DevScene &sc = w.scenes[t.x];
  if (!force && !sc.need_rebuild) return;
  __shared__ int sm[33];
  __shared__ int dlist[512];   // node tile <= 512 nodes
  __shared__ int dcnt[512];
  __shared__ int ndirty;
  const int i = threadIdx.x;
  const int node = t.y + i;
  bool recount = false;
  if (i < t.z) recount = force != 0 || w.N.dirty[node] != 0;
  if (i == 0) ndirty = 0;
  __syncthreads();
  if (recount) dlist[atomicAdd(&ndirty, 1)] = i;
  __syncthreads();
  const int lane = i & 31, wid = i >> 5, nw = blockDim.x >> 5;
  const int *cs = w.N.cell_start + sc.cell_begin;
  for (int j = wid; j < ndirty; j += nw) {
    const int li = dlist[j];
    const int nd = t.y + li;
    int ix, iy, iz;
    node_coords(sc, nd - sc.node_begin, ix, iy, iz);
    int p0 = 0, p1 = 0;
    if (lane < 27) {
      const int bx = ix - lane % 3, by = iy - (lane / 3) % 3, bz = iz - lane / 9;
      if (bx >= 0 && by >= 0 && bz >= 0 && bx < sc.nb[0] && by < sc.nb[1] && bz < sc.nb[2]) {
        const int c = cell_index(sc, bx, by, bz);
        p0 = cs[c];
        p1 = cs[c + 1];
      }
    }
    int cnt = 0;
    bool over = false;
    unsigned long long last = 0;
    bool first = true;
    // a cell of up to KR particles keeps its keys in registers across the
    // passes (the all-ones key is never a code: a cut has one side per particle)
    const bool inreg = p1 - p0 <= KR;
    unsigned long long kr[KR];
#pragma unroll
    for (int j = 0; j < KR; ++j)
      kr[j] = (inreg && p0 + j < p1) ? ((unsigned long long)w.P.s2[p0 + j] << 32) | w.P.s1[p0 + j] : ~0ull;
    for (;;) {
      unsigned long long m = ~0ull;
      if (inreg) {
#pragma unroll
        for (int j = 0; j < KR; ++j)
          if ((first || kr[j] > last) && kr[j] < m) m = kr[j];
      } else {
        for (int p = p0; p < p1; ++p) {
          const unsigned long long k = ((unsigned long long)w.P.s2[p] << 32) | w.P.s1[p];
          if ((first || k > last) && k < m) m = k;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULL, m, o);
        m = y < m ? y : m;
      }
      if (m == ~0ull) break;
      if (cnt < BM_MAXS) {
        if (lane == 0)
          w.N.tmp_codes[(size_t)nd * BM_MAXS + cnt] = make_uint2((uint32_t)m, (uint32_t)(m >> 32));
        ++cnt;
      } else {
        over = true;
        break;
      }
      last = m;
      first = false;
    }
    if (lane == 0) {
      if (over) atomicOr(&sc.err, BM_ERRBIT_SLOT_OVERFLOW);
      w.N.ncodes[nd] = (uint8_t)cnt;
      w.N.dirty[nd] = 0;
      dcnt[li] = cnt;
    }
  }
  __syncthreads();
  int cnt = 0;
  if (i < t.z) cnt = recount ? dcnt[i] : w.N.ncodes[node];
  if (i < t.z) w.N.slot_cnt[node] = (uint8_t)cnt;
  int total;
  block_excl_scan(cnt, sm, total);
  if (threadIdx.x == 0) w.N.tile_sum[t.w] = total;
}

// per brick: slot count and first tile slot of each tile node, and the
// tile's slot total (after the per-node counts are final)
// (one warp per brick, BTILE_WARPS bricks per CTA: lane l takes the tile's
// nodes 7l .. 7l + 6, an exclusive warp scan orders them)
#define BTILE_WARPS 8
__global__ void __launch_bounds__(32 * BTILE_WARPS) k_brick_tiles(World w, LaunchSet ls, int force) {
  const int lane = threadIdx.x & 31;
  const int bi = blockIdx.x * BTILE_WARPS + (threadIdx.x >> 5);
  if (bi >= ls.n_btiles) return;
  const int4 bt = ls.btiles[bi];
  const DevScene &sc = w.scenes[bt.x];
  if (!force && !sc.need_rebuild) return;
  int c0x, c0y, c0z;
  brick_coords(sc, bt.y - sc.brick_begin, c0x, c0y, c0z);
  constexpr int PER = (TN + 31) / 32;  // 7
  int cnt[PER];
  int mine = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int t = lane * PER + j;
    cnt[j] = 0;
    if (t < TN) {
      const int nx = c0x + t % TE, ny = c0y + (t / TE) % TE, nz = c0z + t / (TE * TE);
      if (nx < sc.nn[0] && ny < sc.nn[1] && nz < sc.nn[2])
        cnt[j] = w.N.slot_cnt[sc.node_begin + (nz * sc.nn[1] + ny) * sc.nn[0] + nx];
    }
    mine += cnt[j];
  }
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  int ex = incl - mine;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int t = lane * PER + j;
    if (t < TN) w.B.tdesc[(size_t)bt.y * TN + t] = ex | (cnt[j] << 16);
    ex += cnt[j];
  }
  if (lane == 31) w.B.ptot[bt.y] = incl;
}

// per scene: slot offsets of the node tiles, and partial-sum ranges of the bricks
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
  int pcarry = 0;
  bool pover = false;
  for (int base = 0; base < sc.n_brick; base += blockDim.x) {
    const int j = base + threadIdx.x;
    const int v = j < sc.n_brick ? w.B.ptot[sc.brick_begin + j] : 0;
    int total;
    const int ex = block_excl_scan(v, sm, total);
    if (j < sc.n_brick) {
      const bool fits = pcarry + ex + v <= sc.ppool_cap;
      w.B.poff[sc.brick_begin + j] = fits ? sc.ppool_begin + pcarry + ex : -1;
      pover |= !fits;
    }
    pcarry += total;
    __syncthreads();
  }
  if (pover) atomicOr(&sc.err, BM_ERRBIT_SLOT_OVERFLOW);
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
    int off = w.N.tile_sum[t.w] + ex;
    const bool fits = off + cnt <= sc.slot_cap;
    if (!fits) {
      w.N.slot_cnt[node] = 0;
      off = 0;
    } else {
      for (int a = 0; a < cnt; ++a)
        w.S.code[sc.slot_begin + off + a] = w.N.tmp_codes[(size_t)node * BM_MAXS + a];
    }
    w.N.slot_off[node] = sc.slot_begin + off;
    // the node's first slot in the tile table of every brick whose tile covers it
    int ix, iy, iz, x0, x1, y0, y1, z0, z1;
    node_coords(sc, node - sc.node_begin, ix, iy, iz);
    covering(ix, sc.nbr[0], x0, x1);
    covering(iy, sc.nbr[1], y0, y1);
    covering(iz, sc.nbr[2], z0, z1);
    for (int Bz = z0; Bz <= z1; ++Bz)
      for (int By = y0; By <= y1; ++By)
        for (int Bx = x0; Bx <= x1; ++Bx) {
          const int b = sc.brick_begin + (Bz * sc.nbr[1] + By) * sc.nbr[0] + Bx;
          const int tt = ((iz - Bz * BR) * TE + (iy - By * BR)) * TE + (ix - Bx * BR);
          w.B.tgoff[(size_t)b * TN + tt] = sc.slot_begin + off;
        }
  }
}

// --------------------------------------------------------------------------
// state I/O between pool order and the caller's order
// --------------------------------------------------------------------------
__global__ void k_io(World w, int scene_slot, int p_begin, int n, int field, void *buf, int to_pool) {
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
      if (to_pool) {
        P.D[p] = fb[o];
        P.tflag[p] = 1;  // may be nonzero: the next P2G reads it
      } else {
        fb[o] = P.D[p];
      }
      break;
    case 5:
      for (int a = 0; a < 3; ++a) {
        if (to_pool) P.ut[a][p] = fb[3 * o + a];
        else fb[3 * o + a] = P.ut[a][p];
      }
      if (to_pool) P.tflag[p] = 1;
      break;
    case 7:
      if (to_pool) P.s1[p] = ub[o];
      else ub[o] = P.s1[p];
      break;
    case 8:
      if (to_pool) P.s2[p] = ub[o];
      else ub[o] = P.s2[p];
      break;
    case 9:    // pair history partners (read only): caller indices, -1 ends the list
    case 10: {  // pair history spring displacements (read only)
      if (to_pool || !P.hist_partner[0]) break;
      const int rb = (int)(w.scenes[scene_slot].step & 1);  // the buffer the next substep reads
      bool live = true;
      for (int h = 0; h < BM_HIST; ++h) {
        const int pt = live ? P.hist_partner[rb][(size_t)p * BM_HIST + h] : -1;
        live = pt >= 0;
        if (field == 9) {
          ((int *)buf)[(size_t)o * BM_HIST + h] = live ? P.perm[pt] : -1;
        } else {
          const float *u = P.hist_u[rb] + ((size_t)p * BM_HIST + h) * 3;
          for (int a = 0; a < 3; ++a) fb[((size_t)o * BM_HIST + h) * 3 + a] = live ? u[a] : 0.0f;
        }
      }
      break;
    }
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
    "k_p2g_brick", "k_p2g_node", "k_g2p_musl", "k_musl_node", "k_fupd",
    "k_tool", "k_slot_count", "k_slot_scan", "k_slot_fill", "k_brick_tiles",
    "k_pair_clear", "k_pair_hash", "k_scan_local", "k_scan_top", "k_scan_add", "k_pair_fill",
    "k_pair_sort", "k_pair", "k_pair_list"};

// ev (optional): 2 * BM_NUM_KERNELS events recorded around each launch
static inline void rec(cudaEvent_t *ev, int k, int after, cudaStream_t st) {
  if (ev) cudaEventRecord(ev[2 * k + after], st);
}

static cudaError_t launch_rebuild(const World &w, const LaunchSet &ls, cudaStream_t st, int force,
                                  cudaEvent_t *ev) {
  if (ls.n_ntiles == 0) return cudaSuccess;
  rec(ev, 6, 0, st);
  if (ls.ppc16)
    k_slot_count<16><<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls, force);
  else
    k_slot_count<8><<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls, force);
  rec(ev, 6, 1, st);
  rec(ev, 9, 0, st);
  k_brick_tiles<<<(ls.n_btiles + BTILE_WARPS - 1) / BTILE_WARPS, 32 * BTILE_WARPS, 0, st>>>(w, ls, force);
  rec(ev, 9, 1, st);
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

// Brick-kernel occupancy: the minimum resident CTAs per SM each brick kernel
// is compiled for (launch bounds), chosen per kernel (fewer CTAs leave more
// registers per thread, more CTAs hide more latency).  A launch variant v in [0, 27) picks choice
// v % 3 for k_p2g_brick, (v / 3) % 3 for k_g2p_musl and v / 9 for k_fupd;
// choice 0 is each kernel's default.  The arithmetic is the same in every
// variant, so results are bit-identical; the batch autotuner picks one.
template <int C, bool INELASTIC> struct OccP2G;
template <> struct OccP2G<0, false> { static constexpr int v = 4; };
template <> struct OccP2G<1, false> { static constexpr int v = 3; };
template <> struct OccP2G<2, false> { static constexpr int v = 2; };
template <> struct OccP2G<0, true> { static constexpr int v = 3; };  // the inelastic stress needs the registers
template <> struct OccP2G<1, true> { static constexpr int v = 2; };
template <> struct OccP2G<2, true> { static constexpr int v = 4; };
template <int C> struct OccG2P;
template <> struct OccG2P<0> { static constexpr int v = 5; };
template <> struct OccG2P<1> { static constexpr int v = 4; };
template <> struct OccG2P<2> { static constexpr int v = 6; };
template <int C> struct OccFupd;
template <> struct OccFupd<0> { static constexpr int v = 7; };
template <> struct OccFupd<1> { static constexpr int v = 5; };
template <> struct OccFupd<2> { static constexpr int v = 6; };

// dynamic shared memory of the brick kernels, and the largest shared-memory
// carveout, so that the CTAs per SM their launch bounds aim at fit
template <class K>
static cudaError_t brick_smem(K *kernel, int bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

template <int PPC, int C>
static cudaError_t set_smem_attrs() {
  cudaError_t e = brick_smem(k_p2g_brick<PPC, OccP2G<C, false>::v, false>, (int)sizeof(K2S<PPC>));
  if (e == cudaSuccess) e = brick_smem(k_p2g_brick<PPC, OccP2G<C, true>::v, true>, (int)sizeof(K2S<PPC>));
  if (e == cudaSuccess) e = brick_smem(k_g2p_musl<PPC, OccG2P<C>::v>, (int)sizeof(K4S<PPC>));
  return e;
}

cudaError_t bm_kernels_init() {
  static cudaError_t status = cudaErrorNotReady;
  static int device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (device == dev && status == cudaSuccess) return status;
  if (e == cudaSuccess) e = set_smem_attrs<8, 0>();
  if (e == cudaSuccess) e = set_smem_attrs<8, 1>();
  if (e == cudaSuccess) e = set_smem_attrs<8, 2>();
  if (e == cudaSuccess) e = set_smem_attrs<16, 0>();
  if (e == cudaSuccess) e = set_smem_attrs<16, 1>();
  if (e == cudaSuccess) e = set_smem_attrs<16, 2>();
  status = e;
  device = dev;
  return e;
}

template <int PPC, int C>
static void launch_p2g(const World &w, const LaunchSet &ls, cudaStream_t st) {
  if (ls.any_inelastic)
    k_p2g_brick<PPC, OccP2G<C, true>::v, true><<<ls.n_btiles, BT, sizeof(K2S<PPC>), st>>>(w, ls);
  else
    k_p2g_brick<PPC, OccP2G<C, false>::v, false><<<ls.n_btiles, BT, sizeof(K2S<PPC>), st>>>(w, ls);
}

template <int PPC, int C>
static void launch_g2p(const World &w, const LaunchSet &ls, cudaStream_t st) {
  k_g2p_musl<PPC, OccG2P<C>::v><<<ls.n_btiles, BT, sizeof(K4S<PPC>), st>>>(w, ls);
}

template <int C>
static void launch_fupd(const World &w, const LaunchSet &ls, cudaStream_t st) {
  if (ls.any_inelastic) k_fupd<OccFupd<C>::v, true><<<ls.n_btiles, BT, 0, st>>>(w, ls);
  else k_fupd<OccFupd<C>::v, false><<<ls.n_btiles, BT, 0, st>>>(w, ls);
}

template <int PPC>
static void launch_bricks(const World &w, const LaunchSet &ls, cudaStream_t st, cudaEvent_t *ev) {
  const int cp = ls.variant % 3, cg = (ls.variant / 3) % 3, cf = ls.variant / 9;
  rec(ev, 0, 0, st);
  if (cp == 0) launch_p2g<PPC, 0>(w, ls, st);
  else if (cp == 1) launch_p2g<PPC, 1>(w, ls, st);
  else launch_p2g<PPC, 2>(w, ls, st);
  rec(ev, 0, 1, st);
  rec(ev, 1, 0, st);
  k_p2g_node<<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls);
  rec(ev, 1, 1, st);
  rec(ev, 2, 0, st);
  if (cg == 0) launch_g2p<PPC, 0>(w, ls, st);
  else if (cg == 1) launch_g2p<PPC, 1>(w, ls, st);
  else launch_g2p<PPC, 2>(w, ls, st);
  rec(ev, 2, 1, st);
  rec(ev, 3, 0, st);
  k_musl_node<<<ls.n_ntiles, ls.ntile_size, 0, st>>>(w, ls);
  rec(ev, 3, 1, st);
  rec(ev, 4, 0, st);
  if (cf == 0) launch_fupd<0>(w, ls, st);
  else if (cf == 1) launch_fupd<1>(w, ls, st);
  else launch_fupd<2>(w, ls, st);
  rec(ev, 4, 1, st);
}

static void launch_pairs(const World &w, const LaunchSet &ls, cudaStream_t st, cudaEvent_t *ev) {
  const int nb = w.H.n_buckets;
  const int nblk = (nb + 1023) / 1024;
  rec(ev, 10, 0, st);
  k_pair_reset<<<(ls.n_scenes + 255) / 256, 256, 0, st>>>(w, ls);
  k_pair_vmax<<<ls.n_btiles, BT, 0, st>>>(w, ls);
  k_pair_decide<<<(ls.n_scenes + 63) / 64, 64, 0, st>>>(w, ls);
  cudaMemsetAsync(w.H.bucket_start, 0, sizeof(int) * ((size_t)nb + 1), st);
  cudaMemsetAsync(w.H.bucket_fill, 0, sizeof(int) * (size_t)nb, st);
  rec(ev, 10, 1, st);
  rec(ev, 11, 0, st);
  k_pair_hash<<<ls.n_btiles, BT, 0, st>>>(w, ls);
  rec(ev, 11, 1, st);
  rec(ev, 12, 0, st);
  k_scan_local<<<nblk, 1024, 0, st>>>(w);
  rec(ev, 12, 1, st);
  rec(ev, 13, 0, st);
  k_scan_top<<<1, 1024, 0, st>>>(w, nblk);
  rec(ev, 13, 1, st);
  rec(ev, 14, 0, st);
  k_scan_add<<<nblk, 1024, 0, st>>>(w);
  rec(ev, 14, 1, st);
  rec(ev, 15, 0, st);
  k_pair_fill<<<ls.n_btiles, BT, 0, st>>>(w, ls);
  rec(ev, 15, 1, st);
  rec(ev, 16, 0, st);
  k_pair_sort<<<(nb + 255) / 256, 256, 0, st>>>(w);
  rec(ev, 16, 1, st);
  rec(ev, 18, 0, st);
  const int lgrid = (nb / 32 + 7) / 8;  // 8 warps per CTA, a warp per 32 buckets, at most 8 CTAs per SM
  k_pair_list<<<lgrid < 152 * 8 ? lgrid : 152 * 8, 256, 0, st>>>(w);
  rec(ev, 18, 1, st);
  rec(ev, 17, 0, st);
  k_pair<<<dim3(ls.n_btiles, 4), 128, 0, st>>>(w, ls);
  rec(ev, 17, 1, st);
}

cudaError_t bm_launch_substep_ev(const World &w, const LaunchSet &ls, cudaStream_t st, cudaEvent_t *ev) {
  if (ls.n_btiles == 0) return cudaSuccess;
  if (ls.any_pair && w.H.n_buckets > 0) launch_pairs(w, ls, st, ev);
  if (ls.ppc16) launch_bricks<16>(w, ls, st, ev);
  else launch_bricks<8>(w, ls, st, ev);
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
  if (n == 0) return cudaSuccess;
  k_io<<<(n + 255) / 256, 256, 0, st>>>(w, scene_slot, p_begin, n, field, buf, to_pool);
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
