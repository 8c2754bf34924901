/*
 * FP64 oracle of the TLMPM cutting substep (BladeMaster, arXiv 2609.27342).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what one substep computes.  Only the test suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may build,
 * link or call it; the GPU library shares no code with it.
 *
 * Everything is double precision with plain loops and a scatter-form P2G
 * that follows Eq. 2 literally.  Build with -ffp-contract=off so the few
 * decisions that must agree bit-for-bit with the GPU (side labels, Eq. 4/6)
 * are evaluated with separately rounded multiplies and adds.
 *
 * Readings of points the paper leaves open (they are listed again in the
 * design notes of the repository):
 *   - stress: compressible neo-Hookean (the workloads ask for it; the paper's
 *     own model is fixed-corotated, Sec. III-B);
 *   - shape functions: quadratic B-splines on cell-corner nodes, base node
 *     floor(X/dx - 1/2) relative to the grid origin (Eq. 1);
 *   - substep order: contact -> cutting resistance -> reaction wrench ->
 *     pair contact -> side labels (into the next code) -> stress -> P2G per
 *     logical grid -> coupling -> grid update -> G2P -> MUSL re-scatter with
 *     coupling -> F update -> commit codes -> rigid tool update;
 *   - x update uses the Eq. 9 velocity; F += dt sum_i v*_i (x) grad0 N_ip with
 *     v* from the coupled MUSL re-scatter;
 *   - D release: with D^n < 1 the full impulse is applied and D accumulates;
 *     with D^n = 1 the positive component along d is removed (Eq. 5);
 *   - friction history transport: project onto the tangent plane and rescale
 *     to the previous length; slip stores u = -(f_t + c_t v_t)/k_t (Eq. 12);
 *   - blade = oriented box (half-thickness along n, half-length along e,
 *     height behind the edge along -d), floor = frictionless half-space;
 *   - self-contact exclusion: the reference stencils share a node and the
 *     codes do not conflict (Sec. III-E).
 *
 * Parity status per function is stated in the repository's test suite;
 * whole-run trajectories are parity unpinned beyond the invariants there.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_CUTS 32
#define OR_MAX_SEG 16
#define OR_HIST 16

/* error bits (sticky) */
#define OR_E_INVERTED 1u
#define OR_E_NONFINITE 2u
#define OR_E_HIST_OVERFLOW 4u

typedef struct {
  double E, nu, rho, dx, origin[3], V0, dt, beta, g[3];
  int floor_on;
  double floor_z;
  double s_R, s_n, gamma_k, gamma_c;
  int pair_on;
  double pair_mu_s, pair_mu_d;
  double Gc, zeta, u_min, b_back, b_lead, h;
  int tool_contact_on;
  int single_field; /* 1: P2G/G2P ignore codes (the single-field baseline) */
  int model;        /* 0: compressible neo-Hookean; 1: fixed-corotated (Sec. III-B) */
  double yield_stress; /* > 0: von Mises plasticity projection (Sec. III-B) */
  double viscosity;    /* > 0: Newtonian viscosity eta (Sec. III-B) */
} or_params;

typedef struct {
  int n_steps;
  int cut_id;
  double v[3], w[3];
} or_seg;

typedef struct {
  double edge[3], n[3], e[3], d[3]; /* tool-frame geometry */
  double half_len, thick, height, mu_s, mu_d;
  double mass, inertia[9];
  double x0[3], R0[9];
  double kv;
  int rigid_interval;
  int nseg;
  or_seg seg[OR_MAX_SEG];
} or_blade;

/* One logical grid at one node: S_i^c = (m, p, dp) of Eq. 8 plus results. */
typedef struct {
  int64_t code;
  double m, p[3], dp[3];
  double vold[3], vnew[3];
  double pstar[3], vstar[3];
} or_lgrid;

typedef struct {
  int cnt, cap;
  or_lgrid *g;
} or_node;

typedef struct {
  int64_t partner;
  double u[3];
} or_hist;

typedef struct {
  or_params P;
  or_blade B;
  int has_blade;
  int64_t n;
  double *X, *x, *v, *F, *D, *ut;
  double *Fpi;  /* inverse plastic deformation F_p^{-1} (n x 9), identity without plasticity */
  double *Fdot; /* dF/dt of the last substep (n x 9), for the viscous stress */
  unsigned char *digit, *digit_next; /* n * OR_MAX_CUTS ternary digits */
  double *J;                          /* per-particle total contact+body impulse this step */
  or_hist *hist, *hist_next;
  int *hist_cnt, *hist_cnt_next;
  /* grid */
  int lo[3], dim[3];
  or_node *nodes;
  /* tool state */
  double xB[3], R[9], vB[3], wB[3];
  int64_t step;
  int cur_cut;
  double accF[3], accT[3];
  int acc_cnt;
  double lastF[6];
  double *wrench_hist;
  int64_t wrench_cap;
  double impulse_sum[3]; /* sum of impulses scattered last step (Eq. 18) */
  unsigned err;
  double mp, Rp, mu, lam;
  /* plane of each cut in the world frame at the substep the cut begins:
     unit normal n and offset n . x_e (Sec. III-F uses it as the cut
     faces' Hermite data); bit k of cutpl_set marks cut k as recorded */
  double cutpl[OR_MAX_CUTS][4];
  unsigned cutpl_set;
} or_scene;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
/* y = M x for row-major 3x3 M, summed left to right */
static void matvec(const double M[9], const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i) y[i] = M[3 * i] * x[0] + M[3 * i + 1] * x[1] + M[3 * i + 2] * x[2];
}
static void matmul(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}
static double det3(const double A[9]) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}
static int inv3(const double A[9], double B[9]) {
  double d = det3(A);
  if (d == 0.0) return 0;
  B[0] = (A[4] * A[8] - A[5] * A[7]) / d;
  B[1] = (A[2] * A[7] - A[1] * A[8]) / d;
  B[2] = (A[1] * A[5] - A[2] * A[4]) / d;
  B[3] = (A[5] * A[6] - A[3] * A[8]) / d;
  B[4] = (A[0] * A[8] - A[2] * A[6]) / d;
  B[5] = (A[2] * A[3] - A[0] * A[5]) / d;
  B[6] = (A[3] * A[7] - A[4] * A[6]) / d;
  B[7] = (A[1] * A[6] - A[0] * A[7]) / d;
  B[8] = (A[0] * A[4] - A[1] * A[3]) / d;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: reference-configuration quadratic B-spline                         */
/* ------------------------------------------------------------------------ */

/* xl = (X - origin)/dx.  Returns base node floor(xl - 1/2); w[k], dw[k] are
 * N and dN/dxl of nodes base+k, k = 0, 1, 2 (divide dw by dx for dN/dX). */
int or_bspline(double xl, double w[3], double dw[3]) {
  int base = (int)floor(xl - 0.5);
  double fx = xl - base; /* in [0.5, 1.5) */
  w[0] = 0.5 * (1.5 - fx) * (1.5 - fx);
  w[1] = 0.75 - (fx - 1.0) * (fx - 1.0);
  w[2] = 0.5 * (fx - 0.5) * (fx - 0.5);
  dw[0] = fx - 1.5;
  dw[1] = -2.0 * (fx - 1.0);
  dw[2] = fx - 0.5;
  return base;
}

/* ------------------------------------------------------------------------ */
/* stress: compressible neo-Hookean                                          */
/*   psi = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2                    */
/*   P   = mu (F - F^{-T}) + lam ln J F^{-T}                                 */
/* ------------------------------------------------------------------------ */

#define OR_JMIN 1e-6

double or_psi(const double F[9], double mu, double lam) {
  double J = det3(F);
  if (J < OR_JMIN) J = OR_JMIN;
  double tr = 0;
  for (int k = 0; k < 9; ++k) tr += F[k] * F[k];
  double lj = log(J);
  return 0.5 * mu * (tr - 3.0) - mu * lj + 0.5 * lam * lj * lj;
}

/* returns 1 when J was clamped (inverted or degenerate element) */
int or_piola(const double F[9], double mu, double lam, double P[9]) {
  double J = det3(F);
  int clamped = 0;
  if (!(J > OR_JMIN)) {
    J = OR_JMIN;
    clamped = 1;
  }
  /* F^{-T} = cof(F) / J */
  double c[9];
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
  double lj = log(J);
  for (int k = 0; k < 9; ++k) {
    double FinvT = c[k] / J;
    P[k] = mu * (F[k] - FinvT) + lam * lj * FinvT;
  }
  return clamped;
}

/* ------------------------------------------------------------------------ */
/* stress: fixed-corotated, the paper's elastic model (Sec. III-B)           */
/*   psi = mu |F - R|^2 + lam/2 (J - 1)^2,  F = R S (polar decomposition)     */
/*   P   = 2 mu (F - R) + lam (J - 1) J F^{-T}                               */
/* ------------------------------------------------------------------------ */

/* eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations:
   A = V diag(w) V^T (V orthogonal, columns = eigenvectors) */
static void or_sym_eig3(const double Ain[9], double V[9], double w[3]) {
  double A[9];
  memcpy(A, Ain, sizeof A);
  for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? 1.0 : 0.0;
  static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double diag = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int r = 0; r < 3; ++r) {
      int p = PQ[r][0], q = PQ[r][1];
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      /* rotation angle that zeroes A_pq: tan(2 phi) = 2 A_pq / (A_qq - A_pp) */
      double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
      /* A <- G^T A G, V <- V G with G the rotation in the (p, q) plane */
      for (int k = 0; k < 3; ++k) { /* columns p, q */
        double akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - sn * akq;
        A[3 * k + q] = sn * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) { /* rows p, q */
        double apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - sn * aqk;
        A[3 * q + k] = sn * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        double vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - sn * vkq;
        V[3 * k + q] = sn * vkp + c * vkq;
      }
    }
  }
  w[0] = A[0];
  w[1] = A[4];
  w[2] = A[8];
}

/* polar decomposition F = R S (det F > 0): S = (F^T F)^{1/2}, R = F S^{-1} */
void or_polar(const double F[9], double R[9], double S[9]) {
  double C[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  double V[9], w[3];
  or_sym_eig3(C, V, w);
  double sq[3], isq[3];
  for (int k = 0; k < 3; ++k) {
    sq[k] = sqrt(w[k] > 0 ? w[k] : 0.0);
    isq[k] = sq[k] > 0 ? 1.0 / sq[k] : 0.0;
  }
  double Si[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0, b = 0;
      for (int k = 0; k < 3; ++k) {
        a += V[3 * i + k] * sq[k] * V[3 * j + k];
        b += V[3 * i + k] * isq[k] * V[3 * j + k];
      }
      S[3 * i + j] = a;
      Si[3 * i + j] = b;
    }
  matmul(F, Si, R);
}

double or_psi_fcr(const double F[9], double mu, double lam) {
  double R[9], S[9];
  or_polar(F, R, S);
  double d = 0;
  for (int k = 0; k < 9; ++k) d += (F[k] - R[k]) * (F[k] - R[k]);
  double J = det3(F);
  return mu * d + 0.5 * lam * (J - 1.0) * (J - 1.0);
}

/* returns 1 when the element is inverted or degenerate (J <= 1e-6): the
   rotation is then taken from the clamped-J cofactor form and flagged */
int or_piola_fcr(const double F[9], double mu, double lam, double P[9]) {
  double J = det3(F);
  int clamped = !(J > OR_JMIN);
  double R[9], S[9];
  or_polar(F, R, S);
  double c[9]; /* J F^{-T} = cofactor matrix */
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
  for (int k = 0; k < 9; ++k) P[k] = 2.0 * mu * (F[k] - R[k]) + lam * (J - 1.0) * c[k];
  return clamped;
}

/* the scene's elastic model */
static int or_stress(const or_params *P, const double F[9], double mu, double lam, double Pk[9]) {
  return P->model == 1 ? or_piola_fcr(F, mu, lam, Pk) : or_piola(F, mu, lam, Pk);
}

/* ------------------------------------------------------------------------ */
/* von Mises plasticity projection (Sec. III-B), radial return in principal  */
/* Hencky strains.  Fe = U diag(s) V^T, eps = log s, e = eps - mean(eps);    */
/* the von Mises equivalent of the deviatoric Kirchhoff stress 2 mu e is     */
/* q = sqrt(3/2) |2 mu e|; for q > sigma_y the deviatoric strain is scaled   */
/* back onto the yield surface, e <- e sigma_y / q, which keeps det Fe.      */
/* Returns 1 when the projection acted.                                      */
/* ------------------------------------------------------------------------ */
int or_vonmises(double Fe[9], double mu, double sigma_y) {
  double C[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = Fe[i] * Fe[j] + Fe[3 + i] * Fe[3 + j] + Fe[6 + i] * Fe[6 + j];
  double V[9], w[3];
  or_sym_eig3(C, V, w);
  double sg[3], eps[3];
  for (int k = 0; k < 3; ++k) {
    if (!(w[k] > 0)) return 0; /* degenerate: left to the inversion flag */
    sg[k] = sqrt(w[k]);
    eps[k] = log(sg[k]);
  }
  double mean = (eps[0] + eps[1] + eps[2]) / 3.0;
  double e[3] = {eps[0] - mean, eps[1] - mean, eps[2] - mean};
  double en = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  double q = sqrt(1.5) * 2.0 * mu * en;
  if (!(q > sigma_y)) return 0;
  double scale = sigma_y / q;
  /* U = Fe V diag(1/s); Fe_new = U diag(s_new) V^T = Fe V diag(s_new / s) V^T */
  double M[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0;
      for (int k = 0; k < 3; ++k) {
        double snew = exp(mean + scale * e[k]);
        a += V[3 * i + k] * (snew / sg[k]) * V[3 * j + k];
      }
      M[3 * i + j] = a;
    }
  double out[9];
  matmul(Fe, M, out);
  memcpy(Fe, out, sizeof out);
  return 1;
}

/* Newtonian viscosity (Sec. III-B): Cauchy stress sigma_v = eta (L + L^T)
   with L = dF/dt F^{-1}; its first Piola-Kirchhoff form J sigma_v F^{-T}
   is added to P.  dF/dt is the last substep's rate. */
void or_viscous_piola(const double F[9], const double Fdot[9], double eta, double P[9]) {
  double Fi[9];
  if (!inv3(F, Fi)) return;
  double L[9];
  matmul(Fdot, Fi, L);
  double sv[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) sv[3 * i + j] = eta * (L[3 * i + j] + L[3 * j + i]);
  double c[9]; /* J F^{-T} = cofactor matrix */
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
  double add[9];
  matmul(sv, c, add);
  for (int k = 0; k < 9; ++k) P[k] += add[k];
}

/* stress of particle p at the start of the substep: plastic projection of
   Fe = F Fp^{-1} (updating Fp^{-1}), elastic P(Fe) Fp^{-T}, viscous part */
static int or_particle_stress(or_scene *s, int64_t p, double Pk[9]) {
  const or_params *P = &s->P;
  const double *F = s->F + 9 * p;
  int clamped;
  if (P->yield_stress > 0) {
    double *Fpi = s->Fpi + 9 * p;
    double Fe[9];
    matmul(F, Fpi, Fe);
    if (or_vonmises(Fe, s->mu, P->yield_stress)) {
      double Fi[9];
      if (inv3(F, Fi)) matmul(Fi, Fe, Fpi); /* Fp^{-1} = F^{-1} Fe */
    }
    double Pe[9], FpiT[9];
    clamped = or_stress(P, Fe, s->mu, s->lam, Pe);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) FpiT[3 * i + j] = Fpi[3 * j + i];
    matmul(Pe, FpiT, Pk);
  } else {
    clamped = or_stress(P, F, s->mu, s->lam, Pk);
  }
  if (P->viscosity > 0) or_viscous_piola(F, s->Fdot + 9 * p, P->viscosity, Pk);
  return clamped;
}

/* ------------------------------------------------------------------------ */
/* Eq. 7 and the conflict predicate                                          */
/* ------------------------------------------------------------------------ */

static int64_t pow3(int k) {
  int64_t r = 1;
  while (k-- > 0) r *= 3;
  return r;
}

/* c = sum_k d_k 3^k */
int64_t or_code(const unsigned char *digits, int K) {
  int64_t c = 0;
  for (int k = 0; k < K; ++k) c += (int64_t)digits[k] * pow3(k);
  return c;
}

/* d_k(c): the k-th ternary digit */
int or_digit(int64_t c, int k) { return (int)((c / pow3(k)) % 3); }

/* conflict(a, b) <=> exists k with (d_k(a), d_k(b)) in {(1,2), (2,1)} */
int or_conflict(int64_t a, int64_t b) {
  for (int k = 0; k < OR_MAX_CUTS; ++k) {
    int da = or_digit(a, k), db = or_digit(b, k);
    if ((da == 1 && db == 2) || (da == 2 && db == 1)) return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 8: compatible-state coupling at one node                              */
/*   S_bar^a = S^a + 1/M sum_{b != a, !conflict(a,b)} (m^a S^b - m^b S^a)    */
/* S is ns x nc (row a = logical grid a), updated in place.                  */
/* ------------------------------------------------------------------------ */

void or_couple(int ns, const int64_t *codes, const double *m, int nc, double *S) {
  double M = 0;
  for (int a = 0; a < ns; ++a) M += m[a];
  if (!(M > 0)) return;
  double *Sbar = (double *)malloc(sizeof(double) * (size_t)ns * (size_t)nc);
  for (int a = 0; a < ns; ++a) {
    for (int c = 0; c < nc; ++c) {
      double acc = 0;
      for (int b = 0; b < ns; ++b) {
        if (b == a || or_conflict(codes[a], codes[b])) continue;
        acc += m[a] * S[b * nc + c] - m[b] * S[a * nc + c];
      }
      Sbar[a * nc + c] = S[a * nc + c] + acc / M;
    }
  }
  memcpy(S, Sbar, sizeof(double) * (size_t)ns * (size_t)nc);
  free(Sbar);
}

/* ------------------------------------------------------------------------ */
/* Eq. 12: tangential spring-history Coulomb friction                        */
/* ------------------------------------------------------------------------ */

void or_friction(const double u_hist[3], const double n[3], const double vrel[3], double fn,
                 double meff, double dt, double gk, double gc, double mus, double mud,
                 double ft[3], double u_new[3]) {
  /* transport the stored displacement to the current tangent plane */
  double un = dot3(u_hist, n), ul = norm3(u_hist);
  double tu[3] = {u_hist[0] - un * n[0], u_hist[1] - un * n[1], u_hist[2] - un * n[2]};
  double tl = norm3(tu);
  double ut[3] = {0, 0, 0};
  if (tl > 0) {
    for (int i = 0; i < 3; ++i) ut[i] = tu[i] * (ul / tl);
  }
  double vn = dot3(vrel, n);
  double vt[3] = {vrel[0] - vn * n[0], vrel[1] - vn * n[1], vrel[2] - vn * n[2]};
  double kt = gk * meff / (dt * dt);
  double ct = 2.0 * gc * sqrt(meff * kt);
  double ftr[3];
  for (int i = 0; i < 3; ++i) ftr[i] = -kt * ut[i] - ct * vt[i];
  double fl = norm3(ftr);
  if (fl <= mus * fn) { /* stick: keep the trial force */
    for (int i = 0; i < 3; ++i) {
      ft[i] = ftr[i];
      u_new[i] = ut[i] + dt * vt[i];
    }
  } else { /* slip at the dynamic bound; history matches the applied force */
    for (int i = 0; i < 3; ++i) {
      ft[i] = mud * fn * ftr[i] / fl;
      u_new[i] = -(ft[i] + ct * vt[i]) / kt;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* blade box: closest point, outward normal and sphere gap                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  double xe[3], n[3], e[3], d[3], ve[3]; /* edge point, axes, edge velocity */
  double c[3];                           /* box centre */
  double hext[3];                        /* half extents along n, e, d */
  double Iinv_w[9];                      /* world inverse inertia */
} or_frame;

static void or_make_frame(const or_scene *s, or_frame *fr) {
  const or_blade *B = &s->B;
  double t[3];
  matvec(s->R, B->edge, t);
  for (int i = 0; i < 3; ++i) fr->xe[i] = s->xB[i] + t[i];
  matvec(s->R, B->n, fr->n);
  matvec(s->R, B->e, fr->e);
  matvec(s->R, B->d, fr->d);
  double r[3] = {fr->xe[0] - s->xB[0], fr->xe[1] - s->xB[1], fr->xe[2] - s->xB[2]};
  double wr[3];
  cross3(s->wB, r, wr);
  for (int i = 0; i < 3; ++i) fr->ve[i] = s->vB[i] + wr[i];
  for (int i = 0; i < 3; ++i) fr->c[i] = fr->xe[i] - 0.5 * B->height * fr->d[i];
  fr->hext[0] = 0.5 * B->thick;
  fr->hext[1] = B->half_len;
  fr->hext[2] = 0.5 * B->height;
  memset(fr->Iinv_w, 0, sizeof fr->Iinv_w);
  if (B->mass > 0) {
    double Ib_inv[9], RT[9], tmp[9];
    inv3(B->inertia, Ib_inv);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) RT[3 * i + j] = s->R[3 * j + i];
    matmul(s->R, Ib_inv, tmp);
    matmul(tmp, RT, fr->Iinv_w);
  }
}

/* closest point x_c, outward normal nB, signed sphere-surface gap phi */
void or_box_closest(const double c[3], const double ax_n[3], const double ax_e[3],
                    const double ax_d[3], const double hext[3], const double x[3], double R,
                    double xc[3], double nB[3], double *phi) {
  const double *ax[3] = {ax_n, ax_e, ax_d};
  double r[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
  double q[3], qc[3], nl[3] = {0, 0, 0};
  int outside = 0;
  for (int a = 0; a < 3; ++a) {
    q[a] = dot3(r, ax[a]);
    if (fabs(q[a]) > hext[a]) outside = 1;
  }
  if (outside) {
    double diff[3];
    for (int a = 0; a < 3; ++a) {
      qc[a] = q[a] < -hext[a] ? -hext[a] : (q[a] > hext[a] ? hext[a] : q[a]);
      diff[a] = q[a] - qc[a];
    }
    double dist = norm3(diff);
    for (int a = 0; a < 3; ++a) nl[a] = diff[a] / dist;
    *phi = dist - R;
  } else {
    int best = 0;
    double bd = hext[0] - fabs(q[0]);
    for (int a = 1; a < 3; ++a) {
      double dd = hext[a] - fabs(q[a]);
      if (dd < bd) {
        bd = dd;
        best = a;
      }
    }
    for (int a = 0; a < 3; ++a) qc[a] = q[a];
    double sg = q[best] < 0 ? -1.0 : 1.0;
    qc[best] = sg * hext[best];
    nl[best] = sg;
    *phi = -bd - R;
  }
  for (int i = 0; i < 3; ++i) {
    xc[i] = c[i] + qc[0] * ax[0][i] + qc[1] * ax[1][i] + qc[2] * ax[2][i];
    nB[i] = nl[0] * ax[0][i] + nl[1] * ax[1][i] + nl[2] * ax[2][i];
  }
}

/* ------------------------------------------------------------------------ */
/* Eq. 3, 4, 6: blade coordinates, cutting band and side assignment.         */
/* Evaluated with separately rounded operations in a fixed order.            */
/* Returns the new digit (1 or 2) or 0 when no assignment happens.           */
/* ------------------------------------------------------------------------ */

int or_side_label(const double x[3], const double v[3], const double xe[3], const double n[3],
                  const double e[3], const double d[3], const double ve[3], double h, double L,
                  double b_back, double b_lead, double dt) {
  double r0 = x[0] - xe[0], r1 = x[1] - xe[1], r2 = x[2] - xe[2];
  double s = r0 * n[0] + r1 * n[1] + r2 * n[2];
  double l = r0 * e[0] + r1 * e[1] + r2 * e[2];
  double f = r0 * d[0] + r1 * d[1] + r2 * d[2];
  double uc = (ve[0] - v[0]) * d[0] + (ve[1] - v[1]) * d[1] + (ve[2] - v[2]) * d[2];
  double ucdt = uc * dt;
  double lowb = -b_back - (ucdt > 0.0 ? ucdt : 0.0);
  int band = fabs(s) <= h && fabs(l) <= L && lowb <= f && f <= b_lead;
  if (!band || !(f <= 0.0)) return 0;
  return s < 0.0 ? 1 : 2;
}

/* Eq. 5: one update of the cutting-progress variable */
double or_cut_progress(double D, double Jc, double uc, double Wth) {
  double nd = D + Jc * uc / Wth;
  return nd < 1.0 ? nd : 1.0;
}

/* ------------------------------------------------------------------------ */
/* scene                                                                     */
/* ------------------------------------------------------------------------ */

static void base_of(const or_scene *s, const double X[3], int b[3], double w[3][3],
                    double dw[3][3]) {
  for (int a = 0; a < 3; ++a) {
    double xl = (X[a] - s->P.origin[a]) / s->P.dx;
    b[a] = or_bspline(xl, w[a], dw[a]);
    for (int k = 0; k < 3; ++k) dw[a][k] /= s->P.dx;
  }
}

static int node_index(const or_scene *s, int i, int j, int k) {
  int a = i - s->lo[0], b = j - s->lo[1], c = k - s->lo[2];
  return (c * s->dim[1] + b) * s->dim[0] + a;
}

static or_lgrid *lgrid_find(or_node *nd, int64_t code, int create) {
  for (int a = 0; a < nd->cnt; ++a)
    if (nd->g[a].code == code) return &nd->g[a];
  if (!create) return NULL;
  if (nd->cnt == nd->cap) {
    nd->cap = nd->cap ? 2 * nd->cap : 4;
    nd->g = (or_lgrid *)realloc(nd->g, sizeof(or_lgrid) * (size_t)nd->cap);
  }
  or_lgrid *g = &nd->g[nd->cnt++];
  memset(g, 0, sizeof *g);
  g->code = code;
  return g;
}

static int64_t pcode(const or_scene *s, int64_t p, const unsigned char *dg) {
  if (s->P.single_field) return 0;
  return or_code(dg + p * OR_MAX_CUTS, OR_MAX_CUTS);
}

or_scene *or_create(const or_params *P, const or_blade *B, int64_t n, const double *X,
                    int64_t wrench_cap) {
  or_scene *s = (or_scene *)calloc(1, sizeof(or_scene));
  s->P = *P;
  if (s->P.h <= 0) s->P.h = 6.0 * P->dx;           /* h_k = 6 dx, Sec. III-D */
  if (s->P.b_back <= 0) s->P.b_back = P->dx;
  if (s->P.b_lead <= 0) s->P.b_lead = P->dx;
  s->n = n;
  s->mp = P->rho * P->V0;
  s->Rp = P->s_R * cbrt(P->V0) / 2.0; /* R_p = s_R (V0)^{1/3} / 2, Sec. III-E */
  s->mu = P->E / (2.0 * (1.0 + P->nu));
  s->lam = P->E * P->nu / ((1.0 + P->nu) * (1.0 - 2.0 * P->nu));
  size_t n3 = (size_t)n * 3;
  s->X = (double *)malloc(sizeof(double) * n3);
  s->x = (double *)malloc(sizeof(double) * n3);
  s->v = (double *)calloc(n3, sizeof(double));
  s->F = (double *)calloc((size_t)n * 9, sizeof(double));
  s->Fpi = (double *)calloc((size_t)n * 9, sizeof(double));
  s->Fdot = (double *)calloc((size_t)n * 9, sizeof(double));
  s->D = (double *)calloc((size_t)n, sizeof(double));
  s->ut = (double *)calloc(n3, sizeof(double));
  s->J = (double *)calloc(n3, sizeof(double));
  s->digit = (unsigned char *)calloc((size_t)n * OR_MAX_CUTS, 1);
  s->digit_next = (unsigned char *)calloc((size_t)n * OR_MAX_CUTS, 1);
  s->hist = (or_hist *)calloc((size_t)n * OR_HIST, sizeof(or_hist));
  s->hist_next = (or_hist *)calloc((size_t)n * OR_HIST, sizeof(or_hist));
  s->hist_cnt = (int *)calloc((size_t)n, sizeof(int));
  s->hist_cnt_next = (int *)calloc((size_t)n, sizeof(int));
  memcpy(s->X, X, sizeof(double) * n3);
  memcpy(s->x, X, sizeof(double) * n3);
  for (int64_t p = 0; p < n; ++p) {
    s->F[9 * p] = s->F[9 * p + 4] = s->F[9 * p + 8] = 1.0;
    s->Fpi[9 * p] = s->Fpi[9 * p + 4] = s->Fpi[9 * p + 8] = 1.0;
  }
  /* node range covering every particle's stencil */
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, X + 3 * p, b, w, dw);
    for (int a = 0; a < 3; ++a) {
      if (b[a] < lo[a]) lo[a] = b[a];
      if (b[a] + 2 > hi[a]) hi[a] = b[a] + 2;
    }
  }
  for (int a = 0; a < 3; ++a) {
    s->lo[a] = n > 0 ? lo[a] : 0;
    s->dim[a] = n > 0 ? hi[a] - lo[a] + 1 : 1;
  }
  size_t nn = (size_t)s->dim[0] * s->dim[1] * s->dim[2];
  s->nodes = (or_node *)calloc(nn, sizeof(or_node));
  s->cur_cut = -1;
  s->wrench_cap = wrench_cap;
  s->wrench_hist = (double *)calloc((size_t)(wrench_cap > 0 ? wrench_cap : 1) * 6, sizeof(double));
  if (B) {
    s->B = *B;
    s->has_blade = 1;
    if (s->B.rigid_interval < 1) s->B.rigid_interval = 1;
    if (s->B.kv <= 0) s->B.kv = 1.0 / (10.0 * P->dt);
    memcpy(s->xB, B->x0, sizeof s->xB);
    memcpy(s->R, B->R0, sizeof s->R);
  }
  return s;
}

void or_destroy(or_scene *s) {
  if (!s) return;
  size_t nn = (size_t)s->dim[0] * s->dim[1] * s->dim[2];
  for (size_t i = 0; i < nn; ++i) free(s->nodes[i].g);
  free(s->nodes);
  free(s->X); free(s->x); free(s->v); free(s->F); free(s->D); free(s->ut); free(s->J);
  free(s->Fpi); free(s->Fdot);
  free(s->digit); free(s->digit_next);
  free(s->hist); free(s->hist_next); free(s->hist_cnt); free(s->hist_cnt_next);
  free(s->wrench_hist);
  free(s);
}

/* segment active at substep `step`; NULL when the program has ended */
static const or_seg *seg_at(const or_scene *s, int64_t step) {
  int64_t acc = 0;
  for (int i = 0; i < s->B.nseg; ++i) {
    acc += s->B.seg[i].n_steps;
    if (step < acc) return &s->B.seg[i];
  }
  return NULL;
}

/* Rodrigues rotation by the vector th (angle |th| about th/|th|) */
static void rot_exp(const double th[3], double Rm[9]) {
  double a = norm3(th);
  for (int k = 0; k < 9; ++k) Rm[k] = (k % 4 == 0) ? 1.0 : 0.0;
  if (!(a > 0)) return;
  double k0 = th[0] / a, k1 = th[1] / a, k2 = th[2] / a;
  double K[9] = {0, -k2, k1, k2, 0, -k0, -k1, k0, 0};
  double K2[9];
  matmul(K, K, K2);
  double sa = sin(a), ca = 1.0 - cos(a);
  for (int k = 0; k < 9; ++k) Rm[k] += sa * K[k] + ca * K2[k];
}

/* pair contact candidates: uniform binning of current positions */
typedef struct {
  int64_t *order;
  int64_t *start;
  int nb[3];
  double lo[3], cell;
} or_bins;

static void pair_contact(or_scene *s) {
  int64_t n = s->n;
  double R2 = 2.0 * s->Rp;
  double vmax = 0;
  for (int64_t p = 0; p < n; ++p) {
    double vv = norm3(s->v + 3 * p);
    if (vv > vmax) vmax = vv;
  }
  double cell = R2 + 2.0 * vmax * s->P.dt + 1e-12;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t p = 0; p < n; ++p)
    for (int a = 0; a < 3; ++a) {
      if (s->x[3 * p + a] < lo[a]) lo[a] = s->x[3 * p + a];
      if (s->x[3 * p + a] > hi[a]) hi[a] = s->x[3 * p + a];
    }
  int nb[3];
  for (int a = 0; a < 3; ++a) {
    nb[a] = (int)floor((hi[a] - lo[a]) / cell) + 1;
    if (nb[a] < 1) nb[a] = 1;
  }
  int64_t ncell = (int64_t)nb[0] * nb[1] * nb[2];
  int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t p = 0; p < n; ++p) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = (int)floor((s->x[3 * p + a] - lo[a]) / cell);
      if (c[a] >= nb[a]) c[a] = nb[a] - 1;
    }
    cid[p] = ((int64_t)c[2] * nb[1] + c[1]) * nb[0] + c[0];
    cnt[cid[p] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
  int64_t *fill = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t p = 0; p < n; ++p) order[cnt[cid[p]] + fill[cid[p]]++] = p;

  double meff = s->mp * s->mp / (s->mp + s->mp);
  double dt = s->P.dt;
  for (int64_t p = 0; p < n; ++p) s->hist_cnt_next[p] = 0;
  for (int64_t p = 0; p < n; ++p) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = (int)floor((s->x[3 * p + a] - lo[a]) / cell);
      if (c[a] >= nb[a]) c[a] = nb[a] - 1;
    }
    int bp[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, bp, w, dw);
    int64_t cp = or_code(s->digit + p * OR_MAX_CUTS, OR_MAX_CUTS);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dxx = -1; dxx <= 1; ++dxx) {
          int cc[3] = {c[0] + dxx, c[1] + dy, c[2] + dz};
          if (cc[0] < 0 || cc[1] < 0 || cc[2] < 0 || cc[0] >= nb[0] || cc[1] >= nb[1] ||
              cc[2] >= nb[2])
            continue;
          int64_t ci = ((int64_t)cc[2] * nb[1] + cc[1]) * nb[0] + cc[0];
          for (int64_t t = cnt[ci]; t < cnt[ci + 1]; ++t) {
            int64_t q = order[t];
            if (q <= p) continue; /* each pair once, owned by the lower index */
            double dxv[3] = {s->x[3 * p] - s->x[3 * q], s->x[3 * p + 1] - s->x[3 * q + 1],
                             s->x[3 * p + 2] - s->x[3 * q + 2]};
            double dist = norm3(dxv);
            if (!(dist > 0)) continue;
            double npq[3] = {dxv[0] / dist, dxv[1] / dist, dxv[2] / dist};
            double vrel[3] = {s->v[3 * p] - s->v[3 * q], s->v[3 * p + 1] - s->v[3 * q + 1],
                              s->v[3 * p + 2] - s->v[3 * q + 2]};
            double vn = dot3(vrel, npq);
            /* Eq. 10: predicted overlap */
            double dhat = R2 - (dist + (dt * vn < 0 ? dt * vn : 0.0));
            if (!(dhat > 0)) continue;
            /* self-contact exclusion: reference stencils share a node and the
               codes are compatible */
            int bq[3];
            double wq[3][3], dwq[3][3];
            base_of(s, s->X + 3 * q, bq, wq, dwq);
            int share = abs(bp[0] - bq[0]) <= 2 && abs(bp[1] - bq[1]) <= 2 &&
                        abs(bp[2] - bq[2]) <= 2;
            int64_t cq = or_code(s->digit + q * OR_MAX_CUTS, OR_MAX_CUTS);
            if (share && !or_conflict(cp, cq)) continue;
            /* Eq. 11: normal force */
            double fn = s->P.s_n * meff / (dt * dt) * dhat;
            /* Eq. 12 with the pair history owned by p */
            double uh[3] = {0, 0, 0};
            for (int k = 0; k < s->hist_cnt[p]; ++k)
              if (s->hist[p * OR_HIST + k].partner == q) {
                memcpy(uh, s->hist[p * OR_HIST + k].u, sizeof uh);
                break;
              }
            double ft[3], un[3];
            or_friction(uh, npq, vrel, fn, meff, dt, s->P.gamma_k, s->P.gamma_c,
                        s->P.pair_mu_s, s->P.pair_mu_d, ft, un);
            double Jpq[3];
            for (int i = 0; i < 3; ++i) Jpq[i] = dt * (fn * npq[i] + ft[i]);
            /* Eq. 13: equal and opposite impulses */
            for (int i = 0; i < 3; ++i) {
              s->J[3 * p + i] += Jpq[i];
              s->J[3 * q + i] -= Jpq[i];
            }
            int hc = s->hist_cnt_next[p];
            if (hc < OR_HIST) {
              s->hist_next[p * OR_HIST + hc].partner = q;
              memcpy(s->hist_next[p * OR_HIST + hc].u, un, sizeof un);
              s->hist_cnt_next[p] = hc + 1;
            } else {
              s->err |= OR_E_HIST_OVERFLOW;
            }
          }
        }
  }
  free(cnt); free(cid); free(fill); free(order);
  /* swap history buffers */
  or_hist *th = s->hist; s->hist = s->hist_next; s->hist_next = th;
  int *tc = s->hist_cnt; s->hist_cnt = s->hist_cnt_next; s->hist_cnt_next = tc;
}

static void clear_grid(or_scene *s) {
  size_t nn = (size_t)s->dim[0] * s->dim[1] * s->dim[2];
  for (size_t i = 0; i < nn; ++i) s->nodes[i].cnt = 0;
}

/* one TLMPM substep */
static void substep(or_scene *s) {
  const or_params *P = &s->P;
  int64_t n = s->n;
  double dt = P->dt, mp = s->mp, V0 = P->V0;
  const or_seg *sg = s->has_blade ? seg_at(s, s->step) : NULL;
  int cut = sg ? sg->cut_id : -1;
  or_frame fr;
  memset(&fr, 0, sizeof fr);

  if (s->has_blade) {
    int dynamic = s->B.mass > 0;
    if (!dynamic && sg) { /* prescribed twist of the current segment; with no
                             segment left the last (or externally set) twist holds */
      for (int i = 0; i < 3; ++i) {
        s->vB[i] = sg->v[i];
        s->wB[i] = sg->w[i];
      }
    }
    /* D_p is reset to zero at the beginning of each new cut (Sec. III-A) */
    int started = cut >= 0 && cut != s->cur_cut;
    if (started) {
      for (int64_t p = 0; p < n; ++p) s->D[p] = 0.0;
      s->cur_cut = cut;
    }
    or_make_frame(s, &fr);
    if (started) {
      for (int i = 0; i < 3; ++i) s->cutpl[cut][i] = fr.n[i];
      s->cutpl[cut][3] = dot3(fr.n, fr.xe);
      s->cutpl_set |= 1u << cut;
    }
  }
  double Wth = P->Gc * pow(V0, 2.0 / 3.0) * (1.0 - P->zeta) / P->zeta; /* Eq. 5 */

  memcpy(s->digit_next, s->digit, (size_t)n * OR_MAX_CUTS);
  double Fsum[3] = {0, 0, 0}, Tsum[3] = {0, 0, 0};

  for (int64_t p = 0; p < n; ++p) {
    double *xp = s->x + 3 * p, *vp = s->v + 3 * p;
    double Jp[3] = {0, 0, 0};
    /* --- tool-material contact, Eq. 14-15 with Eq. 12 friction --- */
    if (s->has_blade && P->tool_contact_on) {
      double xc[3], nB[3], phi;
      or_box_closest(fr.c, fr.n, fr.e, fr.d, fr.hext, xp, s->Rp, xc, nB, &phi);
      double rc[3] = {xc[0] - s->xB[0], xc[1] - s->xB[1], xc[2] - s->xB[2]};
      double wr[3];
      cross3(s->wB, rc, wr);
      double vrel[3] = {vp[0] - (s->vB[0] + wr[0]), vp[1] - (s->vB[1] + wr[1]),
                        vp[2] - (s->vB[2] + wr[2])};
      double vn = dot3(vrel, nB);
      double phihat = phi + dt * (vn < 0 ? vn : 0.0);
      double wB = 0;
      if (s->B.mass > 0) {
        double rn[3], t[3];
        cross3(rc, nB, rn);
        matvec(fr.Iinv_w, rn, t);
        wB = 1.0 / s->B.mass + dot3(rn, t);
      }
      double meff = 1.0 / (1.0 / mp + wB);
      double Jn = P->s_n * meff / dt * (phihat < 0 ? -phihat : 0.0); /* Eq. 15 */
      double JpB[3] = {0, 0, 0};
      double *uh = s->ut + 3 * p;
      if (Jn > 0) {
        double ft[3], un[3];
        or_friction(uh, nB, vrel, Jn / dt, meff, dt, P->gamma_k, P->gamma_c, s->B.mu_s,
                    s->B.mu_d, ft, un);
        for (int i = 0; i < 3; ++i) {
          JpB[i] = Jn * nB[i] + dt * ft[i];
          uh[i] = un[i];
        }
        /* --- cutting resistance, Eq. 5 (front band, cut advancing) --- */
        if (cut >= 0) {
          double r[3] = {xp[0] - fr.xe[0], xp[1] - fr.xe[1], xp[2] - fr.xe[2]};
          double sp = dot3(r, fr.n), lp = dot3(r, fr.e), fp = dot3(r, fr.d);
          double dv[3] = {fr.ve[0] - vp[0], fr.ve[1] - vp[1], fr.ve[2] - vp[2]};
          double uc = dot3(dv, fr.d);
          int front = fabs(sp) <= P->h && fabs(lp) <= s->B.half_len && fp >= 0.0 &&
                      fp <= P->b_lead && uc > P->u_min;
          if (front) {
            double Jd = dot3(JpB, fr.d);
            double Jc = Jd > 0 ? Jd : 0.0;
            if (s->D[p] < 1.0) {
              s->D[p] = or_cut_progress(s->D[p], Jc, uc, Wth);
            } else { /* resistance released once D = 1 */
              for (int i = 0; i < 3; ++i) JpB[i] -= Jc * fr.d[i];
            }
          }
        }
      } else {
        uh[0] = uh[1] = uh[2] = 0.0;
      }
      /* --- reaction on the tool, Eq. 16 --- */
      double FB[3] = {-JpB[0] / dt, -JpB[1] / dt, -JpB[2] / dt};
      double tq[3];
      cross3(rc, FB, tq);
      for (int i = 0; i < 3; ++i) {
        Fsum[i] += FB[i];
        Tsum[i] += tq[i];
        Jp[i] += JpB[i];
      }
    }
    /* --- frictionless floor: Eq. 15 with w_B = 0 --- */
    if (P->floor_on) {
      double phi = xp[2] - P->floor_z - s->Rp;
      double vn = vp[2];
      double phihat = phi + dt * (vn < 0 ? vn : 0.0);
      double Jn = P->s_n * mp / dt * (phihat < 0 ? -phihat : 0.0);
      Jp[2] += Jn;
    }
    for (int i = 0; i < 3; ++i) s->J[3 * p + i] = Jp[i];
    /* --- side labels for the next substep, Eq. 3, 4, 6 --- */
    if (cut >= 0 && s->digit[p * OR_MAX_CUTS + cut] == 0) {
      int dnew = or_side_label(xp, vp, fr.xe, fr.n, fr.e, fr.d, fr.ve, P->h, s->B.half_len,
                               P->b_back, P->b_lead, dt);
      if (dnew) s->digit_next[p * OR_MAX_CUTS + cut] = (unsigned char)dnew;
    }
  }
  /* --- material-material contact, Eq. 10-13 --- */
  if (P->pair_on) pair_contact(s);

  /* --- P2G per logical grid, Eq. 2 (+ impulses, Eq. 13 and 16) --- */
  clear_grid(s);
  s->impulse_sum[0] = s->impulse_sum[1] = s->impulse_sum[2] = 0;
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    double Pk[9];
    if (or_particle_stress(s, p, Pk)) s->err |= OR_E_INVERTED;
    int64_t c = pcode(s, p, s->digit);
    double Jb[3];
    for (int i = 0; i < 3; ++i) {
      Jb[i] = s->J[3 * p + i] + mp * P->g[i] * dt;
      s->impulse_sum[i] += Jb[i];
    }
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double N = w[0][i] * w[1][j] * w[2][k];
          double gN[3] = {dw[0][i] * w[1][j] * w[2][k], w[0][i] * dw[1][j] * w[2][k],
                          w[0][i] * w[1][j] * dw[2][k]};
          or_lgrid *g = lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 1);
          g->m += N * mp;
          for (int a = 0; a < 3; ++a) {
            double PgN = Pk[3 * a] * gN[0] + Pk[3 * a + 1] * gN[1] + Pk[3 * a + 2] * gN[2];
            g->p[a] += N * mp * s->v[3 * p + a];
            g->dp[a] += -dt * V0 * PgN + N * Jb[a];
          }
        }
  }
  /* --- coupling (Eq. 8) and grid update (Eq. 9) --- */
  size_t nn = (size_t)s->dim[0] * s->dim[1] * s->dim[2];
  for (size_t i = 0; i < nn; ++i) {
    or_node *nd = &s->nodes[i];
    int ns = nd->cnt;
    if (ns == 0) continue;
    int64_t *codes = (int64_t *)malloc(sizeof(int64_t) * ns);
    double *m = (double *)malloc(sizeof(double) * ns);
    double *S = (double *)malloc(sizeof(double) * ns * 6);
    for (int a = 0; a < ns; ++a) {
      codes[a] = nd->g[a].code;
      m[a] = nd->g[a].m;
      for (int c = 0; c < 3; ++c) {
        S[a * 6 + c] = nd->g[a].p[c];
        S[a * 6 + 3 + c] = nd->g[a].dp[c];
      }
    }
    or_couple(ns, codes, m, 6, S);
    for (int a = 0; a < ns; ++a) {
      or_lgrid *g = &nd->g[a];
      for (int c = 0; c < 3; ++c) {
        double pb = S[a * 6 + c], dpb = S[a * 6 + 3 + c];
        g->vold[c] = g->m > 0 ? pb / g->m : 0.0;
        g->vnew[c] = g->m > 0 ? (pb + dpb) / g->m : 0.0;
        g->p[c] = pb;   /* keep the coupled state for Eq. 17 */
        g->dp[c] = dpb;
      }
    }
    free(codes); free(m); free(S);
  }
  /* --- G2P, Eq. 17, and position update --- */
  double beta = P->beta;
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    double vn[3] = {beta * s->v[3 * p], beta * s->v[3 * p + 1], beta * s->v[3 * p + 2]};
    double dxp[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double N = w[0][i] * w[1][j] * w[2][k];
          or_lgrid *g =
              lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 0);
          if (!g || !(g->m > 0)) continue;
          for (int a = 0; a < 3; ++a) {
            vn[a] += N / g->m * ((1.0 - beta) * g->p[a] + g->dp[a]);
            dxp[a] += N * g->vnew[a];
          }
        }
    for (int a = 0; a < 3; ++a) {
      s->v[3 * p + a] = vn[a];
      s->x[3 * p + a] += dt * dxp[a];
    }
  }
  /* --- MUSL re-scatter of m v^{n+1} per logical grid, with coupling --- */
  for (size_t i = 0; i < nn; ++i)
    for (int a = 0; a < s->nodes[i].cnt; ++a)
      memset(s->nodes[i].g[a].pstar, 0, sizeof(double) * 3);
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double N = w[0][i] * w[1][j] * w[2][k];
          or_lgrid *g =
              lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 0);
          for (int a = 0; a < 3; ++a) g->pstar[a] += N * mp * s->v[3 * p + a];
        }
  }
  for (size_t i = 0; i < nn; ++i) {
    or_node *nd = &s->nodes[i];
    int ns = nd->cnt;
    if (ns == 0) continue;
    int64_t *codes = (int64_t *)malloc(sizeof(int64_t) * ns);
    double *m = (double *)malloc(sizeof(double) * ns);
    double *S = (double *)malloc(sizeof(double) * ns * 3);
    for (int a = 0; a < ns; ++a) {
      codes[a] = nd->g[a].code;
      m[a] = nd->g[a].m;
      for (int c = 0; c < 3; ++c) S[a * 3 + c] = nd->g[a].pstar[c];
    }
    or_couple(ns, codes, m, 3, S);
    for (int a = 0; a < ns; ++a)
      for (int c = 0; c < 3; ++c)
        nd->g[a].vstar[c] = nd->g[a].m > 0 ? S[a * 3 + c] / nd->g[a].m : 0.0;
    free(codes); free(m); free(S);
  }
  /* --- deformation gradient, F += dt sum_i v*_i (x) grad0 N_ip --- */
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    double G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double gN[3] = {dw[0][i] * w[1][j] * w[2][k], w[0][i] * dw[1][j] * w[2][k],
                          w[0][i] * w[1][j] * dw[2][k]};
          or_lgrid *g =
              lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 0);
          for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) G[3 * a + d] += g->vstar[a] * gN[d];
        }
    for (int k = 0; k < 9; ++k) {
      s->F[9 * p + k] += dt * G[k];
      s->Fdot[9 * p + k] = G[k];
    }
    for (int a = 0; a < 3; ++a)
      if (!isfinite(s->x[3 * p + a]) || !isfinite(s->v[3 * p + a])) s->err |= OR_E_NONFINITE;
  }
  /* --- commit the codes assigned this substep (Sec. III-C) --- */
  unsigned char *t = s->digit;
  s->digit = s->digit_next;
  s->digit_next = t;

  /* --- wrench and rigid tool update at the rigid interval (Sec. III-G) --- */
  if (s->has_blade) {
    int64_t st = s->step;
    if (st < s->wrench_cap) {
      for (int i = 0; i < 3; ++i) {
        s->wrench_hist[6 * st + i] = Fsum[i];
        s->wrench_hist[6 * st + 3 + i] = Tsum[i];
      }
    }
    for (int i = 0; i < 3; ++i) {
      s->accF[i] += Fsum[i];
      s->accT[i] += Tsum[i];
    }
    s->acc_cnt++;
    if (s->acc_cnt >= s->B.rigid_interval) {
      double H = dt * s->acc_cnt;
      double Fa[3], Ta[3];
      for (int i = 0; i < 3; ++i) {
        Fa[i] = s->accF[i] / s->acc_cnt;
        Ta[i] = s->accT[i] / s->acc_cnt;
      }
      if (s->B.mass > 0) {
        const or_seg *tg = sg;
        double vt[3] = {0, 0, 0}, wt[3] = {0, 0, 0};
        if (tg)
          for (int i = 0; i < 3; ++i) {
            vt[i] = tg->v[i];
            wt[i] = tg->w[i];
          }
        double kv = s->B.kv;
        /* velocity servo toward the segment twist + interval-averaged reaction */
        double dw_[3];
        matvec(fr.Iinv_w, Ta, dw_);
        for (int i = 0; i < 3; ++i) {
          s->vB[i] += H * (kv * (vt[i] - s->vB[i]) + Fa[i] / s->B.mass);
          s->wB[i] += H * (kv * (wt[i] - s->wB[i]) + dw_[i]);
        }
      }
      double th[3] = {H * s->wB[0], H * s->wB[1], H * s->wB[2]};
      double Rinc[9], Rn[9];
      rot_exp(th, Rinc);
      matmul(Rinc, s->R, Rn);
      memcpy(s->R, Rn, sizeof Rn);
      for (int i = 0; i < 3; ++i) s->xB[i] += H * s->vB[i];
      for (int i = 0; i < 3; ++i) {
        s->lastF[i] = Fa[i];
        s->lastF[3 + i] = Ta[i];
        s->accF[i] = s->accT[i] = 0;
      }
      s->acc_cnt = 0;
    }
  }
  s->step++;
}

int or_step(or_scene *s, int nsteps) {
  for (int k = 0; k < nsteps; ++k) substep(s);
  return (int)s->err;
}

/* ------------------------------------------------------------------------ */
/* state access                                                              */
/* ------------------------------------------------------------------------ */
/* field ids: 0 X, 1 x, 2 v, 3 F, 4 D, 5 ut, 6 code (as double), 7 J, 8 digits (n*32),
   9 pair-contact history (n * OR_HIST entries of {partner or -1, u[3]}; the
   pair list of particle p holds the pairs it owns, i.e. partners q > p) */

int or_get(const or_scene *s, int field, double *out) {
  int64_t n = s->n;
  switch (field) {
    case 0: memcpy(out, s->X, sizeof(double) * n * 3); return 0;
    case 1: memcpy(out, s->x, sizeof(double) * n * 3); return 0;
    case 2: memcpy(out, s->v, sizeof(double) * n * 3); return 0;
    case 3: memcpy(out, s->F, sizeof(double) * n * 9); return 0;
    case 4: memcpy(out, s->D, sizeof(double) * n); return 0;
    case 5: memcpy(out, s->ut, sizeof(double) * n * 3); return 0;
    case 6:
      for (int64_t p = 0; p < n; ++p) out[p] = (double)or_code(s->digit + p * OR_MAX_CUTS, OR_MAX_CUTS);
      return 0;
    case 7: memcpy(out, s->J, sizeof(double) * n * 3); return 0;
    case 8:
      for (int64_t p = 0; p < n * OR_MAX_CUTS; ++p) out[p] = s->digit[p];
      return 0;
    case 9:
      for (int64_t p = 0; p < n; ++p)
        for (int k = 0; k < OR_HIST; ++k) {
          double *o = out + (p * OR_HIST + k) * 4;
          if (k < s->hist_cnt[p]) {
            o[0] = (double)s->hist[p * OR_HIST + k].partner;
            memcpy(o + 1, s->hist[p * OR_HIST + k].u, sizeof(double) * 3);
          } else {
            o[0] = -1.0;
            o[1] = o[2] = o[3] = 0.0;
          }
        }
      return 0;
  }
  return -1;
}

int or_set(or_scene *s, int field, const double *in) {
  int64_t n = s->n;
  switch (field) {
    case 1: memcpy(s->x, in, sizeof(double) * n * 3); return 0;
    case 2: memcpy(s->v, in, sizeof(double) * n * 3); return 0;
    case 3: memcpy(s->F, in, sizeof(double) * n * 9); return 0;
    case 4: memcpy(s->D, in, sizeof(double) * n); return 0;
    case 5: memcpy(s->ut, in, sizeof(double) * n * 3); return 0;
    case 8:
      for (int64_t p = 0; p < n * OR_MAX_CUTS; ++p) s->digit[p] = (unsigned char)in[p];
      return 0;
    case 9:
      for (int64_t p = 0; p < n; ++p) {
        int c = 0;
        for (int k = 0; k < OR_HIST; ++k) {
          const double *e = in + (p * OR_HIST + k) * 4;
          if (e[0] < 0) break;
          s->hist[p * OR_HIST + c].partner = (int64_t)e[0];
          memcpy(s->hist[p * OR_HIST + c].u, e + 1, sizeof(double) * 3);
          ++c;
        }
        s->hist_cnt[p] = c;
      }
      return 0;
  }
  return -1;
}

/* substep counter and the cut in progress (to continue from a state that
   was copied in from elsewhere) */
void or_set_step(or_scene *s, int64_t step, int cur_cut) {
  s->step = step;
  s->cur_cut = cur_cut;
}

/* tool state: xB[3], R[9], vB[3], wB[3] */
void or_get_tool(const or_scene *s, double out[18]) {
  memcpy(out, s->xB, sizeof(double) * 3);
  memcpy(out + 3, s->R, sizeof(double) * 9);
  memcpy(out + 12, s->vB, sizeof(double) * 3);
  memcpy(out + 15, s->wB, sizeof(double) * 3);
}
void or_set_tool(or_scene *s, const double in[18]) {
  memcpy(s->xB, in, sizeof(double) * 3);
  memcpy(s->R, in + 3, sizeof(double) * 9);
  memcpy(s->vB, in + 12, sizeof(double) * 3);
  memcpy(s->wB, in + 15, sizeof(double) * 3);
}
/* blade frame at the current state: xe, n, e, d, ve (15 doubles) */
void or_get_frame(const or_scene *s, double out[15]) {
  or_frame fr;
  or_make_frame(s, &fr);
  memcpy(out, fr.xe, 24); memcpy(out + 3, fr.n, 24); memcpy(out + 6, fr.e, 24);
  memcpy(out + 9, fr.d, 24); memcpy(out + 12, fr.ve, 24);
}

int64_t or_step_count(const or_scene *s) { return s->step; }
unsigned or_errors(const or_scene *s) { return s->err; }

/* recorded cut planes: out[k * 4 + 0..3] = (n, n . x_e) of cut k; returns the
   mask of recorded cuts */
unsigned or_cut_planes(const or_scene *s, double *out) {
  memcpy(out, s->cutpl, sizeof s->cutpl);
  return s->cutpl_set;
}
void or_impulse_sum(const or_scene *s, double out[3]) { memcpy(out, s->impulse_sum, 24); }
void or_last_wrench(const or_scene *s, double out[6]) { memcpy(out, s->lastF, 48); }
int or_wrench_history(const or_scene *s, int64_t first, int64_t count, double *out) {
  if (first < 0 || first + count > s->wrench_cap) return -1;
  memcpy(out, s->wrench_hist + 6 * first, sizeof(double) * 6 * count);
  return 0;
}
void or_grid_dims(const or_scene *s, int lo[3], int dim[3]) {
  memcpy(lo, s->lo, sizeof(int) * 3);
  memcpy(dim, s->dim, sizeof(int) * 3);
}
/* number of logical grids (occupied code slots) after the last P2G */
int64_t or_slot_count(const or_scene *s) {
  size_t nn = (size_t)s->dim[0] * s->dim[1] * s->dim[2];
  int64_t c = 0;
  for (size_t i = 0; i < nn; ++i) c += s->nodes[i].cnt;
  return c;
}
/* momentum sum_p m_p v_p */
void or_momentum(const or_scene *s, double out[3]) {
  out[0] = out[1] = out[2] = 0;
  for (int64_t p = 0; p < s->n; ++p)
    for (int a = 0; a < 3; ++a) out[a] += s->mp * s->v[3 * p + a];
}

/* ======================================================================== */
/* Adjoint of one substep (reverse mode), for calibration of E, nu and the  */
/* blade velocity from reaction-force trajectories.                         */
/*                                                                          */
/* The substep is differentiated with every discrete decision of the       */
/* forward substep held fixed: the codes (side labels), the contact active  */
/* sets (Jn > 0 for the blade and the floor), the sign test of the normal   */
/* velocity in phi_hat, stick or slip (Eq. 12), the front band and the D    */
/* release (Eq. 5), and the face / clamp pattern of the box closest point.  */
/* D itself enters only through those decisions and carries no adjoint.     */
/* Scope: a kinematic blade that translates (no angular velocity), rigid    */
/* interval 1, no material-material contact.                                */
/*                                                                          */
/* Given the scene at the state before substep n and the adjoints of the    */
/* state after it (x, v, F, u_t), plus dL/dF_B^n of this substep's          */
/* reaction force (Eq. 16), or_adj_substep replaces the state adjoints by   */
/* those of the state before the substep and accumulates dL/dmu,            */
/* dL/dlambda, and the adjoints of the tool position and segment velocity.  */
/* ======================================================================== */

typedef struct {
  int64_t n;
  double *xb, *vb, *Fb, *ub;  /* adjoints of x, v, F, u_t (n x 3, 3, 9, 3) */
  double mub, lamb;           /* dL/dmu, dL/dlambda */
  double xBb[3];              /* adjoint of the tool position at the current state */
  double vsegb[OR_MAX_SEG][3];/* dL/d(segment linear velocity) */
} or_adj;

or_adj *or_adj_create(int64_t n) {
  or_adj *a = (or_adj *)calloc(1, sizeof(or_adj));
  a->n = n;
  a->xb = (double *)calloc((size_t)n * 3, sizeof(double));
  a->vb = (double *)calloc((size_t)n * 3, sizeof(double));
  a->Fb = (double *)calloc((size_t)n * 9, sizeof(double));
  a->ub = (double *)calloc((size_t)n * 3, sizeof(double));
  return a;
}

void or_adj_destroy(or_adj *a) {
  if (!a) return;
  free(a->xb); free(a->vb); free(a->Fb); free(a->ub);
  free(a);
}

/* 0: x, 1: v, 2: F, 3: u_t, 4: tool position (3) */
double *or_adj_field(or_adj *a, int which) {
  switch (which) {
    case 0: return a->xb;
    case 1: return a->vb;
    case 2: return a->Fb;
    case 3: return a->ub;
    case 4: return a->xBb;
  }
  return NULL;
}

/* out: dL/dE, dL/dnu, dL/dmu, dL/dlambda, tool-position adjoint (3), then
   the segment velocity adjoints (OR_MAX_SEG x 3) */
void or_adj_theta(const or_adj *a, const or_scene *s, double *out) {
  double E = s->P.E, nu = s->P.nu;
  double Dn = (1.0 + nu) * (1.0 - 2.0 * nu);
  double dmu_dE = 1.0 / (2.0 * (1.0 + nu)), dmu_dnu = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
  double dlam_dE = nu / Dn, dlam_dnu = E * (1.0 + 2.0 * nu * nu) / (Dn * Dn);
  out[0] = a->mub * dmu_dE + a->lamb * dlam_dE;
  out[1] = a->mub * dmu_dnu + a->lamb * dlam_dnu;
  out[2] = a->mub;
  out[3] = a->lamb;
  memcpy(out + 4, a->xBb, sizeof(double) * 3);
  memcpy(out + 7, a->vsegb, sizeof(double) * 3 * OR_MAX_SEG);
}

/* deep copy (a checkpoint); the grid is scratch and starts empty */
or_scene *or_clone(const or_scene *s) {
  or_scene *t = (or_scene *)malloc(sizeof(or_scene));
  *t = *s;
  size_t n = (size_t)s->n, n3 = n * 3;
#define OR_DUP(f, cnt)                                      \
  t->f = malloc(sizeof(*s->f) * (cnt) > 0 ? sizeof(*s->f) * (cnt) : 1); \
  memcpy(t->f, s->f, sizeof(*s->f) * (cnt))
  OR_DUP(X, n3); OR_DUP(x, n3); OR_DUP(v, n3); OR_DUP(F, n * 9); OR_DUP(D, n);
  OR_DUP(Fpi, n * 9); OR_DUP(Fdot, n * 9);
  OR_DUP(ut, n3); OR_DUP(J, n3);
  OR_DUP(digit, n * OR_MAX_CUTS); OR_DUP(digit_next, n * OR_MAX_CUTS);
  OR_DUP(hist, n * OR_HIST); OR_DUP(hist_next, n * OR_HIST);
  OR_DUP(hist_cnt, n); OR_DUP(hist_cnt_next, n);
  OR_DUP(wrench_hist, (size_t)(s->wrench_cap > 0 ? s->wrench_cap : 1) * 6);
#undef OR_DUP
  size_t nn = (size_t)s->dim[0] * s->dim[1] * s->dim[2];
  t->nodes = (or_node *)calloc(nn, sizeof(or_node));
  return t;
}

/* dP^T[Pb] of the neo-Hookean stress: Fb += ..., mub/lamb += ... */
void or_piola_vjp(const double F[9], double mu, double lam, const double Pb[9], double Fb[9],
                      double *mub, double *lamb) {
  double c[9];
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
  double J = det3(F);
  if (!(J > OR_JMIN)) J = OR_JMIN; /* clamped elements are flagged by the forward step */
  double G[9];                     /* F^{-T} */
  for (int k = 0; k < 9; ++k) G[k] = c[k] / J;
  double lj = log(J);
  /* P = mu F + (lam ln J - mu) G, dG = -G dF^T G, d ln J = G : dF */
  double PG = 0, PF = 0;
  for (int k = 0; k < 9; ++k) {
    PG += Pb[k] * G[k];
    PF += Pb[k] * F[k];
  }
  double GPtG[9]; /* (G Pb^T G)_lk = sum_ij G_lj Pb_ij G_ik */
  for (int l = 0; l < 3; ++l)
    for (int k = 0; k < 3; ++k) {
      double acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += G[3 * l + j] * Pb[3 * i + j] * G[3 * i + k];
      GPtG[3 * l + k] = acc;
    }
  for (int k = 0; k < 9; ++k) Fb[k] += mu * Pb[k] - (lam * lj - mu) * GPtG[k] + lam * PG * G[k];
  *mub += PF - PG;
  *lamb += lj * PG;
}

/* (C^T S)^b = S^b + 1/M sum_{a != b, compatible} m^a (S^a - S^b): the
   transpose of the linear map of Eq. 8 (masses and codes fixed) */
void or_couple_T(int ns, const int64_t *codes, const double *m, int nc, double *S) {
  double M = 0;
  for (int a = 0; a < ns; ++a) M += m[a];
  if (!(M > 0)) return;
  double *out = (double *)malloc(sizeof(double) * (size_t)ns * (size_t)nc);
  for (int b = 0; b < ns; ++b)
    for (int c = 0; c < nc; ++c) {
      double acc = 0;
      for (int a = 0; a < ns; ++a) {
        if (a == b || or_conflict(codes[a], codes[b])) continue;
        acc += m[a] * (S[a * nc + c] - S[b * nc + c]);
      }
      out[b * nc + c] = S[b * nc + c] + acc / M;
    }
  memcpy(S, out, sizeof(double) * (size_t)ns * (size_t)nc);
  free(out);
}

/* VJP of the blade contact of particle p (Eq. 12, 14, 15, 5 release).
   Jb: adjoint of the particle's blade impulse J_pB (after release);
   ub_new: adjoint of u_t after the substep.  Adds to xb, vb, xBb, vBb and
   writes ub_old (adjoint of u_t before the substep). */
static void contact_vjp(const or_scene *s, const or_frame *fr, int cut, int64_t p, double Dn,
                        const double Jb_in[3], const double ub_new[3], double xb[3], double vb[3],
                        double ub_old[3], double xBb[3], double vBb[3]) {
  const or_params *P = &s->P;
  const double dt = P->dt, mp = s->mp;
  const double *xp = s->x + 3 * p, *vp = s->v + 3 * p, *uh = s->ut + 3 * p;
  ub_old[0] = ub_old[1] = ub_old[2] = 0.0;
  /* --- forward recomputation --- */
  const double *ax[3] = {fr->n, fr->e, fr->d};
  double y[3] = {xp[0] - fr->c[0], xp[1] - fr->c[1], xp[2] - fr->c[2]};
  double q[3];
  int outside = 0, clampd[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) {
    q[a] = dot3(y, ax[a]);
    if (fabs(q[a]) > fr->hext[a]) outside = clampd[a] = 1;
  }
  double xc[3], nB[3], phi;
  or_box_closest(fr->c, fr->n, fr->e, fr->d, fr->hext, xp, s->Rp, xc, nB, &phi);
  double diff[3] = {0, 0, 0}, dist = 0, nl[3] = {0, 0, 0};
  int best = 0;
  double sg = 1.0;
  if (outside) {
    for (int a = 0; a < 3; ++a) {
      double qc = q[a] < -fr->hext[a] ? -fr->hext[a] : (q[a] > fr->hext[a] ? fr->hext[a] : q[a]);
      diff[a] = q[a] - qc;
    }
    dist = norm3(diff);
    for (int a = 0; a < 3; ++a) nl[a] = diff[a] / dist;
  } else {
    double bd = fr->hext[0] - fabs(q[0]);
    for (int a = 1; a < 3; ++a) {
      double dd = fr->hext[a] - fabs(q[a]);
      if (dd < bd) {
        bd = dd;
        best = a;
      }
    }
    sg = q[best] < 0 ? -1.0 : 1.0;
  }
  double vrel[3] = {vp[0] - s->vB[0], vp[1] - s->vB[1], vp[2] - s->vB[2]};
  double vn = dot3(vrel, nB);
  int neg = vn < 0;
  double phihat = phi + dt * (neg ? vn : 0.0);
  double meff = 1.0 / (1.0 / mp + 0.0);
  double kn = P->s_n * meff / dt;
  double Jn = kn * (phihat < 0 ? -phihat : 0.0);
  if (!(Jn > 0)) return; /* no contact: u_t is reset to zero, nothing flows back */
  double fn = Jn / dt;
  /* friction, Eq. 12 */
  double udn = dot3(uh, nB), ul = norm3(uh);
  double tu[3] = {uh[0] - udn * nB[0], uh[1] - udn * nB[1], uh[2] - udn * nB[2]};
  double tl = norm3(tu);
  double sc = tl > 0 ? ul / tl : 0.0;
  double ut[3] = {tu[0] * sc, tu[1] * sc, tu[2] * sc};
  double vnn = dot3(vrel, nB);
  double vt[3] = {vrel[0] - vnn * nB[0], vrel[1] - vnn * nB[1], vrel[2] - vnn * nB[2]};
  double kt = P->gamma_k * meff / (dt * dt);
  double ct = 2.0 * P->gamma_c * sqrt(meff * kt);
  double ftr[3];
  for (int i = 0; i < 3; ++i) ftr[i] = -kt * ut[i] - ct * vt[i];
  double fl = norm3(ftr);
  int stick = fl <= s->B.mu_s * fn;
  double ft[3];
  for (int i = 0; i < 3; ++i) ft[i] = stick ? ftr[i] : s->B.mu_d * fn * ftr[i] / fl;
  double JpB[3];
  for (int i = 0; i < 3; ++i) JpB[i] = Jn * nB[i] + dt * ft[i];
  int rel = 0;
  if (cut >= 0) {
    double r[3] = {xp[0] - fr->xe[0], xp[1] - fr->xe[1], xp[2] - fr->xe[2]};
    double sp = dot3(r, fr->n), lp = dot3(r, fr->e), fp = dot3(r, fr->d);
    double dv[3] = {fr->ve[0] - vp[0], fr->ve[1] - vp[1], fr->ve[2] - vp[2]};
    double uc = dot3(dv, fr->d);
    int front = fabs(sp) <= P->h && fabs(lp) <= s->B.half_len && fp >= 0.0 && fp <= P->b_lead &&
                uc > P->u_min;
    if (front && !(Dn < 1.0) && dot3(JpB, fr->d) > 0) rel = 1;
  }
  /* --- reverse --- */
  double Jb[3] = {Jb_in[0], Jb_in[1], Jb_in[2]};
  if (rel) { /* J' = (I - d d^T) J */
    double t = dot3(Jb, fr->d);
    for (int i = 0; i < 3; ++i) Jb[i] -= t * fr->d[i];
  }
  double Jnb = dot3(Jb, nB);
  double nBb[3] = {Jn * Jb[0], Jn * Jb[1], Jn * Jb[2]};
  double ftb[3] = {dt * Jb[0], dt * Jb[1], dt * Jb[2]};
  double utb[3] = {0, 0, 0}, vtb[3] = {0, 0, 0}, ftrb[3], fnb = 0;
  if (stick) { /* ft = ftr, u' = ut + dt vt */
    for (int i = 0; i < 3; ++i) {
      ftrb[i] = ftb[i];
      utb[i] += ub_new[i];
      vtb[i] += dt * ub_new[i];
    }
  } else { /* ft = mu_d fn ftr/|ftr|, u' = -(ft + ct vt)/kt */
    double g[3], hh[3], hb[3];
    for (int i = 0; i < 3; ++i) {
      g[i] = ftb[i] - ub_new[i] / kt;
      vtb[i] += -ct * ub_new[i] / kt;
      hh[i] = ftr[i] / fl;
    }
    fnb += s->B.mu_d * dot3(g, hh);
    for (int i = 0; i < 3; ++i) hb[i] = s->B.mu_d * fn * g[i];
    double t = dot3(hb, hh);
    for (int i = 0; i < 3; ++i) ftrb[i] = (hb[i] - t * hh[i]) / fl;
  }
  for (int i = 0; i < 3; ++i) { /* ftr = -kt ut - ct vt */
    utb[i] += -kt * ftrb[i];
    vtb[i] += -ct * ftrb[i];
  }
  double vrelb[3];
  { /* vt = vrel - (vrel.nB) nB */
    double t = dot3(vtb, nB);
    for (int i = 0; i < 3; ++i) {
      vrelb[i] = vtb[i] - t * nB[i];
      nBb[i] += -vnn * vtb[i] - t * vrel[i];
    }
  }
  double uhb[3] = {0, 0, 0};
  if (tl > 0) { /* ut = tu ul/tl; tu = uh - (uh.nB) nB */
    double scb = dot3(utb, tu);
    double ulb = scb / tl, tlb = -scb * ul / (tl * tl);
    double tub[3];
    for (int i = 0; i < 3; ++i) tub[i] = sc * utb[i] + tlb * tu[i] / tl;
    for (int i = 0; i < 3; ++i) uhb[i] += ulb * uh[i] / ul;
    double t = dot3(tub, nB);
    for (int i = 0; i < 3; ++i) {
      uhb[i] += tub[i] - t * nB[i];
      nBb[i] += -udn * tub[i] - t * uh[i];
    }
  }
  Jnb += fnb / dt;
  double phihatb = -kn * Jnb;
  double phib = phihatb, vnb = neg ? dt * phihatb : 0.0;
  for (int i = 0; i < 3; ++i) {
    vrelb[i] += vnb * nB[i];
    nBb[i] += vnb * vrel[i];
  }
  for (int i = 0; i < 3; ++i) {
    vb[i] += vrelb[i];
    vBb[i] -= vrelb[i];
  }
  double qb[3] = {0, 0, 0};
  if (outside) { /* nB = sum_a nl_a ax_a, nl = diff/dist, phi = dist - R */
    double nlb[3], t = 0;
    for (int a = 0; a < 3; ++a) {
      nlb[a] = dot3(nBb, ax[a]);
      t += nlb[a] * nl[a];
    }
    for (int a = 0; a < 3; ++a)
      if (clampd[a]) qb[a] = (nlb[a] - t * nl[a]) / dist + phib * nl[a];
  } else {
    qb[best] = sg * phib; /* phi = sg q_best - h_best - R; nB fixed */
  }
  for (int i = 0; i < 3; ++i) {
    double yb = qb[0] * ax[0][i] + qb[1] * ax[1][i] + qb[2] * ax[2][i];
    xb[i] += yb;
    xBb[i] -= yb; /* box centre = tool position + a fixed offset */
  }
  memcpy(ub_old, uhb, sizeof uhb);
}

int or_adj_substep(const or_scene *s0, or_adj *A, const double Fbar[3]) {
  if (s0->P.pair_on || s0->P.model != 0 || s0->P.yield_stress > 0 || s0->P.viscosity > 0) return -1;
  if (s0->has_blade) {
    if (s0->B.mass > 0 || s0->B.rigid_interval != 1) return -1;
    for (int k = 0; k < s0->B.nseg; ++k)
      if (s0->B.seg[k].w[0] != 0 || s0->B.seg[k].w[1] != 0 || s0->B.seg[k].w[2] != 0) return -1;
    if (s0->wB[0] != 0 || s0->wB[1] != 0 || s0->wB[2] != 0) return -1;
  }
  or_scene *s = or_clone(s0); /* the substep's own set-up is replayed on a copy */
  const or_params *P = &s->P;
  int64_t n = s->n;
  double dt = P->dt, mp = s->mp, V0 = P->V0, beta = P->beta;
  const or_seg *sg = s->has_blade ? seg_at(s, s->step) : NULL;
  int seg_idx = -1;
  if (s->has_blade) { /* segment whose velocity the tool carries this substep */
    int64_t acc = 0;
    for (int k = 0; k < s->B.nseg; ++k) {
      acc += s->B.seg[k].n_steps;
      if (s->step < acc) {
        seg_idx = k;
        break;
      }
    }
    if (seg_idx < 0) seg_idx = s->B.nseg - 1; /* program ended: the last twist holds */
  }
  int cut = sg ? sg->cut_id : -1;
  or_frame fr;
  memset(&fr, 0, sizeof fr);
  if (s->has_blade) {
    if (sg)
      for (int i = 0; i < 3; ++i) {
        s->vB[i] = sg->v[i];
        s->wB[i] = sg->w[i];
      }
    if (cut >= 0 && cut != s->cur_cut) {
      for (int64_t p = 0; p < n; ++p) s->D[p] = 0.0;
      s->cur_cut = cut;
    }
    or_make_frame(s, &fr);
  }
  /* logical grids and their masses (fixed by the codes) */
  clear_grid(s);
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          or_lgrid *g = lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 1);
          g->m += w[0][i] * w[1][j] * w[2][k] * mp;
        }
  }
  size_t nn = (size_t)s->dim[0] * s->dim[1] * s->dim[2];
  /* (a) F' = F + dt sum_i v*_i (x) grad0 N: adjoint of v* per logical grid (in vstar) */
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    const double *Fb = A->Fb + 9 * p;
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double gN[3] = {dw[0][i] * w[1][j] * w[2][k], w[0][i] * dw[1][j] * w[2][k],
                          w[0][i] * w[1][j] * dw[2][k]};
          or_lgrid *g = lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 0);
          for (int a = 0; a < 3; ++a)
            g->vstar[a] += dt * (Fb[3 * a] * gN[0] + Fb[3 * a + 1] * gN[1] + Fb[3 * a + 2] * gN[2]);
        }
  }
  /* (b) v* = C p* / m (coupled MUSL momentum over mass): adjoint of p* per
     logical grid (in pstar) */
  for (size_t i = 0; i < nn; ++i) {
    or_node *nd = &s->nodes[i];
    int ns = nd->cnt;
    if (ns == 0) continue;
    int64_t *codes = (int64_t *)malloc(sizeof(int64_t) * ns);
    double *m = (double *)malloc(sizeof(double) * ns);
    double *S = (double *)malloc(sizeof(double) * ns * 3);
    for (int a = 0; a < ns; ++a) {
      codes[a] = nd->g[a].code;
      m[a] = nd->g[a].m;
      for (int c = 0; c < 3; ++c) S[a * 3 + c] = nd->g[a].m > 0 ? nd->g[a].vstar[c] / nd->g[a].m : 0.0;
    }
    or_couple_T(ns, codes, m, 3, S);
    for (int a = 0; a < ns; ++a)
      for (int c = 0; c < 3; ++c) nd->g[a].pstar[c] = S[a * 3 + c];
    free(codes); free(m); free(S);
  }
  /* (c) p* = sum N m_p v'_p: adjoint of v' (the G2P velocity) */
  double *v1b = (double *)malloc(sizeof(double) * (size_t)n * 3);
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    double acc[3] = {A->vb[3 * p], A->vb[3 * p + 1], A->vb[3 * p + 2]};
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double N = w[0][i] * w[1][j] * w[2][k];
          or_lgrid *g = lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 0);
          for (int a = 0; a < 3; ++a) acc[a] += N * mp * g->pstar[a];
        }
    memcpy(v1b + 3 * p, acc, sizeof acc);
  }
  /* (d) G2P (Eq. 17) and x' = x + dt sum N vnew: adjoints of the coupled
     momentum and momentum change per logical grid (in p and dp) */
  for (size_t i = 0; i < nn; ++i)
    for (int a = 0; a < s->nodes[i].cnt; ++a) {
      memset(s->nodes[i].g[a].p, 0, sizeof(double) * 3);
      memset(s->nodes[i].g[a].dp, 0, sizeof(double) * 3);
    }
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double N = w[0][i] * w[1][j] * w[2][k];
          or_lgrid *g = lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 0);
          if (!(g->m > 0)) continue;
          for (int a = 0; a < 3; ++a) {
            g->p[a] += N / g->m * ((1.0 - beta) * v1b[3 * p + a] + dt * A->xb[3 * p + a]);
            g->dp[a] += N / g->m * (v1b[3 * p + a] + dt * A->xb[3 * p + a]);
          }
        }
  }
  for (size_t i = 0; i < nn; ++i) {
    or_node *nd = &s->nodes[i];
    int ns = nd->cnt;
    if (ns == 0) continue;
    int64_t *codes = (int64_t *)malloc(sizeof(int64_t) * ns);
    double *m = (double *)malloc(sizeof(double) * ns);
    double *S = (double *)malloc(sizeof(double) * ns * 6);
    for (int a = 0; a < ns; ++a) {
      codes[a] = nd->g[a].code;
      m[a] = nd->g[a].m;
      for (int c = 0; c < 3; ++c) {
        S[a * 6 + c] = nd->g[a].p[c];
        S[a * 6 + 3 + c] = nd->g[a].dp[c];
      }
    }
    or_couple_T(ns, codes, m, 6, S);
    for (int a = 0; a < ns; ++a)
      for (int c = 0; c < 3; ++c) {
        nd->g[a].p[c] = S[a * 6 + c];
        nd->g[a].dp[c] = S[a * 6 + 3 + c];
      }
    free(codes); free(m); free(S);
  }
  /* (e) P2G (Eq. 2), stress and contact, per particle */
  double vBb[3] = {0, 0, 0}, xBd[3] = {0, 0, 0};
  for (int64_t p = 0; p < n; ++p) {
    int b[3];
    double w[3][3], dw[3][3];
    base_of(s, s->X + 3 * p, b, w, dw);
    int64_t c = pcode(s, p, s->digit);
    double vb[3], Jbar[3] = {0, 0, 0}, Pb[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 3; ++a) vb[a] = beta * v1b[3 * p + a];
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          double N = w[0][i] * w[1][j] * w[2][k];
          double gN[3] = {dw[0][i] * w[1][j] * w[2][k], w[0][i] * dw[1][j] * w[2][k],
                          w[0][i] * w[1][j] * dw[2][k]};
          or_lgrid *g = lgrid_find(&s->nodes[node_index(s, b[0] + i, b[1] + j, b[2] + k)], c, 0);
          for (int a = 0; a < 3; ++a) {
            vb[a] += N * mp * g->p[a];
            Jbar[a] += N * g->dp[a];
            for (int d = 0; d < 3; ++d) Pb[3 * a + d] += -dt * V0 * g->dp[a] * gN[d];
          }
        }
    double *Fb = A->Fb + 9 * p; /* F' = F + ...: dF'/dF = I */
    or_piola_vjp(s->F + 9 * p, s->mu, s->lam, Pb, Fb, &A->mub, &A->lamb);
    double *xb = A->xb + 3 * p;  /* x' = x + ...: dx'/dx = I */
    double ub_new[3] = {A->ub[3 * p], A->ub[3 * p + 1], A->ub[3 * p + 2]};
    double ub_old[3] = {0, 0, 0};
    if (s->has_blade && P->tool_contact_on) {
      /* J_p = J_pB + floor; F_B^n = -sum_p J_pB / dt (Eq. 16) */
      double JbB[3] = {Jbar[0] - Fbar[0] / dt, Jbar[1] - Fbar[1] / dt, Jbar[2] - Fbar[2] / dt};
      contact_vjp(s, &fr, cut, p, s->D[p], JbB, ub_new, xb, vb, ub_old, xBd, vBb);
    }
    if (P->floor_on) {
      const double *xp = s->x + 3 * p, *vp = s->v + 3 * p;
      double phi = xp[2] - P->floor_z - s->Rp;
      int neg = vp[2] < 0;
      double phihat = phi + dt * (neg ? vp[2] : 0.0);
      double kn = P->s_n * mp / dt;
      if (kn * (phihat < 0 ? -phihat : 0.0) > 0) {
        double phihatb = -kn * Jbar[2];
        xb[2] += phihatb;
        if (neg) vb[2] += dt * phihatb;
      }
    }
    memcpy(A->vb + 3 * p, vb, sizeof vb);
    memcpy(A->ub + 3 * p, ub_old, sizeof ub_old);
  }
  free(v1b);
  /* tool: x_B^{n+1} = x_B^n + dt v_B^n, v_B^n = segment velocity */
  if (s->has_blade) {
    for (int i = 0; i < 3; ++i) {
      double vtot = vBb[i] + dt * A->xBb[i];
      A->xBb[i] += xBd[i];
      if (seg_idx >= 0) A->vsegb[seg_idx][i] += vtot;
    }
  }
  or_destroy(s);
  return 0;
}
