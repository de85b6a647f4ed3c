/*
 * pdg_oracle.c -- TEST INFRASTRUCTURE ONLY (see pdg_oracle.h).
 *
 * Plain, serial, dense FP64 restatement of arXiv 2404.18034:
 *   Sec. 4      6-DoF dynamics F and path constraints g
 *   Sec. 2.1    time dilation and CTCS augmentation (Eq. sys-dyn-dil-aug)
 *   Sec. 2.2    uniform grid, FOH controls, multiple shooting (Eq. disc-dyn)
 *   Sec. 2.3.1  STM ODEs giving A_k, B^-_k, B^+_k (integrated with RK4 here)
 *   Sec. 2.3.2  prescaling and preconditioning (Eq. cvx-subproblem-custom)
 *   Sec. 3      canonical QP (Eq. parsed-data), Alg. 1 (PIPG), Alg. power,
 *               Alg. PIPG_custom, Alg. stopping
 *   Sec. 2.3    prox-linear SCP loop
 * Nothing is blocked, fused or reordered beyond the algorithms as printed.
 *
 * Readings of silent or garbled passages (the CUDA path takes the same ones):
 *  R1  quaternion: Hamilton, scalar first; C_{I<-B} in the 1-2(..) diagonal
 *      form; Omega(w) as in qdot = q (x) (0, w) / 2.
 *  R2  tilt row of g: 2(q2^2 + q3^2) - (1 - cos theta_max)  (the printed row
 *      is positive for every q).
 *  R3  d||T||/dT is taken as 0 at T = 0 (the paper relies on a thrust guess
 *      away from zero).
 *  R4  mu^- update uses (w_ep - phi): the dynamics rows carry +mu^+ - mu^-
 *      (Eq. cvx-subproblem-custom), which also fixes the sign of G_mu.
 *  R5  PIPG_custom: the B^+_{k-1} term of the u_k gradient multiplies the
 *      extrapolated dual of the dynamics rows; superscripts j of the first
 *      node read j+1.  Alg. power: v_k reads theta_k and sigma* accumulates
 *      from sigma* (not sigma); it acts on the full [G; H_y].
 *  R6  the dilation box is the only control box (Sec. 4); H of the canonical
 *      QP holds only the CTCS rows, the box and mu >= 0 are projections.
 *  R7  power iteration starts from the warm-start primal, or from all ones
 *      when that is zero; PIPG stop test compares iterates j+1 and j, with
 *      the warm start as iterate 0.
 *  R8  SCP stop: scaled step, scaled defect and CTCS budget (see orc_solve).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "pdg_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* The problem template of Sec. 2 (F, g, boundary conditions, Mayer cost) is
 * instantiated by a model chosen when this file is compiled:
 *   default          the 6-DoF model of Sec. 4, x = (m, r, v, q, omega, y);
 *   ORC_MODEL_3DOF   the translational (3-DoF) model Sec. 1 contrasts it with,
 *                    x = (m, r, v, y): point mass, thrust in the inertial
 *                    frame, no attitude (readings R18-R19).
 * Everything past the model section uses only NX, XM (the cost's mass) and XY
 * (the CTCS integrator, always last). */
#ifdef ORC_MODEL_3DOF
#define NX 8
enum { XM = 0, XR = 1, XV = 4, XY = 7 };
#else
#define NX 15
enum { XM = 0, XR = 1, XV = 4, XQ = 7, XW = 11, XY = 14 };
#endif

int orc_nx(void) { return NX; }

/* ------------------------------------------------------------------------ */
/* Sec. 4: model                                                             */
/* ------------------------------------------------------------------------ */

/* C_{I<-B}(q), Hamilton scalar-first (R1). */
#ifndef ORC_MODEL_3DOF
static void dcm(const double* q, double C[3][3]) {
  double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
  C[0][0] = 1.0 - 2.0 * (q2 * q2 + q3 * q3);
  C[0][1] = 2.0 * (q1 * q2 - q0 * q3);
  C[0][2] = 2.0 * (q1 * q3 + q0 * q2);
  C[1][0] = 2.0 * (q1 * q2 + q0 * q3);
  C[1][1] = 1.0 - 2.0 * (q1 * q1 + q3 * q3);
  C[1][2] = 2.0 * (q2 * q3 - q0 * q1);
  C[2][0] = 2.0 * (q1 * q3 - q0 * q2);
  C[2][1] = 2.0 * (q2 * q3 + q0 * q1);
  C[2][2] = 1.0 - 2.0 * (q1 * q1 + q2 * q2);
}

/* dC/dq_j for j = 0..3. */
static void dcm_dq(const double* q, double D[4][3][3]) {
  double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
  memset(D, 0, sizeof(double) * 36);
  /* row 0 */
  D[2][0][0] = -4.0 * q2; D[3][0][0] = -4.0 * q3;
  D[0][0][1] = -2.0 * q3; D[1][0][1] = 2.0 * q2; D[2][0][1] = 2.0 * q1; D[3][0][1] = -2.0 * q0;
  D[0][0][2] = 2.0 * q2;  D[1][0][2] = 2.0 * q3; D[2][0][2] = 2.0 * q0; D[3][0][2] = 2.0 * q1;
  /* row 1 */
  D[0][1][0] = 2.0 * q3;  D[1][1][0] = 2.0 * q2; D[2][1][0] = 2.0 * q1; D[3][1][0] = 2.0 * q0;
  D[1][1][1] = -4.0 * q1; D[3][1][1] = -4.0 * q3;
  D[0][1][2] = -2.0 * q1; D[1][1][2] = -2.0 * q0; D[2][1][2] = 2.0 * q3; D[3][1][2] = 2.0 * q2;
  /* row 2 */
  D[0][2][0] = -2.0 * q2; D[1][2][0] = 2.0 * q3; D[2][2][0] = -2.0 * q0; D[3][2][0] = 2.0 * q1;
  D[0][2][1] = 2.0 * q1;  D[1][2][1] = 2.0 * q0; D[2][2][1] = 2.0 * q3; D[3][2][1] = 2.0 * q2;
  D[1][2][2] = -4.0 * q1; D[2][2][2] = -4.0 * q2;
}

/* Omega(w) with qdot = Omega(w) q / 2 (R1). */
static void omega_mat(const double* w, double O[4][4]) {
  double wx = w[0], wy = w[1], wz = w[2];
  O[0][0] = 0;   O[0][1] = -wx; O[0][2] = -wy; O[0][3] = -wz;
  O[1][0] = wx;  O[1][1] = 0;   O[1][2] = wz;  O[1][3] = -wy;
  O[2][0] = wy;  O[2][1] = -wz; O[2][2] = 0;   O[2][3] = wx;
  O[3][0] = wz;  O[3][1] = wy;  O[3][2] = -wx; O[3][3] = 0;
}

/* Xi(q) with Omega(w) q = Xi(q) w. */
static void xi_mat(const double* q, double X[4][3]) {
  double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
  X[0][0] = -q1; X[0][1] = -q2; X[0][2] = -q3;
  X[1][0] = q0;  X[1][1] = -q3; X[1][2] = q2;
  X[2][0] = q3;  X[2][1] = q0;  X[2][2] = -q1;
  X[3][0] = -q2; X[3][1] = q1;  X[3][2] = q0;
}

static void skew(const double* a, double S[3][3]) {
  S[0][0] = 0;     S[0][1] = -a[2]; S[0][2] = a[1];
  S[1][0] = a[2];  S[1][1] = 0;     S[1][2] = -a[0];
  S[2][0] = -a[1]; S[2][1] = a[0];  S[2][2] = 0;
}

static void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* F(xi, zeta) of Sec. 4 (time domain, 14 rows). */
void orc_F(const orc_params* p, const double* x, const double* u, double* Fx) {
  const double m = x[XM];
  const double* v = x + XV;
  const double* q = x + XQ;
  const double* w = x + XW;
  const double* T = u;
  double gam[3] = {0, 0, 0};
  if (p->nu == 7) { gam[0] = u[3]; gam[1] = u[4]; gam[2] = u[5]; }
  double nT = sqrt(dot3(T, T));
  Fx[0] = -p->alpha_mdot * nT;
  for (int i = 0; i < 3; i++) Fx[1 + i] = v[i];
  double C[3][3];
  dcm(q, C);
  for (int i = 0; i < 3; i++) {
    double a = 0;
    for (int j = 0; j < 3; j++) a += C[i][j] * T[j];
    Fx[4 + i] = a / m + p->g_I[i];
  }
  double O[4][4];
  omega_mat(w, O);
  for (int i = 0; i < 4; i++) {
    double a = 0;
    for (int j = 0; j < 4; j++) a += O[i][j] * q[j];
    Fx[7 + i] = 0.5 * a;
  }
  double Jw[3], rxT[3], wxJw[3];
  for (int i = 0; i < 3; i++) Jw[i] = p->J_B[i] * w[i];
  cross(p->r_T_B, T, rxT);
  cross(w, Jw, wxJw);
  for (int i = 0; i < 3; i++) Fx[11 + i] = (rxT[i] - wxJw[i] + gam[i]) / p->J_B[i];
}

/* g(xi, zeta) of Sec. 4 with the tilt reading R2.  nu = 4 drops the gamma row. */
int orc_g(const orc_params* p, const double* x, const double* u, double* g) {
  const double* r = x + XR;
  const double* v = x + XV;
  const double* q = x + XQ;
  const double* w = x + XW;
  const double* T = u;
  double nT = sqrt(dot3(T, T));
  g[0] = p->m_dry - x[XM];
  g[1] = -r[0];
  g[2] = dot3(v, v) - p->v_max * p->v_max;
  g[3] = 2.0 * (q[2] * q[2] + q[3] * q[3]) - (1.0 - cos(p->theta_max));
  g[4] = dot3(w, w) - p->omega_max * p->omega_max;
  g[5] = nT - T[0] / cos(p->delta_max);
  g[6] = nT - p->T_max;
  if (p->soc_thrust) { g[5] = -1.0; g[6] = -1.0; }  /* imposed by projection instead */
  g[7] = p->T_min - nT;
  int ng = 8;
  if (p->nu == 7) {
    const double* gm = u + 3;
    g[ng++] = dot3(gm, gm) - p->gamma_max * p->gamma_max;
  }
  /* glide slope (parameter gamma_gs of Sec. 4; its row is not printed): the
     vehicle stays in the cone tan(gamma_gs) ||(r_y, r_z)|| <= r_x about the
     inertial up axis through the landing site.  Written squared,
     tan^2 (r_y^2 + r_z^2) - r_x^2 <= 0, which with the altitude row r_x >= 0
     is the same cone and is smooth at its apex (the touchdown point). */
  if (p->glide_slope) g[ng++] = p->tan_gs * p->tan_gs * (r[1] * r[1] + r[2] * r[2]) - r[0] * r[0];
  return ng;
}

/* A = df/dx (15x15), B = df/du (15 x nu), dense, analytic. */
void orc_jac(const orc_params* p, const double* x, const double* u, double* A, double* B) {
  const int nu = p->nu;
  const double s = u[nu - 1];
  const double m = x[XM];
  const double* v = x + XV;
  const double* q = x + XQ;
  const double* w = x + XW;
  const double* T = u;
  memset(A, 0, sizeof(double) * NX * NX);
  memset(B, 0, sizeof(double) * NX * nu);
#define AA(i, j) A[(i) * NX + (j)]
#define BB(i, j) B[(i) * nu + (j)]
  double Fx[NX - 1], g[10];
  orc_F(p, x, u, Fx);
  int ng = orc_g(p, x, u, g);
  double gp[10];
  double pen = 0;
  for (int i = 0; i < ng; i++) {
    gp[i] = g[i] > 0 ? g[i] : 0;
    pen += gp[i] * gp[i];
  }
  double nT = sqrt(dot3(T, T));
  double Tu[3] = {0, 0, 0}; /* dn/dT (R3) */
  if (nT > 0) for (int i = 0; i < 3; i++) Tu[i] = T[i] / nT;

  /* --- d/dx of F, times s --- */
  for (int i = 0; i < 3; i++) AA(XR + i, XV + i) = s;
  double C[3][3], D[4][3][3];
  dcm(q, C);
  dcm_dq(q, D);
  for (int i = 0; i < 3; i++) {
    double CT = 0;
    for (int j = 0; j < 3; j++) CT += C[i][j] * T[j];
    AA(XV + i, XM) = s * (-CT / (m * m));
    for (int k = 0; k < 4; k++) {
      double dCT = 0;
      for (int j = 0; j < 3; j++) dCT += D[k][i][j] * T[j];
      AA(XV + i, XQ + k) = s * dCT / m;
    }
  }
  double O[4][4], Xi[4][3];
  omega_mat(w, O);
  xi_mat(q, Xi);
  for (int i = 0; i < 4; i++) {
    for (int j = 0; j < 4; j++) AA(XQ + i, XQ + j) = s * 0.5 * O[i][j];
    for (int j = 0; j < 3; j++) AA(XQ + i, XW + j) = s * 0.5 * Xi[i][j];
  }
  /* d(w x Jw)/dw = [w]x J - [Jw]x */
  double Sw[3][3], SJw[3][3], Jw[3];
  for (int i = 0; i < 3; i++) Jw[i] = p->J_B[i] * w[i];
  skew(w, Sw);
  skew(Jw, SJw);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      AA(XW + i, XW + j) = s * (-(Sw[i][j] * p->J_B[j] - SJw[i][j]) / p->J_B[i]);
  /* y row: sum_i 2 |g_i|_+ dg_i/dx */
  AA(XY, XM) += s * 2.0 * gp[0] * (-1.0);
  AA(XY, XR + 0) += s * 2.0 * gp[1] * (-1.0);
  for (int i = 0; i < 3; i++) AA(XY, XV + i) += s * 2.0 * gp[2] * (2.0 * v[i]);
  AA(XY, XQ + 2) += s * 2.0 * gp[3] * (4.0 * q[2]);
  AA(XY, XQ + 3) += s * 2.0 * gp[3] * (4.0 * q[3]);
  for (int i = 0; i < 3; i++) AA(XY, XW + i) += s * 2.0 * gp[4] * (2.0 * w[i]);
  if (p->glide_slope) {  /* the glide-slope row is the last one */
    const double ggs = gp[ng - 1], t2 = p->tan_gs * p->tan_gs;
    AA(XY, XR + 0) += s * 2.0 * ggs * (-2.0 * x[XR + 0]);
    AA(XY, XR + 1) += s * 2.0 * ggs * (2.0 * t2 * x[XR + 1]);
    AA(XY, XR + 2) += s * 2.0 * ggs * (2.0 * t2 * x[XR + 2]);
  }

  /* --- d/dT --- */
  for (int j = 0; j < 3; j++) BB(XM, j) = s * (-p->alpha_mdot * Tu[j]);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) BB(XV + i, j) = s * C[i][j] / m;
  double Sr[3][3];
  skew(p->r_T_B, Sr);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) BB(XW + i, j) = s * Sr[i][j] / p->J_B[i];
  double secd = 1.0 / cos(p->delta_max);
  for (int j = 0; j < 3; j++) {
    double dg5 = Tu[j] - (j == 0 ? secd : 0.0);
    double dg6 = Tu[j];
    double dg7 = -Tu[j];
    BB(XY, j) = s * 2.0 * (gp[5] * dg5 + gp[6] * dg6 + gp[7] * dg7);
  }
  /* --- d/dgamma (nu = 7) --- */
  if (nu == 7) {
    for (int i = 0; i < 3; i++) BB(XW + i, 3 + i) = s / p->J_B[i];
    for (int j = 0; j < 3; j++) BB(XY, 3 + j) = s * 2.0 * gp[8] * (2.0 * u[3 + j]);
  }
  /* --- d/ds = (F, pen) --- */
  for (int i = 0; i < 14; i++) BB(i, nu - 1) = Fx[i];
  BB(XY, nu - 1) = pen;
#undef AA
#undef BB
}

#else /* ORC_MODEL_3DOF */

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* 3-DoF F(xi, zeta): mass depletion with the thrust magnitude, r' = v,
 * v' = T / m + g; T is an inertial-frame vector (R18). */
void orc_F(const orc_params* p, const double* x, const double* u, double* Fx) {
  const double* v = x + XV;
  const double* T = u;
  Fx[0] = -p->alpha_mdot * sqrt(dot3(T, T));
  for (int i = 0; i < 3; i++) Fx[1 + i] = v[i];
  for (int i = 0; i < 3; i++) Fx[4 + i] = T[i] / x[XM] + p->g_I[i];
}

/* 3-DoF g (R19): dry mass, altitude, speed, thrust pointing within delta_max
 * of the up axis (the 6-DoF gimbal row with the body axis taken as up),
 * thrust magnitude bounds, and the optional glide-slope row of the 6-DoF
 * model.  Row order: m, r_x, v, pointing, T_max, T_min[, glide slope]. */
int orc_g(const orc_params* p, const double* x, const double* u, double* g) {
  const double* r = x + XR;
  const double* v = x + XV;
  const double* T = u;
  double nT = sqrt(dot3(T, T));
  g[0] = p->m_dry - x[XM];
  g[1] = -r[0];
  g[2] = dot3(v, v) - p->v_max * p->v_max;
  g[3] = nT - T[0] / cos(p->delta_max);
  g[4] = nT - p->T_max;
  if (p->soc_thrust) { g[3] = -1.0; g[4] = -1.0; }  /* imposed by projection instead */
  g[5] = p->T_min - nT;
  int ng = 6;
  if (p->glide_slope) g[ng++] = p->tan_gs * p->tan_gs * (r[1] * r[1] + r[2] * r[2]) - r[0] * r[0];
  return ng;
}

/* A = df/dx (8x8), B = df/du (8 x 4), dense, analytic. */
void orc_jac(const orc_params* p, const double* x, const double* u, double* A, double* B) {
  const int nu = p->nu;
  const double s = u[nu - 1];
  const double m = x[XM];
  const double* v = x + XV;
  const double* T = u;
  memset(A, 0, sizeof(double) * NX * NX);
  memset(B, 0, sizeof(double) * NX * nu);
#define AA(i, j) A[(i) * NX + (j)]
#define BB(i, j) B[(i) * nu + (j)]
  double Fx[NX - 1], g[10], gp[10];
  orc_F(p, x, u, Fx);
  int ng = orc_g(p, x, u, g);
  double pen = 0;
  for (int i = 0; i < ng; i++) {
    gp[i] = g[i] > 0 ? g[i] : 0;
    pen += gp[i] * gp[i];
  }
  double nT = sqrt(dot3(T, T));
  double Tu[3] = {0, 0, 0}; /* dn/dT (R3) */
  if (nT > 0) for (int i = 0; i < 3; i++) Tu[i] = T[i] / nT;
  for (int i = 0; i < 3; i++) {
    AA(XR + i, XV + i) = s;
    AA(XV + i, XM) = s * (-T[i] / (m * m));
  }
  /* y row: sum_i 2 |g_i|_+ dg_i/dx */
  AA(XY, XM) += s * 2.0 * gp[0] * (-1.0);
  AA(XY, XR + 0) += s * 2.0 * gp[1] * (-1.0);
  for (int i = 0; i < 3; i++) AA(XY, XV + i) += s * 2.0 * gp[2] * (2.0 * v[i]);
  if (p->glide_slope) {
    const double ggs = gp[ng - 1], t2 = p->tan_gs * p->tan_gs;
    AA(XY, XR + 0) += s * 2.0 * ggs * (-2.0 * x[XR + 0]);
    AA(XY, XR + 1) += s * 2.0 * ggs * (2.0 * t2 * x[XR + 1]);
    AA(XY, XR + 2) += s * 2.0 * ggs * (2.0 * t2 * x[XR + 2]);
  }
  for (int j = 0; j < 3; j++) {
    BB(XM, j) = s * (-p->alpha_mdot * Tu[j]);
    BB(XV + j, j) = s / m;
    double dg3 = Tu[j] - (j == 0 ? 1.0 / cos(p->delta_max) : 0.0);
    BB(XY, j) = s * 2.0 * (gp[3] * dg3 + gp[4] * Tu[j] - gp[5] * Tu[j]);
  }
  for (int i = 0; i < NX - 1; i++) BB(i, nu - 1) = Fx[i];
  BB(XY, nu - 1) = pen;
#undef AA
#undef BB
}

#endif /* ORC_MODEL_3DOF */

/* f(x, u) = s (F, 1^T |g|_+^2), Eq. sys-dyn-dil-aug (no h in this problem). */
void orc_f(const orc_params* p, const double* x, const double* u, double* f) {
  double s = u[p->nu - 1];
  double Fx[NX - 1], g[10];
  orc_F(p, x, u, Fx);
  int ng = orc_g(p, x, u, g);
  double pen = 0;
  for (int i = 0; i < ng; i++) {
    double gp = g[i] > 0 ? g[i] : 0;
    pen += gp * gp;
  }
  for (int i = 0; i < NX - 1; i++) f[i] = s * Fx[i];
  f[XY] = s * pen;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2 / 2.3.1: discretization                                          */
/* ------------------------------------------------------------------------ */

/* FOH control at fraction lp = (tau - tau_k)/(tau_{k+1} - tau_k). */
static void foh(int nu, const double* uk, const double* uk1, double lp, double* u) {
  for (int i = 0; i < nu; i++) u[i] = (1.0 - lp) * uk[i] + lp * uk1[i];
}

/* x_{k+1} = f_k(x_k, u_k, u_{k+1}) by RK4 with nsub substeps on the uniform
 * grid tau_k = (k-1)/(N-1); dtau is passed as 1/(N-1) by the callers. */
static void flow_dtau(const orc_params* p, const double* xk, const double* uk, const double* uk1,
                      double dtau, int nsub, double* xout) {
  const int nu = p->nu;
  double x[NX], xs[NX], k1[NX], k2[NX], k3[NX], k4[NX], u[ORC_NU_MAX];
  double h = dtau / nsub;
  memcpy(x, xk, sizeof x);
  for (int n = 0; n < nsub; n++) {
    double l0 = (double)n / nsub, lh = (n + 0.5) / nsub, l1 = (double)(n + 1) / nsub;
    foh(nu, uk, uk1, l0, u);
    orc_f(p, x, u, k1);
    for (int i = 0; i < NX; i++) xs[i] = x[i] + 0.5 * h * k1[i];
    foh(nu, uk, uk1, lh, u);
    orc_f(p, xs, u, k2);
    for (int i = 0; i < NX; i++) xs[i] = x[i] + 0.5 * h * k2[i];
    orc_f(p, xs, u, k3);
    for (int i = 0; i < NX; i++) xs[i] = x[i] + h * k3[i];
    foh(nu, uk, uk1, l1, u);
    orc_f(p, xs, u, k4);
    for (int i = 0; i < NX; i++) x[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
  memcpy(xout, x, sizeof x);
}

void orc_flow(const orc_params* p, const double* xk, const double* uk, const double* uk1,
              int nsub, double* xout) {
  /* dtau is taken as 1 here; callers scale s instead (used by closed-form tests). */
  flow_dtau(p, xk, uk, uk1, 1.0, nsub, xout);
}

/* Right-hand side of the joint IVP of Sec. 2.3.1: x, Phi_x, Phi_u^-, Phi_u^+. */
static void joint_rhs(const orc_params* p, const double* Z, const double* uk, const double* uk1,
                      double lp, double* dZ) {
  const int nu = p->nu;
  double u[ORC_NU_MAX], A[NX * NX], Bu[NX * ORC_NU_MAX];
  foh(nu, uk, uk1, lp, u);
  const double* x = Z;
  const double* Px = Z + NX;
  const double* Pm = Px + NX * NX;
  const double* Pp = Pm + NX * nu;
  orc_f(p, x, u, dZ);
  orc_jac(p, x, u, A, Bu);
  double* dPx = dZ + NX;
  double* dPm = dPx + NX * NX;
  double* dPp = dPm + NX * nu;
  double lm = 1.0 - lp;
  for (int i = 0; i < NX; i++) {
    for (int j = 0; j < NX; j++) {
      double a = 0;
      for (int r = 0; r < NX; r++) a += A[i * NX + r] * Px[r * NX + j];
      dPx[i * NX + j] = a;
    }
    for (int c = 0; c < nu; c++) {
      double am = 0, ap = 0;
      for (int r = 0; r < NX; r++) {
        am += A[i * NX + r] * Pm[r * nu + c];
        ap += A[i * NX + r] * Pp[r * nu + c];
      }
      dPm[i * nu + c] = am + Bu[i * nu + c] * lm;
      dPp[i * nu + c] = ap + Bu[i * nu + c] * lp;
    }
  }
}

void orc_discretize(const orc_params* p, int N, const double* X, const double* U,
                    double* A, double* Bm, double* Bp, double* xprop) {
  const int nu = p->nu;
  const int nz = NX + NX * NX + 2 * NX * nu;
  const int nsub = p->rk4_substeps;
  const double dtau = 1.0 / (N - 1);
  const double h = dtau / nsub;
  double* Z = malloc(sizeof(double) * nz * 6);
  double* Zs = Z + nz;
  double* k1 = Zs + nz;
  double* k2 = k1 + nz;
  double* k3 = k2 + nz;
  double* k4 = k3 + nz;
  for (int k = 0; k < N - 1; k++) {
    const double* uk = U + k * nu;
    const double* uk1 = U + (k + 1) * nu;
    memset(Z, 0, sizeof(double) * nz);
    memcpy(Z, X + k * NX, sizeof(double) * NX);
    for (int i = 0; i < NX; i++) Z[NX + i * NX + i] = 1.0; /* Phi_x(tau_k) = I */
    for (int n = 0; n < nsub; n++) {
      double l0 = (double)n / nsub, lh = (n + 0.5) / nsub, l1 = (double)(n + 1) / nsub;
      joint_rhs(p, Z, uk, uk1, l0, k1);
      for (int i = 0; i < nz; i++) Zs[i] = Z[i] + 0.5 * h * k1[i];
      joint_rhs(p, Zs, uk, uk1, lh, k2);
      for (int i = 0; i < nz; i++) Zs[i] = Z[i] + 0.5 * h * k2[i];
      joint_rhs(p, Zs, uk, uk1, lh, k3);
      for (int i = 0; i < nz; i++) Zs[i] = Z[i] + h * k3[i];
      joint_rhs(p, Zs, uk, uk1, l1, k4);
      for (int i = 0; i < nz; i++) Z[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    memcpy(xprop + k * NX, Z, sizeof(double) * NX);
    memcpy(A + k * NX * NX, Z + NX, sizeof(double) * NX * NX);
    memcpy(Bm + k * NX * nu, Z + NX + NX * NX, sizeof(double) * NX * nu);
    memcpy(Bp + k * NX * nu, Z + NX + NX * NX + NX * nu, sizeof(double) * NX * nu);
  }
  free(Z);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3.2: scaled subproblem                                             */
/* ------------------------------------------------------------------------ */

int orc_qp_alloc(orc_qp* qp, int N, int nu) {
  memset(qp, 0, sizeof *qp);
  qp->N = N;
  qp->nu = nu;
  qp->Tbar = calloc((size_t)N * 3, sizeof(double));
  qp->Am = calloc((size_t)(N - 1) * NX * NX, sizeof(double));
  qp->Ap = calloc((size_t)(N - 1) * NX * NX, sizeof(double));
  qp->Bm = calloc((size_t)(N - 1) * NX * nu, sizeof(double));
  qp->Bp = calloc((size_t)(N - 1) * NX * nu, sizeof(double));
  qp->w = calloc((size_t)(N - 1) * NX, sizeof(double));
  qp->eps = calloc((size_t)(N - 1), sizeof(double));
  qp->umin = calloc((size_t)N * nu, sizeof(double));
  qp->umax = calloc((size_t)N * nu, sizeof(double));
  return (qp->Tbar && qp->Am && qp->Ap && qp->Bm && qp->Bp && qp->w && qp->eps && qp->umin && qp->umax) ? 0 : -1;
}

void orc_qp_free(orc_qp* qp) {
  free(qp->Am); free(qp->Ap); free(qp->Bm); free(qp->Bp);
  free(qp->w); free(qp->eps); free(qp->umin); free(qp->umax); free(qp->Tbar);
  memset(qp, 0, sizeof *qp);
}

void orc_scale(const orc_params* p, int N, const double* x0, const double* X, const double* U,
               const double* A, const double* Bm, const double* Bp, const double* xprop, orc_qp* qp) {
  const int nu = p->nu;
  const double* Px = p->P_x;
  const double* Pu = p->P_u;
  for (int k = 0; k < N - 1; k++) {
    for (int i = 0; i < NX; i++) {
      for (int j = 0; j < NX; j++) {
        /* hat A^-_k = P_x^{-1} A_k P_x ; hat A^+_k = -I */
        qp->Am[(k * NX + i) * NX + j] = A[(k * NX + i) * NX + j] * Px[j] / Px[i];
        qp->Ap[(k * NX + i) * NX + j] = (i == j) ? -1.0 : 0.0;
      }
      for (int c = 0; c < nu; c++) {
        qp->Bm[(k * NX + i) * nu + c] = Bm[(k * NX + i) * nu + c] * Pu[c] / Px[i];
        qp->Bp[(k * NX + i) * nu + c] = Bp[(k * NX + i) * nu + c] * Pu[c] / Px[i];
      }
      /* hat w_k = P_x^{-1} (xbar^k(tau_{k+1}) - xbar_{k+1}) */
      qp->w[k * NX + i] = (xprop[k * NX + i] - X[(k + 1) * NX + i]) / Px[i];
    }
    /* hat eps_k = eps E_y P_x^{-1} E_y^T - E_y P_x^{-1} (xbar_{k+1} - xbar_k) */
    qp->eps[k] = p->eps_ctcs / Px[XY] - (X[(k + 1) * NX + XY] - X[k * NX + XY]) / Px[XY];
  }
  /* control box on the dilation factor only (Sec. 4, R6).  The time bounds
     of Sec. 2.2 tighten it node-wise: with FOH s, Delta t_k = (s_k + s_{k+1})
     / (2 (N-1)) lies between the node values / (N-1), and t_f = sum Delta t_k
     is at most max_k s_k, so s_k in [dt_min (N-1), min(dt_max (N-1), tf_max)]
     is sufficient for dt_min <= Delta t_k <= dt_max and t_f <= tf_max. */
  double smin = p->s_min, smax = p->s_max;
  if (p->dt_min > 0 && p->dt_min * (N - 1) > smin) smin = p->dt_min * (N - 1);
  if (p->dt_max > 0 && p->dt_max * (N - 1) < smax) smax = p->dt_max * (N - 1);
  if (p->tf_max > 0 && p->tf_max < smax) smax = p->tf_max;
  for (int k = 0; k < N; k++) {
    for (int c = 0; c < nu; c++) {
      if (c == nu - 1) {
        qp->umin[k * nu + c] = (smin - U[k * nu + c]) / Pu[c];
        qp->umax[k * nu + c] = (smax - U[k * nu + c]) / Pu[c];
      } else {
        qp->umin[k * nu + c] = -INFINITY;
        qp->umax[k * nu + c] = INFINITY;
      }
    }
  }
  /* hat z_i: E_i selects all of xi, with y_1 = 0 appended (Eq. disc-ocp) */
  for (int i = 0; i < NX; i++) {
    double zi = (i < NX - 1) ? x0[i] : 0.0;
    qp->zi[i] = (zi - X[i]) / Px[i];
    qp->fixf[i] = p->fix_f[i];
    qp->zf[i] = p->fix_f[i] ? (p->z_f[i] - X[(N - 1) * NX + i]) / Px[i] : 0.0;
    qp->ecost[i] = 0.0;
  }
  qp->ecost[XM] = -1.0; /* propellant-optimal: maximize m_N */
  qp->soc = p->soc_thrust;
  for (int k = 0; k < N; k++)
    for (int i = 0; i < 3; i++) qp->Tbar[k * 3 + i] = U[k * nu + i];
  qp->soc_Tmax = p->T_max;
  qp->soc_tan = tan(p->delta_max);
  qp->soc_PT = p->P_u[0];
  qp->w_cost = p->w_cost;
  qp->w_prox = p->w_prox;
  qp->w_ep = p->w_ep;
}

/* ------------------------------------------------------------------------ */
/* primal-dual state helpers                                                 */
/* ------------------------------------------------------------------------ */

int orc_pd_alloc(orc_pd* s, int N, int nu) {
  s->xh = calloc((size_t)N * NX, sizeof(double));
  s->uh = calloc((size_t)N * nu, sizeof(double));
  s->mup = calloc((size_t)(N - 1) * NX, sizeof(double));
  s->mum = calloc((size_t)(N - 1) * NX, sizeof(double));
  s->phi = calloc((size_t)(N - 1) * NX, sizeof(double));
  s->th = calloc((size_t)(N - 1), sizeof(double));
  return (s->xh && s->uh && s->mup && s->mum && s->phi && s->th) ? 0 : -1;
}

void orc_pd_free(orc_pd* s) {
  free(s->xh); free(s->uh); free(s->mup); free(s->mum); free(s->phi); free(s->th);
  memset(s, 0, sizeof *s);
}

void orc_pd_zero(orc_pd* s, int N, int nu) {
  memset(s->xh, 0, sizeof(double) * N * NX);
  memset(s->uh, 0, sizeof(double) * N * nu);
  memset(s->mup, 0, sizeof(double) * (N - 1) * NX);
  memset(s->mum, 0, sizeof(double) * (N - 1) * NX);
  memset(s->phi, 0, sizeof(double) * (N - 1) * NX);
  memset(s->th, 0, sizeof(double) * (N - 1));
}

void orc_pd_copy(orc_pd* d, const orc_pd* s, int N, int nu) {
  memcpy(d->xh, s->xh, sizeof(double) * N * NX);
  memcpy(d->uh, s->uh, sizeof(double) * N * nu);
  memcpy(d->mup, s->mup, sizeof(double) * (N - 1) * NX);
  memcpy(d->mum, s->mum, sizeof(double) * (N - 1) * NX);
  memcpy(d->phi, s->phi, sizeof(double) * (N - 1) * NX);
  memcpy(d->th, s->th, sizeof(double) * (N - 1));
}

/* small dense helpers */
static void mv(int n, int m, const double* M, const double* x, double* y) { /* y = M x, M n x m */
  for (int i = 0; i < n; i++) {
    double a = 0;
    for (int j = 0; j < m; j++) a += M[i * m + j] * x[j];
    y[i] = a;
  }
}
static void mtv_add(int n, int m, const double* M, const double* x, double* y) { /* y += M^T x */
  for (int j = 0; j < m; j++) {
    double a = 0;
    for (int i = 0; i < n; i++) a += M[i * m + j] * x[i];
    y[j] += a;
  }
}
static double sqn(int n, const double* a) {
  double s = 0;
  for (int i = 0; i < n; i++) s += a[i] * a[i];
  return s;
}
static double infn(int n, const double* a) {
  double s = 0;
  for (int i = 0; i < n; i++) { double t = fabs(a[i]); if (t > s) s = t; }
  return s;
}
static double infd(int n, const double* a, const double* b) {
  double s = 0;
  for (int i = 0; i < n; i++) { double t = fabs(a[i] - b[i]); if (t > s) s = t; }
  return s;
}
static double maxd(double a, double b) { return a > b ? a : b; }

/* ------------------------------------------------------------------------ */
/* Alg. power: customized power iteration                                     */
/* ------------------------------------------------------------------------ */

double orc_power(const orc_params* p, const orc_qp* qp, const orc_pd* start, int force_iters, int* iters) {
  return orc_power_m(p, qp, start, force_iters, iters, NULL);
}

/* Relative margin (a - b) / b of a test a <= b with b > 0: the test passes
 * exactly when the margin is <= 0. */
static double margin(double a, double b) { return (a - b) / b; }

double orc_power_m(const orc_params* p, const orc_qp* qp, const orc_pd* start, int force_iters, int* iters,
                   double* margins) {
  const int N = qp->N, nu = qp->nu;
  orc_pd z;
  orc_pd_alloc(&z, N, nu);
  orc_pd_copy(&z, start, N, nu);
  double* phi = z.phi;
  double* th = z.th;
  /* sigma <- || (x, u, mu+, mu-) ||  (R7: ones if the warm start is zero) */
  double sig = 0;
  for (int k = 0; k < N - 1; k++)
    sig += sqn(NX, z.xh + k * NX) + sqn(nu, z.uh + k * nu) + sqn(NX, z.mup + k * NX) + sqn(NX, z.mum + k * NX);
  sig += sqn(NX, z.xh + (N - 1) * NX) + sqn(nu, z.uh + (N - 1) * nu);
  if (sig == 0.0) {
    for (int i = 0; i < N * NX; i++) z.xh[i] = 1.0;
    for (int i = 0; i < N * nu; i++) z.uh[i] = 1.0;
    for (int i = 0; i < (N - 1) * NX; i++) { z.mup[i] = 1.0; z.mum[i] = 1.0; }
    sig = (double)(N * NX + N * nu + 2 * (N - 1) * NX);
  }
  sig = sqrt(sig);
  int jmax = force_iters > 0 ? force_iters : p->pow_jmax;
  double sstar = sig;
  int j;
  double t[NX];
  for (j = 1; j <= jmax; j++) {
    for (int k = 0; k < N - 1; k++) {
      double* ph = phi + k * NX;
      mv(NX, NX, qp->Am + k * NX * NX, z.xh + k * NX, ph);
      mv(NX, NX, qp->Ap + k * NX * NX, z.xh + (k + 1) * NX, t);
      for (int i = 0; i < NX; i++) ph[i] += t[i];
      mv(NX, nu, qp->Bm + k * NX * nu, z.uh + k * nu, t);
      for (int i = 0; i < NX; i++) ph[i] += t[i];
      mv(NX, nu, qp->Bp + k * NX * nu, z.uh + (k + 1) * nu, t);
      for (int i = 0; i < NX; i++) ph[i] += t[i];
      for (int i = 0; i < NX; i++) ph[i] = (ph[i] + z.mup[k * NX + i] - z.mum[k * NX + i]) / sig;
      th[k] = (z.xh[(k + 1) * NX + XY] - z.xh[k * NX + XY]) / sig;
    }
    /* transposed products */
    memset(z.xh, 0, sizeof(double) * N * NX);
    memset(z.uh, 0, sizeof(double) * N * nu);
    for (int k = 0; k < N - 1; k++) {
      mtv_add(NX, NX, qp->Am + k * NX * NX, phi + k * NX, z.xh + k * NX);
      mtv_add(NX, nu, qp->Bm + k * NX * nu, phi + k * NX, z.uh + k * nu);
      z.xh[k * NX + XY] -= th[k];
      mtv_add(NX, NX, qp->Ap + k * NX * NX, phi + k * NX, z.xh + (k + 1) * NX);
      mtv_add(NX, nu, qp->Bp + k * NX * nu, phi + k * NX, z.uh + (k + 1) * nu);
      z.xh[(k + 1) * NX + XY] += th[k];
      for (int i = 0; i < NX; i++) { z.mup[k * NX + i] = phi[k * NX + i]; z.mum[k * NX + i] = -phi[k * NX + i]; }
    }
    double ss = 0;
    for (int k = 0; k < N - 1; k++)
      ss += sqn(NX, z.xh + k * NX) + sqn(nu, z.uh + k * nu) + sqn(NX, z.mup + k * NX) + sqn(NX, z.mum + k * NX);
    ss += sqn(NX, z.xh + (N - 1) * NX) + sqn(nu, z.uh + (N - 1) * nu);
    sstar = sqrt(ss);
    if (margins) margins[j - 1] = margin(fabs(sstar - sig), p->pow_eps_abs + p->pow_eps_rel * maxd(sstar, sig));
    if (force_iters <= 0 && fabs(sstar - sig) <= p->pow_eps_abs + p->pow_eps_rel * maxd(sstar, sig)) break;
    if (j < jmax) sig = sstar;
  }
  if (j > jmax) j = jmax;
  if (iters) *iters = j;
  orc_pd_free(&z);
  return (1.0 + p->pow_eps_buff) * sstar;
}

/* ------------------------------------------------------------------------ */
/* Alg. PIPG_custom with Alg. stopping                                       */
/* ------------------------------------------------------------------------ */

static int stop_custom(const orc_params* p, const orc_qp* qp, const orc_pd* a, const orc_pd* b) {
  const int N = qp->N, nu = qp->nu;
  int nx = N * NX, nuu = N * nu, nm = (N - 1) * NX;
  double za = maxd(maxd(infn(nx, a->xh), infn(nuu, a->uh)), maxd(infn(nm, a->mup), infn(nm, a->mum)));
  double zb = maxd(maxd(infn(nx, b->xh), infn(nuu, b->uh)), maxd(infn(nm, b->mup), infn(nm, b->mum)));
  double zd = maxd(maxd(infd(nx, a->xh, b->xh), infd(nuu, a->uh, b->uh)),
                   maxd(infd(nm, a->mup, b->mup), infd(nm, a->mum, b->mum)));
  double ra = maxd(infn(nm, a->phi), infn(N - 1, a->th));
  double rb = maxd(infn(nm, b->phi), infn(N - 1, b->th));
  double rd = maxd(infd(nm, a->phi, b->phi), infd(N - 1, a->th, b->th));
  return zd <= p->pipg_eps_abs + p->pipg_eps_rel * maxd(za, zb) &&
         rd <= p->pipg_eps_abs + p->pipg_eps_rel * maxd(ra, rb);
}

/* The same test as a relative margin: the larger of the primal and the dual
 * margins, <= 0 exactly when stop_custom terminates. */
static double stop_margin(const orc_params* p, const orc_qp* qp, const orc_pd* a, const orc_pd* b) {
  const int N = qp->N, nu = qp->nu;
  int nx = N * NX, nuu = N * nu, nm = (N - 1) * NX;
  double za = maxd(maxd(infn(nx, a->xh), infn(nuu, a->uh)), maxd(infn(nm, a->mup), infn(nm, a->mum)));
  double zb = maxd(maxd(infn(nx, b->xh), infn(nuu, b->uh)), maxd(infn(nm, b->mup), infn(nm, b->mum)));
  double zd = maxd(maxd(infd(nx, a->xh, b->xh), infd(nuu, a->uh, b->uh)),
                   maxd(infd(nm, a->mup, b->mup), infd(nm, a->mum, b->mum)));
  double ra = maxd(infn(nm, a->phi), infn(N - 1, a->th));
  double rb = maxd(infn(nm, b->phi), infn(N - 1, b->th));
  double rd = maxd(infd(nm, a->phi, b->phi), infd(N - 1, a->th, b->th));
  return maxd(margin(zd, p->pipg_eps_abs + p->pipg_eps_rel * maxd(za, zb)),
              margin(rd, p->pipg_eps_abs + p->pipg_eps_rel * maxd(ra, rb)));
}

int orc_stop_custom(const orc_params* p, const orc_qp* qp, const orc_pd* a, const orc_pd* b, double* m) {
  if (m) *m = stop_margin(p, qp, a, b);
  return stop_custom(p, qp, a, b);
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

void orc_sector_project(double* T, double Tmax, double tan_delta) {
  /* cone K = {(t, z): ||z|| <= a t}, t = T_x, z = (T_y, T_z), a = tan(delta) */
  double t = T[0], r = sqrt(T[1] * T[1] + T[2] * T[2]), a = tan_delta;
  if (r > a * t) {
    if (a * r <= -t) {
      T[0] = T[1] = T[2] = 0.0;
    } else {
      double tp = (t + a * r) / (1.0 + a * a);
      double rp = a * tp;
      T[0] = tp;
      T[1] = rp * T[1] / r;
      T[2] = rp * T[2] / r;
    }
  }
  /* then the ball of radius Tmax about the apex */
  double n = sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
  if (n > Tmax) {
    double f = Tmax / n;
    T[0] *= f; T[1] *= f; T[2] *= f;
  }
}

/* projection of node k's scaled thrust onto the sector (shifted by the
 * reference and scaled by P_T) */
static void soc_project_uhat(const orc_qp* qp, int k, double* uh) {
  double T[3];
  for (int i = 0; i < 3; i++) T[i] = qp->Tbar[k * 3 + i] + qp->soc_PT * uh[i];
  orc_sector_project(T, qp->soc_Tmax, qp->soc_tan);
  for (int i = 0; i < 3; i++) uh[i] = (T[i] - qp->Tbar[k * 3 + i]) / qp->soc_PT;
}

int orc_pipgc(const orc_params* p, const orc_qp* qp, double sigma, orc_pd* ws, int force_iters) {
  return orc_pipgc_m(p, qp, sigma, ws, force_iters, NULL);
}

int orc_pipgc_m(const orc_params* p, const orc_qp* qp, double sigma, orc_pd* ws, int force_iters,
                double* margins) {
  const int N = qp->N, nu = qp->nu;
  const double wp = qp->w_prox;
  orc_pd cur, prev, til;
  orc_pd_alloc(&cur, N, nu);
  orc_pd_alloc(&prev, N, nu);
  orc_pd_alloc(&til, N, nu);
  /* warm start: tilde variables <- previous solution */
  orc_pd_copy(&til, ws, N, nu);
  orc_pd_copy(&prev, ws, N, nu);
  orc_pd_copy(&cur, ws, N, nu);
  const double alpha = 2.0 / (wp + sqrt(wp * wp + 4.0 * p->pipg_omega * sigma));
  const double beta = p->pipg_omega * alpha;
  const double rho = p->pipg_rho;
  const int jmax = force_iters > 0 ? force_iters : p->pipg_jmax;
  double* xt = til.xh;  double* ut = til.uh;
  double* nup = til.mup; double* num = til.mum;
  double* vph = til.phi; double* vth = til.th;
  double g[NX], gu[ORC_NU_MAX], d1[NX], d2[NX], t[NX];
  int j;
  for (j = 1; j <= jmax; j++) {
    /* projected gradient step, node 1 */
    for (int i = 0; i < NX; i++) g[i] = wp * xt[i];
    mtv_add(NX, NX, qp->Am, vph, g);
    g[XY] -= vth[0];
    for (int i = 0; i < NX; i++) cur.xh[i] = xt[i] - alpha * g[i];
    for (int i = 0; i < NX; i++) cur.xh[i] = qp->zi[i]; /* E_i selects every component */
    for (int c = 0; c < nu; c++) gu[c] = wp * ut[c];
    mtv_add(NX, nu, qp->Bm, vph, gu);
    for (int c = 0; c < nu; c++) cur.uh[c] = clampd(ut[c] - alpha * gu[c], qp->umin[c], qp->umax[c]);
    if (qp->soc) soc_project_uhat(qp, 0, cur.uh);
    /* nodes 2..N-1 */
    for (int k = 1; k < N - 1; k++) {
      for (int i = 0; i < NX; i++) g[i] = wp * xt[k * NX + i];
      mtv_add(NX, NX, qp->Am + k * NX * NX, vph + k * NX, g);
      mtv_add(NX, NX, qp->Ap + (k - 1) * NX * NX, vph + (k - 1) * NX, g);
      g[XY] += -vth[k] + vth[k - 1];
      for (int i = 0; i < NX; i++) cur.xh[k * NX + i] = xt[k * NX + i] - alpha * g[i];
      for (int c = 0; c < nu; c++) gu[c] = wp * ut[k * nu + c];
      mtv_add(NX, nu, qp->Bm + k * NX * nu, vph + k * NX, gu);
      mtv_add(NX, nu, qp->Bp + (k - 1) * NX * nu, vph + (k - 1) * NX, gu); /* R5 */
      for (int c = 0; c < nu; c++)
        cur.uh[k * nu + c] = clampd(ut[k * nu + c] - alpha * gu[c], qp->umin[k * nu + c], qp->umax[k * nu + c]);
      if (qp->soc) soc_project_uhat(qp, k, cur.uh + k * nu);
    }
    /* node N */
    {
      int k = N - 1;
      for (int i = 0; i < NX; i++) g[i] = wp * xt[k * NX + i] + qp->w_cost * qp->ecost[i];
      mtv_add(NX, NX, qp->Ap + (k - 1) * NX * NX, vph + (k - 1) * NX, g);
      g[XY] += vth[k - 1];
      for (int i = 0; i < NX; i++) cur.xh[k * NX + i] = xt[k * NX + i] - alpha * g[i];
      for (int i = 0; i < NX; i++) if (qp->fixf[i]) cur.xh[k * NX + i] = qp->zf[i];
      for (int c = 0; c < nu; c++) gu[c] = wp * ut[k * nu + c];
      mtv_add(NX, nu, qp->Bp + (k - 1) * NX * nu, vph + (k - 1) * NX, gu);
      for (int c = 0; c < nu; c++)
        cur.uh[k * nu + c] = clampd(ut[k * nu + c] - alpha * gu[c], qp->umin[k * nu + c], qp->umax[k * nu + c]);
      if (qp->soc) soc_project_uhat(qp, k, cur.uh + k * nu);
    }
    /* virtual controls (R4) */
    for (int i = 0; i < (N - 1) * NX; i++) {
      double a = nup[i] - alpha * (qp->w_ep + vph[i]);
      double b = num[i] - alpha * (qp->w_ep - vph[i]);
      cur.mup[i] = a > 0 ? a : 0;
      cur.mum[i] = b > 0 ? b : 0;
    }
    /* PI feedback of the affine constraint violation */
    for (int k = 0; k < N - 1; k++) {
      double uk[ORC_NU_MAX], uk1[ORC_NU_MAX];
      for (int i = 0; i < NX; i++) {
        d1[i] = 2.0 * cur.xh[k * NX + i] - xt[k * NX + i];
        d2[i] = 2.0 * cur.xh[(k + 1) * NX + i] - xt[(k + 1) * NX + i];
      }
      for (int c = 0; c < nu; c++) {
        uk[c] = 2.0 * cur.uh[k * nu + c] - ut[k * nu + c];
        uk1[c] = 2.0 * cur.uh[(k + 1) * nu + c] - ut[(k + 1) * nu + c];
      }
      double r[NX];
      mv(NX, NX, qp->Am + k * NX * NX, d1, r);
      mv(NX, NX, qp->Ap + k * NX * NX, d2, t);
      for (int i = 0; i < NX; i++) r[i] += t[i];
      mv(NX, nu, qp->Bm + k * NX * nu, uk, t);
      for (int i = 0; i < NX; i++) r[i] += t[i];
      mv(NX, nu, qp->Bp + k * NX * nu, uk1, t);
      for (int i = 0; i < NX; i++) r[i] += t[i];
      for (int i = 0; i < NX; i++) {
        int ii = k * NX + i;
        r[i] += (2.0 * cur.mup[ii] - nup[ii]) - (2.0 * cur.mum[ii] - num[ii]) + qp->w[ii];
        cur.phi[ii] = vph[ii] + beta * r[i];
      }
      double hy = d2[XY] - d1[XY] - qp->eps[k];
      double th = vth[k] + beta * hy;
      cur.th[k] = th > 0 ? th : 0;
    }
    /* extrapolation */
    for (int i = 0; i < N * NX; i++) xt[i] = (1.0 - rho) * xt[i] + rho * cur.xh[i];
    for (int i = 0; i < N * nu; i++) ut[i] = (1.0 - rho) * ut[i] + rho * cur.uh[i];
    for (int i = 0; i < (N - 1) * NX; i++) {
      nup[i] = (1.0 - rho) * nup[i] + rho * cur.mup[i];
      num[i] = (1.0 - rho) * num[i] + rho * cur.mum[i];
      vph[i] = (1.0 - rho) * vph[i] + rho * cur.phi[i];
    }
    for (int k = 0; k < N - 1; k++) vth[k] = (1.0 - rho) * vth[k] + rho * cur.th[k];
    if (margins && p->pipg_jcheck > 0 && j % p->pipg_jcheck == 0)
      margins[j / p->pipg_jcheck - 1] = stop_margin(p, qp, &cur, &prev);
    if (force_iters <= 0 && p->pipg_jcheck > 0 && j % p->pipg_jcheck == 0) {
      if (stop_custom(p, qp, &cur, &prev)) break;
    }
    orc_pd_copy(&prev, &cur, N, nu);
  }
  if (j > jmax) j = jmax;
  orc_pd_copy(ws, &cur, N, nu);
  orc_pd_free(&cur);
  orc_pd_free(&prev);
  orc_pd_free(&til);
  return j;
}

/* ------------------------------------------------------------------------ */
/* Eq. canonical-QP / parsed-data, dense, and Alg. 1                         */
/* ------------------------------------------------------------------------ */

int orc_qp_dim(int N, int nu) { return (NX + nu) * N + 2 * NX * (N - 1); }

/* z = (x_1..x_N, u_1..u_N, mu^-_1..mu^-_{N-1}, mu^+_1..mu^+_{N-1}) */
void orc_z_pack(const orc_qp* qp, const orc_pd* s, double* z) {
  const int N = qp->N, nu = qp->nu;
  int o = 0;
  for (int i = 0; i < N * NX; i++) z[o++] = s->xh[i];
  for (int i = 0; i < N * nu; i++) z[o++] = s->uh[i];
  for (int i = 0; i < (N - 1) * NX; i++) z[o++] = s->mum[i];
  for (int i = 0; i < (N - 1) * NX; i++) z[o++] = s->mup[i];
}

void orc_z_unpack(const orc_qp* qp, const double* z, orc_pd* s) {
  const int N = qp->N, nu = qp->nu;
  int o = 0;
  for (int i = 0; i < N * NX; i++) s->xh[i] = z[o++];
  for (int i = 0; i < N * nu; i++) s->uh[i] = z[o++];
  for (int i = 0; i < (N - 1) * NX; i++) s->mum[i] = z[o++];
  for (int i = 0; i < (N - 1) * NX; i++) s->mup[i] = z[o++];
}

/* P [nz][nz], pv [nz], G [15(N-1)][nz], gv [15(N-1)], H [N-1][nz], hv [N-1],
 * lo/hi [nz]: the projection set (fixed boundary components, dilation box,
 * mu >= 0; lo = hi where a component is fixed). */
void orc_qp_dense(const orc_qp* qp, double* P, double* pv, double* G, double* gv,
                  double* H, double* hv, double* lo, double* hi) {
  const int N = qp->N, nu = qp->nu;
  const int nz = orc_qp_dim(N, nu);
  const int ox = 0, ou = NX * N, omm = (NX + nu) * N, omp = omm + NX * (N - 1);
  const int ng = NX * (N - 1);
  memset(P, 0, sizeof(double) * nz * nz);
  memset(pv, 0, sizeof(double) * nz);
  memset(G, 0, sizeof(double) * ng * nz);
  memset(H, 0, sizeof(double) * (N - 1) * nz);
  for (int i = 0; i < (NX + nu) * N; i++) P[i * nz + i] = qp->w_prox;
  for (int i = 0; i < NX; i++) pv[ox + (N - 1) * NX + i] = qp->w_cost * qp->ecost[i];
  for (int i = omm; i < nz; i++) pv[i] = qp->w_ep;
  for (int k = 0; k < N - 1; k++) {
    for (int i = 0; i < NX; i++) {
      int row = k * NX + i;
      for (int j = 0; j < NX; j++) {
        G[row * nz + ox + k * NX + j] += qp->Am[(k * NX + i) * NX + j];
        G[row * nz + ox + (k + 1) * NX + j] += qp->Ap[(k * NX + i) * NX + j];
      }
      for (int c = 0; c < nu; c++) {
        G[row * nz + ou + k * nu + c] += qp->Bm[(k * NX + i) * nu + c];
        G[row * nz + ou + (k + 1) * nu + c] += qp->Bp[(k * NX + i) * nu + c];
      }
      G[row * nz + omm + k * NX + i] = -1.0; /* -mu^-  (R4) */
      G[row * nz + omp + k * NX + i] = 1.0;  /* +mu^+ */
      gv[row] = -qp->w[k * NX + i];
    }
    H[k * nz + ox + k * NX + XY] = -1.0;
    H[k * nz + ox + (k + 1) * NX + XY] = 1.0;
    hv[k] = qp->eps[k];
  }
  for (int i = 0; i < nz; i++) { lo[i] = -INFINITY; hi[i] = INFINITY; }
  for (int i = 0; i < NX; i++) { lo[ox + i] = hi[ox + i] = qp->zi[i]; }
  for (int i = 0; i < NX; i++)
    if (qp->fixf[i]) lo[ox + (N - 1) * NX + i] = hi[ox + (N - 1) * NX + i] = qp->zf[i];
  for (int i = 0; i < N * nu; i++) { lo[ou + i] = qp->umin[i]; hi[ou + i] = qp->umax[i]; }
  for (int i = omm; i < nz; i++) lo[i] = 0.0;
}

void orc_pipg_generic(const orc_qp* qp, double alpha, double omega, double rho, int jmax,
                      const double* z1, const double* eta1, const double* chi1,
                      double* zout, double* wout, double* vout) {
  const int N = qp->N, nu = qp->nu;
  const int nz = orc_qp_dim(N, nu), ng = NX * (N - 1), nh = N - 1;
  double* P = malloc(sizeof(double) * nz * nz);
  double* pv = malloc(sizeof(double) * nz);
  double* G = malloc(sizeof(double) * ng * nz);
  double* gv = malloc(sizeof(double) * ng);
  double* H = malloc(sizeof(double) * nh * nz);
  double* hv = malloc(sizeof(double) * nh);
  double* lo = malloc(sizeof(double) * nz);
  double* hi = malloc(sizeof(double) * nz);
  double* zeta = malloc(sizeof(double) * nz);
  double* eta = malloc(sizeof(double) * ng);
  double* chi = malloc(sizeof(double) * nh);
  double* z = malloc(sizeof(double) * nz);
  double* w = malloc(sizeof(double) * ng);
  double* v = malloc(sizeof(double) * nh);
  double* d = malloc(sizeof(double) * nz);
  orc_qp_dense(qp, P, pv, G, gv, H, hv, lo, hi);
  memcpy(zeta, z1, sizeof(double) * nz);
  memcpy(eta, eta1, sizeof(double) * ng);
  memcpy(chi, chi1, sizeof(double) * nh);
  memcpy(z, z1, sizeof(double) * nz);
  memcpy(w, eta1, sizeof(double) * ng);
  memcpy(v, chi1, sizeof(double) * nh);
  const double beta = omega * alpha;
  for (int j = 1; j <= jmax; j++) {
    /* z <- Pi_D(zeta - alpha (P zeta + p + G^T eta + H^T chi)) */
    for (int i = 0; i < nz; i++) {
      double a = pv[i];
      for (int l = 0; l < nz; l++) a += P[i * nz + l] * zeta[l];
      for (int r = 0; r < ng; r++) a += G[r * nz + i] * eta[r];
      for (int r = 0; r < nh; r++) a += H[r * nz + i] * chi[r];
      z[i] = clampd(zeta[i] - alpha * a, lo[i], hi[i]);
    }
    if (qp->soc)
      for (int k = 0; k < N; k++) soc_project_uhat(qp, k, z + NX * N + k * nu);
    for (int i = 0; i < nz; i++) d[i] = 2.0 * z[i] - zeta[i];
    for (int r = 0; r < ng; r++) {
      double a = 0;
      for (int i = 0; i < nz; i++) a += G[r * nz + i] * d[i];
      w[r] = eta[r] + beta * (a - gv[r]);
    }
    for (int r = 0; r < nh; r++) {
      double a = 0;
      for (int i = 0; i < nz; i++) a += H[r * nz + i] * d[i];
      double t = chi[r] + beta * (a - hv[r]);
      v[r] = t > 0 ? t : 0;
    }
    for (int i = 0; i < nz; i++) zeta[i] = (1.0 - rho) * zeta[i] + rho * z[i];
    for (int r = 0; r < ng; r++) eta[r] = (1.0 - rho) * eta[r] + rho * w[r];
    for (int r = 0; r < nh; r++) chi[r] = (1.0 - rho) * chi[r] + rho * v[r];
  }
  memcpy(zout, z, sizeof(double) * nz);
  memcpy(wout, w, sizeof(double) * ng);
  memcpy(vout, v, sizeof(double) * nh);
  free(P); free(pv); free(G); free(gv); free(H); free(hv); free(lo); free(hi);
  free(zeta); free(eta); free(chi); free(z); free(w); free(v); free(d);
}

/* Cyclic Jacobi rotations; M is destroyed; returns the largest eigenvalue. */
double orc_sym_eig_max(int n, double* M) {
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0;
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) off += M[i * n + j] * M[i * n + j];
    if (off < 1e-30) break;
    for (int pp = 0; pp < n; pp++) {
      for (int q = pp + 1; q < n; q++) {
        double apq = M[pp * n + q];
        if (fabs(apq) < 1e-300) continue;
        double app = M[pp * n + pp], aqq = M[q * n + q];
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; k++) {
          double mkp = M[k * n + pp], mkq = M[k * n + q];
          M[k * n + pp] = c * mkp - s * mkq;
          M[k * n + q] = s * mkp + c * mkq;
        }
        for (int k = 0; k < n; k++) {
          double mpk = M[pp * n + k], mqk = M[q * n + k];
          M[pp * n + k] = c * mpk - s * mqk;
          M[q * n + k] = s * mpk + c * mqk;
        }
      }
    }
  }
  double mx = -INFINITY;
  for (int i = 0; i < n; i++) if (M[i * n + i] > mx) mx = M[i * n + i];
  return mx;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: SCP                                                            */
/* ------------------------------------------------------------------------ */

#ifndef ORC_MODEL_3DOF
/* Initial guess (Sec. 4 asks for "an appropriate" one; this reading):
 * straight lines in r, v, omega from x0 to z_f; normalized linear
 * interpolation of q from x0 to z_f; mass linear from m_wet to
 * (m_wet + m_dry)/2; y = 0; hover thrust m ||g|| along body x; gamma = 0;
 * s = tf_guess. */
void orc_init_guess(const orc_params* p, int N, const double* x0, double* X, double* U) {
  const int nu = p->nu;
  double g0 = sqrt(dot3(p->g_I, p->g_I));
  double mf = 0.5 * (x0[XM] + p->m_dry);
  double qf[4] = {p->z_f[XQ], p->z_f[XQ + 1], p->z_f[XQ + 2], p->z_f[XQ + 3]};
  double sg = 0;
  for (int i = 0; i < 4; i++) sg += x0[XQ + i] * qf[i];
  if (sg < 0) for (int i = 0; i < 4; i++) qf[i] = -qf[i];
  for (int k = 0; k < N; k++) {
    double t = (double)k / (N - 1);
    double* x = X + k * NX;
    x[XM] = (1.0 - t) * x0[XM] + t * mf;
    for (int i = 0; i < 3; i++) {
      x[XR + i] = (1.0 - t) * x0[XR + i] + t * p->z_f[XR + i];
      x[XV + i] = (1.0 - t) * x0[XV + i] + t * p->z_f[XV + i];
      x[XW + i] = (1.0 - t) * x0[XW + i] + t * p->z_f[XW + i];
    }
    double qq[4], nq = 0;
    for (int i = 0; i < 4; i++) { qq[i] = (1.0 - t) * x0[XQ + i] + t * qf[i]; nq += qq[i] * qq[i]; }
    nq = sqrt(nq);
    for (int i = 0; i < 4; i++) x[XQ + i] = qq[i] / nq;
    x[XY] = 0.0;
    double* u = U + k * nu;
    for (int c = 0; c < nu; c++) u[c] = 0.0;
    u[0] = x[XM] * g0;
    u[nu - 1] = p->tf_guess;
  }
}
#else
/* Initial guess of the 3-DoF model, the 6-DoF one without attitude: straight
 * lines in r, v from x0 to z_f, mass linear from m_wet to (m_wet + m_dry)/2,
 * y = 0, hover thrust m ||g|| along the up axis, s = tf_guess. */
void orc_init_guess(const orc_params* p, int N, const double* x0, double* X, double* U) {
  const int nu = p->nu;
  double g0 = sqrt(dot3(p->g_I, p->g_I));
  double mf = 0.5 * (x0[XM] + p->m_dry);
  for (int k = 0; k < N; k++) {
    double t = (double)k / (N - 1);
    double* x = X + k * NX;
    x[XM] = (1.0 - t) * x0[XM] + t * mf;
    for (int i = 0; i < 3; i++) {
      x[XR + i] = (1.0 - t) * x0[XR + i] + t * p->z_f[XR + i];
      x[XV + i] = (1.0 - t) * x0[XV + i] + t * p->z_f[XV + i];
    }
    x[XY] = 0.0;
    double* u = U + k * nu;
    for (int c = 0; c < nu; c++) u[c] = 0.0;
    u[0] = x[XM] * g0;
    u[nu - 1] = p->tf_guess;
  }
}
#endif

int orc_scp_iterate(const orc_params* p, int N, const double* x0, double* X, double* U,
                    orc_pd* ws, int force_pow, int force_pipg, double force_sigma,
                    double* sigma, int* pow_it, int* pipg_it, double* defect, double* step) {
  return orc_scp_iterate_m(p, N, x0, X, U, ws, force_pow, force_pipg, force_sigma, sigma, pow_it, pipg_it,
                           defect, step, NULL, NULL);
}

int orc_scp_iterate_m(const orc_params* p, int N, const double* x0, double* X, double* U,
                      orc_pd* ws, int force_pow, int force_pipg, double force_sigma,
                      double* sigma, int* pow_it, int* pipg_it, double* defect, double* step,
                      double* pow_margins, double* pipg_margins) {
  const int nu = p->nu;
  double* A = malloc(sizeof(double) * (N - 1) * NX * NX);
  double* Bm = malloc(sizeof(double) * (N - 1) * NX * nu);
  double* Bp = malloc(sizeof(double) * (N - 1) * NX * nu);
  double* xp = malloc(sizeof(double) * (N - 1) * NX);
  orc_qp qp;
  orc_qp_alloc(&qp, N, nu);
  orc_discretize(p, N, X, U, A, Bm, Bp, xp);
  orc_scale(p, N, x0, X, U, A, Bm, Bp, xp, &qp);
  int pit = 0;
  double sg = force_sigma > 0 ? force_sigma : orc_power_m(p, &qp, ws, force_pow, &pit, pow_margins);
  int jit = orc_pipgc_m(p, &qp, sg, ws, force_pipg, pipg_margins);
  double dfc = infn((N - 1) * NX, qp.w);
  double stp = maxd(infn(N * NX, ws->xh), infn(N * nu, ws->uh));
  for (int k = 0; k < N; k++) {
    for (int i = 0; i < NX; i++) X[k * NX + i] += p->P_x[i] * ws->xh[k * NX + i];
    for (int c = 0; c < nu; c++) U[k * nu + c] += p->P_u[c] * ws->uh[k * nu + c];
  }
  if (sigma) *sigma = sg;
  if (pow_it) *pow_it = pit;
  if (pipg_it) *pipg_it = jit;
  if (defect) *defect = dfc;
  if (step) *step = stp;
  orc_qp_free(&qp);
  free(A); free(Bm); free(Bp); free(xp);
  return 0;
}

/* Touchdown error of a trajectory: the last interval propagated by the same
 * RK4 (Eq. disc-dyn) from (x_{N-1}, u_{N-1}, u_N), compared with z_f on the
 * components E_f fixes, scaled by P_x: 0.5 sum ((x_prop - z_f) / P_x)^2. */
double orc_touchdown(const orc_params* p, int N, const double* X, const double* U) {
  const int nu = p->nu;
  double xp[NX];
  flow_dtau(p, X + (N - 2) * NX, U + (N - 2) * nu, U + (N - 1) * nu, 1.0 / (N - 1), p->rk4_substeps, xp);
  double e = 0;
  for (int i = 0; i < NX; i++)
    if (p->fix_f[i]) {
      double d = (xp[i] - p->z_f[i]) / p->P_x[i];
      e += 0.5 * d * d;
    }
  return e;
}

static int all_finite(int n, const double* a) {
  for (int i = 0; i < n; i++) if (!isfinite(a[i])) return 0;
  return 1;
}

/* SCP convergence (R8): the scaled step ||z_hat||_inf, the scaled defect
 * max_k ||hat w_k||_inf of the reference it was taken about, and the CTCS
 * budget y_N - y_1 <= (N-1) eps all within tolerance. */
int orc_solve(const orc_params* p, int N, const double* x0, double* X, double* U,
              orc_result* res, int* trace, int replay, int replay_scp) {
  return orc_solve_m(p, N, x0, X, U, res, trace, replay, replay_scp, NULL, NULL, NULL);
}

int orc_solve_m(const orc_params* p, int N, const double* x0, double* X, double* U,
                orc_result* res, int* trace, int replay, int replay_scp,
                double* scp_margins, double* pow_margins, double* pipg_margins) {
  const int nu = p->nu;
  orc_pd ws;
  orc_pd_alloc(&ws, N, nu);
  orc_pd_zero(&ws, N, nu);
  orc_init_guess(p, N, x0, X, U);
  memset(res, 0, sizeof *res);
  res->status = 1;
  int jmax = replay ? replay_scp : p->scp_jmax;
  int j;
  for (j = 1; j <= jmax; j++) {
    int fp = 0, fj = 0;
    if (replay) { fp = trace[(j - 1) * 2 + 0]; fj = trace[(j - 1) * 2 + 1]; }
    int pit, jit;
    double sg, dfc, stp;
    orc_scp_iterate_m(p, N, x0, X, U, &ws, fp, fj, 0.0, &sg, &pit, &jit, &dfc, &stp,
                      pow_margins ? pow_margins + (size_t)(j - 1) * p->pow_jmax : NULL,
                      pipg_margins ? pipg_margins + (size_t)(j - 1) * (p->pipg_jmax / p->pipg_jcheck) : NULL);
    if (trace && !replay) { trace[(j - 1) * 2 + 0] = pit; trace[(j - 1) * 2 + 1] = jit; }
    res->pipg_iters += jit;
    res->pow_iters += pit;
    res->defect = dfc;
    res->step = stp;
    if (!all_finite(N * NX, X) || !all_finite(N * nu, U)) { res->status = 2; break; }
    int conv = stp <= p->scp_eps_step && dfc <= p->scp_eps_defect &&
               (X[(N - 1) * NX + XY] - X[XY]) <= (N - 1) * p->eps_ctcs;
    if (scp_margins)
      scp_margins[j - 1] = maxd(maxd(margin(stp, p->scp_eps_step), margin(dfc, p->scp_eps_defect)),
                                margin(X[(N - 1) * NX + XY] - X[XY], (N - 1) * p->eps_ctcs));
    res->status = conv ? 0 : 1;
    if (conv && !replay) break;
  }
  if (j > jmax) j = jmax;
  res->scp_iters = j;
  double tf = 0;
  for (int k = 0; k < N - 1; k++) tf += 0.5 * (U[k * nu + nu - 1] + U[(k + 1) * nu + nu - 1]) / (N - 1);
  res->tf = tf;
  res->fuel = X[XM] - X[(N - 1) * NX + XM];
  orc_pd_free(&ws);
  return 0;
}

int orc_solve_batch(const orc_params* p, int B, int Nmax, const int* Ns, const double* x0s,
                    double* X, double* U, double* tf, double* fuel, int* status,
                    int* scp_iters, long long* pipg_iters, int nthreads) {
  const int nu = p->nu;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
  for (int b = 0; b < B; b++) {
    int N = Ns ? Ns[b] : Nmax;
    orc_result r;
    orc_solve(p, N, x0s + (size_t)b * (NX - 1), X + (size_t)b * Nmax * NX, U + (size_t)b * Nmax * nu, &r, NULL, 0, 0);
    if (tf) tf[b] = r.tf;
    if (fuel) fuel[b] = r.fuel;
    if (status) status[b] = r.status;
    if (scp_iters) scp_iters[b] = r.scp_iters;
    if (pipg_iters) pipg_iters[b] = r.pipg_iters;
  }
  return 0;
}
