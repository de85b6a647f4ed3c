// pdg_model_6dof.cuh -- the 6-DoF powered-descent model of Sec. 4 of arXiv
// 2404.18034 as an instance of the problem template of Sec. 2: state
// x = (m, r, v, q, omega, y), controls (T, [gamma,] s).  Included by
// pdg_device.cuh after DParams; see there for the model interface.
#pragma once

namespace pdg {

constexpr int NX = 15;
// state index
constexpr int IM = 0, IR = 1, IV = 4, IQ = 7, IW = 11, IY = 14;
// compact df/dx slots of the stage buffer (see model_eval)
constexpr int SA_A = 42;
// the model has the RCS-torque controls (nu = 7) and reads the inertia J_B
#define PDG_MODEL_NU_ALT 7
#define PDG_MODEL_USES_INERTIA 1

// Structural sparsity of the interval STM A_k (rows i, columns c): the mass
// depends on no state; r_i on m, r_i, v_i, q, w (through v_i); v_i on m,
// v_i, q, w; q on q, w; w on w; y on everything, and nothing but y on y.
// These are the closure of df/dx's pattern (model_jvp) under the flow, for
// every parameter value (inertia, thrust point, glide slope, nu).
#define PDG_MODEL_HAS_STM_MASK 1
__host__ __device__ constexpr unsigned model_stm_row_mask(int i) {
  constexpr unsigned M = 1u << 0, Q = 0xFu << 7, W = 0x7u << 11;
  return i == 0 ? M
       : i <= 3 ? (M | (1u << i) | (1u << (i + 3)) | Q | W)
       : i <= 6 ? (M | (1u << i) | Q | W)
       : i <= 10 ? (Q | W)
       : i <= 13 ? W
       : 0x7FFFu;
}

// ---------------------------------------------------------------------------
// Sec. 4 model.  One call evaluates, at (x, u): f = s (F, sum |g|_+^2), the
// nonzero pattern of df/dx in compact form, and df/du densely (15 x NU).
// Compact A layout (SA_A slots):
//   [0]  s           (r rows wrt v)
//   [1..3]  dvdot/dm
//   [4..15] dvdot/dq (3 x 4)
//   [16..18] (s/2) w  -> q rows wrt q through Omega(w)
//   [19..22] (s/2) q  -> q rows wrt w through Xi(q)
//   [23..28] dwdot/dw off-diagonals (01, 02, 10, 12, 20, 21)
//   [29..38] y row: m, r_x, v0..2, q2, q3, w0..2
//   [39..40] y row: r_y, r_z (glide slope); [41] unused
// ---------------------------------------------------------------------------
template <typename R, int NU>
__device__ __forceinline__ void model_eval(const DParams& P, const R* x, const R* u, R* f, R* A, R* Bd) {
  const R m = x[IM];
  const R v0 = x[IV], v1 = x[IV + 1], v2 = x[IV + 2];
  const R q0 = x[IQ], q1 = x[IQ + 1], q2 = x[IQ + 2], q3 = x[IQ + 3];
  const R w0 = x[IW], w1 = x[IW + 1], w2 = x[IW + 2];
  const R T0 = u[0], T1 = u[1], T2 = u[2];
  const R s = u[NU - 1];
  R gm0 = 0, gm1 = 0, gm2 = 0;
  if (NU == 7) { gm0 = u[3]; gm1 = u[4]; gm2 = u[5]; }
  const R nT = sqrt(T0 * T0 + T1 * T1 + T2 * T2);
  const R inT = nT > R(0) ? R(1) / nT : R(0);
  const R t0 = T0 * inT, t1 = T1 * inT, t2 = T2 * inT;
  const R im = R(1) / m;
  // C(q) T, Hamilton scalar-first, body -> inertial
  const R C00 = R(1) - R(2) * (q2 * q2 + q3 * q3), C01 = R(2) * (q1 * q2 - q0 * q3), C02 = R(2) * (q1 * q3 + q0 * q2);
  const R C10 = R(2) * (q1 * q2 + q0 * q3), C11 = R(1) - R(2) * (q1 * q1 + q3 * q3), C12 = R(2) * (q2 * q3 - q0 * q1);
  const R C20 = R(2) * (q1 * q3 - q0 * q2), C21 = R(2) * (q2 * q3 + q0 * q1), C22 = R(1) - R(2) * (q1 * q1 + q2 * q2);
  const R CT0 = C00 * T0 + C01 * T1 + C02 * T2;
  const R CT1 = C10 * T0 + C11 * T1 + C12 * T2;
  const R CT2 = C20 * T0 + C21 * T1 + C22 * T2;
  const R J0 = R(P.J[0]), J1 = R(P.J[1]), J2 = R(P.J[2]);
  const R iJ0 = R(P.Jinv[0]), iJ1 = R(P.Jinv[1]), iJ2 = R(P.Jinv[2]);
  const R rT0 = R(P.rT[0]), rT1 = R(P.rT[1]), rT2 = R(P.rT[2]);
  // torque: r_T x T - w x (J w) + gamma
  const R tq0 = rT1 * T2 - rT2 * T1 - (J2 - J1) * w1 * w2 + gm0;
  const R tq1 = rT2 * T0 - rT0 * T2 - (J0 - J2) * w0 * w2 + gm1;
  const R tq2 = rT0 * T1 - rT1 * T0 - (J1 - J0) * w0 * w1 + gm2;
  R F[14];
  F[0] = -R(P.alpha_mdot) * nT;
  F[1] = v0; F[2] = v1; F[3] = v2;
  F[4] = CT0 * im + R(P.g[0]);
  F[5] = CT1 * im + R(P.g[1]);
  F[6] = CT2 * im + R(P.g[2]);
  F[7] = R(0.5) * (-w0 * q1 - w1 * q2 - w2 * q3);
  F[8] = R(0.5) * (w0 * q0 + w2 * q2 - w1 * q3);
  F[9] = R(0.5) * (w1 * q0 - w2 * q1 + w0 * q3);
  F[10] = R(0.5) * (w2 * q0 + w1 * q1 - w0 * q2);
  F[11] = tq0 * iJ0; F[12] = tq1 * iJ1; F[13] = tq2 * iJ2;
  // path constraints (tilt row per the reading 2(q2^2+q3^2) - (1 - cos theta_max))
  R gp[10];
  gp[0] = R(P.m_dry) - m;
  gp[1] = -x[IR];
  gp[2] = v0 * v0 + v1 * v1 + v2 * v2 - R(P.vmax2);
  gp[3] = R(2) * (q2 * q2 + q3 * q3) - R(P.one_m_cos_theta);
  gp[4] = w0 * w0 + w1 * w1 + w2 * w2 - R(P.omega_max2);
  gp[5] = nT - T0 * R(P.sec_delta);
  gp[6] = nT - R(P.T_max);
  gp[7] = R(P.T_min) - nT;
  gp[8] = (NU == 7) ? (gm0 * gm0 + gm1 * gm1 + gm2 * gm2 - R(P.gamma_max2)) : R(-1);
  if (P.soc) { gp[5] = R(-1); gp[6] = R(-1); }  // imposed by projection instead
  // glide slope, squared so that it is smooth at the cone's apex (touchdown)
  const R rx = x[IR], ry = x[IR + 1], rz = x[IR + 2];
  gp[9] = P.gs ? R(P.tan_gs2) * (ry * ry + rz * rz) - rx * rx : R(-1);
  R pen = 0;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    gp[i] = gp[i] > R(0) ? gp[i] : R(0);
    pen += gp[i] * gp[i];
  }
#pragma unroll
  for (int i = 0; i < 14; ++i) f[i] = s * F[i];
  f[14] = s * pen;
  // compact df/dx
  const R sim = s * im;
  A[0] = s;
  A[1] = -sim * im * CT0;
  A[2] = -sim * im * CT1;
  A[3] = -sim * im * CT2;
  // d(C T)/dq_j, rows i
  const R d00 = R(2) * (-q3 * T1 + q2 * T2), d01 = R(2) * (q2 * T1 + q3 * T2);
  const R d02 = R(2) * (-R(2) * q2 * T0 + q1 * T1 + q0 * T2), d03 = R(2) * (-R(2) * q3 * T0 - q0 * T1 + q1 * T2);
  const R d10 = R(2) * (q3 * T0 - q1 * T2), d11 = R(2) * (q2 * T0 - R(2) * q1 * T1 - q0 * T2);
  const R d12 = R(2) * (q1 * T0 + q3 * T2), d13 = R(2) * (q0 * T0 - R(2) * q3 * T1 + q2 * T2);
  const R d20 = R(2) * (-q2 * T0 + q1 * T1), d21 = R(2) * (q3 * T0 + q0 * T1 - R(2) * q1 * T2);
  const R d22 = R(2) * (-q0 * T0 + q3 * T1 - R(2) * q2 * T2), d23 = R(2) * (q1 * T0 + q2 * T1);
  A[4] = sim * d00; A[5] = sim * d01; A[6] = sim * d02; A[7] = sim * d03;
  A[8] = sim * d10; A[9] = sim * d11; A[10] = sim * d12; A[11] = sim * d13;
  A[12] = sim * d20; A[13] = sim * d21; A[14] = sim * d22; A[15] = sim * d23;
  const R hs = R(0.5) * s;
  A[16] = hs * w0; A[17] = hs * w1; A[18] = hs * w2;
  A[19] = hs * q0; A[20] = hs * q1; A[21] = hs * q2; A[22] = hs * q3;
  A[23] = -s * iJ0 * (J2 - J1) * w2;
  A[24] = -s * iJ0 * (J2 - J1) * w1;
  A[25] = -s * iJ1 * (J0 - J2) * w2;
  A[26] = -s * iJ1 * (J0 - J2) * w0;
  A[27] = -s * iJ2 * (J1 - J0) * w1;
  A[28] = -s * iJ2 * (J1 - J0) * w0;
  const R s2 = R(2) * s;
  A[29] = -s2 * gp[0];
  A[30] = -s2 * (gp[1] + gp[9] * R(2) * rx);
  A[31] = s2 * gp[2] * R(2) * v0;
  A[32] = s2 * gp[2] * R(2) * v1;
  A[33] = s2 * gp[2] * R(2) * v2;
  A[34] = s2 * gp[3] * R(4) * q2;
  A[35] = s2 * gp[3] * R(4) * q3;
  A[36] = s2 * gp[4] * R(2) * w0;
  A[37] = s2 * gp[4] * R(2) * w1;
  A[38] = s2 * gp[4] * R(2) * w2;
  A[39] = s2 * gp[9] * R(2) * R(P.tan_gs2) * ry;
  A[40] = s2 * gp[9] * R(2) * R(P.tan_gs2) * rz;
  A[41] = 0;
  // dense df/du
#pragma unroll
  for (int i = 0; i < NX * NU; ++i) Bd[i] = R(0);
  const R sa = -s * R(P.alpha_mdot);
  Bd[0 * NU + 0] = sa * t0; Bd[0 * NU + 1] = sa * t1; Bd[0 * NU + 2] = sa * t2;
  Bd[4 * NU + 0] = sim * C00; Bd[4 * NU + 1] = sim * C01; Bd[4 * NU + 2] = sim * C02;
  Bd[5 * NU + 0] = sim * C10; Bd[5 * NU + 1] = sim * C11; Bd[5 * NU + 2] = sim * C12;
  Bd[6 * NU + 0] = sim * C20; Bd[6 * NU + 1] = sim * C21; Bd[6 * NU + 2] = sim * C22;
  // d(r_T x T)/dT = [r_T]x
  Bd[11 * NU + 1] = -s * iJ0 * rT2; Bd[11 * NU + 2] = s * iJ0 * rT1;
  Bd[12 * NU + 0] = s * iJ1 * rT2;  Bd[12 * NU + 2] = -s * iJ1 * rT0;
  Bd[13 * NU + 0] = -s * iJ2 * rT1; Bd[13 * NU + 1] = s * iJ2 * rT0;
  const R gt = gp[5] + gp[6] - gp[7];
  Bd[14 * NU + 0] = s2 * (gt * t0 - gp[5] * R(P.sec_delta));
  Bd[14 * NU + 1] = s2 * gt * t1;
  Bd[14 * NU + 2] = s2 * gt * t2;
  if (NU == 7) {
    Bd[11 * NU + 3] = s * iJ0; Bd[12 * NU + 4] = s * iJ1; Bd[13 * NU + 5] = s * iJ2;
    Bd[14 * NU + 3] = s2 * gp[8] * R(2) * gm0;
    Bd[14 * NU + 4] = s2 * gp[8] * R(2) * gm1;
    Bd[14 * NU + 5] = s2 * gp[8] * R(2) * gm2;
  }
#pragma unroll
  for (int i = 0; i < 14; ++i) Bd[i * NU + NU - 1] = F[i];
  Bd[14 * NU + NU - 1] = pen;
}

// d = (df/dx) S + lam * (df/du) e_cu, from the compact stage buffer.
template <typename R, int NU>
__device__ __forceinline__ void model_jvp(const R* __restrict__ A, const R* __restrict__ Bd, const R* S,
                                          int cu, R lam, R* d) {
  d[0] = R(0);
  d[1] = A[0] * S[4]; d[2] = A[0] * S[5]; d[3] = A[0] * S[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    d[4 + i] = A[1 + i] * S[0] + A[4 + 4 * i] * S[7] + A[5 + 4 * i] * S[8] + A[6 + 4 * i] * S[9] + A[7 + 4 * i] * S[10];
  const R hw0 = A[16], hw1 = A[17], hw2 = A[18], hq0 = A[19], hq1 = A[20], hq2 = A[21], hq3 = A[22];
  const R a0 = S[7], a1 = S[8], a2 = S[9], a3 = S[10], b0 = S[11], b1 = S[12], b2 = S[13];
  d[7] = -hw0 * a1 - hw1 * a2 - hw2 * a3 - hq1 * b0 - hq2 * b1 - hq3 * b2;
  d[8] = hw0 * a0 + hw2 * a2 - hw1 * a3 + hq0 * b0 - hq3 * b1 + hq2 * b2;
  d[9] = hw1 * a0 - hw2 * a1 + hw0 * a3 + hq3 * b0 + hq0 * b1 - hq1 * b2;
  d[10] = hw2 * a0 + hw1 * a1 - hw0 * a2 - hq2 * b0 + hq1 * b1 + hq0 * b2;
  d[11] = A[23] * b1 + A[24] * b2;
  d[12] = A[25] * b0 + A[26] * b2;
  d[13] = A[27] * b0 + A[28] * b1;
  d[14] = A[29] * S[0] + A[30] * S[1] + A[31] * S[4] + A[32] * S[5] + A[33] * S[6] + A[34] * a2 + A[35] * a3 +
          A[36] * b0 + A[37] * b1 + A[38] * b2 + A[39] * S[2] + A[40] * S[3];
  if (cu >= 0) {
#pragma unroll
    for (int i = 0; i < NX; ++i) d[i] += lam * Bd[i * NU + cu];
  }
}

// xb += (df/dx)^T v, ub += (df/du)^T v from a compact stage buffer (the
// transpose of model_jvp).
template <int NU>
__device__ __forceinline__ void model_vjp(const double* A, const double* Bd, const double* v, double* xb, double* ub) {
  xb[4] += A[0] * v[1]; xb[5] += A[0] * v[2]; xb[6] += A[0] * v[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    xb[0] += A[1 + i] * v[4 + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) xb[7 + j] += A[4 + 4 * i + j] * v[4 + i];
  }
  const double hw0 = A[16], hw1 = A[17], hw2 = A[18], hq0 = A[19], hq1 = A[20], hq2 = A[21], hq3 = A[22];
  const double v7 = v[7], v8 = v[8], v9 = v[9], v10 = v[10];
  xb[7] += hw0 * v8 + hw1 * v9 + hw2 * v10;
  xb[8] += -hw0 * v7 - hw2 * v9 + hw1 * v10;
  xb[9] += -hw1 * v7 + hw2 * v8 - hw0 * v10;
  xb[10] += -hw2 * v7 - hw1 * v8 + hw0 * v9;
  xb[11] += -hq1 * v7 + hq0 * v8 + hq3 * v9 - hq2 * v10;
  xb[12] += -hq2 * v7 - hq3 * v8 + hq0 * v9 + hq1 * v10;
  xb[13] += -hq3 * v7 + hq2 * v8 - hq1 * v9 + hq0 * v10;
  xb[12] += A[23] * v[11]; xb[13] += A[24] * v[11];
  xb[11] += A[25] * v[12]; xb[13] += A[26] * v[12];
  xb[11] += A[27] * v[13]; xb[12] += A[28] * v[13];
  xb[0] += A[29] * v[14]; xb[1] += A[30] * v[14]; xb[2] += A[39] * v[14]; xb[3] += A[40] * v[14];
  xb[4] += A[31] * v[14]; xb[5] += A[32] * v[14]; xb[6] += A[33] * v[14];
  xb[9] += A[34] * v[14]; xb[10] += A[35] * v[14];
  xb[11] += A[36] * v[14]; xb[12] += A[37] * v[14]; xb[13] += A[38] * v[14];
#pragma unroll
  for (int c = 0; c < NU; ++c) {
    double a = 0;
#pragma unroll
    for (int i = 0; i < NX; ++i) a += Bd[i * NU + c] * v[i];
    ub[c] += a;
  }
}

// Initial guess at node fraction t = (k-1)/(N-1) (the paper asks for "an
// appropriate" one; Sec. 4): straight lines in r, v, w from x0 to z_f,
// normalized linear interpolation of q, mass from m_wet to (m_wet + m_dry)/2,
// y = 0, hover thrust m|g| along body x, gamma = 0, s = tf_guess.
template <typename R, int NU>
__device__ __forceinline__ void model_init_node(const DParams& P, const R* x0, R t, R* x, R* u) {
  const R a = R(1) - t;
  const R mf = R(0.5) * (x0[IM] + R(P.m_dry));
  x[IM] = a * x0[IM] + t * mf;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    x[IR + i] = a * x0[IR + i] + t * R(P.z_f[IR + i]);
    x[IV + i] = a * x0[IV + i] + t * R(P.z_f[IV + i]);
    x[IW + i] = a * x0[IW + i] + t * R(P.z_f[IW + i]);
  }
  R dq = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) dq += x0[IQ + i] * R(P.z_f[IQ + i]);
  const R sg = dq < R(0) ? R(-1) : R(1);
  R qq[4], n2 = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    qq[i] = a * x0[IQ + i] + t * sg * R(P.z_f[IQ + i]);
    n2 += qq[i] * qq[i];
  }
  const R inq = R(1) / sqrt(n2);
#pragma unroll
  for (int i = 0; i < 4; ++i) x[IQ + i] = qq[i] * inq;
  x[IY] = 0;
#pragma unroll
  for (int c = 0; c < NU; ++c) u[c] = 0;
  u[0] = x[IM] * R(P.g0);
  u[NU - 1] = R(P.tf_guess);
}

}  // namespace pdg
