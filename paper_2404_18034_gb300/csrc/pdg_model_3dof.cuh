// pdg_model_3dof.cuh -- the translational (3-DoF) powered-descent model as a
// second instance of the problem template of Sec. 2 of arXiv 2404.18034: the
// 6-DoF model of Sec. 4 without attitude.  State x = (m, r, v, y), controls
// (T, s) with T in the inertial frame:
//   m' = -alpha ||T||,  r' = v,  v' = T / m + g,
// path constraints (rows of g): m_dry - m, -r_x, ||v||^2 - v_max^2, the
// thrust-pointing cone ||T|| - sec(delta_max) T_x about the up axis (the 6-DoF
// gimbal row with the body axis taken as up), ||T|| - T_max, T_min - ||T||,
// and the optional squared glide-slope row of the 6-DoF model.  Final r and v
// fixed and the cost -m_N come from the parameters as for 6-DoF.  Included by
// pdg_device.cuh after DParams; see there for the model interface.
#pragma once

namespace pdg {

constexpr int NX = 8;
// state index
constexpr int IM = 0, IR = 1, IV = 4, IY = 7;
// compact df/dx slots of the stage buffer (see model_eval)
constexpr int SA_A = 12;
// no RCS torque, so nu = 4 only
#define PDG_MODEL_NU_ALT 4

// Structural sparsity of the interval STM A_k: the mass depends on no state,
// r_i on m, r_i, v_i; v_i on m, v_i; y on everything, nothing but y on y.
#define PDG_MODEL_HAS_STM_MASK 1
__host__ __device__ constexpr unsigned model_stm_row_mask(int i) {
  return i == 0 ? 1u : i <= 3 ? (1u | (1u << i) | (1u << (i + 3))) : i <= 6 ? (1u | (1u << i)) : 0xFFu;
}

// ---------------------------------------------------------------------------
// One call evaluates, at (x, u): f = s (F, sum |g|_+^2), the nonzero pattern
// of df/dx in compact form, and df/du densely (8 x NU).
// Compact A layout (SA_A slots):
//   [0]      s            (r rows wrt v)
//   [1..3]   dvdot/dm
//   [4..10]  y row: m, r_x, v0..2, r_y, r_z (r_y, r_z: glide slope); [11] unused
// ---------------------------------------------------------------------------
template <typename R, int NU>
__device__ __forceinline__ void model_eval(const DParams& P, const R* x, const R* u, R* f, R* A, R* Bd) {
  const R m = x[IM];
  const R rx = x[IR], ry = x[IR + 1], rz = x[IR + 2];
  const R v0 = x[IV], v1 = x[IV + 1], v2 = x[IV + 2];
  const R T0 = u[0], T1 = u[1], T2 = u[2];
  const R s = u[NU - 1];
  const R nT = sqrt(T0 * T0 + T1 * T1 + T2 * T2);
  const R inT = nT > R(0) ? R(1) / nT : R(0);
  const R t0 = T0 * inT, t1 = T1 * inT, t2 = T2 * inT;
  const R im = R(1) / m;
  R F[7];
  F[0] = -R(P.alpha_mdot) * nT;
  F[1] = v0; F[2] = v1; F[3] = v2;
  F[4] = T0 * im + R(P.g[0]);
  F[5] = T1 * im + R(P.g[1]);
  F[6] = T2 * im + R(P.g[2]);
  R gp[7];
  gp[0] = R(P.m_dry) - m;
  gp[1] = -rx;
  gp[2] = v0 * v0 + v1 * v1 + v2 * v2 - R(P.vmax2);
  gp[3] = nT - T0 * R(P.sec_delta);
  gp[4] = nT - R(P.T_max);
  gp[5] = R(P.T_min) - nT;
  if (P.soc) { gp[3] = R(-1); gp[4] = R(-1); }  // imposed by projection instead
  gp[6] = P.gs ? R(P.tan_gs2) * (ry * ry + rz * rz) - rx * rx : R(-1);
  R pen = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    gp[i] = gp[i] > R(0) ? gp[i] : R(0);
    pen += gp[i] * gp[i];
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) f[i] = s * F[i];
  f[7] = s * pen;
  const R sim = s * im;
  A[0] = s;
  A[1] = -sim * im * T0;
  A[2] = -sim * im * T1;
  A[3] = -sim * im * T2;
  const R s2 = R(2) * s;
  A[4] = -s2 * gp[0];
  A[5] = -s2 * (gp[1] + gp[6] * R(2) * rx);
  A[6] = s2 * gp[2] * R(2) * v0;
  A[7] = s2 * gp[2] * R(2) * v1;
  A[8] = s2 * gp[2] * R(2) * v2;
  A[9] = s2 * gp[6] * R(2) * R(P.tan_gs2) * ry;
  A[10] = s2 * gp[6] * R(2) * R(P.tan_gs2) * rz;
  A[11] = 0;
#pragma unroll
  for (int i = 0; i < NX * NU; ++i) Bd[i] = R(0);
  const R sa = -s * R(P.alpha_mdot);
  Bd[0 * NU + 0] = sa * t0; Bd[0 * NU + 1] = sa * t1; Bd[0 * NU + 2] = sa * t2;
  Bd[4 * NU + 0] = sim; Bd[5 * NU + 1] = sim; Bd[6 * NU + 2] = sim;
  const R gt = gp[3] + gp[4] - gp[5];
  Bd[7 * NU + 0] = s2 * (gt * t0 - gp[3] * R(P.sec_delta));
  Bd[7 * NU + 1] = s2 * gt * t1;
  Bd[7 * NU + 2] = s2 * gt * t2;
#pragma unroll
  for (int i = 0; i < 7; ++i) Bd[i * NU + NU - 1] = F[i];
  Bd[7 * NU + NU - 1] = pen;
}

// d = (df/dx) S + lam * (df/du) e_cu, from the compact stage buffer.
template <typename R, int NU>
__device__ __forceinline__ void model_jvp(const R* __restrict__ A, const R* __restrict__ Bd, const R* S,
                                          int cu, R lam, R* d) {
  d[0] = R(0);
  d[1] = A[0] * S[4]; d[2] = A[0] * S[5]; d[3] = A[0] * S[6];
  d[4] = A[1] * S[0]; d[5] = A[2] * S[0]; d[6] = A[3] * S[0];
  d[7] = A[4] * S[0] + A[5] * S[1] + A[6] * S[4] + A[7] * S[5] + A[8] * S[6] + A[9] * S[2] + A[10] * S[3];
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
  xb[0] += A[1] * v[4] + A[2] * v[5] + A[3] * v[6];
  xb[0] += A[4] * v[7]; xb[1] += A[5] * v[7]; xb[2] += A[9] * v[7]; xb[3] += A[10] * v[7];
  xb[4] += A[6] * v[7]; xb[5] += A[7] * v[7]; xb[6] += A[8] * v[7];
#pragma unroll
  for (int c = 0; c < NU; ++c) {
    double a = 0;
#pragma unroll
    for (int i = 0; i < NX; ++i) a += Bd[i * NU + c] * v[i];
    ub[c] += a;
  }
}

// Initial guess at node fraction t = (k-1)/(N-1): the 6-DoF guess without
// attitude -- straight lines in r, v from x0 to z_f, mass from m_wet to
// (m_wet + m_dry)/2, y = 0, hover thrust m|g| along the up axis, s = tf_guess.
template <typename R, int NU>
__device__ __forceinline__ void model_init_node(const DParams& P, const R* x0, R t, R* x, R* u) {
  const R a = R(1) - t;
  const R mf = R(0.5) * (x0[IM] + R(P.m_dry));
  x[IM] = a * x0[IM] + t * mf;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    x[IR + i] = a * x0[IR + i] + t * R(P.z_f[IR + i]);
    x[IV + i] = a * x0[IV + i] + t * R(P.z_f[IV + i]);
  }
  x[IY] = 0;
#pragma unroll
  for (int c = 0; c < NU; ++c) u[c] = 0;
  u[0] = x[IM] * R(P.g0);
  u[NU - 1] = R(P.tf_guess);
}

}  // namespace pdg
