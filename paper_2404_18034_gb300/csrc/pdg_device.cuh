// pdg_device.cuh -- device side of the batched solver: parameters, per-instance
// shared-memory layout, the 6-DoF model with its compact Jacobians, and the
// phases of one SCP iteration (arXiv 2404.18034, Sec. 2-5).  One CTA owns one
// instance at a time; every block of its subproblem lives in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdg {

constexpr int NX = 15;
constexpr int NMAX = 32;
// state index
constexpr int IM = 0, IR = 1, IV = 4, IQ = 7, IW = 11, IY = 14;
constexpr int ST_RUNNING = -1;

// Parameters as the kernels see them (derived constants precomputed on the host).
struct DParams {
  int nu, nsub, pipg_jmax, pipg_jcheck, pow_jmax, scp_jmax;
  int fix_f[NX];
  double alpha_mdot, g[3], J[3], Jinv[3], rT[3];
  double m_dry, vmax2, one_m_cos_theta, omega_max2, sec_delta, T_min, T_max, gamma_max2;
  double s_min, s_max;
  double z_f[NX];
  double Px[NX], Pxinv[NX], Pu[7], Puinv[7];
  double w_cost, w_prox, w_ep, eps_ctcs;
  double omega, rho, eps_abs, eps_rel;
  double pow_eps_abs, pow_eps_rel, pow_buff;
  double scp_eps_step, scp_eps_defect;
  double tf_guess, g0;
  double budget_ns;  // 0 = none
  int soc;           // thrust sector by projection (T_max, gimbal rows off)
  double soc_tan;    // tan(delta_max)
  int gs;            // glide-slope row on
  double tan_gs2;    // tan^2(gamma_gs)
  double s_lo, s_hi; // node box on the dilation: [s_min, s_max] tightened by the time bounds,
  double dt_lo, dt_hi;  // of which dt_min, dt_max scale with N - 1 (0 = off)
};

// Per-instance shared-memory layout (element offsets in units of R).  The
// "image" prefix is what persists between phases (and what the plain form
// keeps in global memory); the union region is phase-local scratch.
struct Lay {
  int N, nu, ipw, sa;
  int sc, x0, Xb, Ub, Am, Bm, Bp, w, eps, lo, hi, zi, zf, xh, uh, mup, mum, phi, th, img;
  int xt, ut, nup, num, vph, vth, dx, du, td, stage, red, total;
};

// stage buffer of one interval: compact A (40), dense B (15 x nu), then the
// evaluator's RK4 state of x: base P, accumulator, stage input (15 each)
constexpr int SA_A = 42;

// Intervals per discretization wave: warp 0 evaluates the model of up to 32
// intervals, the remaining warps hold one STM column per thread.
__host__ __device__ inline int waves_ipw(int threads, int nu) {
  const int ncol = NX + 2 * nu;
  const int w = (threads - 32) / ncol;
  return w > 32 ? 32 : w;
}

__host__ __device__ inline int round32(int x) { return (x + 31) & ~31; }

__host__ __device__ inline Lay make_lay(int N, int nu, int threads) {
  Lay L;
  L.N = N;
  L.nu = nu;
  L.ipw = waves_ipw(threads, nu);
  L.sa = SA_A + NX * nu + 3 * NX;
  int o = 0;
  L.sc = o; o += 8;
  L.x0 = o; o += 16;
  L.Xb = o; o += N * NX;
  L.Ub = o; o += N * nu;
  L.Am = o; o += (N - 1) * NX * NX;
  L.Bm = o; o += (N - 1) * NX * nu;
  L.Bp = o; o += (N - 1) * NX * nu;
  L.w = o; o += (N - 1) * NX;
  L.eps = o; o += N - 1;
  L.lo = o; o += N;
  L.hi = o; o += N;
  L.zi = o; o += NX;
  L.zf = o; o += NX;
  L.xh = o; o += N * NX;
  L.uh = o; o += N * nu;
  L.mup = o; o += (N - 1) * NX;
  L.mum = o; o += (N - 1) * NX;
  L.phi = o; o += (N - 1) * NX;
  L.th = o; o += N - 1;
  o = (o + 1) & ~1;
  L.img = o;
  int u = o;
  L.xt = u; u += N * NX;
  L.ut = u; u += N * nu;
  L.nup = u; u += (N - 1) * NX;
  L.num = u; u += (N - 1) * NX;
  L.vph = u; u += (N - 1) * NX;
  L.vth = u; u += N - 1;
  L.dx = u; u += N * NX;
  L.du = u; u += N * nu;
  L.td = u; u += (N - 1) * NX;  // PIPG: CTCS-dual difference per node (N used)
  int u2 = o;
  L.stage = u2; u2 += L.ipw * L.sa;
  o = u > u2 ? u : u2;
  o = (o + 1) & ~1;
  L.red = o; o += 6 * 32 + 8;
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// block reductions (every thread of the CTA must call them)
// ---------------------------------------------------------------------------
template <typename R, int K>
__device__ __forceinline__ void block_max_k(R (&v)[K], R* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) red[wid * K + q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    R m = red[q];
    for (int i = 1; i < nw; ++i) m = fmax(m, red[i * K + q]);
    v[q] = m;
  }
  __syncthreads();
}

template <typename R>
__device__ __forceinline__ R block_sum(R v, R* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  R s = red[0];
  for (int i = 1; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Non-negative floating-point numbers order like their bit patterns, so the
// maxima of the PIPG stop test (of |.|, mu >= 0, theta >= 0) are taken exactly
// in integer arithmetic: on GB300 every FP64 warp instruction costs a slot of
// the narrow FP64 pipe whatever its active lanes, integer ones do not.
template <typename R> struct OrdBits;
template <> struct OrdBits<double> {
  using U = unsigned long long;
  __device__ __forceinline__ static U abs(double x) { return U(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull; }
  __device__ __forceinline__ static U nonneg(double x) { return U(__double_as_longlong(x)); }
  __device__ __forceinline__ static double val(U u) { return __longlong_as_double((long long)u); }
};
template <> struct OrdBits<float> {
  using U = unsigned int;
  __device__ __forceinline__ static U abs(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }
  __device__ __forceinline__ static U nonneg(float x) { return __float_as_uint(x); }
  __device__ __forceinline__ static float val(U u) { return __uint_as_float(u); }
};
template <typename U>
__device__ __forceinline__ U umax(U a, U b) { return a > b ? a : b; }

// Block-wide maxima of K unsigned values (every thread calls it; red holds
// K * 32 values of U).
template <typename U, int K>
__device__ __forceinline__ void block_max_u(U (&v)[K], U* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] = umax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) red[wid * K + q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    U m = red[q];
    for (int i = 1; i < nw; ++i) m = umax(m, red[i * K + q]);
    v[q] = m;
  }
  __syncthreads();
}

template <typename R>
__device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
template <typename R>
__device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// Sec. 5 model.  One call evaluates, at (x, u): f = s (F, sum |g|_+^2), the
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

}  // namespace pdg
