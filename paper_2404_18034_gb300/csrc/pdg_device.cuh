// pdg_device.cuh -- device side of the batched solver: parameters, the
// per-instance shared-memory layout, the choice of the model (the 6-DoF model
// of Sec. 4, the 3-DoF model, or a caller's header) and block reductions
// (arXiv 2404.18034, Sec. 2-5).  One CTA owns one instance at a time; every
// block of its subproblem lives in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdg {

constexpr int NMAX = 32;
constexpr int NXMAX = 15;  // largest state size of the models (parameter arrays)
constexpr int ST_RUNNING = -1;

// Parameters as the kernels see them (derived constants precomputed on the host).
struct DParams {
  int nu, nsub, pipg_jmax, pipg_jcheck, pow_jmax, scp_jmax;
  int fix_f[NXMAX];
  double alpha_mdot, g[3], J[3], Jinv[3], rT[3];
  double m_dry, vmax2, one_m_cos_theta, omega_max2, sec_delta, T_min, T_max, gamma_max2;
  double s_min, s_max;
  double z_f[NXMAX];
  double Px[NXMAX], Pxinv[NXMAX], Pu[7], Puinv[7];
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
  double mp[16];     // constants of a model supplied through PDG_MODEL_HEADER
  const int* abort_flag;  // the handle's abort word (host memory mapped into the
                          // device's address space), or null
};

// The handle's abort request, read at system scope so that a store from a
// host thread is seen while a kernel runs.  One thread reads; the callers
// broadcast the answer so that a CTA decides as one.
__device__ __forceinline__ bool abort_requested(const DParams& P) {
  if (!P.abort_flag) return false;
  int v;
  asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(P.abort_flag) : "memory");
  return v != 0;
}

// Per-instance shared-memory layout (element offsets in units of R).  The
// "image" prefix is what persists between phases (and what the plain form
// keeps in global memory); the union region is phase-local scratch.
struct Lay {
  int N, nu, ipw, sa;
  int sc, x0, Xb, Ub, Am, Bm, Bp, w, eps, lo, hi, zi, zf, xh, uh, mup, mum, phi, th, img;
  int xt, ut, nup, num, vph, vth, dx, du, td, stage, red, total;
};

}  // namespace pdg

// The model -- F, g, their compact Jacobians and the initial guess of one
// instance of the problem template of Sec. 2 -- is chosen when the library is
// compiled: the 6-DoF model of Sec. 4 by default, the translational 3-DoF
// model with PDG_MODEL_3DOF, or a model of the caller's with
// PDG_MODEL_HEADER="<path>".  A model header defines, in namespace pdg:
//   NX          state size; the CTCS integrator y is the last state (IY = NX-1)
//   IM          index of the mass, whose final value the cost maximizes
//   IY          NX - 1
//   SA_A        slots of its compact df/dx
//   PDG_MODEL_NU_ALT  a second control size it supports besides 4 (else 4)
//   PDG_MODEL_USES_INERTIA  defined when the model reads J_B (then checked > 0)
//   model_eval<R, NU>(P, x, u, f, A, Bd): f = s (F, sum |g|_+^2), compact
//               df/dx in A[SA_A], dense df/du in Bd[NX][NU]
//   model_jvp<R, NU>(A, Bd, S, cu, lam, d): d = (df/dx) S + lam (df/du) e_cu
//   model_vjp<NU>(A, Bd, v, xb, ub): xb += (df/dx)^T v, ub += (df/du)^T v
//   model_init_node<R, NU>(P, x0, t, x, u): initial guess at node fraction t
// with R in {double, float} and, for the gradient, a dual number type.  The
// phases use nothing else of the model; P.mp holds its own constants.
// Optionally (PDG_MODEL_HAS_STM_MASK defined), the structural sparsity of the
// interval state-transition matrix:
//   model_stm_row_mask(i)  bit c set unless entry (i, c) of every interval's
//               A_k is exactly zero for all states, controls and parameters
//               (the closure of df/dx's pattern under the flow).  The PIPG
//               products then skip the entries outside the mask; without it
//               every entry counts.
#if defined(PDG_MODEL_HEADER)
#include PDG_MODEL_HEADER
#elif defined(PDG_MODEL_3DOF)
#include "pdg_model_3dof.cuh"
#else
#include "pdg_model_6dof.cuh"
#endif
#ifndef PDG_MODEL_NU_ALT
#define PDG_MODEL_NU_ALT 4
#endif
static_assert(pdg::NX >= 2 && pdg::NX <= pdg::NXMAX, "a model's state size must lie in [2, 15]");
static_assert(pdg::IY == pdg::NX - 1, "the CTCS integrator must be the last state");
static_assert(pdg::IM >= 0 && pdg::IM < pdg::NX - 1, "the cost's mass index must be a state of xi");
static_assert(PDG_MODEL_NU_ALT == 4 || PDG_MODEL_NU_ALT == 7, "controls: nu = 4, optionally nu = 7");

namespace pdg {

#ifndef PDG_MODEL_HAS_STM_MASK
__host__ __device__ constexpr unsigned model_stm_row_mask(int) { return (1u << NX) - 1u; }
#endif

// Order in which the PIPG steps visit the entries of hat A^-_k.  A thread of
// the dual step forms row i of hat A^-_k times a vector, one of the primal
// step column i; both skip the structural zeros (model_stm_row_mask).  Tasks
// are sorted by their count of nonzeros, largest first, so that the 32 tasks
// of a warp need about the same number of FMAs and the warp's first task has
// the most (the warp runs that many, on the GB300 FP64 pipe each costs a full
// warp instruction).  A task with fewer entries than its warp's first pads its
// index list with one of its own structural zeros, which adds exactly nothing.
//
// The blocks hold only the structural nonzeros (compact storage): interval k
// keeps its nonzeros row by row, columns ascending, at k * STM_SAS, then one
// zero (offset nnz) and padding to an odd count.  row_off[i] / col_off[i]
// give, in the order of row_list[i] / col_list[i], each entry's offset within
// the interval's block as 8-bit fields (entries 0..7 in word 0, 8..14 in word
// 1); a padding entry points at the zero.
struct StmOrder {
  unsigned char row_order[NXMAX], col_order[NXMAX];  // rows / columns, most nonzeros first
  unsigned char row_nnz[NXMAX], col_nnz[NXMAX];
  unsigned long long row_list[NXMAX], col_list[NXMAX];  // 4-bit indices, ascending, then padding
  unsigned long long row_off[NXMAX][2], col_off[NXMAX][2];
  unsigned row_mask[NXMAX];
  unsigned char row_start[NXMAX];  // offset of row i's first nonzero
  int nnz;
};

__host__ __device__ constexpr bool stm_nz(int i, int c) { return (model_stm_row_mask(i) >> c) & 1u; }

__host__ __device__ constexpr StmOrder make_stm_order() {
  StmOrder S{};
  for (int i = 0; i < NX; ++i) {
    int nr = 0, nc = 0, zr = -1, zc = -1;
    unsigned long long lr = 0, lc = 0;
    for (int c = 0; c < NX; ++c) {
      if (stm_nz(i, c)) { lr |= (unsigned long long)c << (4 * nr); ++nr; } else if (zc < 0) zc = c;
      if (stm_nz(c, i)) { lc |= (unsigned long long)c << (4 * nc); ++nc; } else if (zr < 0) zr = c;
    }
    for (int j = nr; j < NX; ++j) lr |= (unsigned long long)(zc < 0 ? 0 : zc) << (4 * j);
    for (int j = nc; j < NX; ++j) lc |= (unsigned long long)(zr < 0 ? 0 : zr) << (4 * j);
    S.row_nnz[i] = (unsigned char)nr;
    S.col_nnz[i] = (unsigned char)nc;
    S.row_list[i] = lr;
    S.col_list[i] = lc;
    S.row_mask[i] = model_stm_row_mask(i) & ((1u << NX) - 1u);
    S.row_start[i] = (unsigned char)S.nnz;
    S.nnz += nr;
  }
  // offsets of the list entries: (r, c) sits at row_start[r] + (nonzeros of
  // row r left of column c); padding entries at the zero (offset nnz)
  for (int i = 0; i < NX; ++i) {
    for (int j = 0; j < NX; ++j) {
      const int c = int(S.row_list[i] >> (4 * j)) & 15, r = int(S.col_list[i] >> (4 * j)) & 15;
      int oc = S.nnz, orr = S.nnz;
      if (j < S.row_nnz[i]) {
        oc = S.row_start[i];
        for (int q = 0; q < c; ++q) oc += stm_nz(i, q) ? 1 : 0;
      }
      if (j < S.col_nnz[i]) {
        orr = S.row_start[r];
        for (int q = 0; q < i; ++q) orr += stm_nz(r, q) ? 1 : 0;
      }
      S.row_off[i][j >> 3] |= (unsigned long long)oc << (8 * (j & 7));
      S.col_off[i][j >> 3] |= (unsigned long long)orr << (8 * (j & 7));
    }
  }
  for (int a = 0; a < NX; ++a) { S.row_order[a] = (unsigned char)a; S.col_order[a] = (unsigned char)a; }
  for (int a = 1; a < NX; ++a)  // stable insertion sort, most nonzeros first
    for (int b = a; b > 0; --b) {
      if (S.row_nnz[S.row_order[b]] > S.row_nnz[S.row_order[b - 1]]) {
        const unsigned char t = S.row_order[b]; S.row_order[b] = S.row_order[b - 1]; S.row_order[b - 1] = t;
      }
      if (S.col_nnz[S.col_order[b]] > S.col_nnz[S.col_order[b - 1]]) {
        const unsigned char t = S.col_order[b]; S.col_order[b] = S.col_order[b - 1]; S.col_order[b - 1] = t;
      }
    }
  return S;
}
static __constant__ StmOrder kStm = make_stm_order();

// compact block stride per interval: the nonzeros, the zero, and an odd
// count, so that the same entry of consecutive intervals (the tasks of a
// warp) falls in different shared-memory banks
constexpr int STM_SAS = (make_stm_order().nnz + 1) | 1;

// offset of entry j of a row or column list (w = kStm.row_off[i] or col_off[i])
__device__ __forceinline__ int stm_off(unsigned long long w0, unsigned long long w1, int j) {
  return int((j < 8 ? w0 : w1) >> (8 * (j & 7))) & 255;
}
// offset of (r, c) in an interval's compact block (the zero for a structural zero)
__device__ __forceinline__ int stm_index(int r, int c) {
  const unsigned m = kStm.row_mask[r];
  return ((m >> c) & 1u) ? int(kStm.row_start[r]) + __popc(m & ((1u << c) - 1u)) : kStm.nnz;
}

// stage buffer of one interval: two Jacobian buffers, each compact A (SA_A)
// and dense B (NX x nu), then the evaluator's RK4 state of x: base P,
// accumulator, stage input (NX each)

// Intervals per discretization wave: warp 0 evaluates the model of up to 32
// intervals, the remaining warps hold one STM column per thread.
__host__ __device__ inline int waves_ipw(int threads, int nu) {
  const int ncol = NX + 2 * nu;
  const int w = (threads - 32) / ncol;
  return w > 32 ? 32 : w;
}

__host__ __device__ inline int round32(int x) { return (x + 31) & ~31; }

// Elements per interval of hat B^- and hat B^+ (row-major NX x nu): odd, so
// that the same entry of consecutive intervals (the tasks of a warp) falls in
// different shared-memory banks.
__host__ __device__ constexpr int b_stride(int nu) { return (NX * nu) | 1; }

__host__ __device__ inline Lay make_lay(int N, int nu, int threads) {
  Lay L;
  L.N = N;
  L.nu = nu;
  L.ipw = waves_ipw(threads, nu);
  L.sa = 2 * (SA_A + NX * nu) + 3 * NX;
  int o = 0;
  L.sc = o; o += 8;
  L.x0 = o; o += 16;
  L.Xb = o; o += N * NX;
  L.Ub = o; o += N * nu;
  L.Am = o; o += (N - 1) * STM_SAS;  // compact: structural nonzeros, then a zero
  L.Bm = o; o += (N - 1) * b_stride(nu);
  L.Bp = o; o += (N - 1) * b_stride(nu);
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

}  // namespace pdg
