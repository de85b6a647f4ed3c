// pdg_phases.cuh -- the phases of one SCP iteration on one instance, executed
// cooperatively by all threads of a CTA on the instance's shared-memory
// image (arXiv 2404.18034, Sec. 2.3 and Sec. 3).  Every phase is called by
// every thread of the CTA (they contain barriers).
#pragma once
#include "pdg_device.cuh"

namespace pdg {

// max(0, x) by a sign-bit test, kept off the FP64 pipe.
__device__ __forceinline__ double max0(double x) { return __double_as_longlong(x) < 0 ? 0.0 : x; }
__device__ __forceinline__ float max0(float x) { return __float_as_int(x) < 0 ? 0.0f : x; }

// Initial guess of every node (Sec. 4 asks for "an appropriate" one; the
// model's model_init_node says which).
template <typename R, int NU>
__device__ void phase_init_guess(const DParams& P, const Lay& L, R* sm) {
  const int N = L.N;
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    model_init_node<R, NU>(P, sm + L.x0, R(k) / R(N - 1), sm + L.Xb + k * NX, sm + L.Ub + k * NU);
}

// Sec. 2.3.1 + 2.3.2: integrate, on every interval, the joint IVP of x and its
// state-transition matrices with RK4 (nsub substeps, FOH controls), then write
// the prescaled blocks hat A^-_k, hat B^-_k, hat B^+_k, hat w_k.  Thread
// mapping: lane l of warp 0 integrates x on interval k0 + l and evaluates the
// compact Jacobians at each RK4 stage (its RK4 state lives in the interval's
// stage buffer); every thread of warps 1.. holds one STM column (NX + 2 NU per
// interval) in registers.  Intervals are processed in waves of L.ipw.
// Returns max_k |hat w_k|_inf (the scaled defect) on every thread.
#ifdef PDG_DISC_INLINE
#define PDG_DISC_ATTR __forceinline__
#else
#define PDG_DISC_ATTR __noinline__
#endif
template <typename R, int NU>
__device__ __forceinline__ R discretize_body(const DParams& P, const Lay& L, R* sm) {
  constexpr int NCOL = NX + 2 * NU;
  const int N = L.N;
  const R* Xb = sm + L.Xb;
  const R* Ub = sm + L.Ub;
  R* Am = sm + L.Am;
  R* Bm = sm + L.Bm;
  R* Bp = sm + L.Bp;
  R* w = sm + L.w;
  const int nsub = P.nsub;
  const R h = R(1) / (R(N - 1) * R(nsub));
  const R h2 = R(0.5) * h, h6 = h / R(6);
  const bool evaluator = threadIdx.x < 32;
  const int ct = threadIdx.x - 32;
  const int il = evaluator ? threadIdx.x : ct / NCOL;
  const int c = evaluator ? -1 : ct - il * NCOL;
  const int cu = c >= NX ? (c - NX) % NU : -1;
  const bool minus = c >= NX && (c - NX) < NU;
  R dmax = 0;
  constexpr int JS = SA_A + NX * NU;  // one Jacobian buffer: compact df/dx, dense df/du
  const int S = 4 * nsub;              // RK4 stages of the interval
  for (int k0 = 0; k0 < N - 1; k0 += L.ipw) {
    const int k = k0 + il;
    const bool active = il < L.ipw && k < N - 1;
    // two Jacobian buffers, then the evaluator's RK4 state of x
    R* st = sm + L.stage + (active ? il : 0) * L.sa;
    R* xP = st + 2 * JS;
    R* xA = xP + NX;
    R* xS = xA + NX;
    R Pv[NX], Sv[NX], Ac[NX];
    // stage s = 4 n + g of substep n: its time along the interval
    auto stage_t = [&](int s) {
      const int n = s >> 2, g = s & 3;
      return (R(n) + (g == 0 ? R(0) : (g == 3 ? R(1) : R(0.5)))) / R(nsub);
    };
    // the evaluator: f and the Jacobians at stage s into buffer s % 2, then
    // the RK4 update of x
    auto eval_stage = [&](int s) {
      const int g = s & 3;
      const R lp = stage_t(s);
      R* J = st + (s & 1) * JS;
      R u[NU], x[NX], d[NX];
#pragma unroll
      for (int i = 0; i < NU; ++i) u[i] = (R(1) - lp) * Ub[k * NU + i] + lp * Ub[(k + 1) * NU + i];
#pragma unroll
      for (int i = 0; i < NX; ++i) x[i] = xS[i];
      model_eval<R, NU>(P, x, u, d, J, J + SA_A);
      if (g == 0) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { xA[i] = d[i]; xS[i] = xP[i] + h2 * d[i]; }
      } else if (g == 1) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { xA[i] = fma(R(2), d[i], xA[i]); xS[i] = xP[i] + h2 * d[i]; }
      } else if (g == 2) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { xA[i] = fma(R(2), d[i], xA[i]); xS[i] = xP[i] + h * d[i]; }
      } else {
#pragma unroll
        for (int i = 0; i < NX; ++i) { const R v = xP[i] + h6 * (xA[i] + d[i]); xP[i] = v; xS[i] = v; }
      }
    };
    // a column thread: the STM column's RK4 stage s with the Jacobians of
    // buffer s % 2
    auto jvp_stage = [&](int s) {
      const int g = s & 3;
      const R lp = stage_t(s);
      const R* J = st + (s & 1) * JS;
      R d[NX];
      const R lam = minus ? (R(1) - lp) : lp;
      model_jvp<R, NU>(J, J + SA_A, Sv, cu, lam, d);
      if (g == 0) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { Ac[i] = d[i]; Sv[i] = Pv[i] + h2 * d[i]; }
      } else if (g == 1) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { Ac[i] = fma(R(2), d[i], Ac[i]); Sv[i] = Pv[i] + h2 * d[i]; }
      } else if (g == 2) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { Ac[i] = fma(R(2), d[i], Ac[i]); Sv[i] = Pv[i] + h * d[i]; }
      } else {
#pragma unroll
        for (int i = 0; i < NX; ++i) { Pv[i] += h6 * (Ac[i] + d[i]); Sv[i] = Pv[i]; }
      }
    };
    if (active) {
      if (evaluator) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { xP[i] = Xb[k * NX + i]; xS[i] = Xb[k * NX + i]; }
        eval_stage(0);
      } else {
#pragma unroll
        for (int i = 0; i < NX; ++i) { Pv[i] = (c == i) ? R(1) : R(0); Sv[i] = Pv[i]; }
      }
    }
    __syncthreads();
    // software pipeline: while the column threads take stage s, the
    // evaluator warp already evaluates stage s + 1 into the other buffer (it
    // needs only its own x), so a stage costs one barrier and the longer of
    // the two instead of both in turn
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      if (active) {
        if (!evaluator) jvp_stage(s);
        else if (s + 1 < S) eval_stage(s + 1);
      }
      __syncthreads();
    }
    if (active) {
      if (evaluator) {
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          const R wi = (xP[i] - Xb[(k + 1) * NX + i]) * R(P.Pxinv[i]);
          w[k * NX + i] = wi;
          dmax = rmax(dmax, fabs(wi));
        }
      } else if (c < NX) {
        const R pc = R(P.Px[c]);
#pragma unroll
        for (int i = 0; i < NX; ++i)
          if (stm_nz(i, c)) Am[k * STM_SAS + stm_index(i, c)] = Pv[i] * pc * R(P.Pxinv[i]);
        if (c == 0)  // the block's zero and padding
          for (int q = kStm.nnz; q < STM_SAS; ++q) Am[k * STM_SAS + q] = R(0);
      } else {
        const R pc = R(P.Pu[cu]);
        R* Bt = minus ? Bm : Bp;
#pragma unroll
        for (int i = 0; i < NX; ++i) Bt[k * b_stride(NU) + i * NU + cu] = Pv[i] * pc * R(P.Pxinv[i]);
      }
    }
    __syncthreads();
  }
  R v[1] = {dmax};
  block_max_k<R, 1>(v, sm + L.red);
  return v[0];
}
// Out of line (one copy serves every kernel); the persistent kernel of PIPG
// form 3 can inline the body instead (PDG_KS_DISC_INLINE).
template <typename R, int NU>
__device__ PDG_DISC_ATTR R phase_discretize(const DParams& P, const Lay& L, R* sm) {
  return discretize_body<R, NU>(P, L, sm);
}

// Sec. 2.3.2: hat eps_k, the dilation box, hat z_i (every component of
// x_1 = (x0, 0) is fixed) and hat z_f (components selected by E_f).
template <typename R, int NU>
__device__ void phase_scale_extra(const DParams& P, const Lay& L, R* sm) {
  const int N = L.N;
  const R* Xb = sm + L.Xb;
  const R* Ub = sm + L.Ub;
  const R* x0 = sm + L.x0;
  const R iPy = R(P.Pxinv[IY]);
  const R iPs = R(P.Puinv[NU - 1]);
  for (int t = threadIdx.x; t < (N - 1) + N + NX; t += blockDim.x) {
    if (t < N - 1) {
      sm[L.eps + t] = R(P.eps_ctcs) * iPy - (Xb[(t + 1) * NX + IY] - Xb[t * NX + IY]) * iPy;
    } else if (t < 2 * N - 1) {
      // dilation box; the Sec. 2.2 time bounds tighten it (sufficient node box for FOH s)
      const int k = t - (N - 1);
      const R s = Ub[k * NU + NU - 1];
      double lo = P.s_lo, hi = P.s_hi;
      if (P.dt_lo > 0.0 && P.dt_lo * (N - 1) > lo) lo = P.dt_lo * (N - 1);
      if (P.dt_hi > 0.0 && P.dt_hi * (N - 1) < hi) hi = P.dt_hi * (N - 1);
      sm[L.lo + k] = (R(lo) - s) * iPs;
      sm[L.hi + k] = (R(hi) - s) * iPs;
    } else {
      const int i = t - (2 * N - 1);
      sm[L.zi + i] = (x0[i] - Xb[i]) * R(P.Pxinv[i]);
      sm[L.zf + i] = P.fix_f[i] ? (R(P.z_f[i]) - Xb[(N - 1) * NX + i]) * R(P.Pxinv[i]) : R(0);
    }
  }
}

// Alg. power on K = [G; H_y] (readings: v_k is theta_k; sigma* accumulates from
// sigma*; start from the warm-start primal, or all ones when it is zero).  The
// iterate (x, u, mu+, mu-) lives in the xt/ut/nup/num scratch, (phi, theta) in
// vph/vth.  Task ranges are padded to whole warps so that every warp runs one
// kind of task.  Returns the buffered sigma; *iters the iterations run.
template <typename R, int NU>
__device__ R phase_power(const DParams& P, const Lay& L, R* sm, int force, int* iters) {
  const int N = L.N, T = blockDim.x, tid = threadIdx.x;
  const int nx = N * NX, nuu = N * NU, nm = (N - 1) * NX;
  const int PX = round32(nx), PU = round32(nuu), PM = round32(nm);
  const R* Am = sm + L.Am;
  const R* Bm = sm + L.Bm;
  const R* Bp = sm + L.Bp;
  R* px = sm + L.xt;
  R* pu = sm + L.ut;
  R* pp = sm + L.nup;
  R* pn = sm + L.num;
  R* ph = sm + L.vph;
  R* pt = sm + L.vth;
  R ss = 0;
  for (int t = tid; t < nx + nuu + nm; t += T) {
    R a, b = 0;
    if (t < nx) { a = sm[L.xh + t]; px[t] = a; }
    else if (t < nx + nuu) { a = sm[L.uh + t - nx]; pu[t - nx] = a; }
    else {
      const int q = t - nx - nuu;
      a = sm[L.mup + q]; b = sm[L.mum + q];
      pp[q] = a; pn[q] = b;
    }
    ss += a * a + b * b;
  }
  ss = block_sum(ss, sm + L.red);
  if (ss == R(0)) {
    for (int t = tid; t < nx + nuu + nm; t += T) {
      if (t < nx) px[t] = 1;
      else if (t < nx + nuu) pu[t - nx] = 1;
      else { pp[t - nx - nuu] = 1; pn[t - nx - nuu] = 1; }
    }
    ss = R(nx + nuu + 2 * nm);
    __syncthreads();
  }
  R sig = sqrt(ss);
  R sstar = sig;
  const int jmax = force > 0 ? force : P.pow_jmax;
  int j;
  for (j = 1; j <= jmax; ++j) {
    const R isig = R(1) / sig;
    // phi = K z / sigma
    for (int t = tid; t < PM + 32; t += T) {
      if (t < PM) {
        if (t < nm) {
          // rows in kStm.row_order, structural zeros skipped (as in PIPG)
          const int rr = t / (N - 1);
          const int k = t - rr * (N - 1), i = kStm.row_order[rr];
          const int o = k * NX + i;
          const R* a = Am + k * STM_SAS;
          const R* xk = px + k * NX;
          R r = pp[o] - pn[o] - px[(k + 1) * NX + i];
          const int nj = kStm.row_nnz[kStm.row_order[(t & ~31) / (N - 1)]];
          const unsigned long long lst = kStm.row_list[i], w0 = kStm.row_off[i][0], w1 = kStm.row_off[i][1];
#pragma unroll 5
          for (int j = 0; j < nj; ++j) {
            const int cc = int(lst >> (4 * j)) & 15;
            r += a[stm_off(w0, w1, j)] * xk[cc];
          }
          const R* bm = Bm + k * b_stride(NU) + i * NU;
          const R* bp = Bp + k * b_stride(NU) + i * NU;
#pragma unroll
          for (int cc = 0; cc < NU; ++cc) r += bm[cc] * pu[k * NU + cc] + bp[cc] * pu[(k + 1) * NU + cc];
          ph[o] = r * isig;
        }
      } else {
        const int k = t - PM;
        if (k < N - 1) pt[k] = (px[(k + 1) * NX + IY] - px[k * NX + IY]) * isig;
      }
    }
    __syncthreads();
    // z = K^T (phi, theta)
    R s2 = 0;
    for (int t = tid; t < PX + PU + PM; t += T) {
      if (t < PX) {
        if (t < nx) {
          // branch-free, as the PIPG x step: blocks that do not exist (the
          // last node's A, the first node's coupling) run on valid data and
          // selects discard them; the CTCS terms ride on a 0/1-weighted FMA.
          // Columns in kStm.col_order (N nodes each), structural zeros skipped.
          const int cr = t / N;
          const int k = t - cr * N, i = kStm.col_order[cr];
          const bool hasA = k < N - 1, hasP = k > 0;
          const int ka = hasA ? k : 0, kp = hasP ? k - 1 : 0;
          R gc = 0;
          const R* a = Am + ka * STM_SAS;
          const R* f = ph + ka * NX;
          const int nj = kStm.col_nnz[kStm.col_order[(t & ~31) / N]];
          const unsigned long long lst = kStm.col_list[i], w0 = kStm.col_off[i][0], w1 = kStm.col_off[i][1];
#pragma unroll 5
          for (int j = 0; j < nj; ++j) {
            const int r = int(lst >> (4 * j)) & 15;
            gc = fma(a[stm_off(w0, w1, j)], f[r], gc);
          }
          R g = hasA ? gc : R(0);
          const R dth = (hasP ? pt[kp] : R(0)) - (hasA ? pt[ka] : R(0));
          g = fma(i == IY ? R(1) : R(0), dth, g);
          g -= hasP ? ph[kp * NX + i] : R(0);
          px[k * NX + i] = g;
          s2 += g * g;
        }
      } else if (t < PX + PU) {
        const int q = t - PX;
        if (q < nuu) {
          const int k = q / NU, cc = q - NU * k;
          const bool hasM = k < N - 1, hasP = k > 0;
          const int km = hasM ? k : 0, kp = hasP ? k - 1 : 0;
          R gm = 0;
          {
            const R* a = Bm + km * b_stride(NU) + cc;
            const R* f = ph + km * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) gm = fma(a[r * NU], f[r], gm);
          }
          gm = hasM ? gm : R(0);
          R g = gm;
          {
            const R* a = Bp + kp * b_stride(NU) + cc;
            const R* f = ph + kp * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) g = fma(a[r * NU], f[r], g);
          }
          g = hasP ? g : gm;
          pu[q] = g;
          s2 += g * g;
        }
      } else {
        const int q = t - PX - PU;
        if (q < nm) {
          const R f = ph[q];
          pp[q] = f;
          pn[q] = -f;
          s2 += R(2) * f * f;
        }
      }
    }
    s2 = block_sum(s2, sm + L.red);
    sstar = sqrt(s2);
    if (force <= 0 && fabs(sstar - sig) <= R(P.pow_eps_abs) + R(P.pow_eps_rel) * rmax(sstar, sig)) break;
    if (j < jmax) sig = sstar;
  }
  *iters = j > jmax ? jmax : j;
  return (R(1) + R(P.pow_buff)) * sstar;
}

// Alg. PIPG_custom with Alg. stopping, warm-started from (xh, uh, mup, mum,
// phi, th), which hold the solution on return.  Readings: the mu^- step uses
// (w_ep - phi); the B^+_{k-1} term of the u_k gradient multiplies the
// extrapolated dual of the dynamics rows; the stop test compares iterates j+1
// and j (the warm start being iterate 0).
// Work split, every task range padded to whole warps:
//   primal phase: x_hat of nodes 2..N (NX (N-1) tasks), then u_hat (G lanes
//     per node) and the fixed node 1 (NX tasks);
//   dual phase: row i of interval k updates mu^+-, nu^+- (they read the same
//     extrapolated dual entry) and then phi; then the CTCS rows theta_k, whose
//     warp also forms the per-node differences td for the next primal step.
template <bool B> struct ChkTag { static constexpr bool value = B; };

// Returns the iterations run.  Extrapolations 2 z - z~ are written as fma:
// the compiler would otherwise form z + z and subtract (two FP64 adds).
// CK (gradient solves only): before iterations 1, 51, 101, ... the state
// (x~, u~, nu~+-, phi~, theta~; nu~ unshifted) is copied to ck, one record of
// L.dx - L.xt values per 50 iterations, for the adjoint's recomputation.
#ifdef PDG_PIPG_NOINLINE
#define PDG_PIPG_ATTR __noinline__
#else
#define PDG_PIPG_ATTR
#endif
template <typename R, int NU, bool CK = false>
__device__ PDG_PIPG_ATTR int phase_pipg(const DParams& P, const Lay& L, R* sm, R sigma, int force, double* ck = nullptr) {
  using OB = OrdBits<R>;
  using U = typename OB::U;
  const int N = L.N, T = blockDim.x, tid = threadIdx.x;
  constexpr int G = NU <= 4 ? 4 : 8;   // lanes per node for the control step
  const int nxk = (N - 1) * NX, nm = (N - 1) * NX;
  const int PG = round32(N * G);        // grouped control lanes, whole warps
  const int PX = round32(nxk), PU = PG + 32, PM = round32(nm);
  const R* __restrict__ Am = sm + L.Am;
  const R* __restrict__ Bm = sm + L.Bm;
  const R* __restrict__ Bp = sm + L.Bp;
  const R* __restrict__ wv = sm + L.w;
  const R* __restrict__ ep = sm + L.eps;
  const R* lo = sm + L.lo;
  const R* hi = sm + L.hi;
  const R* zi = sm + L.zi;
  const R* zf = sm + L.zf;
  R* xh = sm + L.xh;
  R* uh = sm + L.uh;
  R* mup = sm + L.mup;
  R* mum = sm + L.mum;
  R* phi = sm + L.phi;
  R* th = sm + L.th;
  R* xt = sm + L.xt;
  R* ut = sm + L.ut;
  R* nup = sm + L.nup;
  R* num = sm + L.num;
  R* vph = sm + L.vph;
  R* vth = sm + L.vth;
  R* dx = sm + L.dx;
  R* du = sm + L.du;
  // td[k] = theta~_{k-1} - theta~_k (k < N-1) or theta~_{N-2} (k = N-1): the
  // CTCS rows' contribution to the y component of node k's gradient, formed
  // by the CTCS warp so that the x step carries no per-component branch
  R* td = sm + L.td;
  const R wp = R(P.w_prox);
  const R alpha = R(2) / (wp + sqrt(wp * wp + R(4) * R(P.omega) * sigma));
  const R beta = R(P.omega) * alpha;
  const R c1 = R(1) - alpha * wp;
  const R rho = R(P.rho);
  const R rb = rho * beta;
  const R wcost = R(P.w_cost);
  // The relaxed virtual-control iterates are kept shifted by alpha w_ep
  // (nu~ = nu - alpha w_ep): the projection max{0, nu - alpha (w_ep +- phi)}
  // is then one FMA and the relaxation two; the shift cancels in the
  // extrapolated difference (2 mu+ - nu+) - (2 mu- - nu-).
  const R aw = alpha * R(P.w_ep);
  const R omr = R(1) - rho, raw = rho * aw;
  for (int t = tid; t < N * NX + N * NU + 2 * nm + (N - 1); t += T) {
    if (t < N * NX) xt[t] = xh[t];
    else if (t < N * NX + N * NU) ut[t - N * NX] = uh[t - N * NX];
    else if (t < N * NX + N * NU + nm) { const int q = t - N * NX - N * NU; nup[q] = mup[q] - aw; num[q] = mum[q] - aw; }
    else if (t < N * NX + N * NU + 2 * nm) { const int q = t - N * NX - N * NU - nm; vph[q] = phi[q]; }
    else { const int q = t - N * NX - N * NU - 2 * nm; vth[q] = th[q]; }
  }
  for (int k = 1 + tid; k < N; k += T) td[k] = th[k - 1] - (k < N - 1 ? th[k] : R(0));
  __syncthreads();
  const R sa = R(P.soc_tan), tmax = R(P.T_max), pT = R(P.Pu[0]), ipT = R(P.Puinv[0]);
  const int jmax = force > 0 ? force : P.pipg_jmax;
  const int jcheck = P.pipg_jcheck;
  // One iteration; CHK (compile time) adds the stop test, so that the other
  // iterations carry none of its instructions.  Returns true to stop.
  auto iterate = [&](auto chk_tag) -> bool {
    constexpr bool chk = decltype(chk_tag)::value;
    U zn = 0, zo = 0, zd = 0;
    // ---- projected gradient step (primal)
    for (int t = tid; t < PX + PU; t += T) {
      if (t < PX) {
        if (t < nxk) {
          // branch-free: on GB300 a divergent FP64 instruction costs a full
          // warp slot, and per-component special cases split the warp.
          // Tasks run column by column in kStm.col_order (N - 1 nodes each),
          // so a warp's columns have about as many structural nonzeros as
          // its first task's, which bounds its FMA count.
          const int cr = t / (N - 1);
          const int k = t - cr * (N - 1) + 1, i = kStm.col_order[cr];
          const int o = k * NX + i;
          const bool last = k == N - 1;
          const int km = last ? 0 : k;  // the last node has no A block: any valid one, result discarded
          const R xv = xt[o];
          const R G0 = fma(i == IY ? R(1) : R(0), td[k], -vph[(k - 1) * NX + i]);
          R Gc = G0;
          const R* a = Am + km * STM_SAS;
          const R* f = vph + km * NX;
          const int nj = kStm.col_nnz[kStm.col_order[(t & ~31) / (N - 1)]];
          const unsigned long long lst = kStm.col_list[i], w0 = kStm.col_off[i][0], w1 = kStm.col_off[i][1];
#pragma unroll 5
          for (int j = 0; j < nj; ++j) {
            const int r = int(lst >> (4 * j)) & 15;
            Gc = fma(a[stm_off(w0, w1, j)], f[r], Gc);
          }
          const R G = last ? G0 : Gc;
          // e_cost = -e_m on x_N (maximize m_N) folded into the same FMA
          const R cost = (last && i == IM) ? alpha * wcost : R(0);
          R xn = fma(-alpha, G, fma(c1, xv, cost));
          xn = (last && P.fix_f[i]) ? zf[i] : xn;
          dx[o] = fma(R(2), xn, -xv);
          xt[o] = xv + rho * (xn - xv);
          if constexpr (chk) {
            const R old = xh[o];
            zn = umax(zn, OB::abs(xn)); zo = umax(zo, OB::abs(old)); zd = umax(zd, OB::abs(xn - old));
          }
          xh[o] = xn;
        }
      } else {
        const int q = t - PX;
        if (q < PG) {
          // thrust/control lanes, G per node (aligned within the warp)
          const int k = q / G, cc = q - G * k;
          const bool valid = k < N && cc < NU;
          const int o = k * NU + cc;
          // branch-free like the x step: every lane runs both block products
          // on valid blocks (node 0 has no B^+, node N no B^-, padding lanes
          // neither) and selects discard what does not exist
          const int kv = valid ? k : 0, cv = valid ? cc : 0;
          const int km = kv < N - 1 ? kv : 0, kp = kv > 0 ? kv - 1 : 0;
          const R uv = ut[kv * NU + cv];
          R Gm = 0;
          {
            const R* a = Bm + km * b_stride(NU) + cv;
            const R* f = vph + km * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) Gm = fma(a[r * NU], f[r], Gm);
          }
          Gm = kv < N - 1 ? Gm : R(0);
          R Gs = Gm;
          {
            const R* a = Bp + kp * b_stride(NU) + cv;
            const R* f = vph + kp * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) Gs = fma(a[r * NU], f[r], Gs);
          }
          Gs = kv > 0 ? Gs : Gm;
          R un = c1 * uv - alpha * Gs;
          if (cc == NU - 1) un = rmin(rmax(un, lo[kv]), hi[kv]);
          if (P.soc) {
            // project the node's thrust onto the sector (all lanes of the warp
            // take part in the shuffles; each group of G lanes is one node)
            const R Tb = (valid && cc < 3) ? sm[L.Ub + o] : R(0);
            const R tv = (valid && cc < 3) ? Tb + pT * un : R(0);
            const int base = (threadIdx.x & 31) & ~(G - 1);
            R T0 = __shfl_sync(0xffffffffu, tv, base);
            R T1 = __shfl_sync(0xffffffffu, tv, base + 1);
            R T2 = __shfl_sync(0xffffffffu, tv, base + 2);
            const R rr = ::sqrt(T1 * T1 + T2 * T2);
            if (rr > sa * T0) {
              if (sa * rr <= -T0) {
                T0 = 0; T1 = 0; T2 = 0;
              } else {
                const R tp = (T0 + sa * rr) / (R(1) + sa * sa);
                const R sc = sa * tp / rr;
                T0 = tp; T1 *= sc; T2 *= sc;
              }
            }
            const R nT = ::sqrt(T0 * T0 + T1 * T1 + T2 * T2);
            if (nT > tmax) { const R f = tmax / nT; T0 *= f; T1 *= f; T2 *= f; }
            if (valid && cc < 3) un = ((cc == 0 ? T0 : (cc == 1 ? T1 : T2)) - Tb) * ipT;
          }
          {
            const R dn = fma(R(2), un, -uv), tn = uv + rho * (un - uv);
            if (valid) { du[o] = dn; ut[o] = tn; }
            if constexpr (chk) {
              const R old = uh[kv * NU + cv];
              if (valid) { zn = umax(zn, OB::abs(un)); zo = umax(zo, OB::abs(old)); zd = umax(zd, OB::abs(un - old)); }
            }
            if (valid) uh[o] = un;
          }
        } else if (q < PG + NX) {
          // node 1: every component fixed by E_i
          const int i = q - PG;
          const R xv = xt[i], xn = zi[i];
          dx[i] = fma(R(2), xn, -xv);
          xt[i] = xv + rho * (xn - xv);
          if constexpr (chk) {
            const R old = xh[i];
            zn = umax(zn, OB::abs(xn)); zo = umax(zo, OB::abs(old)); zd = umax(zd, OB::abs(xn - old));
          }
          xh[i] = xn;
        }
      }
    }
    __syncthreads();
    // ---- virtual controls and proportional-integral feedback (dual)
    U rn = 0, ro = 0, rd = 0;
    for (int t = tid; t < PM + 32; t += T) {
      if (t < PM) {
        if (t < nm) {
          // rows in kStm.row_order, N - 1 intervals each (see the x step)
          const int rr = t / (N - 1);
          const int k = t - rr * (N - 1), i = kStm.row_order[rr];
          const int o = k * NX + i;
          const R f = vph[o], a = nup[o], b = num[o];
          const R mp = max0(a - alpha * f);
          const R mm = max0(b + alpha * f);
          nup[o] = omr * a + (rho * mp - raw);
          num[o] = omr * b + (rho * mm - raw);
          if constexpr (chk) {
            const R op = mup[o], om = mum[o];
            zn = umax(zn, umax(OB::nonneg(mp), OB::nonneg(mm)));
            zo = umax(zo, umax(OB::nonneg(op), OB::nonneg(om)));
            zd = umax(zd, umax(OB::abs(mp - op), OB::abs(mm - om)));
          }
          mup[o] = mp;
          mum[o] = mm;
          const R* a_ = Am + k * STM_SAS;
          const R* d = dx + k * NX;
          R r = wv[o] + (fma(R(2), mp, -a) - fma(R(2), mm, -b)) - dx[(k + 1) * NX + i];
          const int nj = kStm.row_nnz[kStm.row_order[(t & ~31) / (N - 1)]];
          const unsigned long long lst = kStm.row_list[i], w0 = kStm.row_off[i][0], w1 = kStm.row_off[i][1];
#pragma unroll 5
          for (int j = 0; j < nj; ++j) {
            const int cc = int(lst >> (4 * j)) & 15;
            r += a_[stm_off(w0, w1, j)] * d[cc];
          }
          const R* bm = Bm + k * b_stride(NU) + i * NU;
          const R* bp = Bp + k * b_stride(NU) + i * NU;
#pragma unroll
          for (int cc = 0; cc < NU; ++cc) { r += bm[cc] * du[k * NU + cc]; r += bp[cc] * du[(k + 1) * NU + cc]; }
          const R pn = f + beta * r;
          vph[o] = f + rb * r;  // = f + rho (pn - f)
          if constexpr (chk) {
            const R old = phi[o];
            rn = umax(rn, OB::abs(pn)); ro = umax(ro, OB::abs(old)); rd = umax(rd, OB::abs(pn - old));
          }
          phi[o] = pn;
        }
      } else {
        // CTCS rows, one warp (N - 1 <= 31 lanes used; all lanes shuffle)
        const int k = t - PM;
        R vn = 0;
        if (k < N - 1) {
          const R hy = dx[(k + 1) * NX + IY] - dx[k * NX + IY] - ep[k];
          const R v = vth[k];
          const R tn = max0(v + beta * hy);
          vn = v + rho * (tn - v);
          vth[k] = vn;
          if constexpr (chk) {
            const R old = th[k];
            rn = umax(rn, OB::nonneg(tn)); ro = umax(ro, OB::abs(old)); rd = umax(rd, OB::abs(tn - old));
          }
          th[k] = tn;
        }
        const R vnext = __shfl_down_sync(0xffffffffu, vn, 1);
        if (k < N - 1) td[k + 1] = vn - (k + 1 < N - 1 ? vnext : R(0));
      }
    }
    if constexpr (chk) {
      U v[6] = {zn, zo, zd, rn, ro, rd};
      block_max_u<U, 6>(v, reinterpret_cast<U*>(sm + L.red));
      const R eabs = R(P.eps_abs), erel = R(P.eps_rel);
      return OB::val(v[2]) <= eabs + erel * rmax(OB::val(v[0]), OB::val(v[1])) &&
             OB::val(v[5]) <= eabs + erel * rmax(OB::val(v[3]), OB::val(v[4]));
    } else {
      (void)zn; (void)zo; (void)zd; (void)rn; (void)ro; (void)rd;
      __syncthreads();
      return false;
    }
  };
  int j;
  for (j = 1; j <= jmax; ++j) {
    if constexpr (CK) {
      if (((j - 1) % 50) == 0) {
        const int ss = L.dx - L.xt, o0 = L.nup - L.xt, o1 = L.vph - L.xt;
        double* c = ck + (size_t)((j - 1) / 50) * ss;
        for (int t = tid; t < ss; t += T) {
          const double v = double(sm[L.xt + t]);
          c[t] = (t >= o0 && t < o1) ? v + double(aw) : v;
        }
        __syncthreads();  // the iteration overwrites the state
      }
    }
    if (force <= 0 && jcheck > 0 && (j % jcheck) == 0) {
      if (iterate(ChkTag<true>{})) break;
    } else {
      iterate(ChkTag<false>{});
    }
  }
  __syncthreads();
  return j > jmax ? jmax : j;
}

// ---------------------------------------------------------------------------
// PIPG_custom with the blocks and the iterates held in registers.
//
// The same iteration as phase_pipg (Alg. PIPG_custom with the stop test of
// Alg. stopping), mapped so that nothing but the two exchanged vectors goes
// through shared memory in the loop.  Thread roles are warp-uniform:
//  * row threads p < RT = round32((N-1) NX): x task p (node p/NX + 1,
//    component i = p%NX; it keeps column i of hat A^-_{node}, zero for the
//    last node) and dual row p (interval p/NX, row i; it keeps row i of
//    hat A^-, hat B^-, hat B^+, hat w and its mu+-, phi entries).
//  * control threads v = tid - RT < UT = round32(N G): node v/G, control
//    component v%G (G lanes per node so a node's thrust is one aligned lane
//    group for the cone projection); they keep column v%G of hat B^-_{node}
//    and hat B^+_{node-1}.  Threads v < NX also own node 1, and in the dual
//    step threads v < N-1 own theta_v.
// Exchanged through shared memory: the relaxed dual phi~ and the per-node
// difference of the relaxed CTCS duals (td, as in phase_pipg) read by the
// primal step, and the extrapolated primal (2 z_{j+1} - z~_j) read by the
// dual step; node vectors are padded to NXS entries (a multiple of four) so
// they load as 16-byte vectors.
// Needs blockDim.x >= pipg_reg_threads(N, NU).
// ---------------------------------------------------------------------------
__host__ __device__ inline int pipg_reg_groups(int nu) { return nu <= 4 ? 4 : 8; }
__host__ __device__ inline int pipg_reg_threads(int N, int nu) {
  return round32((N - 1) * NX) + round32(N * pipg_reg_groups(nu));
}

template <typename R> struct Vec16B;
template <> struct Vec16B<float> {
  static constexpr int n = 4;
  __device__ __forceinline__ static void ld(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <> struct Vec16B<double> {
  static constexpr int n = 2;
  __device__ __forceinline__ static void ld(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
};

// Shared-memory offsets of the exchange vectors (inside the phase-local union
// region, 16-byte aligned): vp[(N-1)][NXS], dx[N][NXS], du[N][NUP], td[N].
constexpr int NXS = (NX + 3) & ~3;
struct RegLay { int vp, dx, du, td, end; };
__host__ __device__ inline RegLay make_reg_lay(const Lay& L) {
  const int nup = L.nu <= 4 ? 4 : 8;
  RegLay Q;
  int o = (L.xt + 3) & ~3;
  Q.vp = o; o += (L.N - 1) * NXS;
  Q.dx = o; o += L.N * NXS;
  Q.du = o; o += L.N * nup;
  Q.td = o; o += (L.N + 3) & ~3;  // CTCS-dual difference per node (as in phase_pipg)
  Q.end = o;
  return Q;
}

// g + sum_{r < NX} a[r] v[r] with v read from shared memory in 16-byte pieces
// (four interleaved accumulators; v is 16-byte aligned, v[NX..NXS) is padding)
template <typename R>
__device__ __forceinline__ R dotx_sm(const R (&a)[NX], const R* v, R g) {
  constexpr int W = Vec16B<R>::n;
  R h[4] = {0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < NXS; q += W) {
    R c[W];
    Vec16B<R>::ld(v + q, c);
#pragma unroll
    for (int e = 0; e < W; ++e) {
      if (q + e < NX) h[(q + e) & 3] = fma(a[q + e], c[e], h[(q + e) & 3]);
    }
  }
  return g + ((h[0] + h[1]) + (h[2] + h[3]));
}

// Out of line by default: the loop then gets the whole register file, not
// what the enclosing kernel leaves over.  The shared-memory image is reached
// through the kernel's dynamic shared array (every kernel places the image at
// its start), so the accesses stay shared-memory loads and stores.
#ifdef PDG_PIPG_REG_NOINLINE
#define PDG_PREG_ATTR __noinline__
#else
#define PDG_PREG_ATTR __forceinline__
#endif
template <typename R, int NU>
__device__ PDG_PREG_ATTR int phase_pipg_reg(const DParams& P, const Lay& L, R* /*image*/, R sigma, int force) {
  using OB = OrdBits<R>;
  using U = typename OB::U;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* const sm = reinterpret_cast<R*>(smraw);
  constexpr int G = NU <= 4 ? 4 : 8;
  constexpr int NUP = NU <= 4 ? 4 : 8;
  const int N = L.N, tid = threadIdx.x;
  const int nm = (N - 1) * NX;
  const int RT = round32(nm), UT = round32(N * G);
  const RegLay Q = make_reg_lay(L);
  R* const vp = sm + Q.vp;
  R* const dxs = sm + Q.dx;
  R* const dus = sm + Q.du;
  R* const tds = sm + Q.td;
  const bool row = tid < RT;
  const bool ctl = !row && tid < RT + UT;
  // row thread p = tid: dual row (interval kd, row i) and x task (node kx = kd + 1, component i)
  const int kd = tid / NX, i = tid - NX * (tid / NX);
  const int kx = kd + 1;
  const bool has_d = row && tid < nm;                 // x task exists exactly when the dual row does
  const bool has_colA = has_d && kx <= N - 2;
  const bool last_x = has_d && kx == N - 1;
  // control thread v: node ku, component cc; theta_v for v < N-1; node-1 entry v for v < NX
  const int v = tid - RT;
  const int ku = v / G, cc = v - G * (v / G);
  const bool has_u = ctl && ku < N && cc < NU;
  const bool has_th = ctl && v < N - 1;
  const bool th_warp = ctl && v < 32;  // the control warp that holds the CTCS rows
  const bool has_x1 = ctl && v < NX;
  // registers.  Arrays: column of hat A^-_{kx} / row of hat A^-_{kd} / row of
  // hat B^-, hat B^+ (row thread); column of hat B^-_{ku} / of hat B^+_{ku-1}
  // (control thread).  Scalars by role:
  //   row:     r0 x~, r1 x_hat, r2 nu~+, r3 nu~-, r4 mu+, r5 mu-, r6 phi~, r7 phi, r8 hat w
  //            (nu~ = nu - alpha w_ep, as in phase_pipg)
  //   control: r0 u~, r1 u_hat, r2 lo, r3 hi, r4 reference thrust,
  //            r5 theta~, r6 theta, r7 hat eps, r8 x~ node 1, r9 x_hat node 1, r10 hat z_i
  const R wp = R(P.w_prox);
  const R alpha = R(2) / (wp + sqrt(wp * wp + R(4) * R(P.omega) * sigma));
  const R beta = R(P.omega) * alpha;
  const R c1 = R(1) - alpha * wp;
  const R rho = R(P.rho);
  const R rb = rho * beta;
  const R aw = alpha * R(P.w_ep);
  const R omr = R(1) - rho, raw = rho * aw;
  R a1[NX], a2[NX], a3[2 * NU];
  R r0 = 0, r1 = 0, r2 = 0, r3 = 0, r4 = 0, r5 = 0, r6 = 0, r7 = 0, r8 = 0, r9 = 0, r10 = 0;
#pragma unroll
  for (int r = 0; r < NX; ++r) { a1[r] = 0; a2[r] = 0; }
#pragma unroll
  for (int r = 0; r < 2 * NU; ++r) a3[r] = 0;
  if (has_d) {
    r0 = r1 = sm[L.xh + kx * NX + i];
    if (has_colA) {
#pragma unroll
      for (int r = 0; r < NX; ++r) a1[r] = sm[L.Am + kx * STM_SAS + stm_index(r, i)];
    }
#pragma unroll
    for (int c = 0; c < NX; ++c) a2[c] = sm[L.Am + kd * STM_SAS + stm_index(i, c)];
#pragma unroll
    for (int c = 0; c < NU; ++c) {
      a3[c] = sm[L.Bm + kd * b_stride(NU) + i * NU + c];
      a3[NU + c] = sm[L.Bp + kd * b_stride(NU) + i * NU + c];
    }
    r8 = sm[L.w + tid];
    r4 = sm[L.mup + tid]; r2 = r4 - aw;
    r5 = sm[L.mum + tid]; r3 = r5 - aw;
    r7 = r6 = sm[L.phi + tid];
    vp[kd * NXS + i] = r6;
  }
  if (has_u) {
    r0 = r1 = sm[L.uh + ku * NU + cc];
    if (ku <= N - 2) {
#pragma unroll
      for (int r = 0; r < NX; ++r) a1[r] = sm[L.Bm + ku * b_stride(NU) + r * NU + cc];
    }
    if (ku >= 1) {
#pragma unroll
      for (int r = 0; r < NX; ++r) a2[r] = sm[L.Bp + (ku - 1) * b_stride(NU) + r * NU + cc];
    }
    if (cc == NU - 1) { r2 = sm[L.lo + ku]; r3 = sm[L.hi + ku]; }
    if (cc < 3) r4 = sm[L.Ub + ku * NU + cc];
  }
  if (has_th) {
    r6 = r5 = sm[L.th + v];
    r7 = sm[L.eps + v];
  }
  if (has_x1) { r8 = r9 = sm[L.xh + v]; r10 = sm[L.zi + v]; }
  if (ctl && v >= 1 && v < N) tds[v] = sm[L.th + v - 1] - (v < N - 1 ? sm[L.th + v] : R(0));
  const R s_iy = (has_d && i == IY) ? R(1) : R(0);
  const R cost = (last_x && i == IM) ? alpha * R(P.w_cost) : R(0);
  const int km = has_colA ? kx : 0;  // the last node has no A block (its column is zero)
  __syncthreads();
  const int jmax = force > 0 ? force : P.pipg_jmax;
  const int jcheck = P.pipg_jcheck;
  auto iterate = [&](auto chk_tag) -> bool {
    constexpr bool chk = decltype(chk_tag)::value;
    U zn = 0, zo = 0, zd = 0, rn = 0, ro = 0, rd = 0;
    // ---- projected gradient step (primal)
    if (has_d) {
      // branch-free (see phase_pipg): zero column for the last node
      const R G = dotx_sm(a1, vp + km * NXS, fma(s_iy, tds[kx], -vp[kd * NXS + i]));
      R xn = fma(-alpha, G, fma(c1, r0, cost));
      xn = (last_x && P.fix_f[i]) ? sm[L.zf + i] : xn;
      dxs[kx * NXS + i] = fma(R(2), xn, -r0);
      r0 += rho * (xn - r0);
      if constexpr (chk) { zn = umax(zn, OB::abs(xn)); zo = umax(zo, OB::abs(r1)); zd = umax(zd, OB::abs(xn - r1)); }
      r1 = xn;
    } else if (ctl) {
      R un = 0;
      if (has_u) {
        R Gs = 0;
        if (ku <= N - 2) Gs = dotx_sm(a1, vp + ku * NXS, Gs);
        if (ku >= 1) Gs = dotx_sm(a2, vp + (ku - 1) * NXS, Gs);
        un = c1 * r0 - alpha * Gs;
        if (cc == NU - 1) un = rmin(rmax(un, r2), r3);
      }
      if (P.soc) {
        // the node's thrust onto the sector: cone about body x, then the ball
        const R sa = R(P.soc_tan), tmax = R(P.T_max), pT = R(P.Pu[0]), ipT = R(P.Puinv[0]);
        const R tv = (has_u && cc < 3) ? r4 + pT * un : R(0);
        const int base = (tid & 31) & ~(G - 1);
        R T0 = __shfl_sync(0xffffffffu, tv, base);
        R T1 = __shfl_sync(0xffffffffu, tv, base + 1);
        R T2 = __shfl_sync(0xffffffffu, tv, base + 2);
        const R rr = ::sqrt(T1 * T1 + T2 * T2);
        if (rr > sa * T0) {
          if (sa * rr <= -T0) {
            T0 = 0; T1 = 0; T2 = 0;
          } else {
            const R tp = (T0 + sa * rr) / (R(1) + sa * sa);
            const R sc = sa * tp / rr;
            T0 = tp; T1 *= sc; T2 *= sc;
          }
        }
        const R nT = ::sqrt(T0 * T0 + T1 * T1 + T2 * T2);
        if (nT > tmax) { const R q = tmax / nT; T0 *= q; T1 *= q; T2 *= q; }
        if (has_u && cc < 3) un = ((cc == 0 ? T0 : (cc == 1 ? T1 : T2)) - r4) * ipT;
      }
      if (has_u) {
        dus[ku * NUP + cc] = fma(R(2), un, -r0);
        r0 += rho * (un - r0);
        if constexpr (chk) { zn = umax(zn, OB::abs(un)); zo = umax(zo, OB::abs(r1)); zd = umax(zd, OB::abs(un - r1)); }
        r1 = un;
      }
      if (has_x1) {  // node 1: every component fixed by E_i
        dxs[v] = fma(R(2), r10, -r8);
        r8 += rho * (r10 - r8);
        if constexpr (chk) { zn = umax(zn, OB::abs(r10)); zo = umax(zo, OB::abs(r9)); zd = umax(zd, OB::abs(r10 - r9)); }
        r9 = r10;
      }
    }
    __syncthreads();
    // ---- virtual controls and proportional-integral feedback (dual)
    if (has_d) {
      const R mp = max0(r2 - alpha * r6);
      const R mm = max0(r3 + alpha * r6);
      const R a = r2, b = r3;
      r2 = omr * a + (rho * mp - raw);
      r3 = omr * b + (rho * mm - raw);
      if constexpr (chk) {
        zn = umax(zn, umax(OB::nonneg(mp), OB::nonneg(mm))); zo = umax(zo, umax(OB::nonneg(r4), OB::nonneg(r5)));
        zd = umax(zd, umax(OB::abs(mp - r4), OB::abs(mm - r5)));
      }
      r4 = mp;
      r5 = mm;
      R r = r8 + (fma(R(2), mp, -a) - fma(R(2), mm, -b)) - dxs[kx * NXS + i];
      r = dotx_sm(a2, dxs + kd * NXS, r);
      R r2b = 0;
#pragma unroll
      for (int c0 = 0; c0 < NU; c0 += Vec16B<R>::n) {
        R d0[Vec16B<R>::n], d1[Vec16B<R>::n];
        Vec16B<R>::ld(dus + kd * NUP + c0, d0);
        Vec16B<R>::ld(dus + kx * NUP + c0, d1);
#pragma unroll
        for (int e = 0; e < Vec16B<R>::n; ++e) {
          if (c0 + e < NU) { r = fma(a3[c0 + e], d0[e], r); r2b = fma(a3[NU + c0 + e], d1[e], r2b); }
        }
      }
      r += r2b;
      const R pn = r6 + beta * r;
      r6 += rb * r;  // = phi~ + rho (phi_new - phi~)
      if constexpr (chk) { rn = umax(rn, OB::abs(pn)); ro = umax(ro, OB::abs(r7)); rd = umax(rd, OB::abs(pn - r7)); }
      r7 = pn;
      vp[kd * NXS + i] = r6;
    } else if (th_warp) {
      if (has_th) {
        const R hy = dxs[(v + 1) * NXS + IY] - dxs[v * NXS + IY] - r7;
        const R tn = max0(r5 + beta * hy);
        r5 += rho * (tn - r5);
        if constexpr (chk) { rn = umax(rn, OB::nonneg(tn)); ro = umax(ro, OB::abs(r6)); rd = umax(rd, OB::abs(tn - r6)); }
        r6 = tn;
      }
      const R vnext = __shfl_down_sync(0xffffffffu, r5, 1);
      if (has_th) tds[v + 1] = r5 - (v + 1 < N - 1 ? vnext : R(0));
    }
    if constexpr (chk) {
      U w6[6] = {zn, zo, zd, rn, ro, rd};
      block_max_u<U, 6>(w6, reinterpret_cast<U*>(sm + L.red));
      const R eabs = R(P.eps_abs), erel = R(P.eps_rel);
      return OB::val(w6[2]) <= eabs + erel * rmax(OB::val(w6[0]), OB::val(w6[1])) &&
             OB::val(w6[5]) <= eabs + erel * rmax(OB::val(w6[3]), OB::val(w6[4]));
    } else {
      (void)zn; (void)zo; (void)zd; (void)rn; (void)ro; (void)rd;
      __syncthreads();
      return false;
    }
  };
  int j;
  for (j = 1; j <= jmax; ++j) {
    if (force <= 0 && jcheck > 0 && (j % jcheck) == 0) {
      if (iterate(ChkTag<true>{})) break;
    } else {
      iterate(ChkTag<false>{});
    }
  }
  // iterates back to the image (warm start of the next SCP iteration)
  if (has_d) {
    sm[L.xh + kx * NX + i] = r1;
    sm[L.mup + tid] = r4; sm[L.mum + tid] = r5; sm[L.phi + tid] = r7;
  }
  if (has_u) sm[L.uh + ku * NU + cc] = r1;
  if (has_th) sm[L.th + v] = r6;
  if (has_x1) sm[L.xh + v] = r9;
  __syncthreads();
  return j > jmax ? jmax : j;
}

// ---------------------------------------------------------------------------
// PIPG_custom with each interval's blocks cut into tiles over a group of
// lanes (form 3).
//
// The same iteration as phase_pipg and phase_pipg_reg (Alg. PIPG_custom with
// the stop test of Alg. stopping).  Node vectors are padded to KS_NXB entries
// (16, or 8 when NX <= 8) and a block to KS_NXB x KS_NXB, cut into tiles of
// KS_TR = 8 rows by KS_TC columns (4, or 2 when NX <= 8).  Group g, KS_GS =
// KS_NR x KS_NC consecutive lanes, owns interval g and node g; its lane
// (rb, cb) = (l / KS_NC, l % KS_NC) keeps, in registers,
//  * tile (rb, cb) of hat A^-_g (zero outside NX, and for the last node,
//    which has no interval), as pairs of rows;
//  * the tile's rows of hat B^-_g and hat B^+_g in the control columns
//    cb + KS_NC s.
// One tile serves both products of an iteration: A^T phi~ in the primal step
// and A (2 x - x~) in the dual step.  A tile's partial sums are combined over
// the lanes of its tile column (primal) or tile row (dual) by butterfly
// shuffles that leave each lane the full sums of KS_WC columns (KS_WR rows);
// that lane owns those x components (dual rows).  The control sums are
// combined on every lane of a tile column, so each of them holds the node's
// controls.  What stays inside a group (phi~_g, the extrapolated x_g and u_g)
// moves by shuffles.  Shared memory carries what the neighbouring groups
// read: phi~_g and hat B^+_g^T phi~_g into the primal step of group g+1, the
// extrapolated x_{g+1} and u_{g+1} into the dual step of group g, and the
// relaxed CTCS duals.  Products run as packed pairs (two FP32 FMAs in one
// instruction on sm_100 and later).
// Needs blockDim.x >= pipg_ks_threads(N).
// ---------------------------------------------------------------------------
constexpr int KS_NXB = NX <= 8 ? 8 : 16;  // node vectors padded to whole tiles
constexpr int KS_TR = 8;                  // tile rows
constexpr int KS_TC = NX <= 8 ? 2 : 4;    // tile columns
constexpr int KS_NR = KS_NXB / KS_TR;     // tile rows per block (lanes of a tile column)
constexpr int KS_NC = KS_NXB / KS_TC;     // tile columns per block (lanes of a tile row)
constexpr int KS_GS = KS_NR * KS_NC;      // lanes per group
constexpr int KS_WR = KS_TR / KS_NC;      // dual rows a lane owns
constexpr int KS_WC = KS_TC / KS_NR;      // x components a lane owns
static_assert(KS_WR >= 1 && KS_WC >= 1 && 32 % KS_GS == 0, "tile shape");
__host__ __device__ inline int pipg_ks_threads(int N) { return round32(N * KS_GS); }

// Shared-memory offsets (inside the phase-local union region, 16-byte
// aligned): vp[N][KS_NXB] (phi~ per interval), dx[N][KS_NXB], du[N][nup],
// bq[N][nup] (hat B^+_{g-1}^T phi~_{g-1}, the control gradient node g gets
// from interval g-1), th[N] (theta~ per interval; th[N-1] stays zero).
struct KsLay { int vp, dx, du, bq, th, end; };
__host__ __device__ inline KsLay make_ks_lay(const Lay& L) {
  const int nup = KS_NC * ((L.nu + KS_NC - 1) / KS_NC);
  KsLay Q;
  int o = (L.xt + 3) & ~3;
  Q.vp = o; o += L.N * KS_NXB;
  Q.dx = o; o += L.N * KS_NXB;
  Q.du = o; o += (L.N * nup + 3) & ~3;
  Q.bq = o; o += (L.N * nup + 3) & ~3;
  Q.th = o; o += (L.N + 3) & ~3;
  Q.end = o;
  return Q;
}

// Two values in one register pair: FP32 uses the packed FMA of sm_100 and
// later, FP64 two scalar FMAs.
template <typename R> struct Pr;
template <> struct Pr<float> {
  using T = float2;
  __device__ __forceinline__ static T mk(float a, float b) { return make_float2(a, b); }
  __device__ __forceinline__ static T mul(T a, T b) { return __fmul2_rn(a, b); }
  __device__ __forceinline__ static T fma(T a, T b, T c) { return __ffma2_rn(a, b, c); }
};
template <> struct Pr<double> {
  struct T { double x, y; };
  __device__ __forceinline__ static T mk(double a, double b) { return T{a, b}; }
  __device__ __forceinline__ static T mul(T a, T b) { return T{a.x * b.x, a.y * b.y}; }
  __device__ __forceinline__ static T fma(T a, T b, T c) { return T{::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)}; }
};

// Butterflies over the M lanes sel = 0..M-1 at stride S (M = 1, 2 or 4).  A
// lane keeps its n partial sums in an order of its own: stored entry s is
// entry s ^ ks_perm<M, n>(sel).  Then every reduce round keeps the first half
// of the stored entries and sends the second half (no per-lane selection),
// and ks_reduce_scatter leaves lane sel the full sums of entries
// (n / M) sel .. (n / M) sel + n / M - 1, in order.  ks_all_gather is its
// inverse and returns the n entries in the lane's stored order.
template <int M, int n>
__host__ __device__ constexpr int ks_perm(int sel) {
  return M == 4 ? (n / 2) * ((sel >> 1) & 1) + (n / 4) * (sel & 1) : (M == 2 ? (n / 2) * (sel & 1) : 0);
}
template <int n, int S, typename R>
__device__ __forceinline__ void ks_rs_round(const R (&v)[n], R (&o)[n / 2]) {
#pragma unroll
  for (int e = 0; e < n / 2; ++e) o[e] = v[e] + __shfl_xor_sync(0xffffffffu, v[n / 2 + e], S);
}
template <int n, int S, typename R>
__device__ __forceinline__ void ks_ag_round(const R (&o)[n], R (&v)[2 * n]) {
#pragma unroll
  for (int e = 0; e < n; ++e) {
    v[e] = o[e];
    v[n + e] = __shfl_xor_sync(0xffffffffu, o[e], S);
  }
}
template <int M, int S, int n, typename R>
__device__ __forceinline__ void ks_reduce_scatter(const R (&v)[n], R (&o)[n / M]) {
  if constexpr (M == 1) {
#pragma unroll
    for (int e = 0; e < n; ++e) o[e] = v[e];
  } else if constexpr (M == 2) {
    ks_rs_round<n, S>(v, o);
  } else {
    static_assert(M == 4, "groups of 1, 2 or 4 lanes");
    R t[n / 2];
    ks_rs_round<n, 2 * S>(v, t);
    ks_rs_round<n / 2, S>(t, o);
  }
}
template <int M, int S, int n, typename R>
__device__ __forceinline__ void ks_all_gather(const R (&o)[n / M], R (&v)[n]) {
  if constexpr (M == 1) {
#pragma unroll
    for (int e = 0; e < n; ++e) v[e] = o[e];
  } else if constexpr (M == 2) {
    ks_ag_round<n / 2, S>(o, v);
  } else {
    static_assert(M == 4, "groups of 1, 2 or 4 lanes");
    R t[n / 2];
    ks_ag_round<n / 4, S>(o, t);
    ks_ag_round<n / 2, 2 * S>(t, v);
  }
}
// every lane of the M gets the same sum (IEEE addition commutes, so the lanes
// agree bit for bit)
template <int M, int S, typename R>
__device__ __forceinline__ R ks_all_sum(R x) {
  if constexpr (M >= 2) x += __shfl_xor_sync(0xffffffffu, x, S);
  if constexpr (M >= 4) x += __shfl_xor_sync(0xffffffffu, x, 2 * S);
  return x;
}

template <int V> struct KsTag { static constexpr int value = V; };

#ifdef PDG_PIPG_KS_NOINLINE
#define PDG_PKS_ATTR __noinline__
#else
#define PDG_PKS_ATTR __forceinline__
#endif
template <typename R, int NU>
__device__ PDG_PKS_ATTR int phase_pipg_ks(const DParams& P, const Lay& L, R* /*image*/, R sigma, int force) {
  using OB = OrdBits<R>;
  using U = typename OB::U;
  using PR = Pr<R>;
  using T2 = typename PR::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* const sm = reinterpret_cast<R*>(smraw);
  constexpr int NXB = KS_NXB, TR = KS_TR, TC = KS_TC, NR = KS_NR, NCB = KS_NC, GS = KS_GS;
  constexpr int WR = KS_WR, WC = KS_WC, TH = TR / 2;
  constexpr int NC = (NU + NCB - 1) / NCB;  // control columns per lane
  constexpr int NUP = NCB * NC;
  const int N = L.N, tid = threadIdx.x;
  const KsLay Q = make_ks_lay(L);
  R* const vps = sm + Q.vp;
  R* const dxs = sm + Q.dx;
  R* const dus = sm + Q.du;
  R* const bqs = sm + Q.bq;
  R* const ths = sm + Q.th;
  const int g = tid / GS, ln = tid - GS * (tid / GS);
  const int rb = ln / NCB, cb = ln - NCB * (ln / NCB);
  // whole warps past the last group only join the barriers; lanes of a group
  // past the last one in a live warp join the shuffles, read clamped
  // addresses and store nothing
  const bool wlive = (tid & ~31) < N * GS;
  const bool live = g < N;
  const bool has_iv = g < N - 1;
  const int gv = live ? g : N - 1;
  const int gm1 = gv > 0 ? gv - 1 : 0, gp1 = gv < N - 1 ? gv + 1 : gv;
  const R wp = R(P.w_prox);
  const R alpha = R(2) / (wp + sqrt(wp * wp + R(4) * R(P.omega) * sigma));
  const R beta = R(P.omega) * alpha;
  const R c1 = R(1) - alpha * wp;
  const R rho = R(P.rho);
  const R rhb = rho * beta;
  const R aw = alpha * R(P.w_ep);  // virtual-control iterates kept shifted (see phase_pipg)
  const R omr = R(1) - rho, raw = rho * aw;
  for (int t = tid; t < Q.end - Q.vp; t += blockDim.x) sm[Q.vp + t] = R(0);
  // ---- tiles, in the lane's stored order (rows permuted by its place in the
  // tile row, columns by its place in the tile column; see ks_perm), as pairs
  // of stored rows 2h, 2h+1
  const int prow = ks_perm<NCB, TR>(cb), pcol = ks_perm<NR, TC>(rb);
  T2 ap[TH][TC], bm[TH][NC], bp[TH][NC];
#pragma unroll
  for (int h = 0; h < TH; ++h) {
    const int r0 = TR * rb + ((2 * h) ^ prow), r1 = TR * rb + ((2 * h + 1) ^ prow);
#pragma unroll
    for (int q = 0; q < TC; ++q) {
      const int c = TC * cb + (q ^ pcol);
      const bool okc = has_iv && c < NX;
      ap[h][q] = PR::mk((okc && r0 < NX) ? sm[L.Am + g * STM_SAS + stm_index(r0, c)] : R(0),
                        (okc && r1 < NX) ? sm[L.Am + g * STM_SAS + stm_index(r1, c)] : R(0));
    }
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const int cc = cb + NCB * s;
      const bool okc = has_iv && cc < NU;
      bm[h][s] = PR::mk((okc && r0 < NX) ? sm[L.Bm + g * b_stride(NU) + r0 * NU + cc] : R(0),
                        (okc && r1 < NX) ? sm[L.Bm + g * b_stride(NU) + r1 * NU + cc] : R(0));
      bp[h][s] = PR::mk((okc && r0 < NX) ? sm[L.Bp + g * b_stride(NU) + r0 * NU + cc] : R(0),
                        (okc && r1 < NX) ? sm[L.Bp + g * b_stride(NU) + r1 * NU + cc] : R(0));
    }
  }
  // ---- iterates.  x components TC cb + WC rb + e of node g, dual rows
  // TR rb + WR cb + e of interval g, controls cb + NCB s of node g (on every
  // lane of the tile column)
  // Only the relaxed iterates stay in registers.  The unextrapolated ones
  // (x_hat, u_hat, mu+-, phi, theta) are what the stop test compares and what
  // the loop returns: the iteration before a tested one and the tested one
  // write them to the image, where the tested one reads them back, and the
  // last iteration leaves them there.
  R xt[WC], zfx[WC], dxn[WC];
  bool fx[WC], okx[WC], okd[WR];
  R nvp[WR], nvm[WR], ft[WR], wv[WR];
  R ut[NC], dun[NC];
  T2 fg[TH];
#pragma unroll
  for (int e = 0; e < WC; ++e) {
    const int c = TC * cb + WC * rb + e;
    okx[e] = live && c < NX;
    xt[e] = okx[e] ? sm[L.xh + g * NX + c] : R(0);
    fx[e] = okx[e] && (g == 0 || (g == N - 1 && P.fix_f[c]));
    zfx[e] = !okx[e] ? R(0) : (g == 0 ? sm[L.zi + c] : (fx[e] ? sm[L.zf + c] : R(0)));
    dxn[e] = 0;
  }
#pragma unroll
  for (int e = 0; e < WR; ++e) {
    const int i = TR * rb + WR * cb + e;
    okd[e] = has_iv && i < NX;
    const int o = g * NX + i;
    wv[e] = okd[e] ? sm[L.w + o] : R(0);
    nvp[e] = okd[e] ? sm[L.mup + o] - aw : R(0);
    nvm[e] = okd[e] ? sm[L.mum + o] - aw : R(0);
    ft[e] = okd[e] ? sm[L.phi + o] : R(0);
  }
#pragma unroll
  for (int h = 0; h < TH; ++h) {
    const int r0 = TR * rb + ((2 * h) ^ prow), r1 = TR * rb + ((2 * h + 1) ^ prow);
    fg[h] = PR::mk((has_iv && r0 < NX) ? sm[L.phi + g * NX + r0] : R(0),
                   (has_iv && r1 < NX) ? sm[L.phi + g * NX + r1] : R(0));
  }
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    const int cc = cb + NCB * s;
    const bool ok = live && cc < NU;
    ut[s] = ok ? sm[L.uh + g * NU + cc] : R(0);
    dun[s] = 0;
  }
  const R lo = sm[L.lo + gv], hi = sm[L.hi + gv];
  // the lane that owns dual row IY of interval g also owns theta_g
  const int iy0 = TR * rb + WR * cb;
  const bool th_lane = has_iv && IY >= iy0 && IY < iy0 + WR;
  R tht = 0;
  if (th_lane) tht = sm[L.th + g];
  __syncthreads();  // the exchange region is zero
#pragma unroll
  for (int e = 0; e < WR; ++e)
    if (okd[e]) vps[g * NXB + TR * rb + WR * cb + e] = ft[e];
  for (int t = tid; t < N - 1; t += blockDim.x) ths[t] = sm[L.th + t];
  // hat B^+_g^T phi~_g for node g+1, summed over the tile column
  auto bq_out = [&]() {
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      T2 acc = PR::mul(bp[0][s], fg[0]);
#pragma unroll
      for (int h = 1; h < TH; ++h) acc = PR::fma(bp[h][s], fg[h], acc);
      const R v = ks_all_sum<NR, NCB>(acc.x + acc.y);
      if (has_iv && rb == 0 && cb + NCB * s < NU) bqs[(g + 1) * NUP + cb + NCB * s] = v;
    }
  };
  if (wlive) bq_out();
  __syncthreads();
  const R acost = alpha * R(P.w_cost);
  const int jmax = force > 0 ? force : P.pipg_jmax;
  const int jcheck = P.pipg_jcheck;
  // V = 0: plain iteration; 1: also stores the unextrapolated iterates in
  // the image; 2: runs the stop test against the stored ones, then stores
  auto iterate = [&](auto v_tag) -> bool {
    constexpr int V = decltype(v_tag)::value;
    constexpr bool chk = V == 2, st = V >= 1;
    U zn = 0, zo = 0, zd = 0, rn = 0, ro = 0, rd = 0;
    // ---- projected gradient step (primal)
    if (wlive) {
      R cx[TC], cu[NC];
#pragma unroll
      for (int q = 0; q < TC; ++q) {
        T2 acc = PR::mul(ap[0][q], fg[0]);
#pragma unroll
        for (int h = 1; h < TH; ++h) acc = PR::fma(ap[h][q], fg[h], acc);
        cx[q] = acc.x + acc.y;
      }
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        T2 acc = PR::mul(bm[0][s], fg[0]);
#pragma unroll
        for (int h = 1; h < TH; ++h) acc = PR::fma(bm[h][s], fg[h], acc);
        cu[s] = ks_all_sum<NR, NCB>(acc.x + acc.y) + bqs[gv * NUP + cb + NCB * s];
      }
      R gx[WC];
      ks_reduce_scatter<NR, NCB>(cx, gx);
      const R tdv = ths[gm1] - ths[gv];  // theta~_{g-1} - theta~_g (th[N-1] = 0)
#pragma unroll
      for (int e = 0; e < WC; ++e) {
        const int c = TC * cb + WC * rb + e;  // padding entries of vp read as zero
        const R G = fma(c == IY ? R(1) : R(0), tdv, gx[e] - vps[gm1 * NXB + c]);
        const R cost = (g == N - 1 && c == IM) ? acost : R(0);
        R xn = fma(-alpha, G, fma(c1, xt[e], cost));
        xn = fx[e] ? zfx[e] : xn;
        dxn[e] = fma(R(2), xn, -xt[e]);
        if (okx[e]) dxs[g * NXB + c] = dxn[e];
        xt[e] += rho * (xn - xt[e]);
        if constexpr (chk) {
          if (okx[e]) {
            const R old = sm[L.xh + g * NX + c];
            zn = umax(zn, OB::abs(xn)); zo = umax(zo, OB::abs(old)); zd = umax(zd, OB::abs(xn - old));
          }
        }
        if constexpr (st) {
          if (okx[e]) sm[L.xh + g * NX + c] = xn;
        }
      }
      R un[NC];
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        const int cc = cb + NCB * s;
        un[s] = c1 * ut[s] - alpha * cu[s];
        if (cc == NU - 1) un[s] = rmin(rmax(un[s], lo), hi);
      }
      if (P.soc) {
        // the node's thrust onto the sector (cone about body x, then the
        // ball); component cc sits on lane cc % NCB of this tile row, in
        // control column cc / NCB, and every tile row projects alike
        // (constants and the reference thrust read here: they would hold
        // registers across the whole loop)
        const R sa = R(P.soc_tan), tmax = R(P.T_max), pT = R(P.Pu[0]), ipT = R(P.Puinv[0]);
        const int base = (tid & 31) & ~(NCB - 1);
        R tv[NC], tref[NC];
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          const int cc = cb + NCB * s;
          tref[s] = (live && cc < 3) ? sm[L.Ub + g * NU + cc] : R(0);
          tv[s] = cc < 3 ? tref[s] + pT * un[s] : R(0);
        }
        R T0 = __shfl_sync(0xffffffffu, tv[0], base);
        R T1 = __shfl_sync(0xffffffffu, tv[1 / NCB], base + 1 % NCB);
        R T2v = __shfl_sync(0xffffffffu, tv[2 / NCB], base + 2 % NCB);
        const R rr = ::sqrt(T1 * T1 + T2v * T2v);
        if (rr > sa * T0) {
          if (sa * rr <= -T0) {
            T0 = 0; T1 = 0; T2v = 0;
          } else {
            const R tp = (T0 + sa * rr) / (R(1) + sa * sa);
            const R sc = sa * tp / rr;
            T0 = tp; T1 *= sc; T2v *= sc;
          }
        }
        const R nT = ::sqrt(T0 * T0 + T1 * T1 + T2v * T2v);
        if (nT > tmax) { const R f = tmax / nT; T0 *= f; T1 *= f; T2v *= f; }
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          const int cc = cb + NCB * s;
          if (cc < 3) un[s] = ((cc == 0 ? T0 : (cc == 1 ? T1 : T2v)) - tref[s]) * ipT;
        }
      }
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        const int cc = cb + NCB * s;
        const bool ok = live && cc < NU;
        dun[s] = fma(R(2), un[s], -ut[s]);
        if (ok && rb == 0) dus[g * NUP + cc] = dun[s];
        ut[s] += rho * (un[s] - ut[s]);
        if constexpr (chk) {
          if (ok) {
            const R old = sm[L.uh + g * NU + cc];
            zn = umax(zn, OB::abs(un[s])); zo = umax(zo, OB::abs(old)); zd = umax(zd, OB::abs(un[s] - old));
          }
        }
        if constexpr (st) {
          if (ok && rb == 0) sm[L.uh + g * NU + cc] = un[s];
        }
      }
    }
    __syncthreads();
    // ---- virtual controls and proportional-integral feedback (dual)
    if (wlive) {
      R dc[TC], rr[TR];
      ks_all_gather<NR, NCB>(dxn, dc);
      T2 du0[NC], du1[NC];
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        const R v1 = dus[gp1 * NUP + cb + NCB * s];
        du0[s] = PR::mk(dun[s], dun[s]);
        du1[s] = PR::mk(v1, v1);
      }
#pragma unroll
      for (int h = 0; h < TH; ++h) {
        T2 acc = PR::mul(ap[h][0], PR::mk(dc[0], dc[0]));
#pragma unroll
        for (int q = 1; q < TC; ++q) acc = PR::fma(ap[h][q], PR::mk(dc[q], dc[q]), acc);
#pragma unroll
        for (int s = 0; s < NC; ++s) { acc = PR::fma(bm[h][s], du0[s], acc); acc = PR::fma(bp[h][s], du1[s], acc); }
        rr[2 * h] = acc.x;
        rr[2 * h + 1] = acc.y;
      }
      R rs[WR];
      ks_reduce_scatter<NCB, 1>(rr, rs);
#pragma unroll
      for (int e = 0; e < WR; ++e) {
        const int i = TR * rb + WR * cb + e;  // padding entries of dx read as zero
        const R f = ft[e], va = nvp[e], vb = nvm[e];
        const R mp = max0(va - alpha * f);
        const R mm = max0(vb + alpha * f);
        nvp[e] = omr * va + (rho * mp - raw);
        nvm[e] = omr * vb + (rho * mm - raw);
        const int o = g * NX + i;
        if constexpr (chk) {
          if (okd[e]) {
            const R op = sm[L.mup + o], om = sm[L.mum + o];
            zn = umax(zn, umax(OB::nonneg(mp), OB::nonneg(mm)));
            zo = umax(zo, umax(OB::nonneg(op), OB::nonneg(om)));
            zd = umax(zd, umax(OB::abs(mp - op), OB::abs(mm - om)));
          }
        }
        if constexpr (st) {
          if (okd[e]) { sm[L.mup + o] = mp; sm[L.mum + o] = mm; }
        }
        const R r0 = wv[e] + (fma(R(2), mp, -va) - fma(R(2), mm, -vb)) - dxs[gp1 * NXB + i] + rs[e];
        const R r = okd[e] ? r0 : R(0);  // rows that do not exist keep phi~ = 0
        const R pn = f + beta * r;
        ft[e] = f + rhb * r;  // = phi~ + rho (phi_new - phi~)
        if constexpr (chk) {
          if (okd[e]) {
            const R old = sm[L.phi + o];
            rn = umax(rn, OB::abs(pn)); ro = umax(ro, OB::abs(old)); rd = umax(rd, OB::abs(pn - old));
          }
        }
        if constexpr (st) {
          if (okd[e]) sm[L.phi + o] = pn;
        }
        if (okd[e]) vps[g * NXB + i] = ft[e];
      }
      {
        R fv[TR];
        ks_all_gather<NCB, 1>(ft, fv);
#pragma unroll
        for (int h = 0; h < TH; ++h) fg[h] = PR::mk(fv[2 * h], fv[2 * h + 1]);
      }
      bq_out();
      if (th_lane) {
        const R hy = dxs[gp1 * NXB + IY] - dxs[g * NXB + IY] - sm[L.eps + g];
        const R tn = max0(tht + beta * hy);
        tht += rho * (tn - tht);
        if constexpr (chk) {
          const R old = sm[L.th + g];
          rn = umax(rn, OB::nonneg(tn)); ro = umax(ro, OB::abs(old)); rd = umax(rd, OB::abs(tn - old));
        }
        if constexpr (st) sm[L.th + g] = tn;
        ths[g] = tht;
      }
    }
    if constexpr (chk) {
      U w6[6] = {zn, zo, zd, rn, ro, rd};
      block_max_u<U, 6>(w6, reinterpret_cast<U*>(sm + L.red));
      const R eabs = R(P.eps_abs), erel = R(P.eps_rel);
      return OB::val(w6[2]) <= eabs + erel * rmax(OB::val(w6[0]), OB::val(w6[1])) &&
             OB::val(w6[5]) <= eabs + erel * rmax(OB::val(w6[3]), OB::val(w6[4]));
    } else {
      (void)zn; (void)zo; (void)zd; (void)rn; (void)ro; (void)rd;
      __syncthreads();
      return false;
    }
  };
  // blocks of jcheck iterations whose last one runs the stop test (the one
  // before it stores the iterates it compares with), so that the loop carries
  // no per-iteration remainder; the last iteration of the loop stores
  const bool chk_on = force <= 0 && jcheck > 0;
  const int per = chk_on ? jcheck : (jmax > 0 ? jmax : 1);
  int j = 0;
  while (j < jmax) {
    const int nb = per < jmax - j ? per : jmax - j;
    const bool tested = chk_on && nb == per;
    const int plain = tested ? nb - 2 : nb - 1;
    for (int k = 0; k < plain; ++k) iterate(KsTag<0>{});
    if (!tested || nb >= 2) iterate(KsTag<1>{});
    j += nb;
    if (tested && iterate(KsTag<2>{})) break;
  }
  __syncthreads();
  return j;
}

// SCP update (Sec. 2.3.2: x = P_x x_hat + xbar) and convergence test
// (reading: scaled step, scaled defect and CTCS budget).  Returns the scaled
// step; *nonfinite is set when X or U holds a non-finite value.
template <typename R, int NU>
__device__ R phase_update(const DParams& P, const Lay& L, R* sm, bool* nonfinite) {
  const int N = L.N, T = blockDim.x, tid = threadIdx.x;
  const int nx = N * NX, nuu = N * NU;
  R* Xb = sm + L.Xb;
  R* Ub = sm + L.Ub;
  R st = 0, bad = 0;
  for (int t = tid; t < nx + nuu; t += T) {
    if (t < nx) {
      const int i = t % NX;
      const R d = sm[L.xh + t];
      st = rmax(st, fabs(d));
      const R nv = Xb[t] + R(P.Px[i]) * d;
      Xb[t] = nv;
      if (!isfinite(nv)) bad = 1;
    } else {
      const int q = t - nx, cc = q % NU;
      const R d = sm[L.uh + q];
      st = rmax(st, fabs(d));
      const R nv = Ub[q] + R(P.Pu[cc]) * d;
      Ub[q] = nv;
      if (!isfinite(nv)) bad = 1;
    }
  }
  R v[2] = {st, bad};
  block_max_k<R, 2>(v, sm + L.red);
  *nonfinite = v[1] > R(0) || !isfinite(v[0]);
  return v[0];
}

}  // namespace pdg
