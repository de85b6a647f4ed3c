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

// Initial guess (the paper asks for "an appropriate" one; Sec. 5): straight
// lines in r, v, w from x0 to z_f, normalized linear interpolation of q, mass
// from m_wet to (m_wet + m_dry)/2, y = 0, hover thrust m|g| along body x,
// gamma = 0, s = tf_guess.
template <typename R, int NU>
__device__ void phase_init_guess(const DParams& P, const Lay& L, R* sm) {
  const int N = L.N;
  const R* x0 = sm + L.x0;
  R* Xb = sm + L.Xb;
  R* Ub = sm + L.Ub;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const R t = R(k) / R(N - 1);
    const R a = R(1) - t;
    R* x = Xb + k * NX;
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
    R* u = Ub + k * NU;
#pragma unroll
    for (int c = 0; c < NU; ++c) u[c] = 0;
    u[0] = x[IM] * R(P.g0);
    u[NU - 1] = R(P.tf_guess);
  }
}

// Sec. 2.3.1 + 2.3.2: integrate, on every interval, the joint IVP of x and its
// state-transition matrices with RK4 (nsub substeps, FOH controls), then write
// the prescaled blocks hat A^-_k, hat B^-_k, hat B^+_k, hat w_k.  Thread
// mapping: lane l of warp 0 integrates x on interval k0 + l and evaluates the
// compact Jacobians at each RK4 stage (its RK4 state lives in the interval's
// stage buffer); every thread of warps 1.. holds one STM column (15 + 2 NU per
// interval) in registers.  Intervals are processed in waves of L.ipw.
// Returns max_k |hat w_k|_inf (the scaled defect) on every thread.
#ifdef PDG_DISC_INLINE
#define PDG_DISC_ATTR __forceinline__
#else
#define PDG_DISC_ATTR __noinline__
#endif
template <typename R, int NU>
__device__ PDG_DISC_ATTR R phase_discretize(const DParams& P, const Lay& L, R* sm) {
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
  for (int k0 = 0; k0 < N - 1; k0 += L.ipw) {
    const int k = k0 + il;
    const bool active = il < L.ipw && k < N - 1;
    R* st = sm + L.stage + (active ? il : 0) * L.sa;
    R* xP = st + SA_A + NX * NU;
    R* xA = xP + NX;
    R* xS = xA + NX;
    R Pv[NX], Sv[NX], Ac[NX];
    if (active) {
      if (evaluator) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { xP[i] = Xb[k * NX + i]; xS[i] = Xb[k * NX + i]; }
      } else {
#pragma unroll
        for (int i = 0; i < NX; ++i) { Pv[i] = (c == i) ? R(1) : R(0); Sv[i] = Pv[i]; }
      }
    }
    for (int n = 0; n < nsub; ++n) {
#pragma unroll 1
      for (int sgi = 0; sgi < 4; ++sgi) {
        const R lp = (R(n) + (sgi == 0 ? R(0) : (sgi == 3 ? R(1) : R(0.5)))) / R(nsub);
        if (active && evaluator) {
          R u[NU], x[NX], d[NX];
#pragma unroll
          for (int i = 0; i < NU; ++i) u[i] = (R(1) - lp) * Ub[k * NU + i] + lp * Ub[(k + 1) * NU + i];
#pragma unroll
          for (int i = 0; i < NX; ++i) x[i] = xS[i];
          model_eval<R, NU>(P, x, u, d, st, st + SA_A);
          if (sgi == 0) {
#pragma unroll
            for (int i = 0; i < NX; ++i) { xA[i] = d[i]; xS[i] = xP[i] + h2 * d[i]; }
          } else if (sgi == 1) {
#pragma unroll
            for (int i = 0; i < NX; ++i) { xA[i] += R(2) * d[i]; xS[i] = xP[i] + h2 * d[i]; }
          } else if (sgi == 2) {
#pragma unroll
            for (int i = 0; i < NX; ++i) { xA[i] += R(2) * d[i]; xS[i] = xP[i] + h * d[i]; }
          } else {
#pragma unroll
            for (int i = 0; i < NX; ++i) { const R v = xP[i] + h6 * (xA[i] + d[i]); xP[i] = v; xS[i] = v; }
          }
        }
        __syncthreads();
        if (active && !evaluator) {
          R d[NX];
          const R lam = minus ? (R(1) - lp) : lp;
          model_jvp<R, NU>(st, st + SA_A, Sv, cu, lam, d);
          if (sgi == 0) {
#pragma unroll
            for (int i = 0; i < NX; ++i) { Ac[i] = d[i]; Sv[i] = Pv[i] + h2 * d[i]; }
          } else if (sgi == 1) {
#pragma unroll
            for (int i = 0; i < NX; ++i) { Ac[i] += R(2) * d[i]; Sv[i] = Pv[i] + h2 * d[i]; }
          } else if (sgi == 2) {
#pragma unroll
            for (int i = 0; i < NX; ++i) { Ac[i] += R(2) * d[i]; Sv[i] = Pv[i] + h * d[i]; }
          } else {
#pragma unroll
            for (int i = 0; i < NX; ++i) { Pv[i] += h6 * (Ac[i] + d[i]); Sv[i] = Pv[i]; }
          }
        }
        __syncthreads();
      }
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
        for (int i = 0; i < NX; ++i) Am[(k * NX + i) * NX + c] = Pv[i] * pc * R(P.Pxinv[i]);
      } else {
        const R pc = R(P.Pu[cu]);
        R* Bt = minus ? Bm : Bp;
#pragma unroll
        for (int i = 0; i < NX; ++i) Bt[(k * NX + i) * NU + cu] = Pv[i] * pc * R(P.Pxinv[i]);
      }
    }
    __syncthreads();
  }
  R v[1] = {dmax};
  block_max_k<R, 1>(v, sm + L.red);
  return v[0];
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
      const int k = t - (N - 1);
      const R s = Ub[k * NU + NU - 1];
      sm[L.lo + k] = (R(P.s_min) - s) * iPs;
      sm[L.hi + k] = (R(P.s_max) - s) * iPs;
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
          const int k = t / NX, i = t - NX * k;
          const R* a = Am + (k * NX + i) * NX;
          const R* xk = px + k * NX;
          R r = pp[t] - pn[t] - px[(k + 1) * NX + i];
#pragma unroll
          for (int cc = 0; cc < NX; ++cc) r += a[cc] * xk[cc];
          const R* bm = Bm + (k * NX + i) * NU;
          const R* bp = Bp + (k * NX + i) * NU;
#pragma unroll
          for (int cc = 0; cc < NU; ++cc) r += bm[cc] * pu[k * NU + cc] + bp[cc] * pu[(k + 1) * NU + cc];
          ph[t] = r * isig;
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
          const int k = t / NX, i = t - NX * k;
          R g = 0;
          if (k < N - 1) {
            const R* a = Am + k * NX * NX + i;
            const R* f = ph + k * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) g += a[r * NX] * f[r];
            if (i == IY) g -= pt[k];
          }
          if (k > 0) {
            g -= ph[(k - 1) * NX + i];
            if (i == IY) g += pt[k - 1];
          }
          px[t] = g;
          s2 += g * g;
        }
      } else if (t < PX + PU) {
        const int q = t - PX;
        if (q < nuu) {
          const int k = q / NU, cc = q - NU * k;
          R g = 0;
          if (k < N - 1) {
            const R* a = Bm + k * NX * NU + cc;
            const R* f = ph + k * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) g += a[r * NU] * f[r];
          }
          if (k > 0) {
            const R* a = Bp + (k - 1) * NX * NU + cc;
            const R* f = ph + (k - 1) * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) g += a[r * NU] * f[r];
          }
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
//   primal phase: x_hat of nodes 2..N (15 (N-1) tasks), then u_hat (N nu
//     tasks) and the fixed node 1 (15 tasks);
//   dual phase: row i of interval k updates mu^+-, nu^+- (they read the same
//     extrapolated dual entry) and then phi; then the CTCS rows theta_k.
// Returns the iterations run.
template <typename R, int NU>
__device__ int phase_pipg(const DParams& P, const Lay& L, R* sm, R sigma, int force) {
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
  for (int t = tid; t < N * NX + N * NU + 2 * nm + (N - 1); t += T) {
    if (t < N * NX) xt[t] = xh[t];
    else if (t < N * NX + N * NU) ut[t - N * NX] = uh[t - N * NX];
    else if (t < N * NX + N * NU + nm) { const int q = t - N * NX - N * NU; nup[q] = mup[q]; num[q] = mum[q]; }
    else if (t < N * NX + N * NU + 2 * nm) { const int q = t - N * NX - N * NU - nm; vph[q] = phi[q]; }
    else { const int q = t - N * NX - N * NU - 2 * nm; vth[q] = th[q]; }
  }
  __syncthreads();
  const R wp = R(P.w_prox);
  const R alpha = R(2) / (wp + sqrt(wp * wp + R(4) * R(P.omega) * sigma));
  const R beta = R(P.omega) * alpha;
  const R c1 = R(1) - alpha * wp;
  const R rho = R(P.rho);
  const R rb = rho * beta;
  const R wcost = R(P.w_cost), wep = R(P.w_ep);
  const R eabs = R(P.eps_abs), erel = R(P.eps_rel);
  const R sa = R(P.soc_tan), tmax = R(P.T_max), pT = R(P.Pu[0]), ipT = R(P.Puinv[0]);
  const int jmax = force > 0 ? force : P.pipg_jmax;
  const int jcheck = P.pipg_jcheck;
  int j;
  for (j = 1; j <= jmax; ++j) {
    const bool chk = force <= 0 && jcheck > 0 && (j % jcheck) == 0;
    R zn = 0, zo = 0, zd = 0;
    // ---- projected gradient step (primal)
    for (int t = tid; t < PX + PU; t += T) {
      if (t < PX) {
        if (t < nxk) {
          const int k = t / NX + 1, i = t - NX * (k - 1);
          const int o = k * NX + i;
          const R xv = xt[o];
          R G = -vph[(k - 1) * NX + i];
          if (k < N - 1) {
            const R* a = Am + k * NX * NX + i;
            const R* f = vph + k * NX;
            R G2 = 0;
#pragma unroll
            for (int r = 0; r < NX; r += 2) {
              G += a[r * NX] * f[r];
              if (r + 1 < NX) G2 += a[(r + 1) * NX] * f[r + 1];
            }
            G += G2;
            if (i == IY) G -= vth[k];
          }
          if (i == IY) G += vth[k - 1];
          if (k == N - 1 && i == IM) G -= wcost;  // e_cost = -e_m (maximize m_N)
          R xn = c1 * xv - alpha * G;
          if (k == N - 1 && P.fix_f[i]) xn = zf[i];
          dx[o] = R(2) * xn - xv;
          xt[o] = xv + rho * (xn - xv);
          if (chk) {
            const R old = xh[o];
            zn = rmax(zn, fabs(xn)); zo = rmax(zo, fabs(old)); zd = rmax(zd, fabs(xn - old));
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
          R uv = 0, un = 0;
          if (valid) {
            uv = ut[o];
            R Gs = 0, G2 = 0;
            if (k < N - 1) {
              const R* a = Bm + k * NX * NU + cc;
              const R* f = vph + k * NX;
#pragma unroll
              for (int r = 0; r < NX; ++r) Gs += a[r * NU] * f[r];
            }
            if (k > 0) {
              const R* a = Bp + (k - 1) * NX * NU + cc;
              const R* f = vph + (k - 1) * NX;
#pragma unroll
              for (int r = 0; r < NX; ++r) G2 += a[r * NU] * f[r];
            }
            Gs += G2;
            un = c1 * uv - alpha * Gs;
            if (cc == NU - 1) un = rmin(rmax(un, lo[k]), hi[k]);
          }
          if (P.soc) {
            // project the node's thrust onto the sector (all lanes of the warp
            // take part in the shuffles; each group of G lanes is one node)
            const R Tb = (valid && cc < 3) ? sm[L.Ub + o] : R(0);
            const R tv = (valid && cc < 3) ? Tb + pT * un : R(0);
            const int base = (threadIdx.x & 31) & ~(G - 1);
            R T0 = __shfl_sync(0xffffffffu, tv, base);
            R T1 = __shfl_sync(0xffffffffu, tv, base + 1);
            R T2 = __shfl_sync(0xffffffffu, tv, base + 2);
            const R rr = sqrt(T1 * T1 + T2 * T2);
            if (rr > sa * T0) {
              if (sa * rr <= -T0) {
                T0 = 0; T1 = 0; T2 = 0;
              } else {
                const R tp = (T0 + sa * rr) / (R(1) + sa * sa);
                const R sc = sa * tp / rr;
                T0 = tp; T1 *= sc; T2 *= sc;
              }
            }
            const R nT = sqrt(T0 * T0 + T1 * T1 + T2 * T2);
            if (nT > tmax) { const R f = tmax / nT; T0 *= f; T1 *= f; T2 *= f; }
            if (valid && cc < 3) un = ((cc == 0 ? T0 : (cc == 1 ? T1 : T2)) - Tb) * ipT;
          }
          if (valid) {
            du[o] = R(2) * un - uv;
            ut[o] = uv + rho * (un - uv);
            if (chk) {
              const R old = uh[o];
              zn = rmax(zn, fabs(un)); zo = rmax(zo, fabs(old)); zd = rmax(zd, fabs(un - old));
            }
            uh[o] = un;
          }
        } else if (q < PG + NX) {
          // node 1: every component fixed by E_i
          const int i = q - PG;
          const R xv = xt[i], xn = zi[i];
          dx[i] = R(2) * xn - xv;
          xt[i] = xv + rho * (xn - xv);
          if (chk) {
            const R old = xh[i];
            zn = rmax(zn, fabs(xn)); zo = rmax(zo, fabs(old)); zd = rmax(zd, fabs(xn - old));
          }
          xh[i] = xn;
        }
      }
    }
    __syncthreads();
    // ---- virtual controls and proportional-integral feedback (dual)
    R rn = 0, ro = 0, rd = 0;
    for (int t = tid; t < PM + 32; t += T) {
      if (t < PM) {
        if (t < nm) {
          const int k = t / NX, i = t - NX * k;
          const R f = vph[t], a = nup[t], b = num[t];
          const R mp = max0(a - alpha * (wep + f));
          const R mm = max0(b - alpha * (wep - f));
          nup[t] = a + rho * (mp - a);
          num[t] = b + rho * (mm - b);
          if (chk) {
            const R op = mup[t], om = mum[t];
            zn = rmax(zn, rmax(mp, mm)); zo = rmax(zo, rmax(op, om));
            zd = rmax(zd, rmax(fabs(mp - op), fabs(mm - om)));
          }
          mup[t] = mp;
          mum[t] = mm;
          const R* a_ = Am + (k * NX + i) * NX;
          const R* d = dx + k * NX;
          R r = wv[t] + ((R(2) * mp - a) - (R(2) * mm - b)) - dx[(k + 1) * NX + i];
          R r2 = 0;
#pragma unroll
          for (int cc = 0; cc < NX; cc += 2) {
            r += a_[cc] * d[cc];
            if (cc + 1 < NX) r2 += a_[cc + 1] * d[cc + 1];
          }
          const R* bm = Bm + (k * NX + i) * NU;
          const R* bp = Bp + (k * NX + i) * NU;
#pragma unroll
          for (int cc = 0; cc < NU; ++cc) { r += bm[cc] * du[k * NU + cc]; r2 += bp[cc] * du[(k + 1) * NU + cc]; }
          r += r2;
          const R pn = f + beta * r;
          vph[t] = f + rb * r;  // = f + rho (pn - f)
          if (chk) {
            const R old = phi[t];
            rn = rmax(rn, fabs(pn)); ro = rmax(ro, fabs(old)); rd = rmax(rd, fabs(pn - old));
          }
          phi[t] = pn;
        }
      } else {
        const int k = t - PM;
        if (k < N - 1) {
          const R hy = dx[(k + 1) * NX + IY] - dx[k * NX + IY] - ep[k];
          const R v = vth[k];
          const R tn = max0(v + beta * hy);
          vth[k] = v + rho * (tn - v);
          if (chk) {
            const R old = th[k];
            rn = rmax(rn, tn); ro = rmax(ro, fabs(old)); rd = rmax(rd, fabs(tn - old));
          }
          th[k] = tn;
        }
      }
    }
    if (chk) {
      R v[6] = {zn, zo, zd, rn, ro, rd};
      block_max_k<R, 6>(v, sm + L.red);
      if (v[2] <= eabs + erel * rmax(v[0], v[1]) && v[5] <= eabs + erel * rmax(v[3], v[4])) break;
    } else {
      __syncthreads();
    }
  }
  __syncthreads();
  return j > jmax ? jmax : j;
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
