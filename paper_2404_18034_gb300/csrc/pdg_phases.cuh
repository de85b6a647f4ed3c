// pdg_phases.cuh -- the phases of one SCP iteration on one instance, executed
// cooperatively by all threads of a CTA on the instance's shared-memory
// image (arXiv 2404.18034, Sec. 2.3 and Sec. 3).  Every phase is called by
// every thread of the CTA (they contain barriers).
#pragma once
#include "pdg_device.cuh"

namespace pdg {

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
// mapping: per interval, one thread per STM column (15 + 2 NU of them, each
// column held in registers) plus one thread integrating x and evaluating the
// compact Jacobians at each RK4 stage.  Intervals are processed in waves of
// L.ipw.  Returns max_k |hat w_k|_inf (the scaled defect) on every thread.
template <typename R, int NU>
__device__ R phase_discretize(const DParams& P, const Lay& L, R* sm) {
  constexpr int NCOL = NX + 2 * NU;
  constexpr int PER = NCOL + 1;
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
  const int my = threadIdx.x / PER;
  const int c = threadIdx.x - my * PER;
  R dmax = 0;
  for (int k0 = 0; k0 < N - 1; k0 += L.ipw) {
    const int k = k0 + my;
    const bool active = my < L.ipw && k < N - 1;
    R* st = sm + L.stage + (my < L.ipw ? my : 0) * L.sa;
    R Pv[NX], Sv[NX], Ac[NX], uk[NU], uk1[NU];
    int cu = -1;
    bool minus = false;
    if (active) {
      if (c == NCOL) {
#pragma unroll
        for (int i = 0; i < NX; ++i) Pv[i] = Xb[k * NX + i];
#pragma unroll
        for (int i = 0; i < NU; ++i) { uk[i] = Ub[k * NU + i]; uk1[i] = Ub[(k + 1) * NU + i]; }
      } else {
#pragma unroll
        for (int i = 0; i < NX; ++i) Pv[i] = (c == i) ? R(1) : R(0);
        if (c >= NX) {
          cu = (c - NX) % NU;
          minus = (c - NX) < NU;
        }
      }
#pragma unroll
      for (int i = 0; i < NX; ++i) Sv[i] = Pv[i];
    }
    for (int n = 0; n < nsub; ++n) {
#pragma unroll 1
      for (int sgi = 0; sgi < 4; ++sgi) {
        const R lp = (R(n) + (sgi == 0 ? R(0) : (sgi == 3 ? R(1) : R(0.5)))) / R(nsub);
        R d[NX];
        if (active && c == NCOL) {
          R u[NU];
#pragma unroll
          for (int i = 0; i < NU; ++i) u[i] = (R(1) - lp) * uk[i] + lp * uk1[i];
          model_eval<R, NU>(P, Sv, u, d, st, st + SA_A);
        }
        __syncthreads();
        if (active && c < NCOL) {
          const R lam = minus ? (R(1) - lp) : lp;
          model_jvp<R, NU>(st, st + SA_A, Sv, cu, lam, d);
        }
        if (active) {
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
      if (c == NCOL) {
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          const R wi = (Pv[i] - Xb[(k + 1) * NX + i]) * R(P.Pxinv[i]);
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
// vph/vth.  Returns the buffered sigma; *iters the iterations run.
template <typename R, int NU>
__device__ R phase_power(const DParams& P, const Lay& L, R* sm, int force, int* iters) {
  const int N = L.N, T = blockDim.x, tid = threadIdx.x;
  const int nx = N * NX, nuu = N * NU, nm = (N - 1) * NX;
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
    for (int t = tid; t < nm + (N - 1); t += T) {
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
      } else {
        const int k = t - nm;
        pt[k] = (px[(k + 1) * NX + IY] - px[k * NX + IY]) * isig;
      }
    }
    __syncthreads();
    // z = K^T (phi, theta)
    R s2 = 0;
    for (int t = tid; t < nx + nuu + nm; t += T) {
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
      } else if (t < nx + nuu) {
        const int q = t - nx, k = q / NU, cc = q - NU * k;
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
      } else {
        const int q = t - nx - nuu;
        const R f = ph[q];
        pp[q] = f;
        pn[q] = -f;
        s2 += R(2) * f * f;
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
// and j (the warm start being iterate 0).  Returns the iterations run.
template <typename R, int NU>
__device__ int phase_pipg(const DParams& P, const Lay& L, R* sm, R sigma, int force) {
  const int N = L.N, T = blockDim.x, tid = threadIdx.x;
  const int nx = N * NX, nuu = N * NU, nm = (N - 1) * NX;
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
  R* dmu = sm + L.dmu;
  for (int t = tid; t < nx + nuu + 2 * nm + (N - 1); t += T) {
    if (t < nx) xt[t] = xh[t];
    else if (t < nx + nuu) ut[t - nx] = uh[t - nx];
    else if (t < nx + nuu + nm) { const int q = t - nx - nuu; nup[q] = mup[q]; num[q] = mum[q]; }
    else if (t < nx + nuu + 2 * nm) { const int q = t - nx - nuu - nm; vph[q] = phi[q]; }
    else { const int q = t - nx - nuu - 2 * nm; vth[q] = th[q]; }
  }
  __syncthreads();
  const R wp = R(P.w_prox);
  const R alpha = R(2) / (wp + sqrt(wp * wp + R(4) * R(P.omega) * sigma));
  const R beta = R(P.omega) * alpha;
  const R c1 = R(1) - alpha * wp;
  const R rho = R(P.rho);
  const R wcost = R(P.w_cost), wep = R(P.w_ep);
  const R eabs = R(P.eps_abs), erel = R(P.eps_rel);
  const int jmax = force > 0 ? force : P.pipg_jmax;
  const int jcheck = P.pipg_jcheck;
  int j;
  for (j = 1; j <= jmax; ++j) {
    const bool chk = force <= 0 && jcheck > 0 && (j % jcheck) == 0;
    R zn = 0, zo = 0, zd = 0;
    // ---- projected gradient step (primal)
    for (int t = tid; t < nx + nuu + nm; t += T) {
      if (t < nx) {
        const int k = t / NX, i = t - NX * k;
        const R xv = xt[t];
        R xn;
        if (k == 0) {
          xn = zi[i];
        } else {
          R G = -vph[(k - 1) * NX + i];
          if (k < N - 1) {
            const R* a = Am + k * NX * NX + i;
            const R* f = vph + k * NX;
#pragma unroll
            for (int r = 0; r < NX; ++r) G += a[r * NX] * f[r];
            if (i == IY) G -= vth[k];
          }
          if (i == IY) G += vth[k - 1];
          if (k == N - 1 && i == IM) G -= wcost;  // e_cost = -e_m (maximize m_N)
          xn = c1 * xv - alpha * G;
          if (k == N - 1 && P.fix_f[i]) xn = zf[i];
        }
        dx[t] = R(2) * xn - xv;
        xt[t] = xv + rho * (xn - xv);
        if (chk) {
          const R o = xh[t];
          zn = rmax(zn, fabs(xn)); zo = rmax(zo, fabs(o)); zd = rmax(zd, fabs(xn - o));
        }
        xh[t] = xn;
      } else if (t < nx + nuu) {
        const int q = t - nx, k = q / NU, cc = q - NU * k;
        const R uv = ut[q];
        R G = 0;
        if (k < N - 1) {
          const R* a = Bm + k * NX * NU + cc;
          const R* f = vph + k * NX;
#pragma unroll
          for (int r = 0; r < NX; ++r) G += a[r * NU] * f[r];
        }
        if (k > 0) {
          const R* a = Bp + (k - 1) * NX * NU + cc;
          const R* f = vph + (k - 1) * NX;
#pragma unroll
          for (int r = 0; r < NX; ++r) G += a[r * NU] * f[r];
        }
        R un = c1 * uv - alpha * G;
        if (cc == NU - 1) un = rmin(rmax(un, lo[k]), hi[k]);
        du[q] = R(2) * un - uv;
        ut[q] = uv + rho * (un - uv);
        if (chk) {
          const R o = uh[q];
          zn = rmax(zn, fabs(un)); zo = rmax(zo, fabs(o)); zd = rmax(zd, fabs(un - o));
        }
        uh[q] = un;
      } else {
        const int q = t - nx - nuu;
        const R f = vph[q], a = nup[q], b = num[q];
        const R mp = rmax(R(0), a - alpha * (wep + f));
        const R mm = rmax(R(0), b - alpha * (wep - f));
        dmu[q] = (R(2) * mp - a) - (R(2) * mm - b);
        nup[q] = a + rho * (mp - a);
        num[q] = b + rho * (mm - b);
        if (chk) {
          const R op = mup[q], om = mum[q];
          zn = rmax(zn, rmax(mp, mm)); zo = rmax(zo, rmax(op, om));
          zd = rmax(zd, rmax(fabs(mp - op), fabs(mm - om)));
        }
        mup[q] = mp;
        mum[q] = mm;
      }
    }
    __syncthreads();
    // ---- proportional-integral feedback (dual)
    R rn = 0, ro = 0, rd = 0;
    for (int t = tid; t < nm + (N - 1); t += T) {
      if (t < nm) {
        const int k = t / NX, i = t - NX * k;
        const R* a = Am + (k * NX + i) * NX;
        const R* d = dx + k * NX;
        R r = wv[t] + dmu[t] - dx[(k + 1) * NX + i];
#pragma unroll
        for (int cc = 0; cc < NX; ++cc) r += a[cc] * d[cc];
        const R* bm = Bm + (k * NX + i) * NU;
        const R* bp = Bp + (k * NX + i) * NU;
#pragma unroll
        for (int cc = 0; cc < NU; ++cc) r += bm[cc] * du[k * NU + cc] + bp[cc] * du[(k + 1) * NU + cc];
        const R v = vph[t];
        const R pn = v + beta * r;
        vph[t] = v + rho * (pn - v);
        if (chk) {
          const R o = phi[t];
          rn = rmax(rn, fabs(pn)); ro = rmax(ro, fabs(o)); rd = rmax(rd, fabs(pn - o));
        }
        phi[t] = pn;
      } else {
        const int k = t - nm;
        const R hy = dx[(k + 1) * NX + IY] - dx[k * NX + IY] - ep[k];
        const R v = vth[k];
        const R tn = rmax(R(0), v + beta * hy);
        vth[k] = v + rho * (tn - v);
        if (chk) {
          const R o = th[k];
          rn = rmax(rn, tn); ro = rmax(ro, fabs(o)); rd = rmax(rd, fabs(tn - o));
        }
        th[k] = tn;
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
