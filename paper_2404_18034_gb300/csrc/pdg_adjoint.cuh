// pdg_adjoint.cuh -- gradient of the final SCP iteration's outputs (fuel and
// touchdown error) with respect to the initial state and wet mass.
//
// Definition (the paper has no gradient; this is the one the solver exports):
// let the last SCP iteration J of a solve start from the reference (Xbar,
// Ubar), the PIPG warm start W, the step-size estimate sigma_J and the PIPG
// count n_J.  Consider that iteration as a function of x0, the reference's
// first node moving with x0 (Xbar_1 = x0), everything else of (Xbar, Ubar, W,
// sigma_J, n_J) held: discretize (Sec. 2.3.1), prescale (Sec. 2.3.2), n_J
// iterations of PIPG_custom, update.  The gradient is that of
//     L = dL_dfuel * (m_1 - m_N) + dL_dtouch * 0.5 sum_{E_f} ((x_prop,N - z_f) / P_x)^2
// of the updated trajectory, x_prop,N being the RK4 propagation of its last
// interval.  x0 reaches L (i) through the discretization of the first
// interval (forward mode: dual numbers over the NX - 1 directions of x0 through
// the same model code), (ii) through the final PIPG loop (reverse mode,
// unrolled, recomputed from checkpoints every 50 iterations, projections
// masked as in the forward pass), (iii) directly through x_1 = x0.
#pragma once
#include "pdg_phases.cuh"

namespace pdg {

// ---------------------------------------------------------------------------
// forward-mode dual numbers (value, derivative along one direction)
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  __device__ __forceinline__ Dual() : v(0), d(0) {}
  __device__ __forceinline__ Dual(double a) : v(a), d(0) {}
  __device__ __forceinline__ Dual(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double iv = 1.0 / b.v;
  return Dual(a.v * iv, (a.d - a.v * iv * b.d) * iv);
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
__device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
__device__ __forceinline__ Dual sqrt(Dual a) {
  const double s = ::sqrt(a.v);
  return Dual(s, s > 0.0 ? 0.5 * a.d / s : 0.0);
}

// Scratch of the gradient kernel, appended after the solve layout.
struct AdjLay {
  int ss;                       // size of the PIPG state (xt .. vth)
  int Sb, rb, hb, Gb, Gub, mup_m, mum_m, th_m, u_m, Xo, Uo, xob, uob, cA, cBm, cBp, cw, gacc, td, tang, total;
};

__host__ __device__ inline AdjLay make_adj(const Lay& L, int nu, int threads) {
  AdjLay A;
  const int N = L.N;
  A.ss = L.dx - L.xt;
  int o = L.total;
  A.Sb = o; o += A.ss;
  A.rb = o; o += (N - 1) * NX;
  A.hb = o; o += N;
  A.Gb = o; o += N * NX;
  A.Gub = o; o += N * nu;
  A.mup_m = o; o += (N - 1) * NX;
  A.mum_m = o; o += (N - 1) * NX;
  A.th_m = o; o += N;
  A.u_m = o; o += N;
  A.Xo = o; o += N * NX;
  A.Uo = o; o += N * nu;
  A.xob = o; o += N * NX;
  A.uob = o; o += N * nu;
  A.cA = o; o += NX * NX;
  A.cBm = o; o += NX * nu;
  A.cBp = o; o += NX * nu;
  A.cw = o; o += NX;
  A.gacc = o; o += 16;
  // touchdown reverse: 4 nsub stage inputs (allowing nsub <= 32) + one stage buffer
  A.td = o; o += 4 * 32 * NX + SA_A + NX * nu;
  // tangent discretization: per group a Dual stage buffer and the evaluator's x state
  const int per = NX + 2 * nu + 1;
  const int groups = threads / per;
  A.tang = o; o += groups * 2 * (SA_A + NX * nu + 3 * NX);
  A.total = o;
  return A;
}

// One PIPG_custom iteration on the state (xt .. vth) in shared memory, with no
// stop test, recording the projection masks; with update = false the state is
// left as it was (the intermediates x_hat, u_hat, mu, phi, theta, 2z - z~ are
// written either way).
template <int NU>
__device__ void grad_pipg_iter(const DParams& P, const Lay& L, const AdjLay& A, double* sm, double alpha,
                               double beta, double c1, double rho, bool update) {
  const int N = L.N, T = blockDim.x, tid = threadIdx.x;
  const int nxk = (N - 1) * NX, nuk = N * NU + NX, nm = (N - 1) * NX;
  const int PX = round32(nxk), PU = round32(nuk), PM = round32(nm);
  const double* Am = sm + L.Am;
  const double* Bm = sm + L.Bm;
  const double* Bp = sm + L.Bp;
  double* xt = sm + L.xt;
  double* ut = sm + L.ut;
  double* nup = sm + L.nup;
  double* num = sm + L.num;
  double* vph = sm + L.vph;
  double* vth = sm + L.vth;
  double* dx = sm + L.dx;
  double* du = sm + L.du;
  const double wcost = P.w_cost, wep = P.w_ep;
  for (int t = tid; t < PX + PU; t += T) {
    if (t < PX) {
      if (t < nxk) {
        const int k = t / NX + 1, i = t - NX * (k - 1), o = k * NX + i;
        const double xv = xt[o];
        double G = -vph[(k - 1) * NX + i];
        if (k < N - 1) {
          for (int r = 0; r < NX; ++r) G += Am[(k * NX + r) * NX + i] * vph[k * NX + r];
          if (i == IY) G -= vth[k];
        }
        if (i == IY) G += vth[k - 1];
        if (k == N - 1 && i == IM) G -= wcost;
        double xn = c1 * xv - alpha * G;
        if (k == N - 1 && P.fix_f[i]) xn = sm[L.zf + i];
        dx[o] = 2.0 * xn - xv;
        sm[L.xh + o] = xn;
        if (update) xt[o] = xv + rho * (xn - xv);
      }
    } else {
      const int q = t - PX;
      if (q < N * NU) {
        const int k = q / NU, cc = q - NU * k;
        const double uv = ut[q];
        double G = 0;
        if (k < N - 1)
          for (int r = 0; r < NX; ++r) G += Bm[(k * NX + r) * NU + cc] * vph[k * NX + r];
        if (k > 0)
          for (int r = 0; r < NX; ++r) G += Bp[((k - 1) * NX + r) * NU + cc] * vph[(k - 1) * NX + r];
        double un = c1 * uv - alpha * G;
        double m = 0;
        if (cc == NU - 1) {
          const double lo = sm[L.lo + k], hi = sm[L.hi + k];
          if (un <= lo) { un = lo; m = 1; }
          else if (un >= hi) { un = hi; m = 1; }
          sm[A.u_m + k] = m;
        }
        du[q] = 2.0 * un - uv;
        sm[L.uh + q] = un;
        if (update) ut[q] = uv + rho * (un - uv);
      } else if (q < nuk) {
        const int i = q - N * NU;
        const double xv = xt[i], xn = sm[L.zi + i];
        dx[i] = 2.0 * xn - xv;
        sm[L.xh + i] = xn;
        if (update) xt[i] = xv + rho * (xn - xv);
      }
    }
  }
  __syncthreads();
  for (int t = tid; t < PM + 32; t += T) {
    if (t < PM) {
      if (t < nm) {
        const int k = t / NX, i = t - NX * k;
        const double f = vph[t], a = nup[t], b = num[t];
        const double pa = a - alpha * (wep + f), pb = b - alpha * (wep - f);
        const double mp = pa > 0 ? pa : 0.0, mm = pb > 0 ? pb : 0.0;
        sm[A.mup_m + t] = pa > 0 ? 1.0 : 0.0;
        sm[A.mum_m + t] = pb > 0 ? 1.0 : 0.0;
        double r = sm[L.w + t] + ((2.0 * mp - a) - (2.0 * mm - b)) - dx[(k + 1) * NX + i];
        for (int c = 0; c < NX; ++c) r += Am[(k * NX + i) * NX + c] * dx[k * NX + c];
        for (int c = 0; c < NU; ++c)
          r += Bm[(k * NX + i) * NU + c] * du[k * NU + c] + Bp[(k * NX + i) * NU + c] * du[(k + 1) * NU + c];
        sm[L.mup + t] = mp;
        sm[L.mum + t] = mm;
        sm[L.phi + t] = f + beta * r;
        if (update) {
          nup[t] = a + rho * (mp - a);
          num[t] = b + rho * (mm - b);
          vph[t] = f + rho * beta * r;
        }
      }
    } else {
      const int k = t - PM;
      if (k < N - 1) {
        const double hy = dx[(k + 1) * NX + IY] - dx[k * NX + IY] - sm[L.eps + k];
        const double v = vth[k];
        const double pt = v + beta * hy;
        const double tn = pt > 0 ? pt : 0.0;
        sm[A.th_m + k] = pt > 0 ? 1.0 : 0.0;
        sm[L.th + k] = tn;
        if (update) vth[k] = v + rho * (tn - v);
      }
    }
  }
  __syncthreads();
}

// Reverse of grad_pipg_iter: the state cotangent in A.Sb (laid out like the
// state) goes from iteration j+1 to iteration j; the intermediates of
// iteration j must be in place (grad_pipg_iter with update = false on S_j).
// last: iteration j produced the output (x_hat, u_hat) whose cotangents are in
// A.xob / A.uob.  Threads 0..NX-1 accumulate the cotangents of the first
// interval's blocks hat A^-_1, hat B^-_1, hat B^+_1, hat w_1 in cA/cBm/cBp/cw.
template <int NU>
__device__ void grad_pipg_reverse(const DParams& P, const Lay& L, const AdjLay& A, double* sm, double alpha,
                                  double beta, double c1, double rho, bool last, double* accA, double* accBm,
                                  double* accBp, double& accW) {
  const int N = L.N, T = blockDim.x, tid = threadIdx.x;
  const int nm = (N - 1) * NX, PM = round32(nm);
  const double* Am = sm + L.Am;
  const double* Bm = sm + L.Bm;
  const double* Bp = sm + L.Bp;
  const double* vph = sm + L.vph;
  const double* dx = sm + L.dx;
  const double* du = sm + L.du;
  double* Sb = sm + A.Sb;
  // state cotangent views (same offsets as the state, relative to L.xt)
  double* xtb = Sb;
  double* utb = Sb + (L.ut - L.xt);
  double* nupb = Sb + (L.nup - L.xt);
  double* numb = Sb + (L.num - L.xt);
  double* vphb = Sb + (L.vph - L.xt);
  double* vthb = Sb + (L.vth - L.xt);
  double* rb = sm + A.rb;
  double* hb = sm + A.hb;
  double* Gb = sm + A.Gb;
  double* Gub = sm + A.Gub;
  const double rhob = rho * beta;
  // R1: dual rows and CTCS rows
  for (int t = tid; t < PM + 32; t += T) {
    if (t < PM) {
      if (t < nm) {
        const double r_ = rhob * vphb[t];
        double fb = vphb[t];
        const double mpb = rho * nupb[t] + 2.0 * r_;
        const double mmb = rho * numb[t] - 2.0 * r_;
        double ab = (1.0 - rho) * nupb[t] - r_;
        double bb = (1.0 - rho) * numb[t] + r_;
        if (sm[A.mup_m + t] > 0) { ab += mpb; fb -= alpha * mpb; }
        if (sm[A.mum_m + t] > 0) { bb += mmb; fb += alpha * mmb; }
        nupb[t] = ab;
        numb[t] = bb;
        vphb[t] = fb;
        rb[t] = r_;
        if (t < NX) {  // interval 1: cotangents of its blocks
          for (int c = 0; c < NX; ++c) accA[c] += r_ * dx[c];
          for (int c = 0; c < NU; ++c) { accBm[c] += r_ * du[c]; accBp[c] += r_ * du[NU + c]; }
          accW += r_;
        }
      }
    } else {
      const int k = t - PM;
      if (k < N - 1) {
        const double tb = rho * vthb[k];
        double vb = (1.0 - rho) * vthb[k];
        double h_ = 0;
        if (sm[A.th_m + k] > 0) { vb += tb; h_ = beta * tb; }
        vthb[k] = vb;
        hb[k] = h_;
      }
    }
  }
  __syncthreads();
  // R2: nodes
  const int nx = N * NX, PX = round32(nx), nuu = N * NU;
  for (int t = tid; t < PX + round32(nuu); t += T) {
    if (t < PX) {
      if (t < nx) {
        const int k = t / NX, i = t - NX * k;
        double d = 0;
        if (k < N - 1) {
          for (int r = 0; r < NX; ++r) d += Am[(k * NX + r) * NX + i] * rb[k * NX + r];
          if (i == IY) d -= hb[k];
        }
        if (k > 0) {
          d -= rb[(k - 1) * NX + i];
          if (i == IY) d += hb[k - 1];
        }
        double xhb = 2.0 * d + rho * xtb[t] + (last ? sm[A.xob + t] : 0.0);
        double xb = -d + (1.0 - rho) * xtb[t];
        double g = 0;
        const bool fixed = (k == 0) || (k == N - 1 && P.fix_f[i]);
        if (!fixed) { xb += c1 * xhb; g = -alpha * xhb; }
        xtb[t] = xb;
        Gb[t] = g;
      }
    } else {
      const int q = t - PX;
      if (q < nuu) {
        const int k = q / NU, cc = q - NU * k;
        double d = 0;
        if (k < N - 1)
          for (int r = 0; r < NX; ++r) d += Bm[(k * NX + r) * NU + cc] * rb[k * NX + r];
        if (k > 0)
          for (int r = 0; r < NX; ++r) d += Bp[((k - 1) * NX + r) * NU + cc] * rb[(k - 1) * NX + r];
        double uhb = 2.0 * d + rho * utb[q] + (last ? sm[A.uob + q] : 0.0);
        double ub = -d + (1.0 - rho) * utb[q];
        double g = 0;
        const bool clamped = (cc == NU - 1) && sm[A.u_m + k] > 0;
        if (!clamped) { ub += c1 * uhb; g = -alpha * uhb; }
        utb[q] = ub;
        Gub[q] = g;
      }
    }
  }
  __syncthreads();
  // R3: the extrapolated duals feed the primal gradients
  for (int t = tid; t < PM + 32; t += T) {
    if (t < PM) {
      if (t < nm) {
        const int k = t / NX, i = t - NX * k;
        double fb = vphb[t];
        if (k >= 1)
          for (int c = 0; c < NX; ++c) fb += Am[(k * NX + i) * NX + c] * Gb[k * NX + c];
        fb -= Gb[(k + 1) * NX + i];
        for (int c = 0; c < NU; ++c)
          fb += Bm[(k * NX + i) * NU + c] * Gub[k * NU + c] + Bp[(k * NX + i) * NU + c] * Gub[(k + 1) * NU + c];
        vphb[t] = fb;
        if (t < NX) {
          const double ph = vph[t];
          for (int c = 0; c < NU; ++c) { accBm[c] += ph * Gub[c]; accBp[c] += ph * Gub[NU + c]; }
        }
      }
    } else {
      const int k = t - PM;
      if (k < N - 1) {
        double vb = vthb[k];
        if (k >= 1) vb -= Gb[k * NX + IY];
        vb += Gb[(k + 1) * NX + IY];
        vthb[k] = vb;
      }
    }
  }
  __syncthreads();
}

// Touchdown functional of the updated trajectory (thread 0 only): returns the
// error and adds its cotangents (times g) to xob / uob (through x_hat, u_hat)
// and to gdir (through x_1 = x0, when the last interval is the first).
template <int NU>
__device__ double touchdown_and_reverse(const DParams& P, const Lay& L, const AdjLay& A, double* sm, double g,
                                        double* gdir) {
  const int N = L.N, nsub = P.nsub;
  const double* Xo = sm + A.Xo;
  const double* Uo = sm + A.Uo;
  double* stg = sm + A.td;                    // stage inputs [nsub][4][NX]
  double* buf = sm + A.td + 4 * 32 * NX;     // one stage buffer
  const double h = 1.0 / (double(N - 1) * nsub), h2 = 0.5 * h, h6 = h / 6.0;
  const double* ua = Uo + (N - 2) * NU;
  const double* ub = Uo + (N - 1) * NU;
  double x[NX], s[NX], acc[NX], d[NX], u[NU];
  for (int i = 0; i < NX; ++i) x[i] = Xo[(N - 2) * NX + i];
  for (int n = 0; n < nsub; ++n) {
    for (int i = 0; i < NX; ++i) s[i] = x[i];
    for (int sg = 0; sg < 4; ++sg) {
      const double lp = (double(n) + (sg == 0 ? 0.0 : (sg == 3 ? 1.0 : 0.5))) / double(nsub);
      for (int i = 0; i < NU; ++i) u[i] = (1.0 - lp) * ua[i] + lp * ub[i];
      for (int i = 0; i < NX; ++i) stg[(n * 4 + sg) * NX + i] = s[i];
      model_eval<double, NU>(P, s, u, d, buf, buf + SA_A);
      if (sg == 0) for (int i = 0; i < NX; ++i) { acc[i] = d[i]; s[i] = x[i] + h2 * d[i]; }
      else if (sg == 1) for (int i = 0; i < NX; ++i) { acc[i] += 2.0 * d[i]; s[i] = x[i] + h2 * d[i]; }
      else if (sg == 2) for (int i = 0; i < NX; ++i) { acc[i] += 2.0 * d[i]; s[i] = x[i] + h * d[i]; }
      else for (int i = 0; i < NX; ++i) x[i] += h6 * (acc[i] + d[i]);
    }
  }
  double e = 0, xb[NX], uab[NU], ubb[NU];
  for (int i = 0; i < NX; ++i) {
    xb[i] = 0;
    if (P.fix_f[i]) {
      const double dd = (x[i] - P.z_f[i]) * P.Pxinv[i];
      e += 0.5 * dd * dd;
      xb[i] = g * dd * P.Pxinv[i];
    }
  }
  for (int c = 0; c < NU; ++c) { uab[c] = 0; ubb[c] = 0; }
  // reverse of the RK4 substeps
  for (int n = nsub - 1; n >= 0; --n) {
    double kb[4][NX], sb[NX];
    for (int i = 0; i < NX; ++i) {
      kb[0][i] = h6 * xb[i]; kb[1][i] = 2.0 * h6 * xb[i]; kb[2][i] = 2.0 * h6 * xb[i]; kb[3][i] = h6 * xb[i];
    }
    for (int sg = 3; sg >= 0; --sg) {
      const double lp = (double(n) + (sg == 0 ? 0.0 : (sg == 3 ? 1.0 : 0.5))) / double(nsub);
      for (int i = 0; i < NU; ++i) u[i] = (1.0 - lp) * ua[i] + lp * ub[i];
      double st[NX];
      for (int i = 0; i < NX; ++i) st[i] = stg[(n * 4 + sg) * NX + i];
      model_eval<double, NU>(P, st, u, d, buf, buf + SA_A);
      double uu[NU];
      for (int i = 0; i < NX; ++i) sb[i] = 0;
      for (int c = 0; c < NU; ++c) uu[c] = 0;
      model_vjp<NU>(buf, buf + SA_A, kb[sg], sb, uu);
      for (int c = 0; c < NU; ++c) { uab[c] += (1.0 - lp) * uu[c]; ubb[c] += lp * uu[c]; }
      // stage input s_sg = x + a h k_{sg-1}
      for (int i = 0; i < NX; ++i) xb[i] += sb[i];
      if (sg == 3) for (int i = 0; i < NX; ++i) kb[2][i] += h * sb[i];
      else if (sg == 2) for (int i = 0; i < NX; ++i) kb[1][i] += h2 * sb[i];
      else if (sg == 1) for (int i = 0; i < NX; ++i) kb[0][i] += h2 * sb[i];
    }
  }
  // x_{N-1} = Xbar_{N-1} + P_x x_hat_{N-1}; the first node is x0 itself
  if (N - 2 == 0) {
    for (int i = 0; i < NX - 1; ++i) gdir[i] += xb[i];
  } else {
    for (int i = 0; i < NX; ++i) sm[A.xob + (N - 2) * NX + i] += P.Px[i] * xb[i];
  }
  for (int c = 0; c < NU; ++c) {
    sm[A.uob + (N - 2) * NU + c] += P.Pu[c] * uab[c];
    sm[A.uob + (N - 1) * NU + c] += P.Pu[c] * ubb[c];
  }
  return e;
}

// Forward-mode derivative of the first interval's discretization (A_1,
// B^-_1, B^+_1, x_prop,1) along the NX - 1 directions of Xbar_1 = x0, contracted
// with their cotangents (cA, cBm, cBp in unscaled units, cw for x_prop):
// adds sum cot * d(block)/dx0_j to gacc[j].  Groups of (NX + 2 nu + 1)
// threads each integrate one direction with dual numbers through the same
// model code as the solve.
template <int NU>
__device__ void tangent_first_interval(const DParams& P, const Lay& L, const AdjLay& AL, double* sm) {
  constexpr int NCOL = NX + 2 * NU;
  constexpr int PER = NCOL + 1;
  constexpr int SAD = SA_A + NX * NU + 3 * NX;  // Dual entries per group
  const int N = L.N, nsub = P.nsub;
  const int groups = blockDim.x / PER;
  const int g = threadIdx.x / PER, c = threadIdx.x - g * PER;
  const bool evaluator = c == NCOL;
  const int cu = (!evaluator && c >= NX) ? (c - NX) % NU : -1;
  const bool minus = !evaluator && c >= NX && (c - NX) < NU;
  Dual* st = reinterpret_cast<Dual*>(sm + AL.tang) + (g < groups ? g : 0) * SAD;
  Dual* xP = st + SA_A + NX * NU;
  Dual* xA = xP + NX;
  Dual* xS = xA + NX;
  const double h = 1.0 / (double(N - 1) * nsub), h2 = 0.5 * h, h6 = h / 6.0;
  const double* Ub = sm + L.Ub;
  for (int d0 = 0; d0 < NX - 1; d0 += groups) {
    const int j = d0 + g;
    const bool active = g < groups && j < NX - 1;
    Dual Pv[NX], Sv[NX], Ac[NX];
    if (active) {
      if (evaluator) {
        for (int i = 0; i < NX; ++i) { xP[i] = Dual(sm[L.Xb + i], i == j ? 1.0 : 0.0); xS[i] = xP[i]; }
      } else {
        for (int i = 0; i < NX; ++i) { Pv[i] = Dual(c == i ? 1.0 : 0.0); Sv[i] = Pv[i]; }
      }
    }
    for (int n = 0; n < nsub; ++n) {
      for (int sgi = 0; sgi < 4; ++sgi) {
        const double lp = (double(n) + (sgi == 0 ? 0.0 : (sgi == 3 ? 1.0 : 0.5))) / double(nsub);
        if (active && evaluator) {
          Dual u[NU], x[NX], dd[NX];
          for (int i = 0; i < NU; ++i) u[i] = Dual((1.0 - lp) * Ub[i] + lp * Ub[NU + i]);
          for (int i = 0; i < NX; ++i) x[i] = xS[i];
          model_eval<Dual, NU>(P, x, u, dd, st, st + SA_A);
          if (sgi == 0) for (int i = 0; i < NX; ++i) { xA[i] = dd[i]; xS[i] = xP[i] + Dual(h2) * dd[i]; }
          else if (sgi == 1) for (int i = 0; i < NX; ++i) { xA[i] += Dual(2.0) * dd[i]; xS[i] = xP[i] + Dual(h2) * dd[i]; }
          else if (sgi == 2) for (int i = 0; i < NX; ++i) { xA[i] += Dual(2.0) * dd[i]; xS[i] = xP[i] + Dual(h) * dd[i]; }
          else for (int i = 0; i < NX; ++i) { const Dual v = xP[i] + Dual(h6) * (xA[i] + dd[i]); xP[i] = v; xS[i] = v; }
        }
        __syncthreads();
        if (active && !evaluator) {
          Dual dd[NX];
          const Dual lam = Dual(minus ? (1.0 - lp) : lp);
          model_jvp<Dual, NU>(st, st + SA_A, Sv, cu, lam, dd);
          if (sgi == 0) for (int i = 0; i < NX; ++i) { Ac[i] = dd[i]; Sv[i] = Pv[i] + Dual(h2) * dd[i]; }
          else if (sgi == 1) for (int i = 0; i < NX; ++i) { Ac[i] += Dual(2.0) * dd[i]; Sv[i] = Pv[i] + Dual(h2) * dd[i]; }
          else if (sgi == 2) for (int i = 0; i < NX; ++i) { Ac[i] += Dual(2.0) * dd[i]; Sv[i] = Pv[i] + Dual(h) * dd[i]; }
          else for (int i = 0; i < NX; ++i) { Pv[i] += Dual(h6) * (Ac[i] + dd[i]); Sv[i] = Pv[i]; }
        }
        __syncthreads();
      }
    }
    if (active) {
      double contrib = 0;
      if (evaluator) {
        for (int i = 0; i < NX; ++i) contrib += sm[AL.cw + i] * xP[i].d;
      } else if (c < NX) {
        for (int i = 0; i < NX; ++i) contrib += sm[AL.cA + i * NX + c] * Pv[i].d;
      } else {
        const double* cb = minus ? sm + AL.cBm : sm + AL.cBp;
        for (int i = 0; i < NX; ++i) contrib += cb[i * NU + cu] * Pv[i].d;
      }
      atomicAdd(sm + AL.gacc + j, contrib);
    }
    __syncthreads();
  }
}

}  // namespace pdg
