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
  int sg;                       // size of one iteration's record for the reverse pass
  int Sb, rb, hb, Gb, Gub, mup_m, mum_m, th_m, u_m, Xo, Uo, xob, uob, cA, cBm, cBp, cw, gacc, td, tang, total;
};

// tangent = false: without the tangent discretization's region (the adjoint
// kernel leaves that part to a kernel of its own).
__host__ __device__ inline AdjLay make_adj(const Lay& L, int nu, int threads, bool tangent = true) {
  AdjLay A;
  const int N = L.N;
  A.ss = L.dx - L.xt;
  // relaxed dual before the update, 2z - z~, the mu and theta masks, the box masks
  A.sg = 3 * (N - 1) * NX + N * NX + N * nu + (N - 1) + N;
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
  A.tang = o; o += tangent ? groups * 2 * (SA_A + NX * nu + 3 * NX) : 0;
  A.total = o;
  return A;
}

// What the tangent kernel needs of an instance, written by the adjoint kernel
// (doubles): the first node of the reference, its first two control nodes,
// the unscaled cotangents of hat A^-_1, hat B^-_1, hat B^+_1, hat w_1, and the
// gradient accumulated so far.
__host__ __device__ constexpr int tangent_rec_size(int nu) { return NX + 2 * nu + NX * NX + 2 * NX * nu + NX + 16; }

// One PIPG_custom iteration on the state (xt .. vth) in shared memory, with no
// stop test, recording the projection masks; with update = false the state is
// left as it was (the intermediates x_hat, u_hat, mu, phi, theta, 2z - z~ are
// written either way).  Like the solve's PIPG step it is branch-free where a
// branch would split a warp: on GB300 every FP64 warp instruction costs a slot
// of the FP64 pipe whatever its active lanes.  Blocks that do not exist (the
// last node's A, the first node's B^+, the last node's B^-) are read at a valid
// index and their products discarded by a select; the CTCS terms of the y
// component and the cost term of m_N ride on 0/1-weighted FMAs.
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
  const double acost = alpha * P.w_cost, wep = P.w_ep;
  for (int t = tid; t < PX + PU; t += T) {
    if (t < PX) {
      if (t < nxk) {
        // columns in kStm.col_order, structural zeros skipped (as in phase_pipg)
        const int cr = t / (N - 1);
        const int k = t - cr * (N - 1) + 1, i = kStm.col_order[cr], o = k * NX + i;
        const bool last = k == N - 1;
        const int km = last ? 0 : k;
        const double xv = xt[o];
        const double tdk = vth[k - 1] - (last ? 0.0 : vth[k]);
        const double G0 = fma(i == IY ? 1.0 : 0.0, tdk, -vph[(k - 1) * NX + i]);
        double Gc = G0;
        const double* a = Am + km * STM_SAS;
        const double* f = vph + km * NX;
        const int nj = kStm.col_nnz[kStm.col_order[(t & ~31) / (N - 1)]];
        const unsigned long long lst = kStm.col_list[i], w0 = kStm.col_off[i][0], w1 = kStm.col_off[i][1];
        for (int j = 0; j < nj; ++j) {
          const int r = int(lst >> (4 * j)) & 15;
          Gc = fma(a[stm_off(w0, w1, j)], f[r], Gc);
        }
        const double G = last ? G0 : Gc;
        const double cost = (last && i == IM) ? acost : 0.0;
        double xn = fma(-alpha, G, fma(c1, xv, cost));
        xn = (last && P.fix_f[i]) ? sm[L.zf + i] : xn;
        dx[o] = fma(2.0, xn, -xv);
        sm[L.xh + o] = xn;
        if (update) xt[o] = xv + rho * (xn - xv);
      }
    } else {
      const int q = t - PX;
      if (q < N * NU) {
        const int k = q / NU, cc = q - NU * k;
        const bool hasM = k < N - 1, hasP = k > 0;
        const int km = hasM ? k : 0, kp = hasP ? k - 1 : 0;
        const double uv = ut[q];
        double Gm = 0;
        {
          const double* a = Bm + km * b_stride(NU) + cc;
          const double* f = vph + km * NX;
          for (int r = 0; r < NX; ++r) Gm = fma(a[r * NU], f[r], Gm);
        }
        Gm = hasM ? Gm : 0.0;
        double Gs = Gm;
        {
          const double* a = Bp + kp * b_stride(NU) + cc;
          const double* f = vph + kp * NX;
          for (int r = 0; r < NX; ++r) Gs = fma(a[r * NU], f[r], Gs);
        }
        double un = fma(-alpha, hasP ? Gs : Gm, c1 * uv);
        if (cc == NU - 1) {
          const double lo = sm[L.lo + k], hi = sm[L.hi + k];
          const bool clo = un <= lo, chi = !clo && un >= hi;
          sm[A.u_m + k] = (clo || chi) ? 1.0 : 0.0;
          un = clo ? lo : (chi ? hi : un);
        }
        du[q] = fma(2.0, un, -uv);
        sm[L.uh + q] = un;
        if (update) ut[q] = uv + rho * (un - uv);
      } else if (q < nuk) {
        const int i = q - N * NU;
        const double xv = xt[i], xn = sm[L.zi + i];
        dx[i] = fma(2.0, xn, -xv);
        sm[L.xh + i] = xn;
        if (update) xt[i] = xv + rho * (xn - xv);
      }
    }
  }
  __syncthreads();
  for (int t = tid; t < PM + 32; t += T) {
    if (t < PM) {
      if (t < nm) {
        // rows in kStm.row_order, structural zeros skipped
        const int rr = t / (N - 1);
        const int k = t - rr * (N - 1), i = kStm.row_order[rr], o = k * NX + i;
        const double f = vph[o], a = nup[o], b = num[o];
        const double pa = a - alpha * (wep + f), pb = b - alpha * (wep - f);
        const bool ma = pa > 0, mb = pb > 0;
        const double mp = ma ? pa : 0.0, mm = mb ? pb : 0.0;
        sm[A.mup_m + o] = ma ? 1.0 : 0.0;
        sm[A.mum_m + o] = mb ? 1.0 : 0.0;
        double r = sm[L.w + o] + (fma(2.0, mp, -a) - fma(2.0, mm, -b)) - dx[(k + 1) * NX + i];
        const int nj = kStm.row_nnz[kStm.row_order[(t & ~31) / (N - 1)]];
        const unsigned long long lst = kStm.row_list[i], w0 = kStm.row_off[i][0], w1 = kStm.row_off[i][1];
        for (int j = 0; j < nj; ++j) {
          const int c = int(lst >> (4 * j)) & 15;
          r = fma(Am[k * STM_SAS + stm_off(w0, w1, j)], dx[k * NX + c], r);
        }
        for (int c = 0; c < NU; ++c)
          r = fma(Bp[k * b_stride(NU) + i * NU + c], du[(k + 1) * NU + c],
                  fma(Bm[k * b_stride(NU) + i * NU + c], du[k * NU + c], r));
        sm[L.mup + o] = mp;
        sm[L.mum + o] = mm;
        sm[L.phi + o] = fma(beta, r, f);
        if (update) {
          nup[o] = a + rho * (mp - a);
          num[o] = b + rho * (mm - b);
          vph[o] = f + rho * beta * r;
        }
      }
    } else {
      const int k = t - PM;
      if (k < N - 1) {
        const double hy = dx[(k + 1) * NX + IY] - dx[k * NX + IY] - sm[L.eps + k];
        const double v = vth[k];
        const double pt = fma(beta, hy, v);
        const bool m = pt > 0;
        const double tn = m ? pt : 0.0;
        sm[A.th_m + k] = m ? 1.0 : 0.0;
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
// A.xob / A.uob.  Threads 0..NX-1 (dual rows of the first interval) add the
// cotangents of its blocks hat A^-_1, hat B^-_1, hat B^+_1, hat w_1 to their
// rows of A.cA / A.cBm / A.cBp / A.cw in shared memory (no register carries
// them through the reverse pass).
// Branch-free like grad_pipg_iter: the recorded 0/1 projection masks weight
// FMAs, and blocks that do not exist are read at a valid index and selected
// away.
template <int NU>
__device__ void grad_pipg_reverse(const DParams& P, const Lay& L, const AdjLay& A, double* sm, double alpha,
                                  double beta, double c1, double rho, bool last) {
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
  const double rhob = rho * beta, omr = 1.0 - rho;
  // R1: dual rows and CTCS rows
  for (int t = tid; t < PM + 32; t += T) {
    if (t < PM) {
      if (t < nm) {
        const double r_ = rhob * vphb[t];
        const double m1 = sm[A.mup_m + t], m2 = sm[A.mum_m + t];  // 0 or 1
        const double mpb = fma(rho, nupb[t], 2.0 * r_);
        const double mmb = fma(rho, numb[t], -2.0 * r_);
        nupb[t] = fma(m1, mpb, fma(omr, nupb[t], -r_));
        numb[t] = fma(m2, mmb, fma(omr, numb[t], r_));
        vphb[t] = fma(alpha * m2, mmb, fma(-alpha * m1, mpb, vphb[t]));
        rb[t] = r_;
        if (t < NX) {  // interval 1: cotangents of its blocks (row t)
          for (int c = 0; c < NX; ++c) sm[A.cA + t * NX + c] = fma(r_, dx[c], sm[A.cA + t * NX + c]);
          for (int c = 0; c < NU; ++c) {
            sm[A.cBm + t * NU + c] = fma(r_, du[c], sm[A.cBm + t * NU + c]);
            sm[A.cBp + t * NU + c] = fma(r_, du[NU + c], sm[A.cBp + t * NU + c]);
          }
          sm[A.cw + t] += r_;
        }
      }
    } else {
      const int k = t - PM;
      if (k < N - 1) {
        const double m = sm[A.th_m + k];
        const double tb = rho * vthb[k];
        vthb[k] = fma(m, tb, omr * vthb[k]);
        hb[k] = m * beta * tb;
      }
    }
  }
  __syncthreads();
  // R2: nodes
  const int nx = N * NX, PX = round32(nx), nuu = N * NU;
  for (int t = tid; t < PX + round32(nuu); t += T) {
    if (t < PX) {
      if (t < nx) {
        // columns in kStm.col_order (N nodes each), structural zeros skipped
        const int cr = t / N;
        const int k = t - cr * N, i = kStm.col_order[cr], o = k * NX + i;
        const bool hasA = k < N - 1, hasP = k > 0;
        const int ka = hasA ? k : 0, kp = hasP ? k - 1 : 0;
        double dA = 0;
        const double* a = Am + ka * STM_SAS;
        const double* f = rb + ka * NX;
        const int nj = kStm.col_nnz[kStm.col_order[(t & ~31) / N]];
        const unsigned long long lst = kStm.col_list[i], w0 = kStm.col_off[i][0], w1 = kStm.col_off[i][1];
        for (int j = 0; j < nj; ++j) {
          const int r = int(lst >> (4 * j)) & 15;
          dA = fma(a[stm_off(w0, w1, j)], f[r], dA);
        }
        const double hd = (hasP ? hb[kp] : 0.0) - (hasA ? hb[ka] : 0.0);
        double d = fma(i == IY ? 1.0 : 0.0, hd, hasA ? dA : 0.0);
        d -= hasP ? rb[kp * NX + i] : 0.0;
        const double xhb = fma(2.0, d, fma(rho, xtb[o], last ? sm[A.xob + o] : 0.0));
        const bool fixed = (k == 0) || (k == N - 1 && P.fix_f[i]);
        const double nf = fixed ? 0.0 : 1.0;
        xtb[o] = fma(nf * c1, xhb, fma(omr, xtb[o], -d));
        Gb[o] = (-alpha * nf) * xhb;
      }
    } else {
      const int q = t - PX;
      if (q < nuu) {
        const int k = q / NU, cc = q - NU * k;
        const bool hasM = k < N - 1, hasP = k > 0;
        const int km = hasM ? k : 0, kp = hasP ? k - 1 : 0;
        double dm = 0;
        for (int r = 0; r < NX; ++r) dm = fma(Bm[km * b_stride(NU) + r * NU + cc], rb[km * NX + r], dm);
        dm = hasM ? dm : 0.0;
        double dp = dm;
        for (int r = 0; r < NX; ++r) dp = fma(Bp[kp * b_stride(NU) + r * NU + cc], rb[kp * NX + r], dp);
        const double d = hasP ? dp : dm;
        const double uhb = fma(2.0, d, fma(rho, utb[q], last ? sm[A.uob + q] : 0.0));
        // the mask is 0.0 or 1.0: test its bit pattern, not on the FP64 pipe
        const bool clamped = (cc == NU - 1) && __double_as_longlong(sm[A.u_m + k]) != 0;
        const double nc = clamped ? 0.0 : 1.0;
        utb[q] = fma(nc * c1, uhb, fma(omr, utb[q], -d));
        Gub[q] = (-alpha * nc) * uhb;
      }
    }
  }
  __syncthreads();
  // R3: the extrapolated duals feed the primal gradients
  for (int t = tid; t < PM + 32; t += T) {
    if (t < PM) {
      if (t < nm) {
        // rows in kStm.row_order, structural zeros skipped
        const int rr = t / (N - 1);
        const int k = t - rr * (N - 1), i = kStm.row_order[rr], o = k * NX + i;
        const int kk = k >= 1 ? k : 0;
        double fb = vphb[o];
        double fa = fb;
        const int nj = kStm.row_nnz[kStm.row_order[(t & ~31) / (N - 1)]];
        const unsigned long long lst = kStm.row_list[i], w0 = kStm.row_off[i][0], w1 = kStm.row_off[i][1];
        for (int j = 0; j < nj; ++j) {
          const int c = int(lst >> (4 * j)) & 15;
          fa = fma(Am[kk * STM_SAS + stm_off(w0, w1, j)], Gb[kk * NX + c], fa);
        }
        fb = k >= 1 ? fa : fb;
        fb -= Gb[(k + 1) * NX + i];
        for (int c = 0; c < NU; ++c)
          fb = fma(Bp[k * b_stride(NU) + i * NU + c], Gub[(k + 1) * NU + c],
                   fma(Bm[k * b_stride(NU) + i * NU + c], Gub[k * NU + c], fb));
        vphb[o] = fb;
        if (k == 0) {  // interval 1: cotangents of hat B^-_1, hat B^+_1 (row i)
          const double ph = vph[o];
          for (int c = 0; c < NU; ++c) {
            sm[A.cBm + i * NU + c] = fma(ph, Gub[c], sm[A.cBm + i * NU + c]);
            sm[A.cBp + i * NU + c] = fma(ph, Gub[NU + c], sm[A.cBp + i * NU + c]);
          }
        }
      }
    } else {
      const int k = t - PM;
      if (k < N - 1) vthb[k] = vthb[k] - (k >= 1 ? Gb[k * NX + IY] : 0.0) + Gb[(k + 1) * NX + IY];
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
