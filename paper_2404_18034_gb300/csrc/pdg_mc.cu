// pdg_mc.cu -- kernels and C ABI of the batched GB300 solver for Monte Carlo
// powered-descent guidance (arXiv 2404.18034).  See include/pdg_mc.h.  The
// model (6-DoF of Sec. 4, or 3-DoF with PDG_MODEL_3DOF) is fixed at compile
// time by pdg_device.cuh; nothing in this file depends on which.
//
// Two execution forms share the device phases of pdg_phases.cuh:
//  * persistent: one launch; each CTA takes instance ids from a global work
//    queue (atomicAdd), runs the whole SCP solve with every block of the
//    instance in shared memory, writes the result and takes the next id, so
//    instances of uneven size and iteration count retire and refill freely;
//  * plain: one launch per phase (discretize+scale, power iteration, PIPG,
//    update) per SCP iteration, the per-instance image kept in global memory
//    between launches; the four launches of an SCP iteration are captured
//    once in a CUDA graph and replayed until every instance is done.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pdg_mc.h"
#include "pdg_adjoint.cuh"

using namespace pdg;

// CTAs per SM the FP32 solve kernels are compiled for (register cap)
#ifndef PDG_FP32_MIN_BLOCKS
#define PDG_FP32_MIN_BLOCKS 3
#endif
// ... and the plain-form discretization kernel (its STM columns and model
// evaluation want more registers than the other per-phase kernels)
#ifndef PDG_FP32_DISC_MIN_BLOCKS
#define PDG_FP32_DISC_MIN_BLOCKS 2
#endif

// PIPG forms: 1 = blocks in shared memory (phase_pipg), 2 = blocks and
// iterates in registers (phase_pipg_reg), 3 = blocks in register tiles over
// lane groups (phase_pipg_ks).  The register form runs one thread per dual
// row plus the control lanes, so its kernels are built for up to
// PDG_REG_MAXT threads (FP32) or 512 (FP64).  Form 3 is built for up to 512
// threads and one CTA per SM, so its FP32 kernels may take 128 registers: four
// CTAs per SM at N <= 16 (128 threads).
#define PDG_REG_MAXT_F32 576
// FP64 solve kernels: compiled for up to PDG_FP64_MAXT threads with at least
// PDG_FP64_MINB CTAs per SM (the register budget is 65536 / (threads x CTAs))
#ifndef PDG_FP64_MAXT
#define PDG_FP64_MAXT 512
#endif
#ifndef PDG_FP64_MINB
#define PDG_FP64_MINB 1
#endif
// The persistent kernel of form 3 (FP32) is built for at most
// PDG_KS_PERS_MAXT threads (N <= 32 needs 256) and so takes up to 65536 /
// PDG_KS_PERS_MAXT registers.  At 512 (128 registers) its PIPG loop reloads
// some of its tiles from local memory; at 384 (168 registers) it does not,
// but N = 15 then fits three CTAs per SM instead of four and N = 30 one
// instead of two: 25 677 against 25 374 solves/s at N = 15, 7461 against
// 10 553 on the uneven batch, so 512 is the build.
// PDG_KS_DISC_INLINE=1 inlines the discretization into that kernel instead
// of calling it (the call costs the PIPG loop registers, the inlined body
// spills in turn; measured slower with the pipelined discretization).
#ifndef PDG_KS_DISC_INLINE
#define PDG_KS_DISC_INLINE 0
#endif
#ifndef PDG_KS_PERS_MAXT
#define PDG_KS_PERS_MAXT 512
#endif
#define PDG_LB_PERS(R, PV)                                                                  \
  __launch_bounds__((PV) == 3 && sizeof(R) == 4 ? PDG_KS_PERS_MAXT                            \
                    : ((PV) == 2 && sizeof(R) == 4 ? PDG_REG_MAXT_F32 : (sizeof(R) == 8 ? PDG_FP64_MAXT : 512)), \
                    sizeof(R) == 8 ? PDG_FP64_MINB : ((PV) == 1 ? PDG_FP32_MIN_BLOCKS : 1))
#define PDG_LB(R, PV)                                                                       \
  __launch_bounds__((PV) == 2 && sizeof(R) == 4 ? PDG_REG_MAXT_F32 : (sizeof(R) == 8 ? PDG_FP64_MAXT : 512), \
                    sizeof(R) == 8 ? PDG_FP64_MINB : ((PV) == 1 ? PDG_FP32_MIN_BLOCKS : 1))

namespace {

template <typename R, int NU, int PV, bool CK = false>
__device__ __forceinline__ int run_pipg(const DParams& P, const Lay& L, R* sm, R sigma, int force,
                                        double* ck = nullptr) {
  if constexpr (PV == 2) return phase_pipg_reg<R, NU>(P, L, sm, sigma, force);
  else if constexpr (PV == 3) return phase_pipg_ks<R, NU>(P, L, sm, sigma, force);
  else return phase_pipg<R, NU, CK>(P, L, sm, sigma, force, ck);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename R>
__device__ __forceinline__ void copy_g2s(R* dst, const R* src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
template <typename R>
__device__ __forceinline__ void copy_s2g(R* dst, const R* src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Load x0 of instance b into the image (x0[NX-1], y = 0); returns false when it
// is not finite.  Every thread returns the same value.
template <typename R>
__device__ bool load_x0(const Lay& L, R* sm, const double* __restrict__ x0, int b) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  if (threadIdx.x < 16) {
    double v = threadIdx.x < NX - 1 ? x0[(size_t)b * (NX - 1) + threadIdx.x] : 0.0;
    if (!isfinite(v)) atomicOr(&bad, 1);
    sm[L.x0 + threadIdx.x] = R(v);
  }
  __syncthreads();
  const bool ok = bad == 0;
  __syncthreads();
  return ok;
}

template <typename R, int NU>
__device__ void write_outputs(const Lay& L, const R* sm, int b, int Nmax, int status, int scp, long long pipg,
                              double* X, double* U, double* tf, double* fuel, int* st, int* sit, long long* pit) {
  const int N = L.N;
  double* Xo = X + (size_t)b * Nmax * NX;
  double* Uo = U + (size_t)b * Nmax * NU;
  const bool ok = status != PDG_BAD_INPUT;
  for (int t = threadIdx.x; t < Nmax * NX; t += blockDim.x) Xo[t] = (ok && t < N * NX) ? double(sm[L.Xb + t]) : 0.0;
  for (int t = threadIdx.x; t < Nmax * NU; t += blockDim.x) Uo[t] = (ok && t < N * NU) ? double(sm[L.Ub + t]) : 0.0;
  if (threadIdx.x == 0) {
    double t_f = 0.0, fu = 0.0;
    if (ok) {
      for (int k = 0; k < N - 1; ++k)
        t_f += 0.5 * (double(sm[L.Ub + k * NU + NU - 1]) + double(sm[L.Ub + (k + 1) * NU + NU - 1])) / double(N - 1);
      fu = double(sm[L.Xb + IM]) - double(sm[L.Xb + (N - 1) * NX + IM]);
    }
    tf[b] = t_f;
    fuel[b] = fu;
    st[b] = status;
    sit[b] = scp;
    pit[b] = pipg;
  }
}

// ---------------------------------------------------------------------------
// persistent form
// ---------------------------------------------------------------------------
// CK: the gradient solve's instantiation (FP64, PIPG form 1, rec set): each
// SCP iteration also records the PIPG state every 50 iterations and the
// final x_hat, u_hat in the instance's record, so that the adjoint does not
// rerun the last PIPG loop forward.  Record of an instance (offsets for its N):
// X_bar, U_bar | warm start | sigma, PIPG count | x_hat, u_hat | checkpoints.
template <typename R, int NU, int PV, bool CK = false>
__global__ void PDG_LB_PERS(R, PV)
k_persistent(const DParams P, int B, int Nmax, const double* __restrict__ x0, const int* __restrict__ Ns,
             double* X, double* U, double* tf, double* fuel, int* status, int* scp_iters, long long* pipg_iters,
             int* trace, int* queue, double* rec, int rec_stride, const int* perm, const int* class_off, int cls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  __shared__ int inst;
  // Per-instance layout and scalars live in shared memory and are re-read
  // after the phases (which end in barriers), so that no register is held
  // across the PIPG loop: it gets the whole register budget.
  __shared__ Lay Ls;
  __shared__ struct {
    unsigned long long t_start;
    long long ptot;
    double defect, sigma;
    int b, pit, over;
  } C;
  // shape-class launch: this grid serves the instances perm[class_off[cls] ..
  // class_off[cls + 1]) (all of one node count)
  const int nq = perm ? class_off[cls + 1] - class_off[cls] : B;
  for (;;) {
    if (threadIdx.x == 0) inst = atomicAdd(queue, 1);
    __syncthreads();
    const int qi = inst;
    __syncthreads();
    if (qi >= nq) break;
    const int b = perm ? perm[class_off[cls] + qi] : qi;
    const int N = Ns ? Ns[b] : Nmax;
    if (N < 2 || N > Nmax) {
      Lay L0 = make_lay(2, NU, blockDim.x);
      write_outputs<R, NU>(L0, sm, b, Nmax, PDG_BAD_INPUT, 0, 0, X, U, tf, fuel, status, scp_iters, pipg_iters);
      __syncthreads();
      continue;
    }
    // the layout lives in shared memory: read field by field after each
    // barrier instead of occupying registers across the phases
    if (threadIdx.x == 0) Ls = make_lay(N, NU, blockDim.x);
    __syncthreads();
    const Lay& L = Ls;
    if (!load_x0<R>(L, sm, x0, b)) {
      write_outputs<R, NU>(L, sm, b, Nmax, PDG_BAD_INPUT, 0, 0, X, U, tf, fuel, status, scp_iters, pipg_iters);
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) { C.b = b; C.t_start = globaltimer_ns(); C.ptot = 0; }
    phase_init_guess<R, NU>(P, L, sm);
    for (int t = threadIdx.x; t < L.img - L.xh; t += blockDim.x) sm[L.xh + t] = R(0);
    __syncthreads();
    int stat = PDG_MAX_SCP, j;
    for (j = 1; j <= P.scp_jmax; ++j) {
      if (P.budget_ns > 0.0 || P.abort_flag) {
        // one clock reading and one read of the abort word decide for the
        // whole CTA: threads that read either on both sides of a change would
        // part at the next barrier
        if (threadIdx.x == 0) {
          int over = 0;
          if (P.budget_ns > 0.0 && double(globaltimer_ns() - C.t_start) > P.budget_ns) over = PDG_BUDGET;
          if (abort_requested(P)) over = PDG_ABORTED;
          C.over = over;
        }
        __syncthreads();
        if (C.over) { stat = C.over; --j; break; }
      }
      if (rec) {  // reference and warm start of this SCP iteration (the last one is kept)
        double* rc = rec + (size_t)C.b * rec_stride;
        const int n = L.N, ow = n * (NX + NU), nw = L.img - L.xh;
        for (int t = threadIdx.x; t < n * NX; t += blockDim.x) rc[t] = double(sm[L.Xb + t]);
        for (int t = threadIdx.x; t < n * NU; t += blockDim.x) rc[n * NX + t] = double(sm[L.Ub + t]);
        for (int t = threadIdx.x; t < nw; t += blockDim.x) rc[ow + t] = double(sm[L.xh + t]);
      }
      {
        R defect;
        if constexpr (PV == 3 && PDG_KS_DISC_INLINE) defect = discretize_body<R, NU>(P, L, sm);
        else defect = phase_discretize<R, NU>(P, L, sm);
        if (threadIdx.x == 0) C.defect = double(defect);
      }
      phase_scale_extra<R, NU>(P, L, sm);
      __syncthreads();
      int jit;
      {
        int pit;
        const R sigma = phase_power<R, NU>(P, L, sm, 0, &pit);
        if (threadIdx.x == 0) { C.sigma = double(sigma); C.pit = pit; }
        if constexpr (CK) {
          const int ow = L.N * (NX + NU), nw = L.img - L.xh;
          double* ckp = rec + (size_t)C.b * rec_stride + ow + nw + 2 + ow;
          jit = run_pipg<R, NU, PV, true>(P, L, sm, sigma, 0, ckp);
          double* rf = rec + (size_t)C.b * rec_stride + ow + nw + 2;
          for (int t = threadIdx.x; t < ow; t += blockDim.x)
            rf[t] = double(t < L.N * NX ? sm[L.xh + t] : sm[L.uh + t - L.N * NX]);
        } else {
          jit = run_pipg<R, NU, PV>(P, L, sm, sigma, 0);
        }
      }
      const int bb = C.b;
      if (rec && threadIdx.x == 0) {
        const int ow = L.N * (NX + NU), nw = L.img - L.xh;
        double* rc = rec + (size_t)bb * rec_stride;
        rc[ow + nw] = C.sigma;
        rc[ow + nw + 1] = double(jit);
      }
      bool bad;
      const R step = phase_update<R, NU>(P, L, sm, &bad);
      if (threadIdx.x == 0) {
        C.ptot += jit;
        if (trace) {
          trace[((size_t)bb * P.scp_jmax + (j - 1)) * 2 + 0] = C.pit;
          trace[((size_t)bb * P.scp_jmax + (j - 1)) * 2 + 1] = jit;
        }
      }
      if (bad) { stat = PDG_NONFINITE; break; }
      const int n = L.N;
      const R dy = sm[L.Xb + (n - 1) * NX + IY] - sm[L.Xb + IY];
      if (step <= R(P.scp_eps_step) && R(C.defect) <= R(P.scp_eps_defect) && dy <= R(n - 1) * R(P.eps_ctcs)) {
        stat = PDG_CONVERGED;
        break;
      }
    }
    if (j > P.scp_jmax) j = P.scp_jmax;
    __syncthreads();  // C.ptot written by thread 0 above
    const int bb = C.b;
    if (trace) {
      for (int t = threadIdx.x + 2 * j; t < 2 * P.scp_jmax; t += blockDim.x) trace[(size_t)bb * P.scp_jmax * 2 + t] = 0;
    }
    write_outputs<R, NU>(L, sm, bb, Nmax, stat, j, C.ptot, X, U, tf, fuel, status, scp_iters, pipg_iters);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// plain form: per-instance image in global memory between launches
// ---------------------------------------------------------------------------
// The abort request, read once per CTA and broadcast (every thread of the CTA
// returns the same answer).
__device__ bool plain_aborted(const DParams& P) {
  if (!P.abort_flag) return false;
  __shared__ int ab;
  if (threadIdx.x == 0) ab = abort_requested(P);
  __syncthreads();
  const bool r = ab != 0;
  __syncthreads();
  return r;
}

struct PlainWs {
  void* img;           // [B][istride] of R
  int istride;         // elements of R per instance
  int* st;             // [B] running / final status
  int* sit;            // [B] SCP iterations done
  long long* lit;      // [B] PIPG iterations summed
  int* pow_it;         // [B] last power iterations
  int* pipg_it;        // [B] last PIPG iterations
  int* done;           // [1] instances finished
};

template <typename R, int NU>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? PDG_FP32_MIN_BLOCKS : 1)
k_plain_init(const DParams P, int B, int Nmax, const double* __restrict__ x0, const int* __restrict__ Ns, PlainWs W,
             double* X, double* U, double* tf, double* fuel, int* status, int* scp_iters, long long* pipg_iters) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  const int b = blockIdx.x;
  const int N = Ns ? Ns[b] : Nmax;
  R* img = reinterpret_cast<R*>(W.img) + (size_t)b * W.istride;
  if (threadIdx.x == 0) { W.sit[b] = 0; W.lit[b] = 0; }
  if (N < 2 || N > Nmax) {
    Lay L0 = make_lay(2, NU, blockDim.x);
    if (threadIdx.x == 0) { W.st[b] = PDG_BAD_INPUT; atomicAdd(W.done, 1); }
    write_outputs<R, NU>(L0, sm, b, Nmax, PDG_BAD_INPUT, 0, 0, X, U, tf, fuel, status, scp_iters, pipg_iters);
    return;
  }
  const Lay L = make_lay(N, NU, blockDim.x);
  if (!load_x0<R>(L, sm, x0, b)) {
    if (threadIdx.x == 0) { W.st[b] = PDG_BAD_INPUT; atomicAdd(W.done, 1); }
    write_outputs<R, NU>(L, sm, b, Nmax, PDG_BAD_INPUT, 0, 0, X, U, tf, fuel, status, scp_iters, pipg_iters);
    return;
  }
  phase_init_guess<R, NU>(P, L, sm);
  for (int t = threadIdx.x; t < L.img - L.xh; t += blockDim.x) sm[L.xh + t] = R(0);
  __syncthreads();
  copy_s2g(img, sm, L.img);
  if (threadIdx.x == 0) W.st[b] = ST_RUNNING;
}

template <typename R, int NU>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? PDG_FP32_DISC_MIN_BLOCKS : 1)
k_plain_disc(const DParams P, int B, int Nmax, const int* __restrict__ Ns, PlainWs W) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  const int b = blockIdx.x;
  if (W.st[b] != ST_RUNNING) return;
  if (plain_aborted(P)) return;  // k_plain_update ends the instance
  const int N = Ns ? Ns[b] : Nmax;
  const Lay L = make_lay(N, NU, blockDim.x);
  R* img = reinterpret_cast<R*>(W.img) + (size_t)b * W.istride;
  copy_g2s(sm + L.x0, img + L.x0, L.Am - L.x0);  // x0, Xb, Ub
  __syncthreads();
  const R defect = phase_discretize<R, NU>(P, L, sm);
  phase_scale_extra<R, NU>(P, L, sm);
  __syncthreads();
  copy_s2g(img + L.Am, sm + L.Am, L.xh - L.Am);  // Am .. zf
  if (threadIdx.x == 0) img[L.sc + 1] = defect;
}

template <typename R, int NU>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? PDG_FP32_MIN_BLOCKS : 1)
k_plain_power(const DParams P, int B, int Nmax, const int* __restrict__ Ns, PlainWs W, const int* force) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  const int b = blockIdx.x;
  if (W.st[b] != ST_RUNNING) return;
  if (plain_aborted(P)) return;  // k_plain_update ends the instance
  const int N = Ns ? Ns[b] : Nmax;
  const Lay L = make_lay(N, NU, blockDim.x);
  R* img = reinterpret_cast<R*>(W.img) + (size_t)b * W.istride;
  copy_g2s(sm + L.Am, img + L.Am, L.w - L.Am);        // Am, Bm, Bp
  copy_g2s(sm + L.xh, img + L.xh, L.phi - L.xh);      // xh, uh, mup, mum
  __syncthreads();
  int it;
  const R sigma = phase_power<R, NU>(P, L, sm, force ? force[2 * b] : 0, &it);
  if (threadIdx.x == 0) { img[L.sc + 0] = sigma; W.pow_it[b] = it; }
}

template <typename R, int NU, int PV>
__global__ void PDG_LB(R, PV)
k_plain_pipg(const DParams P, int B, int Nmax, const int* __restrict__ Ns, PlainWs W, const int* force) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  const int b = blockIdx.x;
  if (W.st[b] != ST_RUNNING) return;
  if (plain_aborted(P)) return;  // k_plain_update ends the instance
  const int N = Ns ? Ns[b] : Nmax;
  const Lay L = make_lay(N, NU, blockDim.x);
  R* img = reinterpret_cast<R*>(W.img) + (size_t)b * W.istride;
  copy_g2s(sm + L.Am, img + L.Am, L.img - L.Am);     // subproblem + warm start
  __syncthreads();
  const R sigma = img[L.sc + 0];
  const int it = run_pipg<R, NU, PV>(P, L, sm, sigma, force ? force[2 * b + 1] : 0);
  copy_s2g(img + L.xh, sm + L.xh, L.img - L.xh);
  if (threadIdx.x == 0) W.pipg_it[b] = it;
}

// step_only: the one-iteration API (no status, no outputs).  An abort
// request ends a running instance here, before its step is applied: its
// outputs are the reference after the SCP iterations it completed.
template <typename R, int NU>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? PDG_FP32_MIN_BLOCKS : 1)
k_plain_update(const DParams P, int B, int Nmax, const int* __restrict__ Ns, PlainWs W, int step_only,
               double* X, double* U, double* tf, double* fuel, int* status, int* scp_iters, long long* pipg_iters,
               int* trace, double* step_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  const int b = blockIdx.x;
  if (W.st[b] != ST_RUNNING) return;
  const int N = Ns ? Ns[b] : Nmax;
  const Lay L = make_lay(N, NU, blockDim.x);
  R* img = reinterpret_cast<R*>(W.img) + (size_t)b * W.istride;
  copy_g2s(sm + L.Xb, img + L.Xb, L.Am - L.Xb);      // Xb, Ub
  copy_g2s(sm + L.xh, img + L.xh, L.mup - L.xh);     // xh, uh
  __syncthreads();
  if (!step_only && plain_aborted(P)) {
    const int j = W.sit[b];
    if (trace) {
      for (int t = threadIdx.x + 2 * j; t < 2 * P.scp_jmax; t += blockDim.x) trace[(size_t)b * P.scp_jmax * 2 + t] = 0;
    }
    write_outputs<R, NU>(L, sm, b, Nmax, PDG_ABORTED, j, W.lit[b], X, U, tf, fuel, status, scp_iters, pipg_iters);
    if (threadIdx.x == 0) { W.st[b] = PDG_ABORTED; atomicAdd(W.done, 1); }
    return;
  }
  bool bad;
  const R step = phase_update<R, NU>(P, L, sm, &bad);
  copy_s2g(img + L.Xb, sm + L.Xb, L.Am - L.Xb);
  if (step_only) {
    if (threadIdx.x == 0) step_out[b] = double(step);
    return;
  }
  const int j = W.sit[b] + 1;
  const long long ptot = W.lit[b] + W.pipg_it[b];
  if (trace && threadIdx.x == 0) {
    trace[((size_t)b * P.scp_jmax + (j - 1)) * 2 + 0] = W.pow_it[b];
    trace[((size_t)b * P.scp_jmax + (j - 1)) * 2 + 1] = W.pipg_it[b];
  }
  const R defect = img[L.sc + 1];
  const R dy = sm[L.Xb + (N - 1) * NX + IY] - sm[L.Xb + IY];
  int stat = ST_RUNNING;
  if (bad) stat = PDG_NONFINITE;
  else if (step <= R(P.scp_eps_step) && defect <= R(P.scp_eps_defect) && dy <= R(N - 1) * R(P.eps_ctcs)) stat = PDG_CONVERGED;
  else if (j >= P.scp_jmax) stat = PDG_MAX_SCP;
  __syncthreads();
  if (threadIdx.x == 0) { W.sit[b] = j; W.lit[b] = ptot; }
  if (stat != ST_RUNNING) {
    if (trace) {
      for (int t = threadIdx.x + 2 * j; t < 2 * P.scp_jmax; t += blockDim.x) trace[(size_t)b * P.scp_jmax * 2 + t] = 0;
    }
    write_outputs<R, NU>(L, sm, b, Nmax, stat, j, ptot, X, U, tf, fuel, status, scp_iters, pipg_iters);
    if (threadIdx.x == 0) { W.st[b] = stat; atomicAdd(W.done, 1); }
  }
}

// ---------------------------------------------------------------------------
// API helpers: subproblem data and one-iteration packing
// ---------------------------------------------------------------------------
template <typename R, int NU>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? PDG_FP32_MIN_BLOCKS : 1)
k_subproblem(const DParams P, int B, int Nmax, const double* __restrict__ x0, const int* __restrict__ Ns,
             const double* __restrict__ X, const double* __restrict__ U, double* Am, double* Bm, double* Bp, double* w) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  const int b = blockIdx.x;
  const int N = Ns ? Ns[b] : Nmax;
  const size_t oA = (size_t)b * (Nmax - 1) * NX * NX, oB = (size_t)b * (Nmax - 1) * NX * NU, ow = (size_t)b * (Nmax - 1) * NX;
  if (N < 2 || N > Nmax) return;
  const Lay L = make_lay(N, NU, blockDim.x);
  load_x0<R>(L, sm, x0, b);
  for (int t = threadIdx.x; t < N * NX; t += blockDim.x) sm[L.Xb + t] = R(X[(size_t)b * Nmax * NX + t]);
  for (int t = threadIdx.x; t < N * NU; t += blockDim.x) sm[L.Ub + t] = R(U[(size_t)b * Nmax * NU + t]);
  __syncthreads();
  phase_discretize<R, NU>(P, L, sm);
  __syncthreads();
  for (int t = threadIdx.x; t < (Nmax - 1) * NX * NX; t += blockDim.x) {  // compact block -> dense
    const int k = t / (NX * NX), rc = t - k * NX * NX, r = rc / NX, c = rc - r * NX;
    Am[oA + t] = k < N - 1 ? double(sm[L.Am + k * STM_SAS + stm_index(r, c)]) : 0.0;
  }
  for (int t = threadIdx.x; t < (Nmax - 1) * NX * NU; t += blockDim.x) {  // strided blocks -> dense
    const int k = t / (NX * NU), o = k * b_stride(NU) + (t - k * NX * NU);
    Bm[oB + t] = k < N - 1 ? double(sm[L.Bm + o]) : 0.0;
    Bp[oB + t] = k < N - 1 ? double(sm[L.Bp + o]) : 0.0;
  }
  for (int t = threadIdx.x; t < (Nmax - 1) * NX; t += blockDim.x) w[ow + t] = t < (N - 1) * NX ? double(sm[L.w + t]) : 0.0;
}

// dir = 0: user buffers -> image (and mark running); dir = 1: image -> user.
template <typename R, int NU>
__global__ void k_pack(int B, int Nmax, int threads, const double* __restrict__ x0, const int* __restrict__ Ns, PlainWs W,
                       int dir, double* X, double* U, double* xh, double* uh, double* mup, double* mum, double* phi,
                       double* th, double* sigma, double* defect, int* iters) {
  const int b = blockIdx.x;
  const int N = Ns ? Ns[b] : Nmax;
  if (N < 2 || N > Nmax) {
    if (dir == 0 && threadIdx.x == 0) W.st[b] = PDG_BAD_INPUT;
    return;
  }
  const Lay L = make_lay(N, NU, threads);
  R* img = reinterpret_cast<R*>(W.img) + (size_t)b * W.istride;
  struct Seg { int off, n; double* p; size_t stride; };
  const Seg segs[8] = {
      {L.Xb, N * NX, X, (size_t)Nmax * NX},          {L.Ub, N * NU, U, (size_t)Nmax * NU},
      {L.xh, N * NX, xh, (size_t)Nmax * NX},         {L.uh, N * NU, uh, (size_t)Nmax * NU},
      {L.mup, (N - 1) * NX, mup, (size_t)(Nmax - 1) * NX}, {L.mum, (N - 1) * NX, mum, (size_t)(Nmax - 1) * NX},
      {L.phi, (N - 1) * NX, phi, (size_t)(Nmax - 1) * NX}, {L.th, N - 1, th, (size_t)(Nmax - 1)}};
  for (int s = 0; s < 8; ++s) {
    double* p = segs[s].p + (size_t)b * segs[s].stride;
    for (int t = threadIdx.x; t < segs[s].n; t += blockDim.x) {
      if (dir == 0) img[segs[s].off + t] = R(p[t]);
      else p[t] = double(img[segs[s].off + t]);
    }
  }
  if (dir == 0) {
    for (int t = threadIdx.x; t < 16; t += blockDim.x) img[L.x0 + t] = t < NX - 1 ? R(x0[(size_t)b * (NX - 1) + t]) : R(0);
    if (threadIdx.x == 0) W.st[b] = ST_RUNNING;
  } else if (threadIdx.x == 0) {
    sigma[b] = double(img[L.sc + 0]);
    defect[b] = double(img[L.sc + 1]);
    iters[2 * b] = W.pow_it[b];
    iters[2 * b + 1] = W.pipg_it[b];
  }
}

// ---------------------------------------------------------------------------
// gradient of the last SCP iteration (see pdg_adjoint.cuh), FP64
// ---------------------------------------------------------------------------
// k_grad runs everything but the forward-mode discretization of the first
// interval, whose dual-number arithmetic needs far more registers than the
// reverse PIPG loop: that part runs in k_grad_tangent, after it, so that the
// reverse loop keeps two CTAs per SM.  tg receives the record
// k_grad_tangent starts from (tangent_rec_size doubles per instance).
template <int NU>
__global__ void __launch_bounds__(256, 2)
k_grad(const DParams P, int B, int Nmax, const double* __restrict__ x0, const int* __restrict__ Ns,
       const double* __restrict__ rec, int rec_stride, const int* __restrict__ status,
       const double* __restrict__ gf_in, const double* __restrict__ gt_in, double* ck, long long ck_stride,
       int nck_max, int ckrec, double* tg, double* fuel_out, double* touch_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sm = reinterpret_cast<double*>(smraw);
  const int b = blockIdx.x;
  const int N = Ns ? Ns[b] : Nmax;
  const int st = status[b];
  if (N < 2 || N > Nmax || !(st == PDG_CONVERGED || st == PDG_MAX_SCP)) {
    if (threadIdx.x == 0) {
      if (fuel_out) fuel_out[b] = 0.0;
      if (touch_out) touch_out[b] = 0.0;
    }
    return;
  }
  const Lay L = make_lay(N, NU, blockDim.x);
  const AdjLay AL = make_adj(L, NU, blockDim.x, false);
  const double gf = gf_in ? gf_in[b] : 0.0, gt = gt_in ? gt_in[b] : 0.0;
  const double* rc = rec + (size_t)b * rec_stride;
  const int ow = N * (NX + NU), nw = L.img - L.xh;
  load_x0<double>(L, sm, x0, b);
  for (int t = threadIdx.x; t < N * NX; t += blockDim.x) sm[L.Xb + t] = rc[t];
  for (int t = threadIdx.x; t < N * NU; t += blockDim.x) sm[L.Ub + t] = rc[N * NX + t];
  for (int t = threadIdx.x; t < nw; t += blockDim.x) sm[L.xh + t] = rc[ow + t];
  for (int t = threadIdx.x; t < AL.total - AL.Sb; t += blockDim.x) sm[AL.Sb + t] = 0.0;
  const double sigma = rc[ow + nw];
  const int n = int(rc[ow + nw + 1]);
  __syncthreads();
  phase_discretize<double, NU>(P, L, sm);
  phase_scale_extra<double, NU>(P, L, sm);
  __syncthreads();
  const int ss = AL.ss;
  double* state = sm + L.xt;
  {
    const int nx = N * NX, nuu = N * NU, nm = (N - 1) * NX;
    for (int t = threadIdx.x; t < nx + nuu + 2 * nm + (N - 1); t += blockDim.x) {
      if (t < nx) sm[L.xt + t] = sm[L.xh + t];
      else if (t < nx + nuu) sm[L.ut + t - nx] = sm[L.uh + t - nx];
      else if (t < nx + nuu + nm) { const int q = t - nx - nuu; sm[L.nup + q] = sm[L.mup + q]; sm[L.num + q] = sm[L.mum + q]; }
      else if (t < nx + nuu + 2 * nm) { const int q = t - nx - nuu - nm; sm[L.vph + q] = sm[L.phi + q]; }
      else { const int q = t - nx - nuu - 2 * nm; sm[L.vth + q] = sm[L.th + q]; }
    }
  }
  __syncthreads();
  const double wp = P.w_prox;
  const double alpha = 2.0 / (wp + sqrt(wp * wp + 4.0 * P.omega * sigma));
  const double beta = P.omega * alpha;
  const double c1 = 1.0 - alpha * wp;
  const double rho = P.rho;
  double* ckb = ck + (size_t)b * ck_stride;
  double* seg = ckb + (ckrec ? (size_t)0 : (size_t)nck_max * ss);
  const int nck = (n + 49) / 50;
  const double* cks = ckrec ? rc + (ow + nw + 2 + ow) : ckb;  // the checkpoints
  if (ckrec) {
    // the solve recorded the last PIPG loop's final iterate and checkpoints
    for (int t = threadIdx.x; t < N * NX; t += blockDim.x) sm[L.xh + t] = rc[ow + nw + 2 + t];
    for (int t = threadIdx.x; t < N * NU; t += blockDim.x) sm[L.uh + t] = rc[ow + nw + 2 + N * NX + t];
    __syncthreads();
  } else {
    // forward pass of the final PIPG loop with a checkpoint every 50 iterations
    for (int j = 0; j < n; ++j) {
      if (j % 50 == 0) {
        for (int t = threadIdx.x; t < ss; t += blockDim.x) ckb[(size_t)(j / 50) * ss + t] = state[t];
        __syncthreads();
      }
      grad_pipg_iter<NU>(P, L, AL, sm, alpha, beta, c1, rho, true);
    }
  }
  // updated trajectory and the output functionals
  for (int t = threadIdx.x; t < N * NX; t += blockDim.x) sm[AL.Xo + t] = sm[L.Xb + t] + P.Px[t % NX] * sm[L.xh + t];
  for (int t = threadIdx.x; t < N * NU; t += blockDim.x) sm[AL.Uo + t] = sm[L.Ub + t] + P.Pu[t % NU] * sm[L.uh + t];
  __syncthreads();
  if (threadIdx.x == 0) {
    double gdir[NX - 1];
    for (int i = 0; i < NX - 1; ++i) gdir[i] = 0.0;
    const double fu = sm[AL.Xo + IM] - sm[AL.Xo + (N - 1) * NX + IM];
    gdir[IM] += gf;                                      // m_1 = m_wet
    sm[AL.xob + (N - 1) * NX + IM] += -gf * P.Px[IM];    // m_N through x_hat_N
    const double e = touchdown_and_reverse<NU>(P, L, AL, sm, gt, gdir);
    for (int i = 0; i < NX - 1; ++i) sm[AL.gacc + i] = gdir[i];
    if (fuel_out) fuel_out[b] = fu;
    if (touch_out) touch_out[b] = e;
  }
  __syncthreads();
  // reverse pass, segment by segment; the first interval's block cotangents
  // accumulate in shared memory (cA, cBm, cBp, cw are contiguous)
  for (int t = threadIdx.x; t < AL.gacc - AL.cA; t += blockDim.x) sm[AL.cA + t] = 0.0;
  __syncthreads();
  // Within a segment the recomputation records, per iteration, what its
  // reverse step reads (the relaxed dual before the update, 2z - z~ and the
  // projection masks), so the reverse steps need no second recomputation.
  const int nm = (N - 1) * NX, o1 = nm, o2 = o1 + N * NX, o3 = o2 + N * NU, o4 = o3 + nm, o5 = o4 + nm,
            o6 = o5 + (N - 1);
  for (int sgm = nck - 1; sgm >= 0; --sgm) {
    const int j0 = sgm * 50, j1 = min(n, j0 + 50);
    for (int t = threadIdx.x; t < ss; t += blockDim.x) state[t] = cks[(size_t)sgm * ss + t];
    __syncthreads();
    for (int j = j0; j < j1; ++j) {
      double* e = seg + (size_t)(j - j0) * AL.sg;
      // the iteration's first write to vph comes after the barrier that ends its primal phase
      for (int t = threadIdx.x; t < nm; t += blockDim.x) e[t] = sm[L.vph + t];
      grad_pipg_iter<NU>(P, L, AL, sm, alpha, beta, c1, rho, true);
      for (int t = threadIdx.x; t < AL.sg - o1; t += blockDim.x) {
        const int u = o1 + t;
        e[u] = u < o2 ? sm[L.dx + (u - o1)]
             : u < o3 ? sm[L.du + (u - o2)]
             : u < o4 ? sm[AL.mup_m + (u - o3)]
             : u < o5 ? sm[AL.mum_m + (u - o4)]
             : u < o6 ? sm[AL.th_m + (u - o5)]
                      : sm[AL.u_m + (u - o6)];
      }
      __syncthreads();  // the next iteration overwrites 2z - z~ and the masks
    }
    for (int j = j1 - 1; j >= j0; --j) {
      const double* e = seg + (size_t)(j - j0) * AL.sg;
      for (int u = threadIdx.x; u < AL.sg; u += blockDim.x) {
        const double v = e[u];
        if (u < o1) sm[L.vph + u] = v;
        else if (u < o2) sm[L.dx + (u - o1)] = v;
        else if (u < o3) sm[L.du + (u - o2)] = v;
        else if (u < o4) sm[AL.mup_m + (u - o3)] = v;
        else if (u < o5) sm[AL.mum_m + (u - o4)] = v;
        else if (u < o6) sm[AL.th_m + (u - o5)] = v;
        else sm[AL.u_m + (u - o6)] = v;
      }
      __syncthreads();
      grad_pipg_reverse<NU>(P, L, AL, sm, alpha, beta, c1, rho, j == n - 1);
    }
  }
  // cotangents of the first interval's blocks, unscaled
  if (threadIdx.x < NX) {
    const int i = threadIdx.x;
    for (int c = 0; c < NX; ++c) sm[AL.cA + i * NX + c] *= P.Px[c] * P.Pxinv[i];
    for (int c = 0; c < NU; ++c) {
      sm[AL.cBm + i * NU + c] *= P.Pu[c] * P.Pxinv[i];
      sm[AL.cBp + i * NU + c] *= P.Pu[c] * P.Pxinv[i];
    }
    sm[AL.cw + i] *= P.Pxinv[i];
  }
  __syncthreads();
  // the tangent kernel's record: x_bar_1, u_bar_1, u_bar_2, then cA .. gacc
  // (contiguous in the layout)
  double* r = tg + (size_t)b * tangent_rec_size(NU);
  for (int t = threadIdx.x; t < tangent_rec_size(NU); t += blockDim.x)
    r[t] = t < NX ? sm[L.Xb + t] : t < NX + 2 * NU ? sm[L.Ub + t - NX] : sm[AL.cA + t - NX - 2 * NU];
}

// The forward-mode part of the gradient: the first interval's RK4
// discretization in dual arithmetic along every direction of x0, its
// sensitivities contracted with the block cotangents k_grad recorded, added
// to the gradient k_grad accumulated (see tangent_first_interval).
template <int NU>
__global__ void __launch_bounds__(256, 1)
k_grad_tangent(const DParams P, int B, int Nmax, const int* __restrict__ Ns, const int* __restrict__ status,
               const double* __restrict__ tg, double* grad) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sm = reinterpret_cast<double*>(smraw);
  const int b = blockIdx.x;
  const int N = Ns ? Ns[b] : Nmax;
  const int st = status[b];
  if (N < 2 || N > Nmax || !(st == PDG_CONVERGED || st == PDG_MAX_SCP)) {
    if (threadIdx.x < NX - 1) grad[(size_t)b * (NX - 1) + threadIdx.x] = 0.0;
    return;
  }
  // a layout holding only what tangent_first_interval reads: the record, then
  // the dual-number stage buffers
  Lay L{};
  L.N = N;
  L.Xb = 0;
  L.Ub = NX;
  AdjLay A{};
  A.cA = NX + 2 * NU;
  A.cBm = A.cA + NX * NX;
  A.cBp = A.cBm + NX * NU;
  A.cw = A.cBp + NX * NU;
  A.gacc = A.cw + NX;
  A.tang = (A.gacc + 16 + 1) & ~1;
  const double* r = tg + (size_t)b * tangent_rec_size(NU);
  for (int t = threadIdx.x; t < tangent_rec_size(NU); t += blockDim.x) sm[t] = r[t];
  __syncthreads();
  tangent_first_interval<NU>(P, L, A, sm);
  __syncthreads();
  if (threadIdx.x < NX - 1) grad[(size_t)b * (NX - 1) + threadIdx.x] = sm[A.gacc + threadIdx.x];
}


// Counting sort of the instance ids by node count (shape classes 0..32):
// class_off[c] .. class_off[c+1] index perm for N = c.  One CTA.
__global__ void k_class_sort(int B, const int* __restrict__ Ns, int n_max, int* perm, int* class_off) {
  __shared__ int cnt[NMAX + 2], off[NMAX + 2];
  for (int i = threadIdx.x; i < NMAX + 2; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int N = Ns[b];
    if (N < 2 || N > n_max) N = n_max;  // bad inputs go with the largest class and are rejected there
    atomicAdd(&cnt[N], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0;
    for (int c = 0; c <= NMAX + 1; ++c) { off[c] = o; class_off[c] = o; o += (c <= NMAX ? cnt[c] : 0); }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int N = Ns[b];
    if (N < 2 || N > n_max) N = n_max;
    perm[atomicAdd(&off[N], 1)] = b;
  }
}

// FMA-chain probe for the roofline denominator: every thread runs 8
// independent dependency chains of `iters` FMAs each (16 flops per step).
// Lanes >= active of every warp return at once (active = 32: all work).
template <typename R>
__global__ void k_fma_probe(int iters, int active, R seed, R* out) {
  if ((threadIdx.x & 31) >= active) return;
  R a0 = seed + R(threadIdx.x), a1 = a0 + R(1), a2 = a0 + R(2), a3 = a0 + R(3);
  R a4 = a0 + R(4), a5 = a0 + R(5), a6 = a0 + R(6), a7 = a0 + R(7);
  const R m = R(0.999999), c = R(1e-7);
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  const R s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == R(-12345)) out[0] = s;  // keeps the chains live; never true
}

}  // namespace

// ===========================================================================
// scratch for pdg_mc_solve_batch_noalloc: a fixed device array, so that the
// entry point never allocates (see include/pdg_mc.h)
// ===========================================================================
static constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// ===========================================================================
// host side
// ===========================================================================
struct pdg_handle {
  pdg_params p;
  DParams dp;
  int n_max;
  int threads_override;
  int pipg_variant = 0;        // 0 auto, 1 shared-memory PIPG, 2 register PIPG
  int device;
  int num_sms;
  std::string err;
  // plain-form workspace
  void* img = nullptr;
  size_t img_bytes = 0;
  int* ints = nullptr;        // st, sit, pow_it, pipg_it, done, queue
  size_t ints_count = 0;
  long long* lit = nullptr;
  size_t lit_count = 0;
  int* pinned_done = nullptr;
  cudaStream_t cap = nullptr;  // plain form runs (and is captured) here
  // gradient workspace
  int* cls = nullptr;          // shape classes: perm, class offsets, queues
  size_t cls_count = 0;
  cudaStream_t cls_streams[NMAX + 1] = {};
  cudaEvent_t cls_events[NMAX + 1] = {};
  double* rec_ptr = nullptr;   // set only while a gradient solve runs
  int rec_stride = 0;
  bool ck_rec = false;         // ... and whose record also holds the PIPG checkpoints
  void* gws = nullptr;
  size_t gws_bytes = 0;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // host-buffer API staging
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // last launch
  int last_threads = 0, last_ctas = 0, last_smem = 0, last_variant = 0;
  // abort word: pinned host memory mapped into the device's address space
  int* abort_host = nullptr;
  // plain form: the instantiated graph of one SCP iteration, kept between
  // calls and updated in place when only the kernels' arguments change
  cudaGraphExec_t plain_exec = nullptr;
  long long plain_graph_builds = 0, plain_graph_updates = 0;
};

static std::string g_init_err;

// NVTX range for profilers (nsys, ncu's NVTX filters): the entry points and,
// in the plain form, each SCP iteration.  Costs nothing without a tool.
struct NvtxRange {
  explicit NvtxRange(const char* m) { nvtxRangePushA(m); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define PDG_CUDA(h, call)                                                        \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
      return PDG_ECUDA;                                                          \
    }                                                                            \
  } while (0)

static int fail(pdg_handle* h, int code, const std::string& msg) {
  h->err = msg;
  return code;
}

static bool fill_dparams(const pdg_params* p, DParams* d, std::string* why) {
  memset(d, 0, sizeof *d);
  if (!(p->nu == 4 || p->nu == PDG_MODEL_NU_ALT)) {
    *why = PDG_MODEL_NU_ALT == 7 ? "nu must be 4 or 7" : "nu must be 4 (this model has no RCS torque)"; return false;
  }
  if (!(p->precision == 0 || p->precision == 1)) { *why = "precision must be 0 (FP64) or 1 (FP32)"; return false; }
  if (p->rk4_substeps < 1 || p->pipg_jmax < 1 || p->pipg_jcheck < 1 || p->pow_jmax < 1 || p->scp_jmax < 1) {
    *why = "iteration counts and rk4_substeps must be >= 1"; return false;
  }
#ifdef PDG_MODEL_USES_INERTIA
  for (int i = 0; i < 3; ++i) if (!(p->J_B[i] > 0)) { *why = "J_B must be positive"; return false; }
#endif
  for (int i = 0; i < NX; ++i) if (!(p->P_x[i] > 0)) { *why = "P_x must be positive"; return false; }
  for (int i = 0; i < 3; ++i) if (!(p->P_u[i] > 0)) { *why = "P_u must be positive"; return false; }
  if (p->nu == 7) for (int i = 3; i < 6; ++i) if (!(p->P_u[i] > 0)) { *why = "P_u must be positive"; return false; }
  if (!(p->P_u[p->nu - 1] > 0)) { *why = "P_u must be positive"; return false; }
  if (!(p->w_prox > 0) || !(p->pipg_omega > 0) || !(p->s_max >= p->s_min)) { *why = "w_prox, pipg_omega > 0 and s_min <= s_max required"; return false; }
  d->nu = p->nu;
  d->nsub = p->rk4_substeps;
  d->pipg_jmax = p->pipg_jmax;
  d->pipg_jcheck = p->pipg_jcheck;
  d->pow_jmax = p->pow_jmax;
  d->scp_jmax = p->scp_jmax;
  for (int i = 0; i < NX; ++i) d->fix_f[i] = p->fix_f[i] ? 1 : 0;
  d->alpha_mdot = p->alpha_mdot;
  for (int i = 0; i < 3; ++i) {
    d->g[i] = p->g_I[i];
    d->J[i] = p->J_B[i];
    d->Jinv[i] = p->J_B[i] > 0 ? 1.0 / p->J_B[i] : 0.0;  // the 3-DoF model has no inertia
    d->rT[i] = p->r_T_B[i];
  }
  d->m_dry = p->m_dry;
  d->vmax2 = p->v_max * p->v_max;
  d->one_m_cos_theta = 1.0 - cos(p->theta_max);
  d->omega_max2 = p->omega_max * p->omega_max;
  d->sec_delta = 1.0 / cos(p->delta_max);
  d->T_min = p->T_min;
  d->T_max = p->T_max;
  d->gamma_max2 = p->gamma_max * p->gamma_max;
  d->s_min = p->s_min;
  d->s_max = p->s_max;
  for (int i = 0; i < NX; ++i) {
    d->z_f[i] = p->z_f[i];
    d->Px[i] = p->P_x[i];
    d->Pxinv[i] = 1.0 / p->P_x[i];
  }
  for (int i = 0; i < 7; ++i) {
    d->Pu[i] = p->P_u[i];
    d->Puinv[i] = p->P_u[i] > 0 ? 1.0 / p->P_u[i] : 0.0;
  }
  d->w_cost = p->w_cost;
  d->w_prox = p->w_prox;
  d->w_ep = p->w_ep;
  d->eps_ctcs = p->eps_ctcs;
  d->omega = p->pipg_omega;
  d->rho = p->pipg_rho;
  d->eps_abs = p->pipg_eps_abs;
  d->eps_rel = p->pipg_eps_rel;
  d->pow_eps_abs = p->pow_eps_abs;
  d->pow_eps_rel = p->pow_eps_rel;
  d->pow_buff = p->pow_eps_buff;
  d->scp_eps_step = p->scp_eps_step;
  d->scp_eps_defect = p->scp_eps_defect;
  d->tf_guess = p->tf_guess;
  d->g0 = sqrt(p->g_I[0] * p->g_I[0] + p->g_I[1] * p->g_I[1] + p->g_I[2] * p->g_I[2]);
  d->budget_ns = p->budget_seconds > 0 ? p->budget_seconds * 1e9 : 0.0;
  d->gs = p->glide_slope ? 1 : 0;
  if (d->gs && !(p->gamma_gs > 0 && p->gamma_gs < 1.5707963267948966)) {
    *why = "gamma_gs must lie in (0, pi/2) with glide_slope on"; return false;
  }
  d->tan_gs2 = d->gs ? tan(p->gamma_gs) * tan(p->gamma_gs) : 0.0;
  if (p->dt_min < 0 || p->dt_max < 0 || p->tf_max < 0) { *why = "dt_min, dt_max, tf_max must be >= 0 (0 = off)"; return false; }
  d->s_lo = p->s_min;
  d->s_hi = p->tf_max > 0 && p->tf_max < p->s_max ? p->tf_max : p->s_max;
  d->dt_lo = p->dt_min;
  d->dt_hi = p->dt_max;
  for (int i = 0; i < 16; ++i) d->mp[i] = p->model_params[i];
  d->soc = p->soc_thrust ? 1 : 0;
  d->soc_tan = tan(p->delta_max);
  if (d->soc && !(p->P_u[0] == p->P_u[1] && p->P_u[1] == p->P_u[2])) {
    *why = "soc_thrust needs the same P_u on the three thrust components"; return false;
  }
  return true;
}


// Threads per CTA for instances of N nodes.  FP32: one thread per dual row
// (whole warps) plus the warp of CTCS rows.  FP64: as many CTAs per SM as
// shared memory holds (at most four; more keep the FP64 pipe busier), each
// with the threads that the kernels' 128 registers per thread leave for that
// many (128, 160, 256 or 512), but no more than the FP32 count.  Within
// [128, 512].
static int threads_for(int N, int nu, int precision) {
  const int full = round32((N - 1) * NX) + 32;
  int t = full;
  if (precision == 0) {
    for (int c = 4; c >= 1; --c) {
      int tc = (65536 / (128 * c)) & ~31;
      if (tc > full) tc = full;
      if (tc < 128) tc = 128;
      const Lay L = make_lay(N, nu, tc);
      if (L.ipw >= 1 && (size_t)c * ((size_t)L.total * 8 + 1024) <= 228 * 1024) { t = tc; break; }
    }
  }
  if (t > 512) t = 512;
  if (t < 128) t = 128;
  return t;
}

// PIPG form and CTA size for instances of up to N nodes.  Auto (variant 0):
// FP32 takes the tiled register form (form 3; the shared-memory form is bound
// by shared-memory bandwidth, form 2 by its operand loads), FP64 the
// shared-memory form (bound by the FP64 pipe, it gains nothing from registers
// and keeps three CTAs per SM).  In auto mode a thread-count override outside
// what form 3 accepts selects the shared form; with form 2 or 3 requested it
// is an error.
// The non-PIPG kernels of the plain form run with at most 512 threads.
struct Plan {
  int T;   // threads of the solve kernel (and of k_plain_pipg)
  int Tr;  // threads of the other plain-form kernels
  int pv;  // 1 shared-memory PIPG, 2 register PIPG, 3 register tiles
};

static bool plan_for(const pdg_handle* h, int N, Plan* out, std::string* why, bool use_override = true) {
  const int treg = pipg_reg_threads(N, h->p.nu);
  const int maxt = h->p.precision == 1 ? PDG_REG_MAXT_F32 : 512;
  const int ov = use_override ? h->threads_override : 0;
  const int tks = pipg_ks_threads(N);
  int pv = h->pipg_variant;
  if (pv == 0) pv = (h->p.precision == 1 && (ov == 0 || (ov >= tks && ov <= PDG_KS_PERS_MAXT))) ? 3 : 1;
  if (pv == 2) {
    const int T = ov > 0 ? ov : treg;
    if (T < treg || T > maxt) {
      *why = "the register PIPG form needs " + std::to_string(treg) + " to " + std::to_string(maxt) +
             " threads per CTA at N = " + std::to_string(N);
      return false;
    }
    *out = {T, T < 512 ? T : 512, 2};
  } else if (pv == 3) {
    // the lane groups' threads, at least two warps (the discretization wants
    // one interval per wave); the plain form's other kernels at least 128
    const int T = ov > 0 ? ov : (tks < 64 ? 64 : tks);
    const int tmax = h->p.precision == 1 ? PDG_KS_PERS_MAXT : 512;
    if (T < tks || T > tmax) {
      *why = "PIPG form 3 needs " + std::to_string(tks) + " to " + std::to_string(tmax) +
             " threads per CTA at N = " + std::to_string(N);
      return false;
    }
    *out = {T, T < 128 ? 128 : T, 3};
  } else {
    const int T = ov > 0 ? ov : threads_for(N, h->p.nu, h->p.precision);
    if (T > 512) { *why = "the shared-memory PIPG form runs at most 512 threads per CTA"; return false; }
    *out = {T, T, 1};
  }
  return true;
}

template <typename R, int NU>
using PersistentFn = void (*)(const DParams, int, int, const double*, const int*, double*, double*, double*, double*,
                              int*, int*, long long*, int*, int*, double*, int, const int*, const int*, int);
template <typename R, int NU>
using PlainPipgFn = void (*)(const DParams, int, int, const int*, PlainWs, const int*);
template <typename R, int NU>
static PersistentFn<R, NU> persistent_fn(int pv, bool ck = false) {
  if constexpr (sizeof(R) == 8) {
    if (ck && pv == 1) return k_persistent<R, NU, 1, true>;
  }
  return pv == 3 ? k_persistent<R, NU, 3> : (pv == 2 ? k_persistent<R, NU, 2> : k_persistent<R, NU, 1>);
}
template <typename R, int NU>
static PlainPipgFn<R, NU> plain_pipg_fn(int pv) {
  return pv == 3 ? k_plain_pipg<R, NU, 3> : (pv == 2 ? k_plain_pipg<R, NU, 2> : k_plain_pipg<R, NU, 1>);
}

template <typename R, int NU>
struct Kern {
  static int prepare(pdg_handle* h, int threads, size_t smem) {
    const void* fns[] = {(const void*)k_persistent<R, NU, 1>, (const void*)k_persistent<R, NU, 2>,
                         (const void*)k_persistent<R, NU, 3>, (const void*)k_plain_init<R, NU>,
                         (const void*)k_plain_disc<R, NU>, (const void*)k_plain_power<R, NU>,
                         (const void*)k_plain_pipg<R, NU, 1>, (const void*)k_plain_pipg<R, NU, 2>,
                         (const void*)k_plain_pipg<R, NU, 3>, (const void*)k_plain_update<R, NU>,
                         (const void*)k_subproblem<R, NU>};
    for (const void* f : fns) PDG_CUDA(h, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if constexpr (sizeof(R) == 8)
      PDG_CUDA(h, cudaFuncSetAttribute(k_persistent<R, NU, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    return 0;
  }
};

template <typename R, int NU>
static int run_solve(pdg_handle* h, int B, const double* x0, const int* Ns, int mode, double* X, double* U, double* tf,
                     double* fuel, int* status, int* scp_iters, long long* pipg_iters, int* trace, cudaStream_t s) {
  Plan pl;
  std::string why;
  if (!plan_for(h, h->n_max, &pl, &why)) return fail(h, PDG_EINVAL, why);
  const int T = pl.T;
  const Lay L = make_lay(h->n_max, NU, T);
  const size_t smem = (size_t)L.total * sizeof(R);
  if (L.ipw < 1 || make_lay(h->n_max, NU, pl.Tr).ipw < 1)
    return fail(h, PDG_EINVAL, "threads per CTA too small for one discretization interval");
  if (int rc = Kern<R, NU>::prepare(h, T, smem)) return rc;
  const PersistentFn<R, NU> kp = persistent_fn<R, NU>(pl.pv, h->ck_rec && mode == 1);
  int occ = 0;
  PDG_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kp, T, smem));
  if (occ < 1) return fail(h, PDG_EINVAL, "solve kernel does not fit on an SM with this configuration");
  h->last_threads = T;
  h->last_ctas = occ;
  h->last_smem = (int)smem;
  h->last_variant = pl.pv;
  // integer workspace: st, sit, pow_it, pipg_it [B each], done, queue
  const size_t nints = (size_t)4 * B + 2;
  if (h->ints_count < nints) {
    if (h->ints) cudaFree(h->ints);
    h->ints = nullptr;
    h->ints_count = 0;
    PDG_CUDA(h, cudaMalloc(&h->ints, nints * sizeof(int)));
    h->ints_count = nints;
  }
  int* queue = h->ints + 4 * (size_t)B + 1;
  if (mode == 1 || (mode == 2 && !Ns)) {
    PDG_CUDA(h, cudaMemsetAsync(queue, 0, sizeof(int), s));
    const int grid = (int)((long long)occ * h->num_sms < B ? (long long)occ * h->num_sms : B);
    kp<<<grid, T, smem, s>>>(h->dp, B, h->n_max, x0, Ns, X, U, tf, fuel, status, scp_iters, pipg_iters, trace, queue,
                             h->rec_ptr, h->rec_stride, nullptr, nullptr, 0);
    PDG_CUDA(h, cudaGetLastError());
    return 0;
  }
  if (mode == 2) {
    // shape classes: one persistent grid per node count, all on forked streams
    const size_t ncls = NMAX + 2;
    if (h->cls_count < (size_t)B + ncls + NMAX + 1) {
      if (h->cls) cudaFree(h->cls);
      h->cls = nullptr;
      h->cls_count = 0;
      PDG_CUDA(h, cudaMalloc(&h->cls, sizeof(int) * ((size_t)B + ncls + NMAX + 1)));
      h->cls_count = (size_t)B + ncls + NMAX + 1;
    }
    int* perm = h->cls;
    int* class_off = h->cls + B;
    int* queues = class_off + ncls;
    if (!h->ev_in) PDG_CUDA(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    PDG_CUDA(h, cudaMemsetAsync(queues, 0, sizeof(int) * (NMAX + 1), s));
    k_class_sort<<<1, 1024, 0, s>>>(B, Ns, h->n_max, perm, class_off);
    PDG_CUDA(h, cudaGetLastError());
    PDG_CUDA(h, cudaEventRecord(h->ev_in, s));
    for (int N = h->n_max; N >= 2; --N) {
      Plan pn;
      if (!plan_for(h, N, &pn, &why, N == h->n_max)) return fail(h, PDG_EINVAL, why);
      const int Tn = pn.T;
      const PersistentFn<R, NU> kpn = persistent_fn<R, NU>(pn.pv);
      const Lay Ln = make_lay(N, NU, Tn);
      const size_t smem_n = (size_t)Ln.total * sizeof(R);
      if (Ln.ipw < 1) continue;
      int occ_n = 0;
      PDG_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_n, kpn, Tn, smem_n));
      if (occ_n < 1) return fail(h, PDG_EINVAL, "a shape class does not fit on an SM");
      cudaStream_t cs = h->cls_streams[N];
      if (!cs) {
        PDG_CUDA(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        h->cls_streams[N] = cs;
        PDG_CUDA(h, cudaEventCreateWithFlags(&h->cls_events[N], cudaEventDisableTiming));
      }
      PDG_CUDA(h, cudaStreamWaitEvent(cs, h->ev_in, 0));
      const int grid = (int)((long long)occ_n * h->num_sms < B ? (long long)occ_n * h->num_sms : B);
      kpn<<<grid, Tn, smem_n, cs>>>(h->dp, B, h->n_max, x0, Ns, X, U, tf, fuel, status, scp_iters, pipg_iters, trace,
                                    queues + N, h->rec_ptr, h->rec_stride, perm, class_off, N);
      PDG_CUDA(h, cudaGetLastError());
      PDG_CUDA(h, cudaEventRecord(h->cls_events[N], cs));
      PDG_CUDA(h, cudaStreamWaitEvent(s, h->cls_events[N], 0));
    }
    return 0;
  }
  // plain form
  const Lay Li = make_lay(h->n_max, NU, T);
  const size_t istride = (size_t)Li.img;
  const size_t need = istride * sizeof(R) * B;
  if (h->img_bytes < need) {
    if (h->img) cudaFree(h->img);
    h->img = nullptr;
    h->img_bytes = 0;
    PDG_CUDA(h, cudaMalloc(&h->img, need));
    h->img_bytes = need;
  }
  if (h->lit_count < (size_t)B) {
    if (h->lit) cudaFree(h->lit);
    h->lit = nullptr;
    h->lit_count = 0;
    PDG_CUDA(h, cudaMalloc(&h->lit, sizeof(long long) * B));
    h->lit_count = B;
  }
  if (!h->pinned_done) PDG_CUDA(h, cudaMallocHost(&h->pinned_done, sizeof(int)));
  if (!h->cap) PDG_CUDA(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  if (!h->ev_in) PDG_CUDA(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  if (!h->ev_out) PDG_CUDA(h, cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  // the caller's stream may be the legacy default stream, which cannot be
  // captured: run on the handle's stream, ordered after and before the caller's
  const cudaStream_t us = s;
  PDG_CUDA(h, cudaEventRecord(h->ev_in, us));
  PDG_CUDA(h, cudaStreamWaitEvent(h->cap, h->ev_in, 0));
  s = h->cap;
  PlainWs W;
  W.img = h->img;
  W.istride = (int)istride;
  W.st = h->ints;
  W.sit = h->ints + B;
  W.pow_it = h->ints + 2 * (size_t)B;
  W.pipg_it = h->ints + 3 * (size_t)B;
  W.done = h->ints + 4 * (size_t)B;
  W.lit = h->lit;
  PDG_CUDA(h, cudaMemsetAsync(W.done, 0, sizeof(int), s));
  const int Tr = pl.Tr;
  const PlainPipgFn<R, NU> kpp = plain_pipg_fn<R, NU>(pl.pv);
  k_plain_init<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, x0, Ns, W, X, U, tf, fuel, status, scp_iters, pipg_iters);
  PDG_CUDA(h, cudaGetLastError());
  cudaGraph_t graph = nullptr;
  PDG_CUDA(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  k_plain_disc<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W);
  k_plain_power<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W, nullptr);
  kpp<<<B, T, smem, s>>>(h->dp, B, h->n_max, Ns, W, nullptr);
  k_plain_update<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W, 0, X, U, tf, fuel, status, scp_iters, pipg_iters,
                                             trace, nullptr);
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (ce != cudaSuccess) return fail(h, PDG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  // Capturing is cheap; instantiating is not.  A graph with the same four
  // kernels (same functions and launch shapes) only changes arguments from
  // call to call (batch size, buffers), which cudaGraphExecUpdate applies to
  // the kept executable; anything else instantiates it anew.
  if (h->plain_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(h->plain_exec, graph, &info) == cudaSuccess) {
      ++h->plain_graph_updates;
    } else {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(h->plain_exec);
      h->plain_exec = nullptr;
    }
  }
  if (!h->plain_exec) {
    ce = cudaGraphInstantiate(&h->plain_exec, graph, 0);
    if (ce != cudaSuccess) {
      h->plain_exec = nullptr;
      cudaGraphDestroy(graph);
      return fail(h, PDG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    }
    ++h->plain_graph_builds;
  }
  cudaGraphDestroy(graph);
  cudaGraphExec_t exec = h->plain_exec;
  int rc = 0;
  for (int j = 0; j < h->p.scp_jmax; ++j) {
    NvtxRange r("pdg_mc plain SCP iteration");
    ce = cudaGraphLaunch(exec, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h->pinned_done, W.done, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) { rc = fail(h, PDG_ECUDA, std::string("plain SCP step: ") + cudaGetErrorString(ce)); break; }
    if (*h->pinned_done >= B) break;
  }
  if (rc == 0) {
    PDG_CUDA(h, cudaEventRecord(h->ev_out, s));
    PDG_CUDA(h, cudaStreamWaitEvent(us, h->ev_out, 0));
  }
  return rc;
}

template <typename R, int NU>
static int run_subproblem(pdg_handle* h, int B, const double* x0, const int* Ns, const double* X, const double* U,
                          double* Am, double* Bm, double* Bp, double* w, cudaStream_t s) {
  Plan pl;
  std::string why;
  if (!plan_for(h, h->n_max, &pl, &why)) return fail(h, PDG_EINVAL, why);
  const int T = pl.Tr;
  const Lay L = make_lay(h->n_max, NU, T);
  const size_t smem = (size_t)L.total * sizeof(R);
  if (int rc = Kern<R, NU>::prepare(h, T, smem)) return rc;
  k_subproblem<R, NU><<<B, T, smem, s>>>(h->dp, B, h->n_max, x0, Ns, X, U, Am, Bm, Bp, w);
  PDG_CUDA(h, cudaGetLastError());
  return 0;
}

template <typename R, int NU>
static int run_step(pdg_handle* h, int B, const double* x0, const int* Ns, double* X, double* U, double* xh, double* uh,
                    double* mup, double* mum, double* phi, double* th, const int* force, double* sigma, double* defect,
                    double* step, int* iters, cudaStream_t s) {
  Plan pl;
  std::string why;
  if (!plan_for(h, h->n_max, &pl, &why)) return fail(h, PDG_EINVAL, why);
  const int T = pl.T, Tr = pl.Tr;
  const PlainPipgFn<R, NU> kpp = plain_pipg_fn<R, NU>(pl.pv);
  h->last_variant = pl.pv;
  const Lay L = make_lay(h->n_max, NU, T);
  const size_t smem = (size_t)L.total * sizeof(R);
  if (int rc = Kern<R, NU>::prepare(h, T, smem)) return rc;
  const size_t istride = (size_t)L.img;
  const size_t need = istride * sizeof(R) * B;
  if (h->img_bytes < need) {
    if (h->img) cudaFree(h->img);
    h->img = nullptr;
    h->img_bytes = 0;
    PDG_CUDA(h, cudaMalloc(&h->img, need));
    h->img_bytes = need;
  }
  const size_t nints = (size_t)4 * B + 2;
  if (h->ints_count < nints) {
    if (h->ints) cudaFree(h->ints);
    h->ints = nullptr;
    h->ints_count = 0;
    PDG_CUDA(h, cudaMalloc(&h->ints, nints * sizeof(int)));
    h->ints_count = nints;
  }
  if (h->lit_count < (size_t)B) {
    if (h->lit) cudaFree(h->lit);
    h->lit = nullptr;
    h->lit_count = 0;
    PDG_CUDA(h, cudaMalloc(&h->lit, sizeof(long long) * B));
    h->lit_count = B;
  }
  PlainWs W;
  W.img = h->img;
  W.istride = (int)istride;
  W.st = h->ints;
  W.sit = h->ints + B;
  W.pow_it = h->ints + 2 * (size_t)B;
  W.pipg_it = h->ints + 3 * (size_t)B;
  W.done = h->ints + 4 * (size_t)B;
  W.lit = h->lit;
  k_pack<R, NU><<<B, 128, 0, s>>>(B, h->n_max, T, x0, Ns, W, 0, X, U, xh, uh, mup, mum, phi, th, sigma, defect, iters);
  k_plain_disc<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W);
  k_plain_power<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W, force);
  kpp<<<B, T, smem, s>>>(h->dp, B, h->n_max, Ns, W, force);
  k_plain_update<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W, 1, nullptr, nullptr, nullptr, nullptr, nullptr,
                                             nullptr, nullptr, nullptr, step);
  k_pack<R, NU><<<B, 128, 0, s>>>(B, h->n_max, T, x0, Ns, W, 1, X, U, xh, uh, mup, mum, phi, th, sigma, defect, iters);
  PDG_CUDA(h, cudaGetLastError());
  return 0;
}

// Device address of g_noalloc_scratch for the current device, looked up once
// per device (the host-side name of the array is not a device address).
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];

static int noalloc_scratch(pdg_handle* h, void** out) {
  int dev = 0;
  PDG_CUDA(h, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(h, PDG_EINVAL, "device index out of range for the static scratch table");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(h, PDG_ECUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return 0;
}

template <typename R, int NU>
static int run_noalloc(pdg_handle* h, int B, const double* x0, const int* Ns, double* X, double* U, double* tf,
                       double* fuel, int* status, int* scp_iters, long long* pipg_iters, cudaStream_t s) {
  Plan pl;
  std::string why;
  if (!plan_for(h, h->n_max, &pl, &why)) return fail(h, PDG_EINVAL, why);
  const int T = pl.T, Tr = pl.Tr;
  const PlainPipgFn<R, NU> kpp = plain_pipg_fn<R, NU>(pl.pv);
  const Lay L = make_lay(h->n_max, NU, T);
  const size_t smem = (size_t)L.total * sizeof(R);
  if (L.ipw < 1) return fail(h, PDG_EINVAL, "threads per CTA too small for one discretization interval");
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t istride = (size_t)L.img;
  const size_t per = istride * sizeof(R) + sizeof(long long) + 4 * sizeof(int);
  const size_t fixed = al(sizeof(int) * 2) + 3 * 256;
  const size_t need = al(sizeof(int) * (4 * (size_t)B + 2)) + al(sizeof(long long) * (size_t)B) + al(istride * sizeof(R) * B);
  if (need > kNoAllocBytes) {
    const size_t bmax = (kNoAllocBytes - fixed) / per;
    char msg[200];
    snprintf(msg, sizeof msg, "batch of %d needs %zu bytes of scratch; the static scratch holds %zu bytes (at most about %zu instances for this n_max and precision)",
             B, need, kNoAllocBytes, bmax);
    return fail(h, PDG_EINVAL, msg);
  }
  void* base = nullptr;
  if (int rc = noalloc_scratch(h, &base)) return rc;
  if (int rc = Kern<R, NU>::prepare(h, T, smem)) return rc;
  char* c = (char*)base;
  PlainWs W;
  W.st = (int*)c;
  W.sit = W.st + B;
  W.pow_it = W.st + 2 * (size_t)B;
  W.pipg_it = W.st + 3 * (size_t)B;
  W.done = W.st + 4 * (size_t)B;
  c += al(sizeof(int) * (4 * (size_t)B + 2));
  W.lit = (long long*)c;
  c += al(sizeof(long long) * (size_t)B);
  W.img = c;
  W.istride = (int)istride;
  // the array keeps the previous call's contents: clear the counter (every
  // per-instance field is written by k_plain_init before it is read)
  PDG_CUDA(h, cudaMemsetAsync(W.done, 0, sizeof(int), s));
  k_plain_init<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, x0, Ns, W, X, U, tf, fuel, status, scp_iters, pipg_iters);
  for (int j = 0; j < h->p.scp_jmax; ++j) {
    k_plain_disc<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W);
    k_plain_power<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W, nullptr);
    kpp<<<B, T, smem, s>>>(h->dp, B, h->n_max, Ns, W, nullptr);
    k_plain_update<R, NU><<<B, Tr, smem, s>>>(h->dp, B, h->n_max, Ns, W, 0, X, U, tf, fuel, status, scp_iters,
                                               pipg_iters, nullptr, nullptr);
  }
  PDG_CUDA(h, cudaGetLastError());
  h->last_threads = T;
  h->last_smem = (int)smem;
  h->last_variant = pl.pv;
  return 0;
}

template <int NU>
static int run_grad(pdg_handle* h, int B, const double* x0, const int* Ns, const double* gf, const double* gt,
                    double* grad, double* fuel_out, double* touch_out, int* status_out, cudaStream_t s) {
  const int Tg = 256;
  const Lay Lg = make_lay(h->n_max, NU, Tg);
  const AdjLay Ag = make_adj(Lg, NU, Tg, false);
  const size_t smem_g = (size_t)Ag.total * sizeof(double);
  // the tangent kernel: as many groups of one evaluator and NX + 2 nu columns
  // as fit in 256 threads, and their dual-number stage buffers after the record
  constexpr int PER = NX + 2 * NU + 1;
  const int Tt = (256 / PER) * PER;
  const int tang_off = (tangent_rec_size(NU) + 1) & ~1;
  const size_t smem_t = sizeof(double) * ((size_t)tang_off + 2 * (size_t)(256 / PER) * (SA_A + NX * NU + 3 * NX));
  if (smem_g > 232448) return fail(h, PDG_EINVAL, "gradient kernel does not fit in shared memory for this n_max");
  if (h->p.rk4_substeps > 32) return fail(h, PDG_EINVAL, "gradients support at most 32 RK4 substeps");
  const int ss = Ag.ss;
  const int nck_max = (h->p.pipg_jmax + 49) / 50;
  // With the shared-memory PIPG form the solve itself records the last PIPG
  // loop's checkpoints and final iterate (k_persistent's CK instantiation);
  // otherwise k_grad reruns that loop forward and writes the checkpoints.
  Plan pl;
  std::string why;
  if (!plan_for(h, h->n_max, &pl, &why)) return fail(h, PDG_EINVAL, why);
  const bool ckrec = pl.pv == 1;
  const int rec_stride = h->n_max * (NX + NU) + (Lg.img - Lg.xh) + 2 +
                         (ckrec ? h->n_max * (NX + NU) + nck_max * ss : 0);
  // per instance: [checkpoints of the state every 50 iterations,] one segment's records
  const long long ck_stride = (ckrec ? 0LL : (long long)nck_max * ss) + 50LL * Ag.sg;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bX = sizeof(double) * (size_t)B * h->n_max * NX, bU = sizeof(double) * (size_t)B * h->n_max * NU;
  const size_t bB = sizeof(double) * B, bI = sizeof(int) * B, bL = sizeof(long long) * B;
  const size_t bR = sizeof(double) * (size_t)B * rec_stride, bC = sizeof(double) * (size_t)B * ck_stride;
  const size_t bT = sizeof(double) * (size_t)B * tangent_rec_size(NU);
  const size_t need = al(bX) + al(bU) + 2 * al(bB) + 2 * al(bI) + al(bL) + al(bR) + al(bC) + al(bT);
  if (h->gws_bytes < need) {
    if (h->gws) cudaFree(h->gws);
    h->gws = nullptr;
    h->gws_bytes = 0;
    PDG_CUDA(h, cudaMalloc(&h->gws, need));
    h->gws_bytes = need;
  }
  char* c = (char*)h->gws;
  double* X = (double*)c; c += al(bX);
  double* U = (double*)c; c += al(bU);
  double* tf = (double*)c; c += al(bB);
  double* fu = (double*)c; c += al(bB);
  int* st = (int*)c; c += al(bI);
  int* sc = (int*)c; c += al(bI);
  long long* pi = (long long*)c; c += al(bL);
  double* rec = (double*)c; c += al(bR);
  double* tgr = (double*)c; c += al(bT);
  double* ck = (double*)c;
  h->rec_ptr = rec;
  h->rec_stride = rec_stride;
  h->ck_rec = ckrec;
  int rc = run_solve<double, NU>(h, B, x0, Ns, 1, X, U, tf, fu, st, sc, pi, nullptr, s);
  h->rec_ptr = nullptr;
  h->rec_stride = 0;
  h->ck_rec = false;
  if (rc) return rc;
  PDG_CUDA(h, cudaFuncSetAttribute(k_grad<NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_g));
  k_grad<NU><<<B, Tg, smem_g, s>>>(h->dp, B, h->n_max, x0, Ns, rec, rec_stride, st, gf, gt, ck, ck_stride, nck_max,
                                   ckrec ? 1 : 0, tgr, fuel_out, touch_out);
  PDG_CUDA(h, cudaGetLastError());
  PDG_CUDA(h, cudaFuncSetAttribute(k_grad_tangent<NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t));
  k_grad_tangent<NU><<<B, Tt, smem_t, s>>>(h->dp, B, h->n_max, Ns, st, tgr, grad);
  PDG_CUDA(h, cudaGetLastError());
  if (status_out) PDG_CUDA(h, cudaMemcpyAsync(status_out, st, sizeof(int) * B, cudaMemcpyDeviceToDevice, s));
  return 0;
}

#define PDG_DISPATCH(h, fn, ...)                                         \
  ((h)->p.precision == 0                                                 \
       ? ((h)->p.nu == 4 ? fn<double, 4>(__VA_ARGS__) : fn<double, PDG_MODEL_NU_ALT>(__VA_ARGS__)) \
       : ((h)->p.nu == 4 ? fn<float, 4>(__VA_ARGS__) : fn<float, PDG_MODEL_NU_ALT>(__VA_ARGS__)))

extern "C" {

int pdg_mc_init(const pdg_params* p, int n_max, pdg_handle** out) {
  if (!out) { g_init_err = "out is NULL"; return PDG_EINVAL; }
  *out = nullptr;
  if (!p) { g_init_err = "params is NULL"; return PDG_EINVAL; }
  if (n_max < 2 || n_max > NMAX) { g_init_err = "n_max must be in [2, 32]"; return PDG_EINVAL; }
  DParams d;
  std::string why;
  if (!fill_dparams(p, &d, &why)) { g_init_err = why; return PDG_EINVAL; }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { g_init_err = std::string("no usable CUDA device: ") + cudaGetErrorString(e); return PDG_ECUDA; }
  pdg_handle* h = new (std::nothrow) pdg_handle();
  if (!h) { g_init_err = "out of host memory"; return PDG_ENOMEM; }
  h->p = *p;
  h->dp = d;
  h->n_max = n_max;
  h->threads_override = 0;
  h->device = dev;
  h->num_sms = sms;
  {
    void* dptr = nullptr;
    cudaError_t ea = cudaHostAlloc((void**)&h->abort_host, sizeof(int), cudaHostAllocMapped);
    if (ea == cudaSuccess) {
      __atomic_store_n(h->abort_host, 0, __ATOMIC_SEQ_CST);
      ea = cudaHostGetDevicePointer(&dptr, h->abort_host, 0);
    }
    if (ea != cudaSuccess) {
      if (h->abort_host) cudaFreeHost(h->abort_host);
      delete h;
      g_init_err = std::string("abort word (mapped pinned host memory): ") + cudaGetErrorString(ea);
      return PDG_ECUDA;
    }
    h->dp.abort_flag = static_cast<const int*>(dptr);
  }
  *out = h;
  g_init_err.clear();
  return PDG_OK;
}

void pdg_mc_destroy(pdg_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->img) cudaFree(h->img);
  if (h->ints) cudaFree(h->ints);
  if (h->lit) cudaFree(h->lit);
  if (h->stage) cudaFree(h->stage);
  if (h->gws) cudaFree(h->gws);
  if (h->cls) cudaFree(h->cls);
  for (int i = 0; i <= NMAX; ++i) {
    if (h->cls_streams[i]) cudaStreamDestroy(h->cls_streams[i]);
    if (h->cls_events[i]) cudaEventDestroy(h->cls_events[i]);
  }
  if (h->pinned_done) cudaFreeHost(h->pinned_done);
  if (h->abort_host) cudaFreeHost(h->abort_host);
  if (h->plain_exec) cudaGraphExecDestroy(h->plain_exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  delete h;
}

const char* pdg_mc_last_error(const pdg_handle* h) { return h ? h->err.c_str() : g_init_err.c_str(); }

int pdg_mc_abort(pdg_handle* h) {
  if (!h) return PDG_EINVAL;
  __atomic_store_n(h->abort_host, 1, __ATOMIC_SEQ_CST);
  return PDG_OK;
}

int pdg_mc_clear_abort(pdg_handle* h) {
  if (!h) return PDG_EINVAL;
  __atomic_store_n(h->abort_host, 0, __ATOMIC_SEQ_CST);
  return PDG_OK;
}

int pdg_mc_solve_batch(pdg_handle* h, int B, const double* x0, const int* n_nodes, int mode, double* X, double* U,
                       double* tf, double* fuel, int* status, int* scp_iters, long long* pipg_iters, int* trace,
                       void* cuda_stream) {
  if (!h) return PDG_EINVAL;
  h->err.clear();
  if (B < 0) return fail(h, PDG_EINVAL, "B must be >= 0");
  if (B == 0) return PDG_OK;
  if (mode < 0 || mode > 2) return fail(h, PDG_EINVAL, "mode must be 0 (plain), 1 (persistent) or 2 (persistent, shape classes)");
  if (!x0 || !X || !U || !tf || !fuel || !status || !scp_iters || !pipg_iters) return fail(h, PDG_EINVAL, "NULL buffer");
  PDG_CUDA(h, cudaSetDevice(h->device));
  NvtxRange r(mode == 0 ? "pdg_mc_solve_batch plain" : mode == 1 ? "pdg_mc_solve_batch persistent"
                                                                   : "pdg_mc_solve_batch shape classes");
  return PDG_DISPATCH(h, run_solve, h, B, x0, n_nodes, mode, X, U, tf, fuel, status, scp_iters, pipg_iters, trace,
                      (cudaStream_t)cuda_stream);
}

int pdg_mc_solve_batch_host(pdg_handle* h, int B, const double* x0, const int* n_nodes, int mode, double* X,
                            double* U, double* tf, double* fuel, int* status, int* scp_iters, long long* pipg_iters,
                            void* cuda_stream) {
  if (!h) return PDG_EINVAL;
  h->err.clear();
  if (B < 0) return fail(h, PDG_EINVAL, "B must be >= 0");
  if (B == 0) return PDG_OK;
  if (!x0 || !X || !U || !tf || !fuel || !status || !scp_iters || !pipg_iters) return fail(h, PDG_EINVAL, "NULL buffer");
  PDG_CUDA(h, cudaSetDevice(h->device));
  const int nu = h->p.nu, Nm = h->n_max;
  const size_t bx0 = sizeof(double) * (NX - 1) * B, bN = sizeof(int) * B, bX = sizeof(double) * (size_t)B * Nm * NX,
               bU = sizeof(double) * (size_t)B * Nm * nu, bs = sizeof(double) * B, bi = sizeof(int) * B,
               bl = sizeof(long long) * B;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t need = al(bx0) + al(bN) + al(bX) + al(bU) + 2 * al(bs) + 2 * al(bi) + al(bl);
  if (h->stage_bytes < need) {
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    PDG_CUDA(h, cudaMalloc(&h->stage, need));
    h->stage_bytes = need;
  }
  char* c = (char*)h->stage;
  double* dx0 = (double*)c; c += al(bx0);
  int* dN = (int*)c; c += al(bN);
  double* dX = (double*)c; c += al(bX);
  double* dU = (double*)c; c += al(bU);
  double* dtf = (double*)c; c += al(bs);
  double* dfu = (double*)c; c += al(bs);
  int* dst = (int*)c; c += al(bi);
  int* dsc = (int*)c; c += al(bi);
  long long* dpi = (long long*)c;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  NvtxRange r("pdg_mc_solve_batch_host");
  PDG_CUDA(h, cudaMemcpyAsync(dx0, x0, bx0, cudaMemcpyHostToDevice, s));
  if (n_nodes) PDG_CUDA(h, cudaMemcpyAsync(dN, n_nodes, bN, cudaMemcpyHostToDevice, s));
  int rc = pdg_mc_solve_batch(h, B, dx0, n_nodes ? dN : nullptr, mode, dX, dU, dtf, dfu, dst, dsc, dpi, nullptr, s);
  if (rc) return rc;
  PDG_CUDA(h, cudaMemcpyAsync(X, dX, bX, cudaMemcpyDeviceToHost, s));
  PDG_CUDA(h, cudaMemcpyAsync(U, dU, bU, cudaMemcpyDeviceToHost, s));
  PDG_CUDA(h, cudaMemcpyAsync(tf, dtf, bs, cudaMemcpyDeviceToHost, s));
  PDG_CUDA(h, cudaMemcpyAsync(fuel, dfu, bs, cudaMemcpyDeviceToHost, s));
  PDG_CUDA(h, cudaMemcpyAsync(status, dst, bi, cudaMemcpyDeviceToHost, s));
  PDG_CUDA(h, cudaMemcpyAsync(scp_iters, dsc, bi, cudaMemcpyDeviceToHost, s));
  PDG_CUDA(h, cudaMemcpyAsync(pipg_iters, dpi, bl, cudaMemcpyDeviceToHost, s));
  PDG_CUDA(h, cudaStreamSynchronize(s));
  return PDG_OK;
}

int pdg_mc_subproblem(pdg_handle* h, int B, const double* x0, const int* n_nodes, const double* X, const double* U,
                      double* Am, double* Bm, double* Bp, double* w, void* cuda_stream) {
  if (!h) return PDG_EINVAL;
  h->err.clear();
  if (B < 0) return fail(h, PDG_EINVAL, "B must be >= 0");
  if (B == 0) return PDG_OK;
  if (!x0 || !X || !U || !Am || !Bm || !Bp || !w) return fail(h, PDG_EINVAL, "NULL buffer");
  PDG_CUDA(h, cudaSetDevice(h->device));
  return PDG_DISPATCH(h, run_subproblem, h, B, x0, n_nodes, X, U, Am, Bm, Bp, w, (cudaStream_t)cuda_stream);
}

int pdg_mc_scp_step(pdg_handle* h, int B, const double* x0, const int* n_nodes, double* X, double* U, double* xh,
                    double* uh, double* mup, double* mum, double* phi, double* th, const int* force, double* sigma,
                    double* defect, double* step, int* iters, void* cuda_stream) {
  if (!h) return PDG_EINVAL;
  h->err.clear();
  if (B < 0) return fail(h, PDG_EINVAL, "B must be >= 0");
  if (B == 0) return PDG_OK;
  if (!x0 || !X || !U || !xh || !uh || !mup || !mum || !phi || !th || !sigma || !defect || !step || !iters)
    return fail(h, PDG_EINVAL, "NULL buffer");
  PDG_CUDA(h, cudaSetDevice(h->device));
  return PDG_DISPATCH(h, run_step, h, B, x0, n_nodes, X, U, xh, uh, mup, mum, phi, th, force, sigma, defect, step,
                      iters, (cudaStream_t)cuda_stream);
}

int pdg_mc_launch_info(pdg_handle* h, int* threads, int* ctas_per_sm, int* smem_bytes) {
  if (!h) return PDG_EINVAL;
  if (threads) *threads = h->last_threads;
  if (ctas_per_sm) *ctas_per_sm = h->last_ctas;
  if (smem_bytes) *smem_bytes = h->last_smem;
  return PDG_OK;
}

int pdg_mc_set_pipg_form(pdg_handle* h, int form) {
  if (!h) return PDG_EINVAL;
  if (form < 0 || form > 3)
    return fail(h, PDG_EINVAL, "PIPG form must be 0 (auto), 1 (shared memory), 2 (registers) or 3 (register tiles)");
  h->pipg_variant = form;
  return PDG_OK;
}

int pdg_mc_pipg_form(const pdg_handle* h) { return h ? h->last_variant : PDG_EINVAL; }

int pdg_mc_autotune(pdg_handle* h, int B, const double* x0, const int* n_nodes, int mode, int* threads_out,
                    int* form_out, double* solves_per_s, void* cuda_stream) {
  if (!h) return PDG_EINVAL;
  h->err.clear();
  if (B < 1 || !x0) return fail(h, PDG_EINVAL, "autotune needs B >= 1 and x0");
  if (mode < 0 || mode > 2) return fail(h, PDG_EINVAL, "mode must be 0, 1 or 2");
  PDG_CUDA(h, cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nu = h->p.nu, n = h->n_max;
  // caller-invisible outputs of the trial solves
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bX = sizeof(double) * (size_t)B * n * NX, bU = sizeof(double) * (size_t)B * n * nu;
  const size_t need = al(bX) + al(bU) + 2 * al(sizeof(double) * B) + 2 * al(sizeof(int) * B) + al(sizeof(long long) * B);
  char* buf = nullptr;
  PDG_CUDA(h, cudaMalloc(&buf, need));
  char* c = buf;
  double* X = (double*)c; c += al(bX);
  double* U = (double*)c; c += al(bU);
  double* tf = (double*)c; c += al(sizeof(double) * B);
  double* fu = (double*)c; c += al(sizeof(double) * B);
  int* st = (int*)c; c += al(sizeof(int) * B);
  int* sc = (int*)c; c += al(sizeof(int) * B);
  long long* pi = (long long*)c;
  int* hst = (int*)malloc(sizeof(int) * B);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int keep_t = h->threads_override, keep_f = h->pipg_variant;
  double best = -1.0;
  int best_t = 0, best_f = 0, rc = PDG_OK;
  const int treg = pipg_reg_threads(n, nu), maxt = h->p.precision == 1 ? PDG_REG_MAXT_F32 : 512;
  const int tks = pipg_ks_threads(n);
  // candidates: (form 1, 128..512), (form 2, its minimum .. its limit) and
  // (form 3, its minimum .. 512), multiples of 32
  for (int form = 1; form <= 3 && rc == PDG_OK; ++form) {
    const int t_lo = form == 1 ? 128 : (form == 2 ? treg : tks);
    const int t_hi = form == 2 ? maxt : (form == 3 && h->p.precision == 1 ? PDG_KS_PERS_MAXT : 512);
    for (int T = t_lo; T <= t_hi && rc == PDG_OK; T += 32) {
      h->pipg_variant = form;
      h->threads_override = T;
      // a candidate that does not fit (shared memory, threads) is skipped
      if (pdg_mc_solve_batch(h, B, x0, n_nodes, mode, X, U, tf, fu, st, sc, pi, nullptr, s) != PDG_OK) {
        h->err.clear();
        if (cudaGetLastError() != cudaSuccess) { rc = fail(h, PDG_ECUDA, "autotune: CUDA error after a skipped candidate"); }
        continue;
      }
      if (cudaEventRecord(e0, s) != cudaSuccess) { rc = fail(h, PDG_ECUDA, "autotune: event"); break; }
      int r2 = pdg_mc_solve_batch(h, B, x0, n_nodes, mode, X, U, tf, fu, st, sc, pi, nullptr, s);
      if (r2 != PDG_OK) { rc = r2; break; }
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess ||
          cudaMemcpy(hst, st, sizeof(int) * B, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = fail(h, PDG_ECUDA, "autotune: timing or status copy failed");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      int conv = 0;
      for (int b = 0; b < B; ++b) conv += hst[b] == PDG_CONVERGED;
      const double rate = ms > 0 ? conv / (ms * 1e-3) : 0.0;
      if (rate > best) { best = rate; best_t = T; best_f = form; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free(hst);
  cudaFree(buf);
  if (rc != PDG_OK || best_t == 0) {
    h->threads_override = keep_t;
    h->pipg_variant = keep_f;
    return rc != PDG_OK ? rc : fail(h, PDG_EINVAL, "autotune: no candidate ran");
  }
  h->threads_override = best_t;
  h->pipg_variant = best_f;
  if (threads_out) *threads_out = best_t;
  if (form_out) *form_out = best_f;
  if (solves_per_s) *solves_per_s = best;
  return PDG_OK;
}

int pdg_mc_set_threads(pdg_handle* h, int threads) {
  if (!h) return PDG_EINVAL;
  if (threads < 0 || threads > PDG_REG_MAXT_F32 || (threads % 32) != 0)
    return fail(h, PDG_EINVAL, "threads must be 0 or a multiple of 32 up to " + std::to_string(PDG_REG_MAXT_F32));
  h->threads_override = threads;
  return PDG_OK;
}

int pdg_mc_solve_batch_noalloc(pdg_handle* h, int B, const double* x0, const int* n_nodes, double* X, double* U,
                               double* tf, double* fuel, int* status, int* scp_iters, long long* pipg_iters,
                               void* cuda_stream) {
  if (!h) return PDG_EINVAL;
  h->err.clear();
  if (B < 0) return fail(h, PDG_EINVAL, "B must be >= 0");
  if (B == 0) return PDG_OK;
  if (!x0 || !X || !U || !tf || !fuel || !status || !scp_iters || !pipg_iters) return fail(h, PDG_EINVAL, "NULL buffer");
  PDG_CUDA(h, cudaSetDevice(h->device));
  return PDG_DISPATCH(h, run_noalloc, h, B, x0, n_nodes, X, U, tf, fuel, status, scp_iters, pipg_iters,
                      (cudaStream_t)cuda_stream);
}

int pdg_mc_grad_batch(pdg_handle* h, int B, const double* x0, const int* n_nodes, const double* dL_dfuel,
                      const double* dL_dtouch, double* grad_x0, double* fuel, double* touch, int* status,
                      void* cuda_stream) {
  if (!h) return PDG_EINVAL;
  h->err.clear();
  if (B < 0) return fail(h, PDG_EINVAL, "B must be >= 0");
  if (B == 0) return PDG_OK;
  if (!x0 || !grad_x0) return fail(h, PDG_EINVAL, "NULL buffer");
  if (h->p.precision != 0) return fail(h, PDG_EINVAL, "gradients are computed in FP64 only (precision 0)");
  if (h->p.soc_thrust) return fail(h, PDG_EINVAL, "gradients are not available with soc_thrust");
  PDG_CUDA(h, cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  return h->p.nu == 4 ? run_grad<4>(h, B, x0, n_nodes, dL_dfuel, dL_dtouch, grad_x0, fuel, touch, status, s)
                      : run_grad<PDG_MODEL_NU_ALT>(h, B, x0, n_nodes, dL_dfuel, dL_dtouch, grad_x0, fuel, touch, status, s);
}

static int probe_fma_run(int precision, int active, double* best_ms, long long* lane_fma, void* cuda_stream) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PDG_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int threads = 512, blocks = sms * 4;
  const int iters = precision == 0 ? 1 << 14 : 1 << 18;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 16) != cudaSuccess) return PDG_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    if (precision == 0) k_fma_probe<double><<<blocks, threads, 0, s>>>(iters, active, 1.0, (double*)buf);
    else k_fma_probe<float><<<blocks, threads, 0, s>>>(iters, active, 1.0f, (float*)buf);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return PDG_ECUDA;
  *best_ms = best;
  *lane_fma = 8LL * iters * blocks * threads;
  return PDG_OK;
}

int pdg_mc_probe_fma(int precision, double* tflops, void* cuda_stream) {
  if (!tflops || (precision != 0 && precision != 1)) return PDG_EINVAL;
  double ms = 0;
  long long n = 0;
  if (int rc = probe_fma_run(precision, 32, &ms, &n, cuda_stream)) return rc;
  *tflops = 2.0 * (double)n / (ms * 1e-3) / 1e12;
  return PDG_OK;
}

int pdg_mc_model_nx(void) { return NX; }

int pdg_mc_probe_fma_lanes(int precision, int active_lanes, double* ms, void* cuda_stream) {
  if (!ms || (precision != 0 && precision != 1) || active_lanes < 1 || active_lanes > 32) return PDG_EINVAL;
  long long n = 0;
  return probe_fma_run(precision, active_lanes, ms, &n, cuda_stream);
}

}  // extern "C"
