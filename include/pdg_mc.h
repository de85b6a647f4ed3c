/*
 * pdg_mc.h -- C ABI of the batched GB300 solver for Monte Carlo 6-DoF
 * powered-descent guidance (arXiv 2404.18034).
 *
 * Each instance is a free-final-time 6-DoF landing problem (Sec. 4) solved by
 * prox-linear sequential convex programming (Sec. 2.3, Eq. cvx-subproblem)
 * with the CTCS reformulation (Sec. 2.1, Eq. sys-dyn-dil-aug).  Every SCP
 * iteration discretizes the augmented dynamics with their state-transition
 * matrices (Sec. 2.3.1), prescales the subproblem (Sec. 2.3.2), estimates the
 * step size by the customized power iteration (Alg. power) and solves the
 * subproblem by customized PIPG (Alg. PIPG_custom with Alg. stopping).
 *
 * Models.  The problem template of Sec. 2 (dynamics F, path constraints g,
 * boundary conditions, Mayer cost) is instantiated by a model fixed when the
 * library is compiled, and every entry point below has the same meaning in
 * each library:
 *   libpdg_mc.so       the 6-DoF model of Sec. 4, state size NX = 15;
 *   libpdg_mc_3dof.so  the translational 3-DoF model, NX = 8: the 6-DoF model
 *                      without attitude, thrust in the inertial frame, nu = 4,
 *                      path rows m_dry, altitude, v_max, thrust pointing within
 *                      delta_max of the up axis, T_min/T_max, optional glide
 *                      slope.  J_B, r_T_B, theta_max, omega_max and gamma_max
 *                      are not read.
 * pdg_mc_model_nx() returns the library's NX.  A library for another model is
 * built from a user header passed as -DPDG_MODEL_HEADER="<path>" that defines
 * the same model interface (see csrc/pdg_device.cuh); its constants come in
 * through pdg_params.model_params.
 *
 * Conventions
 *   - Layouts are row-major, double precision, instance-major:
 *       x0[B][NX-1]          6-DoF: (m_wet, r[3], v[3], q[4] scalar first, w[3]);
 *                            3-DoF: (m_wet, r[3], v[3])
 *       X[B][n_max][NX]      6-DoF: (m, r, v, q, w, y); 3-DoF: (m, r, v, y);
 *                            y is the CTCS integrator
 *       U[B][n_max][nu]      (T[3], s) for nu = 4; (T[3], gamma[3], s) for nu = 7
 *     Rows k >= n_nodes[b] of X and U are written as zero.  Arrays of
 *     pdg_params indexed like x hold 15 entries; a library reads its first NX.
 *   - Pointers named "device" must point to device memory of the current
 *     device; the caller owns every buffer it passes.  The handle owns its
 *     workspace (allocated by pdg_mc_init and grown on demand).
 *   - All calls are asynchronous on the given CUDA stream (NULL: the legacy
 *     default stream) unless stated otherwise.
 *   - Return 0 on success, a negative PDG_E* code on error; the message is
 *     available from pdg_mc_last_error.  Per-instance solver outcomes are in
 *     status[], never in the return code.  Nothing throws across the ABI.
 *   - precision = 1 computes in FP32 (inputs and outputs stay double).
 */
#ifndef PDG_MC_H
#define PDG_MC_H

#ifdef __cplusplus
extern "C" {
#endif

#define PDG_OK 0
#define PDG_EINVAL (-1)   /* bad argument */
#define PDG_ENOMEM (-2)   /* device allocation failed */
#define PDG_ECUDA (-3)    /* CUDA runtime error */

/* per-instance status */
#define PDG_CONVERGED 0
#define PDG_MAX_SCP 1     /* SCP iteration cap reached without convergence */
#define PDG_NONFINITE 2   /* a non-finite value appeared */
#define PDG_BUDGET 3      /* the device-side wall-clock budget ran out */
#define PDG_BAD_INPUT 4   /* n_nodes out of range or non-finite x0 */
#define PDG_ABORTED 5     /* stopped by pdg_mc_abort at an SCP iteration boundary */

/* Problem and solver parameters; angles in radians.  Sec. 4 lists the model
 * quantities, Sec. 2.3.2 the scalings P_x, P_u and Sec. 3 the PIPG inputs. */
typedef struct pdg_params {
  int nu;                 /* 4 or 7 */
  int precision;          /* 0 = FP64, 1 = FP32 */
  double alpha_mdot;      /* mass depletion per unit thrust magnitude */
  double g_I[3];          /* gravity (inertial) */
  double J_B[3];          /* diagonal inertia */
  double r_T_B[3];        /* thrust point (body) */
  double m_dry, v_max, theta_max, omega_max, delta_max, T_min, T_max, gamma_max;
  double s_min, s_max;    /* dilation bounds (the only control box) */
  double z_f[15];         /* final targets, indexed as x */
  int fix_f[15];          /* 1 where the final component is fixed (E_f) */
  double P_x[15], P_u[7]; /* diagonal scalings */
  double w_cost, w_prox, w_ep, eps_ctcs;
  double pipg_omega, pipg_rho, pipg_eps_abs, pipg_eps_rel;
  int pipg_jmax, pipg_jcheck;
  double pow_eps_abs, pow_eps_rel, pow_eps_buff;
  int pow_jmax;
  int scp_jmax;
  double scp_eps_step, scp_eps_defect;
  int rk4_substeps;
  double tf_guess;        /* dilation of the initial guess */
  double budget_seconds;  /* device wall-clock cap per instance (persistent forms); 0 = none */
  int soc_thrust;         /* 1: T_max and the gimbal cone as a per-node projection of the
                             thrust onto {||T|| <= T_max, ||T|| cos(delta_max) <= T_x}
                             inside PIPG (second-order cone then ball, Alg. 1's
                             projection step) instead of CTCS rows; needs P_u equal on
                             the three thrust components; no gradients */
  int glide_slope;        /* 1: add the glide-slope row tan^2(gamma_gs) (r_y^2 + r_z^2) - r_x^2
                             <= 0 to g (CTCS), the bound gamma_gs named in Sec. 4 */
  double gamma_gs;        /* glide-slope angle from the horizontal (rad), in (0, pi/2) */
  double dt_min, dt_max, tf_max;  /* Sec. 2.2 time bounds, 0 = off: imposed as the node box
                             s_k in [dt_min (N-1), min(dt_max (N-1), tf_max)] on the
                             dilation (sufficient for FOH s) */
  double model_params[16]; /* constants of a model supplied at build time through
                             PDG_MODEL_HEADER (read by its device code as P.mp[i]);
                             the built-in models do not read them */
} pdg_params;

typedef struct pdg_handle pdg_handle;

/* Create a solver for instances of at most n_max nodes (2 <= n_max <= 32)
 * on the current device.  Copies *p; validates it (PDG_EINVAL on nonsense).
 * Allocates nothing large; workspaces grow on first use. */
int pdg_mc_init(const pdg_params* p, int n_max, pdg_handle** out);

/* Release the handle and its device workspace (synchronizes the device). */
void pdg_mc_destroy(pdg_handle* h);

/* Last error message of this handle ("" if none).  With h == NULL, the last
 * error of pdg_mc_init. */
const char* pdg_mc_last_error(const pdg_handle* h);

/* Abort request (failure handling; no counterpart in the paper).  Sets the
 * handle's abort word, a word of pinned host memory that pdg_mc_init maps into
 * the device's address space.  Safe to call from any host thread, also while
 * a solve of this handle runs on the GPU; it returns at once and waits for
 * nothing.  Every solve of the handle reads the word at each SCP iteration
 * boundary (the persistent forms once per CTA before each SCP iteration; the
 * plain form and the no-allocation entry point once per instance in each SCP
 * iteration's kernels) and never waits on it: an instance still running stops
 * there with status PDG_ABORTED, X and U holding its trajectory after the
 * scp_iters SCP iterations it completed, and instances not yet started stop
 * before their first iteration (scp_iters 0, X and U the initial guess).
 * The request stays set, and later solves abort at once, until
 * pdg_mc_clear_abort.  Gradients of aborted instances are zero.  Returns
 * PDG_EINVAL for a NULL handle. */
int pdg_mc_abort(pdg_handle* h);

/* Clear the abort request.  Make sure no solve of the handle is running, or
 * it may see either value.  Returns PDG_EINVAL for a NULL handle. */
int pdg_mc_clear_abort(pdg_handle* h);

/* Solve B instances (Sec. 2.3 SCP loop; all of Sec. 2.3.1-3 per iteration).
 *   x0        device [B][NX-1]
 *   n_nodes   device [B] (2..n_max) or NULL for n_max everywhere
 *   mode      0: plain form, one launch per phase per SCP iteration, the
 *                iteration captured once in a CUDA graph and replayed;
 *             1: persistent form, one launch, each CTA takes instances from
 *                a work queue until none is left;
 *             2: persistent form by shape class: the instances are sorted by
 *                node count on the device and every node count gets its own
 *                persistent grid (shared memory and CTA size for that count),
 *                all grids running concurrently on forked streams.  Same as
 *                mode 1 when n_nodes is NULL.
 *   X, U      device outputs (see layouts)
 *   tf, fuel  device [B]: final time sum_k dtau (s_k + s_{k+1})/2 and m_1 - m_N
 *   status    device [B] PDG_CONVERGED ... PDG_ABORTED
 *   scp_iters device [B]; pipg_iters device [B] (sum over SCP iterations)
 *   trace     device [B][scp_jmax][2] (power iterations, PIPG iterations per
 *             SCP iteration; zero past the last) or NULL
 * The plain form synchronizes the stream once per SCP iteration to stop early
 * when every instance is done. */
int pdg_mc_solve_batch(pdg_handle* h, int B, const double* x0, const int* n_nodes, int mode,
                       double* X, double* U, double* tf, double* fuel, int* status,
                       int* scp_iters, long long* pipg_iters, int* trace, void* cuda_stream);

/* Same as pdg_mc_solve_batch with HOST buffers (pageable or pinned): copies
 * x0 / n_nodes in and the outputs back through handle-owned device buffers on
 * the stream, and returns after the stream has drained. */
int pdg_mc_solve_batch_host(pdg_handle* h, int B, const double* x0, const int* n_nodes, int mode,
                            double* X, double* U, double* tf, double* fuel, int* status,
                            int* scp_iters, long long* pipg_iters, void* cuda_stream);

/* Scaled subproblem data about a reference (X, U) (Sec. 2.3.1 STM IVP by RK4
 * with rk4_substeps substeps per interval, then the prescaling of Sec. 2.3.2):
 *   Am  device [B][n_max-1][NX][NX]   hat A^-_k = P_x^-1 A_k P_x
 *   Bm  device [B][n_max-1][NX][nu]   hat B^-_k = P_x^-1 B^-_k P_u
 *   Bp  device [B][n_max-1][NX][nu]   hat B^+_k
 *   w   device [B][n_max-1][NX]       hat w_k = P_x^-1 (xbar^k(tau_{k+1}) - xbar_{k+1})
 * Inputs x0, n_nodes, X, U as above (device).  Rows past n_nodes-1 are zero. */
int pdg_mc_subproblem(pdg_handle* h, int B, const double* x0, const int* n_nodes,
                      const double* X, const double* U,
                      double* Am, double* Bm, double* Bp, double* w, void* cuda_stream);

/* One SCP iteration in place (plain-form kernels): discretize and scale about
 * (X, U), power iteration, PIPG_custom warm-started from (xh, uh, mup, mum,
 * phi, th), then X += P_x xh, U += P_u uh.  Device buffers:
 *   X [B][n_max][NX], U [B][n_max][nu]         reference in / updated out
 *   xh [B][n_max][NX], uh [B][n_max][nu], mup, mum, phi [B][n_max-1][NX],
 *   th [B][n_max-1]                             warm start in / solution out
 *   force [B][2] (power, PIPG) iteration counts to run exactly, or NULL
 *   sigma [B], defect [B] (max |hat w|), step [B] (max |xh|, |uh|) outputs
 *   iters [B][2] (power, PIPG) outputs. */
int pdg_mc_scp_step(pdg_handle* h, int B, const double* x0, const int* n_nodes,
                    double* X, double* U, double* xh, double* uh, double* mup, double* mum,
                    double* phi, double* th, const int* force,
                    double* sigma, double* defect, double* step, int* iters, void* cuda_stream);

/* One-step gradients of the converged outputs with respect to the initial
 * state and wet mass (FP64 handles only).  Solves the batch (persistent form),
 * then differentiates the solve's last SCP iteration as a function of x0 -- the
 * reference's first node moving with x0, the rest of that iteration's
 * reference, its PIPG warm start, step size and iteration count held --
 * through the RK4 discretization of the first interval (Sec. 2.3.1, forward
 * mode), the prescaling (Sec. 2.3.2) and the final PIPG_custom loop (reverse
 * mode, recomputed from checkpoints every 50 iterations, projections masked as
 * in the forward pass).  The paper has no gradient; this definition is the
 * solver's own.  It is not the total derivative through the SCP fixed point:
 * the earlier iterations' dependence on x0 is not followed.  Device buffers:
 *   dL_dfuel, dL_dtouch [B]  upstream cotangents (NULL = zero)
 *   grad_x0 [B][NX-1]        d L / d x0 (6-DoF: m_wet, r, v, q, w), with
 *                            L = dL_dfuel fuel + dL_dtouch touchdown
 *   fuel [B], touch [B]      outputs (NULL = not written): fuel = m_1 - m_N and
 *                            touchdown = 0.5 sum_{E_f} ((x_prop,N - z_f)/P_x)^2,
 *                            x_prop,N the RK4 propagation of the last interval
 *   status [B]               solve status (NULL = not written); instances that
 *                            end non-finite or with bad input get zero gradient
 * The handle's gradient workspace (grown on demand, kept until destroy) holds,
 * per instance, the last SCP iteration's record with its PIPG checkpoints and
 * one 50-iteration segment of the adjoint's records: about 0.7 MB at
 * n_max = 15 and pipg_jmax = 2000 (2.8 GB for 4096 instances). */
int pdg_mc_grad_batch(pdg_handle* h, int B, const double* x0, const int* n_nodes,
                      const double* dL_dfuel, const double* dL_dtouch, double* grad_x0,
                      double* fuel, double* touch, int* status, void* cuda_stream);

/* Shape of the last launch configuration chosen for (n_max, nu, precision):
 * threads per CTA, CTAs per SM and dynamic shared memory per CTA (bytes).
 * Synchronous; no device work. */
int pdg_mc_launch_info(pdg_handle* h, int* threads, int* ctas_per_sm, int* smem_bytes);

/* Override the threads-per-CTA of the solve kernels (multiple of 32 up to
 * 576, 0 = automatic).  Used by the autotuner.  PIPG forms 1 and 3 run at
 * most 512; forms 2 and 3 need a minimum (see pdg_mc_set_pipg_form); a solve
 * whose setting does not fit returns PDG_EINVAL. */
int pdg_mc_set_threads(pdg_handle* h, int threads);

/* Autotune the launch shape for this handle's n_max, nu and precision on a
 * caller batch (no counterpart in the paper).  Times one solve of the batch
 * (device x0 [B][NX-1], n_nodes as in pdg_mc_solve_batch, execution mode 0/1/2)
 * for every candidate: PIPG form 1 at 128..512 threads, forms 2 and 3 from
 * the threads they need up to their limits, multiples of 32; candidates that do not
 * fit on an SM are skipped.  Each candidate runs one untimed solve, then one
 * solve timed with CUDA events on cuda_stream, scored by converged solves per
 * second.  The fastest (form, threads) is applied to the handle (as by
 * pdg_mc_set_pipg_form and pdg_mc_set_threads) and written to *threads_out,
 * *form_out, *solves_per_s (each may be NULL).  Allocates and frees its
 * scratch outputs; synchronizes the stream.  Returns PDG_EINVAL for B < 1 or
 * no x0, or when no candidate ran (the handle's settings are then kept). */
int pdg_mc_autotune(pdg_handle* h, int B, const double* x0, const int* n_nodes, int mode, int* threads_out,
                    int* form_out, double* solves_per_s, void* cuda_stream);

/* Choose how the PIPG loop (Alg. PIPG_custom, Sec. 3) is laid out on the
 * CTA.  Results agree to rounding; only speed differs.
 *   form 1: blocks hat A^-, hat B^+- and the iterates in shared memory, any
 *           thread count (one thread per block row or column, looped);
 *   form 2: every thread keeps its block rows/columns and iterate entries in
 *           registers for the whole loop; only the vectors exchanged between
 *           the primal and dual steps go through shared memory.  Needs
 *           round32(NX (N-1)) + round32(N G) threads, G = 4 (nu = 4) or 8,
 *           at most 576 (FP32) or 512 (FP64);
 *   form 3: blocks padded to 16 x 16 (8 x 8 when NX <= 8) and cut into tiles
 *           of 8 rows by 4 (2) columns, one tile per lane, so that a group
 *           of 8 (4) lanes holds one interval's blocks and owns one node;
 *           products run as packed pairs and their partial sums combine
 *           by shuffles within the group.  Needs round32(8 N) threads
 *           (round32(4 N) when NX <= 8), at least 64, at most 512;
 *   form 0: automatic (default) -- form 3 for FP32 when the thread setting
 *           allows it, else form 1.
 * Returns PDG_EINVAL for another value.  Synchronous; no device work. */
int pdg_mc_set_pipg_form(pdg_handle* h, int form);

/* The PIPG form (1, 2 or 3) of the handle's last solve or SCP step, 0 before
 * the first; PDG_EINVAL for a NULL handle. */
int pdg_mc_pipg_form(const pdg_handle* h);

/* Solve without allocating: for callers that cannot call cudaMalloc while
 * they run, e.g. code inside a region that a memory pool or allocator owns,
 * or a host that must not grow its device footprint after start-up.  The
 * paper has no counterpart.  Same arguments, results and status codes as
 * pdg_mc_solve_batch in plain form (mode 0), except: no trace; every SCP
 * iteration up to scp_jmax is launched (finished instances return at once)
 * and the call never synchronizes the stream.  The per-instance workspace
 * lives in a fixed 32 MiB device array that the library defines, so every
 * GPU that loads the library holds those 32 MiB until the process exits (each
 * model library has its own array: a process using both holds 64 MiB).
 *   - Batches that need more than the 32 MiB (about 870 instances at
 *     n_max = 15 in FP64, twice that in FP32) are rejected with PDG_EINVAL
 *     and a message that states the limit; nothing is launched.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture on that device.
 *   - Under CUDA's lazy module loading (the default since CUDA 12) the
 *     library's kernels and this array are put on a device at their first
 *     use there.  If this entry point is that first use, its first call does
 *     that loading, which takes the 32 MiB and the code's memory.  Callers
 *     that must not allocate at all make one call (or one solve of any kind)
 *     during set-up; every later call allocates nothing.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (other streams, other threads) race and corrupt each other.  Serialize
 *     them, e.g. on one stream.
 * Apart from that first loading, no cudaMalloc, cudaFree or other allocating
 * call is made. */
int pdg_mc_solve_batch_noalloc(pdg_handle* h, int B, const double* x0, const int* n_nodes,
                               double* X, double* U, double* tf, double* fuel, int* status,
                               int* scp_iters, long long* pipg_iters, void* cuda_stream);

/* Roofline denominator probe (no counterpart in the paper): runs an FMA-chain
 * kernel on all SMs of the current device in FP64 (precision 0) or FP32 (1)
 * and writes the best of three timed launches, in TFLOP/s, to *tflops.
 * Synchronizes the stream; allocates 16 bytes of device memory. */
int pdg_mc_probe_fma(int precision, double* tflops, void* cuda_stream);

/* The same probe with only the first active_lanes (1..32) lanes of every warp
 * running their chains; writes the best time in milliseconds to *ms.  The
 * number of warp instructions does not depend on active_lanes, so equal times
 * for 1 and 32 lanes show a pipe whose cost is per warp instruction (GB300's
 * FP64 pipe).  PDG_EINVAL for other arguments.  Synchronizes the stream. */
int pdg_mc_probe_fma_lanes(int precision, int active_lanes, double* ms, void* cuda_stream);

/* State size NX of the library's model (15: 6-DoF of Sec. 4; 8: 3-DoF).
 * Needs no device and no handle; the binding checks it against the model it
 * expects before any call. */
int pdg_mc_model_nx(void);

#ifdef __cplusplus
}
#endif
#endif
