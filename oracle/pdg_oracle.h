/*
 * pdg_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, serial, FP64 CPU restatement of the method of arXiv 2404.18034
 * (6-DoF powered-descent guidance solved by prox-linear SCP with the CTCS
 * reformulation and a customized PIPG subproblem solver).  It exists to check
 * the CUDA solver; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header or constant
 * table with the CUDA path: its parameter struct below is its own.
 *
 * Every routine follows a passage of the paper, cited as "Sec.", "Eq." or
 * "Alg." in the implementation.  Readings of silent or garbled passages are
 * listed next to the code that takes them.
 *
 * The model (F, g and the initial guess of the problem template of Sec. 2)
 * is chosen when the library is compiled: libpdg_oracle.so holds the 6-DoF
 * model of Sec. 4, libpdg_oracle_3dof.so (-DORC_MODEL_3DOF) the translational
 * 3-DoF model.  orc_nx() returns the library's state size NX.
 *
 * Layouts (row-major, double):
 *   6-DoF state x[15] = (m, r[3], v[3], q[4], omega[3], y)   (Sec. 2.1, Sec. 4)
 *   3-DoF state x[8]  = (m, r[3], v[3], y)
 *   control u[nu] = (T[3], [gamma[3],] s), nu in {4, 7}; the 3-DoF model has nu = 4
 *   X[N][NX], U[N][nu]; A[N-1][NX][NX]; Bm, Bp[N-1][NX][nu]; xprop[N-1][NX]
 *   x0 (the initial condition of a solve) is the first NX - 1 entries of x.
 * Parameter arrays below are sized for the 6-DoF model; the 3-DoF model reads
 * the first NX entries of z_f, fix_f and P_x, and uses delta_max as the
 * half-angle of its thrust-pointing cone about the up axis.
 */
#ifndef PDG_ORACLE_H
#define PDG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NX 15
#define ORC_NU_MAX 7

typedef struct orc_params {
  int nu;                 /* 4: (T, s); 7: (T, gamma, s) */
  double alpha_mdot;      /* mass depletion per unit thrust */
  double g_I[3];          /* gravity, inertial frame */
  double J_B[3];          /* diagonal inertia */
  double r_T_B[3];        /* thrust point, body frame */
  double m_dry, v_max, theta_max, omega_max, delta_max, T_min, T_max, gamma_max;
  double s_min, s_max;    /* dilation box */
  double z_f[15];         /* final-state targets (index as x) */
  int fix_f[15];          /* 1 where the final state component is fixed */
  double P_x[15], P_u[7]; /* diagonal scalings */
  double w_cost, w_prox, w_ep, eps_ctcs;
  double pipg_omega, pipg_rho, pipg_eps_abs, pipg_eps_rel;
  int pipg_jmax, pipg_jcheck;
  double pow_eps_abs, pow_eps_rel, pow_eps_buff;
  int pow_jmax;
  int scp_jmax;
  double scp_eps_step, scp_eps_defect;
  int rk4_substeps;
  double tf_guess;        /* initial guess of the final time */
  int soc_thrust;         /* 1: T_max and gimbal bounds as a per-node second-order-cone
                             projection in PIPG instead of CTCS rows */
  int glide_slope;        /* 1: glide-slope row tan(gamma_gs) ||(r_y, r_z)|| - r_x <= 0 in g */
  double tan_gs;          /* tan(gamma_gs), gamma_gs measured from the horizontal */
  double dt_min, dt_max, tf_max;  /* Sec. 2.2 time bounds; 0 = off (node box on s) */
} orc_params;

/* Scaled convex subproblem data (Eq. cvx-subproblem-custom). */
typedef struct orc_qp {
  int N, nu;
  double *Am;   /* [N-1][NX][NX]  hat A^-_k */
  double *Ap;   /* [N-1][NX][NX]  hat A^+_k = -I */
  double *Bm;   /* [N-1][NX][nu]  hat B^-_k */
  double *Bp;   /* [N-1][NX][nu]  hat B^+_k */
  double *w;    /* [N-1][NX]      hat w_k */
  double *eps;  /* [N-1]          hat epsilon_k */
  double *umin; /* [N][nu]        hat u_{k,min} (-inf where unbounded) */
  double *umax; /* [N][nu]        hat u_{k,max} (+inf where unbounded) */
  double zi[15];
  double zf[15];
  int fixf[15];
  double w_cost, w_prox, w_ep;
  double ecost[15]; /* e_cost on the scaled x_N (Eq. cvx-subproblem-custom objective) */
  int soc;          /* thrust sector projection on (see orc_params.soc_thrust) */
  double *Tbar;     /* [N][3] reference thrust (unscaled) */
  double soc_Tmax, soc_tan, soc_PT;
} orc_qp;

/* PIPG primal-dual state (warm start in, solution out), Alg. PIPG_custom. */
typedef struct orc_pd {
  double *xh;   /* [N][NX] */
  double *uh;   /* [N][nu] */
  double *mup;  /* [N-1][NX] */
  double *mum;  /* [N-1][NX] */
  double *phi;  /* [N-1][NX] */
  double *th;   /* [N-1] */
} orc_pd;

/* ---- model (Sec. 4) ---- */
int  orc_nx(void);                                                                /* NX */
void orc_F(const orc_params* p, const double* x, const double* u, double* Fx);   /* dxi/dt, NX - 1 */
int  orc_g(const orc_params* p, const double* x, const double* u, double* g);    /* returns n_g */
void orc_f(const orc_params* p, const double* x, const double* u, double* f);    /* Eq. sys-dyn-dil-aug, NX */
void orc_jac(const orc_params* p, const double* x, const double* u, double* A, double* B);

/* ---- discretization (Sec. 2.2, Sec. 2.3.1) ---- */
void orc_flow(const orc_params* p, const double* xk, const double* uk, const double* uk1,
              int nsub, double* xout);
void orc_discretize(const orc_params* p, int N, const double* X, const double* U,
                    double* A, double* Bm, double* Bp, double* xprop);

/* ---- scaled subproblem (Sec. 2.3.2) ---- */
int  orc_qp_alloc(orc_qp* qp, int N, int nu);
void orc_qp_free(orc_qp* qp);
void orc_scale(const orc_params* p, int N, const double* x0, const double* X, const double* U,
               const double* A, const double* Bm, const double* Bp, const double* xprop, orc_qp* qp);

int  orc_pd_alloc(orc_pd* s, int N, int nu);
void orc_pd_free(orc_pd* s);
void orc_pd_zero(orc_pd* s, int N, int nu);
void orc_pd_copy(orc_pd* dst, const orc_pd* src, int N, int nu);

/* ---- solver (Sec. 3) ---- */
/* Alg. power.  force_iters > 0 runs exactly that many iterations. Returns sigma. */
double orc_power(const orc_params* p, const orc_qp* qp, const orc_pd* start, int force_iters, int* iters);
/* Alg. PIPG_custom + Alg. stopping.  ws is warm start in / solution out.
 * force_iters > 0 runs exactly that many iterations without the stop test.
 * Returns the number of iterations run. */
int orc_pipgc(const orc_params* p, const orc_qp* qp, double sigma, orc_pd* ws, int force_iters);

/* Stop-decision report (test aid for checking another solver's stop decisions
 * against the oracle's own).  Each test "a <= b" of the solver is reported as
 * the relative margin (a - b) / b, which is <= 0 exactly when the test passes;
 * a test of several conditions reports the largest margin.
 *   orc_power_m:  margins[i]  = Alg. power's test after iteration i + 1
 *   orc_pipgc_m:  margins[c]  = Alg. stopping at the check after iteration
 *                 (c + 1) pipg_jcheck (iterates j and j - 1, unextrapolated)
 * They are written for every iteration run, including under force_iters (the
 * test is then evaluated but does not stop the loop); NULL skips the report.
 * orc_stop_custom evaluates Alg. stopping on the iterate pair (a, b): returns
 * 1 to terminate, and its margin in *m (may be NULL). */
double orc_power_m(const orc_params* p, const orc_qp* qp, const orc_pd* start, int force_iters, int* iters,
                   double* margins);
int orc_pipgc_m(const orc_params* p, const orc_qp* qp, double sigma, orc_pd* ws, int force_iters,
                double* margins);
int orc_stop_custom(const orc_params* p, const orc_qp* qp, const orc_pd* a, const orc_pd* b, double* m);

/* Dense canonical QP (Eq. canonical-QP / parsed-data) and generic PIPG (Alg. 1). */
int  orc_qp_dim(int N, int nu);  /* n_z */
void orc_qp_dense(const orc_qp* qp, double* P, double* pv, double* G, double* gv,
                  double* H, double* hv, double* lo, double* hi);
void orc_pipg_generic(const orc_qp* qp, double alpha, double omega, double rho, int jmax,
                      const double* z1, const double* eta1, const double* chi1,
                      double* zout, double* wout, double* vout);
void orc_z_pack(const orc_qp* qp, const orc_pd* s, double* z);
void orc_z_unpack(const orc_qp* qp, const double* z, orc_pd* s);

/* Euclidean projection of T onto {||T|| <= Tmax, ||(T_y, T_z)|| <= tan_delta T_x}
 * (second-order cone about body x, then the ball about its apex), in place. */
void orc_sector_project(double* T, double Tmax, double tan_delta);

/* Jacobi eigenvalues of a dense symmetric matrix (in place; returns the largest). */
double orc_sym_eig_max(int n, double* M);

/* ---- SCP (Sec. 2.3) ---- */
void orc_init_guess(const orc_params* p, int N, const double* x0, double* X, double* U);

typedef struct orc_result {
  double tf, fuel;
  int status;          /* 0 converged, 1 max SCP iterations, 2 non-finite */
  int scp_iters;
  long long pipg_iters;
  long long pow_iters;
  double defect, step;  /* last convergence measures */
} orc_result;

/* One SCP iteration about (X, U): discretize, scale, power iteration, PIPG.
 * ws: warm start in / subproblem solution out.  Outputs the subproblem data
 * measures and counts.  force_pipg / force_pow > 0 replay given counts;
 * force_sigma > 0 replaces the power iteration's estimate. */
int orc_scp_iterate(const orc_params* p, int N, const double* x0, double* X, double* U,
                    orc_pd* ws, int force_pow, int force_pipg, double force_sigma,
                    double* sigma, int* pow_it, int* pipg_it, double* defect, double* step);

/* orc_scp_iterate with the stop-decision report of its power iteration
 * ([pow_jmax]) and PIPG loop ([pipg_jmax / pipg_jcheck]); either may be NULL. */
int orc_scp_iterate_m(const orc_params* p, int N, const double* x0, double* X, double* U,
                      orc_pd* ws, int force_pow, int force_pipg, double force_sigma,
                      double* sigma, int* pow_it, int* pipg_it, double* defect, double* step,
                      double* pow_margins, double* pipg_margins);

/* Touchdown error 0.5 sum_{E_f} ((x_prop,N - z_f) / P_x)^2 of a trajectory,
 * x_prop,N the RK4 propagation of the last interval. */
double orc_touchdown(const orc_params* p, int N, const double* X, const double* U);

/* Full solve.  trace (may be NULL) is [scp_jmax][2] = (power iters, PIPG iters)
 * per SCP iteration, written on output; when replay != 0 it is read instead and
 * forces those counts, and replay_scp forces the SCP iteration count. */
int orc_solve(const orc_params* p, int N, const double* x0, double* X, double* U,
              orc_result* res, int* trace, int replay, int replay_scp);

/* orc_solve with the stop-decision report of every SCP iteration j (0-based):
 * scp_margins [scp_cap] the SCP convergence test (R8) after iteration j + 1,
 * pow_margins [scp_cap][pow_jmax] and pipg_margins [scp_cap][pipg_jmax /
 * pipg_jcheck] as for orc_scp_iterate_m; scp_cap = max(scp_jmax, replay_scp).
 * Entries of iterations not run are left untouched.  Any may be NULL. */
int orc_solve_m(const orc_params* p, int N, const double* x0, double* X, double* U,
                orc_result* res, int* trace, int replay, int replay_scp,
                double* scp_margins, double* pow_margins, double* pipg_margins);

/* Batch over instances with OpenMP (nthreads <= 0: library default).
 * x0s: [B][NX-1], X: [B][Nmax][NX], U: [B][Nmax][nu]; N may differ per instance. */
int orc_solve_batch(const orc_params* p, int B, int Nmax, const int* Ns, const double* x0s,
                    double* X, double* U, double* tf, double* fuel, int* status,
                    int* scp_iters, long long* pipg_iters, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
