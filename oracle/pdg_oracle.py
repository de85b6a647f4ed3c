"""ctypes front end of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It builds ``libpdg_oracle.so`` (the
6-DoF model of Sec. 4) and ``libpdg_oracle_3dof.so`` (the translational 3-DoF
model) from ``pdg_oracle.c`` with gcc and exposes the oracle's routines on
numpy arrays; every routine picks the library by the parameter dict's
``model`` ("6dof" when absent), and state arrays have that model's size NX.
It shares no code with the CUDA solver; the two meet only in the parameter
dict and the initial conditions produced by ``paper_2404_18034_gb300.inputs``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdg_oracle.c")
_LIBS = {"6dof": os.path.join(_HERE, "libpdg_oracle.so"), "3dof": os.path.join(_HERE, "libpdg_oracle_3dof.so")}
_DEFS = {"6dof": [], "3dof": ["-DORC_MODEL_3DOF"]}
NXS = {"6dof": 15, "3dof": 8}
NX = NXS["6dof"]
_lock = threading.Lock()
_libs: Dict = {}


def model_of(p: Dict) -> str:
    m = p.get("model", "6dof")
    if m not in NXS:
        raise ValueError(f"unknown model {m!r}")
    return m


def nx_of(p: Dict) -> int:
    """State size NX of the parameter dict's model (15 or 8)."""
    return NXS[model_of(p)]


def _build_one(model: str, force: bool) -> str:
    out = _LIBS[model]
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(os.path.join(_HERE, "pdg_oracle.h")))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall"] + _DEFS[model] + \
        [_SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile both model libraries of the oracle (plain C, -O2, OpenMP)
    next to their source; returns the 6-DoF one's path."""
    for m in ("3dof", "6dof"):
        path = _build_one(m, force)
    return path


class Params(C.Structure):
    _fields_ = [
        ("nu", C.c_int),
        ("alpha_mdot", C.c_double), ("g_I", C.c_double * 3), ("J_B", C.c_double * 3),
        ("r_T_B", C.c_double * 3),
        ("m_dry", C.c_double), ("v_max", C.c_double), ("theta_max", C.c_double),
        ("omega_max", C.c_double), ("delta_max", C.c_double), ("T_min", C.c_double),
        ("T_max", C.c_double), ("gamma_max", C.c_double),
        ("s_min", C.c_double), ("s_max", C.c_double),
        ("z_f", C.c_double * 15), ("fix_f", C.c_int * 15),
        ("P_x", C.c_double * 15), ("P_u", C.c_double * 7),
        ("w_cost", C.c_double), ("w_prox", C.c_double), ("w_ep", C.c_double), ("eps_ctcs", C.c_double),
        ("pipg_omega", C.c_double), ("pipg_rho", C.c_double), ("pipg_eps_abs", C.c_double),
        ("pipg_eps_rel", C.c_double),
        ("pipg_jmax", C.c_int), ("pipg_jcheck", C.c_int),
        ("pow_eps_abs", C.c_double), ("pow_eps_rel", C.c_double), ("pow_eps_buff", C.c_double),
        ("pow_jmax", C.c_int),
        ("scp_jmax", C.c_int),
        ("scp_eps_step", C.c_double), ("scp_eps_defect", C.c_double),
        ("rk4_substeps", C.c_int),
        ("tf_guess", C.c_double),
        ("soc_thrust", C.c_int),
        ("glide_slope", C.c_int), ("tan_gs", C.c_double),
        ("dt_min", C.c_double), ("dt_max", C.c_double), ("tf_max", C.c_double),
    ]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


class QP(C.Structure):
    _fields_ = [("N", C.c_int), ("nu", C.c_int),
                ("Am", _DP), ("Ap", _DP), ("Bm", _DP), ("Bp", _DP), ("w", _DP), ("eps", _DP),
                ("umin", _DP), ("umax", _DP),
                ("zi", C.c_double * 15), ("zf", C.c_double * 15), ("fixf", C.c_int * 15),
                ("w_cost", C.c_double), ("w_prox", C.c_double), ("w_ep", C.c_double),
                ("ecost", C.c_double * 15),
                ("soc", C.c_int), ("Tbar", _DP), ("soc_Tmax", C.c_double), ("soc_tan", C.c_double),
                ("soc_PT", C.c_double)]


class PD(C.Structure):
    _fields_ = [("xh", _DP), ("uh", _DP), ("mup", _DP), ("mum", _DP), ("phi", _DP), ("th", _DP)]


class Result(C.Structure):
    _fields_ = [("tf", C.c_double), ("fuel", C.c_double), ("status", C.c_int), ("scp_iters", C.c_int),
                ("pipg_iters", C.c_longlong), ("pow_iters", C.c_longlong),
                ("defect", C.c_double), ("step", C.c_double)]


def lib(model: str = "6dof"):
    with _lock:
        if model not in _libs:
            L = C.CDLL(_build_one(model, False))
            L.orc_nx.restype = C.c_int
            if L.orc_nx() != NXS[model]:
                raise RuntimeError(f"oracle library for {model} reports NX = {L.orc_nx()}")
            P = C.POINTER(Params)
            L.orc_F.argtypes = [P, _DP, _DP, _DP]
            L.orc_g.argtypes = [P, _DP, _DP, _DP]
            L.orc_g.restype = C.c_int
            L.orc_f.argtypes = [P, _DP, _DP, _DP]
            L.orc_jac.argtypes = [P, _DP, _DP, _DP, _DP]
            L.orc_flow.argtypes = [P, _DP, _DP, _DP, C.c_int, _DP]
            L.orc_discretize.argtypes = [P, C.c_int, _DP, _DP, _DP, _DP, _DP, _DP]
            L.orc_scale.argtypes = [P, C.c_int, _DP, _DP, _DP, _DP, _DP, _DP, _DP, C.POINTER(QP)]
            L.orc_power.argtypes = [P, C.POINTER(QP), C.POINTER(PD), C.c_int, _IP]
            L.orc_power.restype = C.c_double
            L.orc_pipgc.argtypes = [P, C.POINTER(QP), C.c_double, C.POINTER(PD), C.c_int]
            L.orc_pipgc.restype = C.c_int
            L.orc_qp_dim.argtypes = [C.c_int, C.c_int]
            L.orc_qp_dim.restype = C.c_int
            L.orc_qp_dense.argtypes = [C.POINTER(QP)] + [_DP] * 8
            L.orc_pipg_generic.argtypes = [C.POINTER(QP), C.c_double, C.c_double, C.c_double, C.c_int,
                                           _DP, _DP, _DP, _DP, _DP, _DP]
            L.orc_z_pack.argtypes = [C.POINTER(QP), C.POINTER(PD), _DP]
            L.orc_sector_project.argtypes = [_DP, C.c_double, C.c_double]
            L.orc_sym_eig_max.argtypes = [C.c_int, _DP]
            L.orc_sym_eig_max.restype = C.c_double
            L.orc_init_guess.argtypes = [P, C.c_int, _DP, _DP, _DP]
            L.orc_scp_iterate.argtypes = [P, C.c_int, _DP, _DP, _DP, C.POINTER(PD), C.c_int, C.c_int, C.c_double,
                                          _DP, _IP, _IP, _DP, _DP]
            L.orc_touchdown.argtypes = [P, C.c_int, _DP, _DP]
            L.orc_touchdown.restype = C.c_double
            L.orc_solve.argtypes = [P, C.c_int, _DP, _DP, _DP, C.POINTER(Result), _IP, C.c_int, C.c_int]
            L.orc_solve_m.argtypes = [P, C.c_int, _DP, _DP, _DP, C.POINTER(Result), _IP, C.c_int, C.c_int,
                                      _DP, _DP, _DP]
            L.orc_pipgc_m.argtypes = [P, C.POINTER(QP), C.c_double, C.POINTER(PD), C.c_int, _DP]
            L.orc_pipgc_m.restype = C.c_int
            L.orc_stop_custom.argtypes = [P, C.POINTER(QP), C.POINTER(PD), C.POINTER(PD), _DP]
            L.orc_stop_custom.restype = C.c_int
            L.orc_solve_batch.argtypes = [P, C.c_int, C.c_int, _IP, _DP, _DP, _DP, _DP, _DP, _IP, _IP,
                                          C.POINTER(C.c_longlong), C.c_int]
            _libs[model] = L
    return _libs[model]


def _L(p: Dict):
    return lib(model_of(p))


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_IP)


def make_params(p: Dict) -> Params:
    s = Params()
    s.nu = int(p["nu"])
    for k in ("alpha_mdot", "m_dry", "v_max", "theta_max", "omega_max", "delta_max", "T_min", "T_max",
              "gamma_max", "s_min", "s_max", "w_cost", "w_prox", "w_ep", "eps_ctcs", "pipg_omega",
              "pipg_rho", "pipg_eps_abs", "pipg_eps_rel", "pow_eps_abs", "pow_eps_rel", "pow_eps_buff",
              "scp_eps_step", "scp_eps_defect", "tf_guess"):
        setattr(s, k, float(p[k]))
    for k in ("pipg_jmax", "pipg_jcheck", "pow_jmax", "scp_jmax", "rk4_substeps"):
        setattr(s, k, int(p[k]))
    for k, n in (("g_I", 3), ("J_B", 3), ("r_T_B", 3), ("z_f", 15), ("P_x", 15), ("P_u", 7)):
        arr = getattr(s, k)
        for i in range(min(n, len(p[k]))):  # state vectors hold the model's NX entries
            arr[i] = float(p[k][i])
    for i in range(len(p["fix_f"])):
        s.fix_f[i] = int(p["fix_f"][i])
    s.soc_thrust = int(p.get("soc_thrust", 0))
    s.glide_slope = int(p.get("glide_slope", 0))
    s.tan_gs = math.tan(float(p.get("gamma_gs", 0.0)))
    for k in ("dt_min", "dt_max", "tf_max"):
        setattr(s, k, float(p.get(k, 0.0)))
    return s


# ---------------------------------------------------------------------------
# model
# ---------------------------------------------------------------------------

def F(p, x, u):
    out = np.zeros(nx_of(p) - 1)
    _L(p).orc_F(C.byref(make_params(p)), _d(np.ascontiguousarray(x, np.float64)),
                _d(np.ascontiguousarray(u, np.float64)), _d(out))
    return out


def g(p, x, u):
    out = np.zeros(10)
    n = _L(p).orc_g(C.byref(make_params(p)), _d(np.ascontiguousarray(x, np.float64)),
                    _d(np.ascontiguousarray(u, np.float64)), _d(out))
    return out[:n]


def f(p, x, u):
    out = np.zeros(nx_of(p))
    _L(p).orc_f(C.byref(make_params(p)), _d(np.ascontiguousarray(x, np.float64)),
                _d(np.ascontiguousarray(u, np.float64)), _d(out))
    return out


def jac(p, x, u):
    nu, NX = int(p["nu"]), nx_of(p)
    A = np.zeros((NX, NX))
    B = np.zeros((NX, nu))
    _L(p).orc_jac(C.byref(make_params(p)), _d(np.ascontiguousarray(x, np.float64)),
                  _d(np.ascontiguousarray(u, np.float64)), _d(A), _d(B))
    return A, B


def flow(p, xk, uk, uk1, nsub):
    """RK4 flow of Eq. sys-dyn-dil-aug over a unit tau interval (nsub substeps)."""
    out = np.zeros(nx_of(p))
    _L(p).orc_flow(C.byref(make_params(p)), _d(np.ascontiguousarray(xk, np.float64)),
                   _d(np.ascontiguousarray(uk, np.float64)), _d(np.ascontiguousarray(uk1, np.float64)),
                   int(nsub), _d(out))
    return out


def discretize(p, X, U):
    X = np.ascontiguousarray(X, np.float64)
    U = np.ascontiguousarray(U, np.float64)
    N, nu, NX = X.shape[0], int(p["nu"]), nx_of(p)
    A = np.zeros((N - 1, NX, NX))
    Bm = np.zeros((N - 1, NX, nu))
    Bp = np.zeros((N - 1, NX, nu))
    xp = np.zeros((N - 1, NX))
    _L(p).orc_discretize(C.byref(make_params(p)), N, _d(X), _d(U), _d(A), _d(Bm), _d(Bp), _d(xp))
    return A, Bm, Bp, xp


# ---------------------------------------------------------------------------
# subproblem
# ---------------------------------------------------------------------------

class QPData:
    """Scaled subproblem data (Eq. cvx-subproblem-custom) held in numpy arrays."""

    def __init__(self, N: int, nu: int, model: str = "6dof"):
        self.N, self.nu, self.model = N, nu, model
        NX = NXS[model]
        self.Am = np.zeros((N - 1, NX, NX))
        self.Ap = np.zeros((N - 1, NX, NX))
        self.Bm = np.zeros((N - 1, NX, nu))
        self.Bp = np.zeros((N - 1, NX, nu))
        self.w = np.zeros((N - 1, NX))
        self.eps = np.zeros(N - 1)
        self.umin = np.zeros((N, nu))
        self.umax = np.zeros((N, nu))
        self.zi = np.zeros(NX)
        self.zf = np.zeros(NX)
        self.fixf = np.zeros(NX, np.int32)
        self.ecost = np.zeros(NX)
        self.w_cost = self.w_prox = self.w_ep = 0.0
        self.Tbar = np.zeros((N, 3))
        self.soc = 0
        self.soc_Tmax = self.soc_tan = self.soc_PT = 0.0

    def cstruct(self) -> QP:
        q = QP()
        q.N, q.nu = self.N, self.nu
        for k in ("Am", "Ap", "Bm", "Bp", "w", "eps", "umin", "umax"):
            setattr(q, k, _d(getattr(self, k)))
        for i in range(NXS[self.model]):
            q.zi[i] = self.zi[i]
            q.zf[i] = self.zf[i]
            q.fixf[i] = int(self.fixf[i])
            q.ecost[i] = self.ecost[i]
        q.w_cost, q.w_prox, q.w_ep = self.w_cost, self.w_prox, self.w_ep
        q.soc = int(self.soc)
        q.Tbar = _d(self.Tbar)
        q.soc_Tmax, q.soc_tan, q.soc_PT = self.soc_Tmax, self.soc_tan, self.soc_PT
        return q

    def pull(self, q: QP):
        n = NXS[self.model]
        self.zi[:] = list(q.zi)[:n]
        self.zf[:] = list(q.zf)[:n]
        self.fixf[:] = list(q.fixf)[:n]
        self.ecost[:] = list(q.ecost)[:n]
        self.w_cost, self.w_prox, self.w_ep = q.w_cost, q.w_prox, q.w_ep
        self.soc = q.soc
        self.soc_Tmax, self.soc_tan, self.soc_PT = q.soc_Tmax, q.soc_tan, q.soc_PT


class PDState:
    """Primal-dual PIPG state (x_hat, u_hat, mu+, mu-, phi, theta)."""

    def __init__(self, N: int, nu: int, model: str = "6dof"):
        self.N, self.nu, self.model = N, nu, model
        NX = NXS[model]
        self.xh = np.zeros((N, NX))
        self.uh = np.zeros((N, nu))
        self.mup = np.zeros((N - 1, NX))
        self.mum = np.zeros((N - 1, NX))
        self.phi = np.zeros((N - 1, NX))
        self.th = np.zeros(N - 1)

    def cstruct(self) -> PD:
        s = PD()
        for k in ("xh", "uh", "mup", "mum", "phi", "th"):
            setattr(s, k, _d(getattr(self, k)))
        return s

    def copy(self) -> "PDState":
        o = PDState(self.N, self.nu, self.model)
        for k in ("xh", "uh", "mup", "mum", "phi", "th"):
            getattr(o, k)[...] = getattr(self, k)
        return o


def scale(p, x0, X, U, A, Bm, Bp, xp) -> QPData:
    N, nu = X.shape[0], int(p["nu"])
    qp = QPData(N, nu, model_of(p))
    qs = qp.cstruct()
    _L(p).orc_scale(C.byref(make_params(p)), N, _d(np.ascontiguousarray(x0, np.float64)),
                    _d(np.ascontiguousarray(X, np.float64)), _d(np.ascontiguousarray(U, np.float64)),
                    _d(np.ascontiguousarray(A)), _d(np.ascontiguousarray(Bm)),
                    _d(np.ascontiguousarray(Bp)), _d(np.ascontiguousarray(xp)), C.byref(qs))
    qp.pull(qs)
    return qp


def power(p, qp: QPData, start: PDState, force_iters: int = 0):
    it = C.c_int(0)
    qs = qp.cstruct()
    ss = start.cstruct()
    sig = _L(p).orc_power(C.byref(make_params(p)), C.byref(qs), C.byref(ss), int(force_iters), C.byref(it))
    return sig, it.value


def pipgc(p, qp: QPData, sigma: float, ws: PDState, force_iters: int = 0, margins: bool = False):
    """Runs Alg. PIPG_custom in place on ws; returns the iteration count, and
    with margins=True also the stop test's margin at every check (NaN where
    no check ran; see orc_pipgc_m)."""
    qs = qp.cstruct()
    ss = ws.cstruct()
    if not margins:
        return _L(p).orc_pipgc(C.byref(make_params(p)), C.byref(qs), float(sigma), C.byref(ss), int(force_iters))
    m = np.full(max(int(p["pipg_jmax"]), int(force_iters)) // int(p["pipg_jcheck"]), np.nan)
    n = _L(p).orc_pipgc_m(C.byref(make_params(p)), C.byref(qs), float(sigma), C.byref(ss), int(force_iters), _d(m))
    return n, m


def stop_custom(p, qp: QPData, a: PDState, b: PDState):
    """Alg. stopping on the iterate pair (a, b): (terminate?, margin)."""
    m = C.c_double()
    qs = qp.cstruct()
    r = _L(p).orc_stop_custom(C.byref(make_params(p)), C.byref(qs), C.byref(a.cstruct()), C.byref(b.cstruct()),
                              C.byref(m))
    return bool(r), m.value


def qp_dim(N, nu, model: str = "6dof"):
    return lib(model).orc_qp_dim(int(N), int(nu))


def qp_dense(qp: QPData):
    N, nu, NX = qp.N, qp.nu, NXS[qp.model]
    nz = qp_dim(N, nu, qp.model)
    P = np.zeros((nz, nz)); pv = np.zeros(nz)
    G = np.zeros((NX * (N - 1), nz)); gv = np.zeros(NX * (N - 1))
    H = np.zeros((N - 1, nz)); hv = np.zeros(N - 1)
    lo = np.zeros(nz); hi = np.zeros(nz)
    qs = qp.cstruct()
    lib(qp.model).orc_qp_dense(C.byref(qs), _d(P), _d(pv), _d(G), _d(gv), _d(H), _d(hv), _d(lo), _d(hi))
    return dict(P=P, p=pv, G=G, g=gv, H=H, h=hv, lo=lo, hi=hi)


def z_pack(qp: QPData, s: PDState) -> np.ndarray:
    z = np.zeros(qp_dim(qp.N, qp.nu, qp.model))
    qs = qp.cstruct()
    ss = s.cstruct()
    lib(qp.model).orc_z_pack(C.byref(qs), C.byref(ss), _d(z))
    return z


def pipg_generic(qp: QPData, alpha, omega, rho, jmax, z1, eta1, chi1):
    nz = qp_dim(qp.N, qp.nu, qp.model)
    z = np.zeros(nz); w = np.zeros(NXS[qp.model] * (qp.N - 1)); v = np.zeros(qp.N - 1)
    qs = qp.cstruct()
    lib(qp.model).orc_pipg_generic(C.byref(qs), float(alpha), float(omega), float(rho), int(jmax),
                           _d(np.ascontiguousarray(z1, np.float64)), _d(np.ascontiguousarray(eta1, np.float64)),
                           _d(np.ascontiguousarray(chi1, np.float64)), _d(z), _d(w), _d(v))
    return z, w, v


def sector_project(T, Tmax, tan_delta):
    T = np.array(T, dtype=np.float64)
    lib().orc_sector_project(_d(T), float(Tmax), float(tan_delta))
    return T


def sym_eig_max(M: np.ndarray) -> float:
    M = np.array(M, dtype=np.float64, order="C", copy=True)
    return lib().orc_sym_eig_max(M.shape[0], _d(M))


def init_guess(p, N, x0):
    nu, NX = int(p["nu"]), nx_of(p)
    X = np.zeros((N, NX)); U = np.zeros((N, nu))
    _L(p).orc_init_guess(C.byref(make_params(p)), int(N), _d(np.ascontiguousarray(x0, np.float64)), _d(X), _d(U))
    return X, U


def scp_iterate(p, x0, X, U, ws: PDState, force_pow=0, force_pipg=0, force_sigma=0.0):
    """One SCP iteration in place on (X, U, ws)."""
    sig = C.c_double(); pit = C.c_int(); jit = C.c_int(); dfc = C.c_double(); stp = C.c_double()
    ss = ws.cstruct()
    _L(p).orc_scp_iterate(C.byref(make_params(p)), X.shape[0], _d(np.ascontiguousarray(x0, np.float64)),
                          _d(X), _d(U), C.byref(ss), int(force_pow), int(force_pipg), float(force_sigma),
                          C.byref(sig), C.byref(pit), C.byref(jit), C.byref(dfc), C.byref(stp))
    return dict(sigma=sig.value, pow_iters=pit.value, pipg_iters=jit.value, defect=dfc.value, step=stp.value)


def touchdown(p, X, U):
    """Touchdown error of a trajectory (see orc_touchdown)."""
    X = np.ascontiguousarray(X, np.float64); U = np.ascontiguousarray(U, np.float64)
    return _L(p).orc_touchdown(C.byref(make_params(p)), X.shape[0], _d(X), _d(U))


def final_iteration_state(p, N, x0, trace, scp_iters):
    """Replay a solve's recorded counts up to (not including) its last SCP
    iteration; returns the reference (X, U), the PIPG warm start of the last
    iteration, and that iteration's sigma and PIPG count."""
    nu = int(p["nu"])
    X, U = init_guess(p, N, x0)
    ws = PDState(N, nu, model_of(p))
    for j in range(scp_iters - 1):
        scp_iterate(p, x0, X, U, ws, force_pow=int(trace[j][0]), force_pipg=int(trace[j][1]))
    A, Bm, Bp, xp = discretize(p, X, U)
    qp = scale(p, x0, X, U, A, Bm, Bp, xp)
    sig, _ = power(p, qp, ws, force_iters=int(trace[scp_iters - 1][0]))
    return X, U, ws, sig, int(trace[scp_iters - 1][1])


def final_iteration_outputs(p, x0, X, U, ws: PDState, sigma, n_pipg):
    """The last SCP iteration as a function of x0 (the reference's first node
    moving with it): returns (fuel, touchdown error) of its updated trajectory."""
    X = X.copy(); U = U.copy(); w = ws.copy()
    X[0, :nx_of(p) - 1] = x0
    scp_iterate(p, x0, X, U, w, force_pow=1, force_pipg=n_pipg, force_sigma=sigma)
    return X[0, 0] - X[-1, 0], touchdown(p, X, U)


def solve(p, N, x0, trace: Optional[np.ndarray] = None, replay_scp: int = 0, margins: bool = False):
    """Full SCP solve of one instance.  With replay_scp > 0, trace[j] = (power
    iterations, PIPG iterations) of SCP iteration j is replayed exactly.
    margins=True adds the oracle's own stop-test margins (orc_solve_m):
    "scp_margin" [scp_iters], "pow_margin" [scp_iters][pow_jmax] and
    "pipg_margin" [scp_iters][pipg_jmax // pipg_jcheck], NaN where no test ran."""
    nu, NX = int(p["nu"]), nx_of(p)
    X = np.zeros((N, NX)); U = np.zeros((N, nu))
    res = Result()
    jm = max(int(p["scp_jmax"]), int(replay_scp))
    tr = np.zeros((jm, 2), np.int32) if trace is None else np.ascontiguousarray(trace, np.int32)
    args = (C.byref(make_params(p)), int(N), _d(np.ascontiguousarray(x0, np.float64)), _d(X), _d(U),
            C.byref(res), _i(tr), 1 if replay_scp > 0 else 0, int(replay_scp))
    if margins:
        ms = np.full(jm, np.nan)
        mp = np.full((jm, int(p["pow_jmax"])), np.nan)
        mj = np.full((jm, int(p["pipg_jmax"]) // int(p["pipg_jcheck"])), np.nan)
        _L(p).orc_solve_m(*args, _d(ms), _d(mp), _d(mj))
    else:
        _L(p).orc_solve(*args)
    out = dict(X=X, U=U, tf=res.tf, fuel=res.fuel, status=res.status, scp_iters=res.scp_iters,
               pipg_iters=res.pipg_iters, pow_iters=res.pow_iters, defect=res.defect, step=res.step,
               trace=tr[:res.scp_iters].copy())
    if margins:
        n = res.scp_iters
        out.update(scp_margin=ms[:n].copy(), pow_margin=mp[:n].copy(), pipg_margin=mj[:n].copy())
    return out


def solve_batch(p, x0s, Ns, Nmax=None, nthreads=0):
    x0s = np.ascontiguousarray(x0s, np.float64)
    B = x0s.shape[0]
    Ns = np.ascontiguousarray(Ns, np.int32)
    Nmax = int(Nmax or Ns.max())
    nu, NX = int(p["nu"]), nx_of(p)
    X = np.zeros((B, Nmax, NX)); U = np.zeros((B, Nmax, nu))
    tf = np.zeros(B); fuel = np.zeros(B)
    st = np.zeros(B, np.int32); sc = np.zeros(B, np.int32); pi = np.zeros(B, np.int64)
    _L(p).orc_solve_batch(C.byref(make_params(p)), B, Nmax, _i(Ns), _d(x0s), _d(X), _d(U), _d(tf), _d(fuel),
                          _i(st), _i(sc), pi.ctypes.data_as(C.POINTER(C.c_longlong)), int(nthreads))
    return dict(X=X, U=U, tf=tf, fuel=fuel, status=st, scp_iters=sc, pipg_iters=pi)
