"""Python binding of the C ABI in include/pdg_mc.h (ctypes; marshalling only).

Every computation runs in the CUDA library of the parameter dict's model
(libpdg_mc.so: 6-DoF; libpdg_mc_3dof.so: 3-DoF); there is no fallback.
Importing this module does not touch the GPU; creating a Solver loads the
library and raises if it is missing or no CUDA device is usable.  Device
buffers are torch CUDA tensors (float64 / int32 / int64), host buffers numpy
arrays; the stream is torch's current stream unless one is given.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PDG_MC_LIB", os.path.join(HERE, "libpdg_mc.so"))
LIB_PATHS = {"6dof": LIB_PATH, "3dof": os.path.join(HERE, "libpdg_mc_3dof.so")}
NXS = {"6dof": 15, "3dof": 8}

PDG_CONVERGED, PDG_MAX_SCP, PDG_NONFINITE, PDG_BUDGET, PDG_BAD_INPUT, PDG_ABORTED = 0, 1, 2, 3, 4, 5
ERRORS = {-1: "PDG_EINVAL", -2: "PDG_ENOMEM", -3: "PDG_ECUDA"}
EXPORTS = ("pdg_mc_init", "pdg_mc_destroy", "pdg_mc_last_error", "pdg_mc_solve_batch",
           "pdg_mc_solve_batch_host", "pdg_mc_subproblem", "pdg_mc_scp_step", "pdg_mc_launch_info",
           "pdg_mc_set_threads", "pdg_mc_probe_fma", "pdg_mc_solve_batch_noalloc",
           "pdg_mc_grad_batch", "pdg_mc_set_pipg_form", "pdg_mc_pipg_form", "pdg_mc_probe_fma_lanes",
           "pdg_mc_autotune", "pdg_mc_model_nx", "pdg_mc_abort", "pdg_mc_clear_abort")


class PdgParams(C.Structure):
    """Mirror of struct pdg_params."""
    _fields_ = [
        ("nu", C.c_int), ("precision", C.c_int),
        ("alpha_mdot", C.c_double), ("g_I", C.c_double * 3), ("J_B", C.c_double * 3), ("r_T_B", C.c_double * 3),
        ("m_dry", C.c_double), ("v_max", C.c_double), ("theta_max", C.c_double), ("omega_max", C.c_double),
        ("delta_max", C.c_double), ("T_min", C.c_double), ("T_max", C.c_double), ("gamma_max", C.c_double),
        ("s_min", C.c_double), ("s_max", C.c_double),
        ("z_f", C.c_double * 15), ("fix_f", C.c_int * 15),
        ("P_x", C.c_double * 15), ("P_u", C.c_double * 7),
        ("w_cost", C.c_double), ("w_prox", C.c_double), ("w_ep", C.c_double), ("eps_ctcs", C.c_double),
        ("pipg_omega", C.c_double), ("pipg_rho", C.c_double), ("pipg_eps_abs", C.c_double),
        ("pipg_eps_rel", C.c_double),
        ("pipg_jmax", C.c_int), ("pipg_jcheck", C.c_int),
        ("pow_eps_abs", C.c_double), ("pow_eps_rel", C.c_double), ("pow_eps_buff", C.c_double),
        ("pow_jmax", C.c_int), ("scp_jmax", C.c_int),
        ("scp_eps_step", C.c_double), ("scp_eps_defect", C.c_double),
        ("rk4_substeps", C.c_int),
        ("tf_guess", C.c_double), ("budget_seconds", C.c_double),
        ("soc_thrust", C.c_int),
        ("glide_slope", C.c_int), ("gamma_gs", C.c_double),
        ("dt_min", C.c_double), ("dt_max", C.c_double), ("tf_max", C.c_double),
        ("model_params", C.c_double * 16),
    ]


_VP = C.c_void_p
_libs: Dict = {}


def model_of(p: Dict) -> str:
    m = p.get("model", "6dof")
    if m not in NXS and m != "custom":
        raise ValueError(f"unknown model {m!r}")
    return m


def load_library(path: Optional[str] = None, model: str = "6dof"):
    """Load the model's library (libpdg_mc.so for 6-DoF, libpdg_mc_3dof.so for
    3-DoF, or `path`); raises RuntimeError when it has not been built or its
    state size is not the model's.  model="custom" loads a library built
    from a model header of the caller's (build.build_model) and takes its
    state size from the library."""
    path = path or LIB_PATHS[model]
    if (path, model) in _libs:
        return _libs[(path, model)]
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_2404_18034_gb300.build.build())")
    L = C.CDLL(path)
    L.pdg_mc_model_nx.argtypes = []
    L.pdg_mc_model_nx.restype = C.c_int
    if model != "custom" and L.pdg_mc_model_nx() != NXS[model]:
        raise RuntimeError(f"{path} implements NX = {L.pdg_mc_model_nx()}, not the {model} model")
    L.pdg_mc_init.argtypes = [C.POINTER(PdgParams), C.c_int, C.POINTER(_VP)]
    L.pdg_mc_destroy.argtypes = [_VP]
    L.pdg_mc_destroy.restype = None
    L.pdg_mc_last_error.argtypes = [_VP]
    L.pdg_mc_last_error.restype = C.c_char_p
    L.pdg_mc_solve_batch.argtypes = [_VP, C.c_int, _VP, _VP, C.c_int] + [_VP] * 8 + [_VP]
    L.pdg_mc_solve_batch_host.argtypes = [_VP, C.c_int, _VP, _VP, C.c_int] + [_VP] * 7 + [_VP]
    L.pdg_mc_subproblem.argtypes = [_VP, C.c_int] + [_VP] * 8 + [_VP]
    L.pdg_mc_scp_step.argtypes = [_VP, C.c_int] + [_VP] * 14 + [_VP]
    L.pdg_mc_launch_info.argtypes = [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.pdg_mc_set_threads.argtypes = [_VP, C.c_int]
    L.pdg_mc_probe_fma.argtypes = [C.c_int, C.POINTER(C.c_double), _VP]
    L.pdg_mc_solve_batch_noalloc.argtypes = [_VP, C.c_int, _VP, _VP] + [_VP] * 7 + [_VP]
    L.pdg_mc_grad_batch.argtypes = [_VP, C.c_int] + [_VP] * 8 + [_VP]
    L.pdg_mc_set_pipg_form.argtypes = [_VP, C.c_int]
    L.pdg_mc_probe_fma_lanes.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), _VP]
    L.pdg_mc_autotune.argtypes = [_VP, C.c_int, _VP, _VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_double), _VP]
    L.pdg_mc_pipg_form.argtypes = [_VP]
    L.pdg_mc_abort.argtypes = [_VP]
    L.pdg_mc_clear_abort.argtypes = [_VP]
    for name in ("pdg_mc_init", "pdg_mc_solve_batch", "pdg_mc_solve_batch_host", "pdg_mc_subproblem",
                 "pdg_mc_scp_step", "pdg_mc_launch_info", "pdg_mc_set_threads", "pdg_mc_probe_fma",
                 "pdg_mc_solve_batch_noalloc", "pdg_mc_grad_batch", "pdg_mc_set_pipg_form", "pdg_mc_pipg_form",
                 "pdg_mc_probe_fma_lanes", "pdg_mc_autotune", "pdg_mc_abort", "pdg_mc_clear_abort"):
        getattr(L, name).restype = C.c_int
    _libs[(path, model)] = L
    return L


def make_params(p: Dict, precision: int = 0, budget_seconds: float = 0.0) -> PdgParams:
    s = PdgParams()
    s.nu = int(p["nu"])
    s.precision = int(precision)
    for k in ("alpha_mdot", "m_dry", "v_max", "theta_max", "omega_max", "delta_max", "T_min", "T_max",
              "gamma_max", "s_min", "s_max", "w_cost", "w_prox", "w_ep", "eps_ctcs", "pipg_omega", "pipg_rho",
              "pipg_eps_abs", "pipg_eps_rel", "pow_eps_abs", "pow_eps_rel", "pow_eps_buff", "scp_eps_step",
              "scp_eps_defect", "tf_guess"):
        setattr(s, k, float(p[k]))
    for k in ("pipg_jmax", "pipg_jcheck", "pow_jmax", "scp_jmax", "rk4_substeps"):
        setattr(s, k, int(p[k]))
    for k, n in (("g_I", 3), ("J_B", 3), ("r_T_B", 3), ("z_f", 15), ("P_x", 15), ("P_u", 7)):
        arr = getattr(s, k)
        for i in range(min(n, len(p[k]))):  # state vectors hold the model's NX entries
            arr[i] = float(p[k][i])
    for i in range(len(p["fix_f"])):
        s.fix_f[i] = int(p["fix_f"][i])
    s.budget_seconds = float(budget_seconds)
    s.soc_thrust = int(p.get("soc_thrust", 0))
    s.glide_slope = int(p.get("glide_slope", 0))
    s.gamma_gs = float(p.get("gamma_gs", 0.0))
    for k in ("dt_min", "dt_max", "tf_max"):
        setattr(s, k, float(p.get(k, 0.0)))
    for i, v in enumerate(p.get("model_params", ())):
        s.model_params[i] = float(v)
    return s


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def probe_fma(precision: int = 0, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (pdg_mc_probe_fma)."""
    import torch
    L = load_library()
    out = C.c_double()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.pdg_mc_probe_fma(int(precision), C.byref(out), C.c_void_p(s.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"pdg_mc_probe_fma: {ERRORS.get(rc, rc)}")
    return out.value


def probe_fma_lanes(precision: int = 0, lanes=(32, 16, 8, 1), stream=None) -> Dict[int, float]:
    """Best time (ms) of the FMA-chain probe with only `k` active lanes per
    warp, for each k in lanes (pdg_mc_probe_fma_lanes).  The warp-instruction
    count is the same for every k."""
    import torch
    L = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    res = {}
    for k in lanes:
        out = C.c_double()
        rc = L.pdg_mc_probe_fma_lanes(int(precision), int(k), C.byref(out), C.c_void_p(s.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"pdg_mc_probe_fma_lanes: {ERRORS.get(rc, rc)}")
        res[int(k)] = out.value
    return res


class Solver:
    """Handle on the batched solver (pdg_mc_init / pdg_mc_destroy)."""

    def __init__(self, params: Dict, n_max: int, precision: int = 0, budget_seconds: float = 0.0,
                 tune_cache: Optional[str] = None, mode: int = 1, library: Optional[str] = None):
        """library: path of a library built from a model header of the
        caller's (build.build_model); params["model"] is then "custom"."""
        self.model = model_of(params)
        if self.model == "custom" and library is None:
            raise ValueError('params["model"] == "custom" needs library= (a library from build.build_model)')
        self.lib = load_library(library, model=self.model)
        self.nx = int(self.lib.pdg_mc_model_nx())
        self.params = params
        self.nu = int(params["nu"])
        self.n_max = int(n_max)
        self.precision = int(precision)
        self._p = make_params(params, precision, budget_seconds)
        h = _VP()
        rc = self.lib.pdg_mc_init(C.byref(self._p), self.n_max, C.byref(h))
        if rc != 0:
            raise RuntimeError(f"pdg_mc_init: {ERRORS.get(rc, rc)}: {self.lib.pdg_mc_last_error(None).decode()}")
        self.h = h
        self.tuned_threads = None
        self.tuned_form = None
        if tune_cache:
            import torch

            from .autotune import lookup
            e = lookup(torch.cuda.get_device_name(), self.n_max, self.nu, self.precision, mode, tune_cache,
                       self.model)
            if e:
                self.set_pipg_form(e[1])
                self.set_threads(e[0])
                self.tuned_threads = e[0]
                self.tuned_form = e[1]

    def close(self):
        if getattr(self, "h", None):
            self.lib.pdg_mc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what}: {ERRORS.get(rc, rc)}: {self.lib.pdg_mc_last_error(self.h).decode()}")

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def alloc_outputs(self, B: int, device="cuda"):
        import torch
        f = dict(dtype=torch.float64, device=device)
        return dict(X=torch.empty(B, self.n_max, self.nx, **f), U=torch.empty(B, self.n_max, self.nu, **f),
                    tf=torch.empty(B, **f), fuel=torch.empty(B, **f),
                    status=torch.empty(B, dtype=torch.int32, device=device),
                    scp_iters=torch.empty(B, dtype=torch.int32, device=device),
                    pipg_iters=torch.empty(B, dtype=torch.int64, device=device))

    def solve(self, x0, n_nodes=None, mode: int = 1, out=None, trace: bool = False, stream=None):
        """pdg_mc_solve_batch on device tensors; returns the output dict."""
        import torch
        B = int(x0.shape[0])
        out = out or self.alloc_outputs(B, x0.device)
        tr = None
        if trace:
            tr = torch.zeros(B, int(self.params["scp_jmax"]), 2, dtype=torch.int32, device=x0.device)
            out["trace"] = tr
        rc = self.lib.pdg_mc_solve_batch(self.h, B, _ptr(x0), _ptr(n_nodes), int(mode), _ptr(out["X"]),
                                         _ptr(out["U"]), _ptr(out["tf"]), _ptr(out["fuel"]), _ptr(out["status"]),
                                         _ptr(out["scp_iters"]), _ptr(out["pipg_iters"]), _ptr(tr),
                                         self._stream(stream))
        self._check(rc, "pdg_mc_solve_batch")
        return out

    def solve_noalloc(self, x0, n_nodes=None, out=None, stream=None):
        """pdg_mc_solve_batch_noalloc: the plain-form solve with its workspace in
        the library's fixed device scratch array (no allocation in the call)."""
        B = int(x0.shape[0])
        out = out or self.alloc_outputs(B, x0.device)
        rc = self.lib.pdg_mc_solve_batch_noalloc(self.h, B, _ptr(x0), _ptr(n_nodes), _ptr(out["X"]), _ptr(out["U"]),
                                                 _ptr(out["tf"]), _ptr(out["fuel"]), _ptr(out["status"]),
                                                 _ptr(out["scp_iters"]), _ptr(out["pipg_iters"]),
                                                 self._stream(stream))
        self._check(rc, "pdg_mc_solve_batch_noalloc")
        return out

    def grad(self, x0, n_nodes=None, dL_dfuel=None, dL_dtouch=None, stream=None):
        """pdg_mc_grad_batch: returns grad (B x NX-1), fuel, touch, status."""
        import torch
        B = int(x0.shape[0])
        f = dict(dtype=torch.float64, device=x0.device)
        o = dict(grad=torch.empty(B, self.nx - 1, **f), fuel=torch.empty(B, **f), touch=torch.empty(B, **f),
                 status=torch.empty(B, dtype=torch.int32, device=x0.device))
        rc = self.lib.pdg_mc_grad_batch(self.h, B, _ptr(x0), _ptr(n_nodes), _ptr(dL_dfuel), _ptr(dL_dtouch),
                                        _ptr(o["grad"]), _ptr(o["fuel"]), _ptr(o["touch"]), _ptr(o["status"]),
                                        self._stream(stream))
        self._check(rc, "pdg_mc_grad_batch")
        return o

    def solve_host(self, x0: np.ndarray, n_nodes: Optional[np.ndarray] = None, mode: int = 1, out=None,
                   stream=None):
        """pdg_mc_solve_batch_host on host numpy arrays (returns when done)."""
        x0 = np.ascontiguousarray(x0, np.float64)
        B = x0.shape[0]
        if n_nodes is not None:
            n_nodes = np.ascontiguousarray(n_nodes, np.int32)
        out = out or dict(X=np.empty((B, self.n_max, self.nx)), U=np.empty((B, self.n_max, self.nu)),
                          tf=np.empty(B), fuel=np.empty(B), status=np.empty(B, np.int32),
                          scp_iters=np.empty(B, np.int32), pipg_iters=np.empty(B, np.int64))
        rc = self.lib.pdg_mc_solve_batch_host(self.h, B, _np(x0), _np(n_nodes), int(mode), _np(out["X"]),
                                              _np(out["U"]), _np(out["tf"]), _np(out["fuel"]), _np(out["status"]),
                                              _np(out["scp_iters"]), _np(out["pipg_iters"]),
                                              self._stream(stream))
        self._check(rc, "pdg_mc_solve_batch_host")
        return out

    def subproblem(self, x0, X, U, n_nodes=None, stream=None):
        import torch
        B = int(x0.shape[0])
        f = dict(dtype=torch.float64, device=x0.device)
        nm = self.n_max - 1
        nx = self.nx
        o = dict(Am=torch.empty(B, nm, nx, nx, **f), Bm=torch.empty(B, nm, nx, self.nu, **f),
                 Bp=torch.empty(B, nm, nx, self.nu, **f), w=torch.empty(B, nm, nx, **f))
        rc = self.lib.pdg_mc_subproblem(self.h, B, _ptr(x0), _ptr(n_nodes), _ptr(X), _ptr(U), _ptr(o["Am"]),
                                        _ptr(o["Bm"]), _ptr(o["Bp"]), _ptr(o["w"]), self._stream(stream))
        self._check(rc, "pdg_mc_subproblem")
        return o

    def scp_step(self, x0, X, U, ws: Dict, n_nodes=None, force=None, stream=None):
        """pdg_mc_scp_step: X, U and the warm-start tensors in ws are updated in place."""
        import torch
        B = int(x0.shape[0])
        f = dict(dtype=torch.float64, device=x0.device)
        o = dict(sigma=torch.empty(B, **f), defect=torch.empty(B, **f), step=torch.empty(B, **f),
                 iters=torch.empty(B, 2, dtype=torch.int32, device=x0.device))
        rc = self.lib.pdg_mc_scp_step(self.h, B, _ptr(x0), _ptr(n_nodes), _ptr(X), _ptr(U), _ptr(ws["xh"]),
                                      _ptr(ws["uh"]), _ptr(ws["mup"]), _ptr(ws["mum"]), _ptr(ws["phi"]),
                                      _ptr(ws["th"]), _ptr(force), _ptr(o["sigma"]), _ptr(o["defect"]),
                                      _ptr(o["step"]), _ptr(o["iters"]), self._stream(stream))
        self._check(rc, "pdg_mc_scp_step")
        return o

    def launch_info(self):
        t, c, s = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.pdg_mc_launch_info(self.h, C.byref(t), C.byref(c), C.byref(s)), "pdg_mc_launch_info")
        return dict(threads=t.value, ctas_per_sm=c.value, smem_bytes=s.value,
                    pipg_form=int(self.lib.pdg_mc_pipg_form(self.h)))

    def autotune(self, x0, n_nodes=None, mode: int = 1, stream=None):
        """pdg_mc_autotune on a device batch: returns (threads, form,
        converged solves/s) of the fastest candidate, applied to the handle."""
        t, f, r = C.c_int(), C.c_int(), C.c_double()
        rc = self.lib.pdg_mc_autotune(self.h, int(x0.shape[0]), _ptr(x0), _ptr(n_nodes), int(mode), C.byref(t),
                                      C.byref(f), C.byref(r), self._stream(stream))
        self._check(rc, "pdg_mc_autotune")
        self.tuned_threads, self.tuned_form = t.value, f.value
        return t.value, f.value, r.value

    def abort(self):
        """pdg_mc_abort: ask every running or later solve of this handle to stop
        at its next SCP iteration boundary (any thread; returns at once)."""
        self._check(self.lib.pdg_mc_abort(self.h), "pdg_mc_abort")

    def clear_abort(self):
        """pdg_mc_clear_abort."""
        self._check(self.lib.pdg_mc_clear_abort(self.h), "pdg_mc_clear_abort")

    def set_pipg_form(self, form: int):
        """0 automatic, 1 blocks in shared memory, 2 blocks in registers,
        3 blocks in register tiles over lane groups."""
        self._check(self.lib.pdg_mc_set_pipg_form(self.h, int(form)), "pdg_mc_set_pipg_form")

    def set_threads(self, threads: int):
        self._check(self.lib.pdg_mc_set_threads(self.h, int(threads)), "pdg_mc_set_threads")
