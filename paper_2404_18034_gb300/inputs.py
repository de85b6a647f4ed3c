"""Seeded, synthetic inputs shared by the CUDA solver's tests and the oracle.

This module holds no arithmetic of the guidance method: it only loads the
parameter set (plain numbers) and draws dispersed initial conditions from a
counter-based generator, so that both sides of a parity check see the same
inputs.  It imports neither the CUDA binding nor the oracle.

State layout (Sec. 4 of arXiv 2404.18034): x = (m, r[3], v[3], q[4], w[3], y);
the initial condition passed to a solve is the first 14 entries (m_wet, r, v,
q, w).  Controls: (T[3], s) for nu = 4, (T[3], gamma[3], s) for nu = 7.  The
translational 3-DoF model ("model": "3dof" in its parameter file) has
x = (m, r[3], v[3], y), initial conditions (m_wet, r, v) and nu = 4.

Dispersions:
  "bj"       r, v scaled by 1 + U(-0.1, 0.1) per component; attitude tilted
             about a uniform random axis by an angle U(0, 5 deg); w drawn
             U(-2, 2) deg per time unit per axis; wet mass scaled by
             1 + U(-0.02, 0.02).  The 3-DoF model draws the same m, r, v.
  "paper256" r(0) ~ (U(6, 9), U(3, 6), U(1, 2)) with the rest nominal, the
             Monte Carlo distribution of Sec. 6 of the paper.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PARAMS = os.path.join(_HERE, "params", "pdg_default.json")
PARAMS_3DOF = os.path.join(_HERE, "params", "pdg_3dof.json")

NX = 15
IDX = {"m": [0], "r": [1, 2, 3], "v": [4, 5, 6], "q": [7, 8, 9, 10], "w": [11, 12, 13], "y": [14],
       "q0": [7], "q1": [8], "q2": [9], "q3": [10], "wx": [11], "wy": [12], "wz": [13]}
NX_3DOF = 8
IDX_3DOF = {"m": [0], "r": [1, 2, 3], "v": [4, 5, 6], "y": [7]}


def nx_of(p: Dict) -> int:
    """State size of the parameter dict's model: 15 (6-DoF) or 8 (3-DoF)."""
    return NX_3DOF if p.get("model", "6dof") == "3dof" else NX

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def load_params(path: Optional[str] = None, nu: Optional[int] = None, model: Optional[str] = None,
                **overrides) -> Dict:
    """Load a parameter file into a flat dict with the derived vectors.

    Returns keys used by both the oracle and the CUDA binding: model, nu,
    alpha_mdot, g_I, J_B, r_T_B, m_dry, v_max, theta_max, omega_max,
    delta_max (radians), T_min, T_max, gamma_max, s_min, s_max, z_f[NX],
    fix_f[NX], P_x[NX], P_u[7], weights and solver settings; plus m_wet,
    x0_nominal[NX - 1].  model="3dof" loads the 3-DoF parameter file when no
    path is given; the file's own "model" entry decides the model.
    """
    if path is None:
        path = PARAMS_3DOF if model == "3dof" else DEFAULT_PARAMS
    with open(path) as fh:
        raw = json.load(fh)
    if nu is not None:
        raw["nu"] = int(nu)
    nu = int(raw["nu"])
    mdl = raw.get("model", "6dof")
    if mdl not in ("6dof", "3dof"):
        raise ValueError(f"unknown model {mdl!r}")
    if nu not in (4, 7) or (mdl == "3dof" and nu != 4):
        raise ValueError("nu must be 4 or 7 (6-DoF) or 4 (3-DoF)")
    if mdl == "3dof":
        return _load_3dof(raw, overrides)
    d2r = math.pi / 180.0
    p: Dict = {}
    p["model"] = "6dof"
    p["nu"] = nu
    for k in ("alpha_mdot", "m_dry", "v_max", "T_min", "T_max", "gamma_max", "s_min", "s_max",
              "w_cost", "w_prox", "w_ep", "eps_ctcs", "pipg_omega", "pipg_rho", "pipg_eps_abs",
              "pipg_eps_rel", "pow_eps_abs", "pow_eps_rel", "pow_eps_buff", "scp_eps_step",
              "scp_eps_defect", "tf_guess", "m_wet"):
        p[k] = float(raw[k])
    for k in ("pipg_jmax", "pipg_jcheck", "pow_jmax", "scp_jmax", "rk4_substeps"):
        p[k] = int(raw[k])
    p["soc_thrust"] = int(raw.get("soc_thrust", 0))
    # glide slope (gamma_gs of Sec. 4, from the horizontal) and the Sec. 2.2
    # time bounds (0 = off); off in the default workloads
    p["glide_slope"] = int(raw.get("glide_slope", 0))
    p["dt_min"] = float(raw.get("dt_min", 0.0))
    p["dt_max"] = float(raw.get("dt_max", 0.0))
    p["tf_max"] = float(raw.get("tf_max", 0.0))
    for k in ("g_I", "J_B", "r_T_B"):
        p[k] = np.asarray(raw[k], dtype=np.float64)
    p["theta_max"] = raw["theta_max_deg"] * d2r
    p["omega_max"] = raw["omega_max_deg"] * d2r
    p["delta_max"] = raw["delta_max_deg"] * d2r
    p["gamma_gs"] = float(raw.get("gamma_gs_deg", 30.0)) * d2r
    zf = np.zeros(NX)
    zf[1:4] = raw["r_f"]
    zf[4:7] = raw["v_f"]
    zf[7:11] = raw["q_f"]
    zf[11:14] = np.asarray(raw["w_f_deg"]) * d2r
    p["z_f"] = zf
    fix = np.zeros(NX, dtype=np.int32)
    for name in raw["fix_f_nu4" if nu == 4 else "fix_f_nu7"]:
        fix[IDX[name]] = 1
    p["fix_f"] = fix
    px = np.zeros(NX)
    for name, val in raw["P_x"].items():
        px[IDX[name]] = float(val)
    p["P_x"] = px
    pu = np.zeros(7)
    pu[0:3] = raw["P_u"]["T"]
    if nu == 7:
        pu[3:6] = raw["P_u"]["gamma"]
    pu[nu - 1] = raw["P_u"]["s"]
    p["P_u"] = pu
    x0 = np.zeros(14)
    x0[0] = raw["m_wet"]
    x0[1:4] = raw["r0"]
    x0[4:7] = raw["v0"]
    x0[7:11] = raw["q0"]
    x0[11:14] = np.asarray(raw["w0_deg"]) * d2r
    p["x0_nominal"] = x0
    return _override(p, overrides)


def _override(p: Dict, overrides: Dict) -> Dict:
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = type(p[k])(v) if isinstance(p[k], (int, float)) else np.asarray(v, dtype=p[k].dtype)
    return p


def _load_3dof(raw: Dict, overrides: Dict) -> Dict:
    """The 3-DoF parameter set: the 6-DoF keys without the attitude ones
    (J_B, r_T_B, theta_max, omega_max, gamma_max are kept at 0, unused)."""
    d2r = math.pi / 180.0
    p: Dict = {"model": "3dof", "nu": 4}
    for k in ("alpha_mdot", "m_dry", "v_max", "T_min", "T_max", "s_min", "s_max",
              "w_cost", "w_prox", "w_ep", "eps_ctcs", "pipg_omega", "pipg_rho", "pipg_eps_abs",
              "pipg_eps_rel", "pow_eps_abs", "pow_eps_rel", "pow_eps_buff", "scp_eps_step",
              "scp_eps_defect", "tf_guess", "m_wet"):
        p[k] = float(raw[k])
    for k in ("pipg_jmax", "pipg_jcheck", "pow_jmax", "scp_jmax", "rk4_substeps"):
        p[k] = int(raw[k])
    p["soc_thrust"] = int(raw.get("soc_thrust", 0))
    p["glide_slope"] = int(raw.get("glide_slope", 0))
    for k in ("dt_min", "dt_max", "tf_max"):
        p[k] = float(raw.get(k, 0.0))
    p["g_I"] = np.asarray(raw["g_I"], dtype=np.float64)
    p["J_B"] = np.zeros(3)
    p["r_T_B"] = np.zeros(3)
    p["theta_max"] = p["omega_max"] = p["gamma_max"] = 0.0
    p["delta_max"] = raw["delta_max_deg"] * d2r
    p["gamma_gs"] = float(raw.get("gamma_gs_deg", 30.0)) * d2r
    zf = np.zeros(NX_3DOF)
    zf[1:4] = raw["r_f"]
    zf[4:7] = raw["v_f"]
    p["z_f"] = zf
    fix = np.zeros(NX_3DOF, dtype=np.int32)
    for name in raw["fix_f_nu4"]:
        fix[IDX_3DOF[name]] = 1
    p["fix_f"] = fix
    px = np.zeros(NX_3DOF)
    for name, val in raw["P_x"].items():
        px[IDX_3DOF[name]] = float(val)
    p["P_x"] = px
    pu = np.zeros(7)
    pu[0:3] = raw["P_u"]["T"]
    pu[3] = raw["P_u"]["s"]
    p["P_u"] = pu
    x0 = np.zeros(NX_3DOF - 1)
    x0[0] = raw["m_wet"]
    x0[1:4] = raw["r0"]
    x0[4:7] = raw["v0"]
    p["x0_nominal"] = x0
    return _override(p, overrides)


# ---------------------------------------------------------------------------
# counter-based generator: SplitMix64 (Steele, Lea, Flood 2014), one 64-bit
# output per (seed, instance, slot) counter.
# ---------------------------------------------------------------------------

def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, B: int, slot: int) -> np.ndarray:
    """U[0, 1) for instances 0..B-1 at a fixed slot; 53-bit resolution."""
    key = _splitmix64(np.asarray([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    ctr = np.arange(B, dtype=np.uint64) * np.uint64(64) + np.uint64(slot)
    z = _splitmix64(ctr ^ key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _uniform(seed, B, slot, lo, hi):
    return lo + (hi - lo) * uniform01(seed, B, slot)


def _qmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a0, av = a[..., :1], a[..., 1:]
    b0, bv = b[..., :1], b[..., 1:]
    return np.concatenate([a0 * b0 - np.sum(av * bv, axis=-1, keepdims=True),
                           a0 * bv + b0 * av + np.cross(av, bv)], axis=-1)


def dispersion(params: Dict, B: int, seed: int, kind: str = "bj") -> np.ndarray:
    """Dispersed initial conditions x0[B][NX - 1] (float64)."""
    x0n = params["x0_nominal"]
    x0 = np.tile(x0n, (B, 1))
    if kind == "bj":
        x0[:, 0] = x0n[0] * (1.0 + _uniform(seed, B, 0, -0.02, 0.02))
        for i in range(3):
            x0[:, 1 + i] = x0n[1 + i] * (1.0 + _uniform(seed, B, 1 + i, -0.1, 0.1))
            x0[:, 4 + i] = x0n[4 + i] * (1.0 + _uniform(seed, B, 4 + i, -0.1, 0.1))
        if x0.shape[1] < 14:  # 3-DoF: no attitude
            return np.ascontiguousarray(x0)
        zc = _uniform(seed, B, 7, -1.0, 1.0)
        ph = _uniform(seed, B, 8, 0.0, 2.0 * math.pi)
        ang = _uniform(seed, B, 9, 0.0, 5.0 * math.pi / 180.0)
        sr = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
        axis = np.stack([sr * np.cos(ph), sr * np.sin(ph), zc], axis=1)
        dq = np.concatenate([np.cos(ang / 2)[:, None], np.sin(ang / 2)[:, None] * axis], axis=1)
        q = _qmul(np.tile(x0n[7:11], (B, 1)), dq)
        x0[:, 7:11] = q / np.linalg.norm(q, axis=1, keepdims=True)
        d2r = math.pi / 180.0
        for i in range(3):
            x0[:, 11 + i] = x0n[11 + i] + _uniform(seed, B, 10 + i, -2.0 * d2r, 2.0 * d2r)
    elif kind == "paper256":
        x0[:, 1] = _uniform(seed, B, 1, 6.0, 9.0)
        x0[:, 2] = _uniform(seed, B, 2, 3.0, 6.0)
        x0[:, 3] = _uniform(seed, B, 3, 1.0, 2.0)
    elif kind == "nominal":
        pass
    else:
        raise ValueError(f"unknown dispersion {kind!r}")
    return np.ascontiguousarray(x0)


def node_counts(B: int, seed: int, choices: Sequence[int] = (10, 15, 20, 30)) -> np.ndarray:
    """Per-instance node counts N drawn uniformly from `choices` (int32)."""
    u = uniform01(seed, B, 13)
    idx = np.minimum((u * len(choices)).astype(np.int64), len(choices) - 1)
    return np.asarray(choices, dtype=np.int32)[idx]


def config_seed(index: int) -> int:
    """Seed of a named workload: 2404_18034 + workload index."""
    return 240418034 + int(index)
