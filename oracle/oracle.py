"""ctypes wrapper of the CPU oracle (``aero_oracle.c``) -- TEST INFRASTRUCTURE.

The oracle is a plain double-precision restatement of one AERO-MPPI planning
step, used only by the test suite, the smoke check and the benchmark's CPU
baseline.  The CUDA planner never imports this module.  ``build()`` compiles the
C file with gcc (``-ffp-contract=off``: no fused multiply-adds, so the binary32
partition decisions follow the stated operation order).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "aero_oracle.c")
LIB = os.path.join(HERE, "liborc.so")
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liborc.so`` (gcc, plain C11; with OpenMP
    for the per-sample loop of a planning step when gcc offers it, else serial)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                "-o", tmp, SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, LIB)
    return LIB


def set_threads(n: int) -> int:
    """Threads of the per-sample loop of ``plan_step`` (results do not depend on
    it); returns the count in use (1 when built without OpenMP)."""
    return int(lib().orc_set_threads(C.c_int(int(n))))


class Params(C.Structure):
    _fields_ = [
        ("E", C.c_int32), ("K", C.c_int32), ("T", C.c_int32), ("iters", C.c_int32),
        ("dt", C.c_double), ("lam", C.c_double), ("mass", C.c_double), ("g", C.c_double),
        ("sigma", C.c_double * 4), ("u_min", C.c_double * 4), ("u_max", C.c_double * 4),
        ("Q_track", C.c_double), ("Q_vnorm", C.c_double), ("Q_c", C.c_double),
        ("Q_cd", C.c_double), ("Q_p", C.c_double), ("Q_v", C.c_double), ("Q_q", C.c_double),
        ("C_col", C.c_double), ("a_col", C.c_double), ("d_min", C.c_double), ("d_max", C.c_double),
        ("r_max", C.c_double), ("ell", C.c_double), ("v_end", C.c_double),
        ("A_f", C.c_int32), ("E_f", C.c_int32), ("P_a", C.c_int32), ("P_e", C.c_int32),
        ("M_h", C.c_int32), ("M_v", C.c_int32),
        ("el_lo", C.c_double), ("el_hi", C.c_double),
        ("collision_set", C.c_int32), ("pad_", C.c_int32),
        ("v_goal", C.c_double * 3), ("q_goal", C.c_double * 4),
        ("seed", C.c_uint64), ("step_id", C.c_uint64),
        ("refine_steps", C.c_int32), ("pad2_", C.c_int32), ("refine_step", C.c_double),
    ]


def params(d: dict) -> Params:
    """Marshal a parameter dictionary (see ``inputs.default_params``)."""
    p = Params()
    for k in ("E", "K", "T", "iters", "collision_set"):
        setattr(p, k, int(d[k]))
    for k in ("dt", "mass", "g", "Q_track", "Q_vnorm", "Q_c", "Q_cd", "Q_p", "Q_v", "Q_q",
              "C_col", "a_col", "d_min", "d_max", "r_max", "ell", "v_end", "el_lo", "el_hi"):
        setattr(p, k, float(d[k]))
    p.lam = float(d["lam"])
    p.A_f, p.E_f, p.P_a, p.P_e = int(d["fine_az"]), int(d["fine_el"]), int(d["pool_az"]), int(d["pool_el"])
    p.M_h, p.M_v = int(d["M_h"]), int(d["M_v"])
    for k in ("sigma", "u_min", "u_max", "v_goal", "q_goal"):
        arr = getattr(p, k)
        for i, v in enumerate(d[k]):
            arr[i] = float(v)
    p.seed, p.step_id = int(d["seed"]), int(d["step_id"])
    p.refine_steps = int(d.get("refine_steps", 0))
    p.refine_step = float(d.get("refine_step", 0.05))
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            vp = C.c_void_p
            L.orc_partition.restype = C.c_int64
            L.orc_collision_set.restype = C.c_int64
            L.orc_nn_dist.restype = C.c_double
            L.orc_jcol.restype = C.c_double
            L.orc_attitude_err.restype = C.c_double
            L.orc_poly_eval.restype = C.c_double
            L.orc_goal_fine_cell.restype = C.c_int
            for name in ("orc_partition", "orc_collision_set"):
                getattr(L, name).argtypes = None
            L.orc_nn_dist.argtypes = [vp, vp, C.c_int64]
            L.orc_jcol.argtypes = [C.c_double, vp]
            L.orc_attitude_err.argtypes = [vp, vp]
            L.orc_poly_eval.argtypes = [vp, C.c_double]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ----------------------------------------------------------------- primitives

def philox(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def noise(P: dict, e: int, k: int, j: int, it: int = 0) -> np.ndarray:
    out = np.zeros(4)
    pp = params(P)
    lib().orc_noise(C.byref(pp), e, k, j, it, _p(out))
    return out


def noise_block(P: dict, e: int, ks, it: int = 0) -> np.ndarray:
    """delta for samples ks of instance e: len(ks) x T x 4."""
    T = P["T"]
    out = np.zeros((len(ks), T, 4))
    pp = params(P)
    L = lib()
    buf = np.zeros(4)
    for a, k in enumerate(ks):
        for j in range(T):
            L.orc_noise(C.byref(pp), e, int(k), j, it, _p(buf))
            out[a, j] = buf
    return out


def noise_range(P: dict, e: int, k0: int, nk: int, it: int = 0) -> np.ndarray:
    """delta for samples k0 .. k0+nk-1 of instance e: nk x T x 4."""
    out = np.zeros((nk, P["T"], 4))
    pp = params(P)
    lib().orc_noise_fill(C.byref(pp), C.c_int(e), C.c_int(k0), C.c_int(nk), C.c_int(it), _p(out))
    return out


def quat_mul(a, b) -> np.ndarray:
    r = np.zeros(4)
    lib().orc_quat_mul(_p(_f64(a)), _p(_f64(b)), _p(r))
    return r


def rotation(q) -> np.ndarray:
    R = np.zeros(9)
    lib().orc_rotation(_p(_f64(q)), _p(R))
    return R.reshape(3, 3)


def dynamics(x, u, m=1.0, g=9.81) -> np.ndarray:
    xd = np.zeros(10)
    lib().orc_dynamics(_p(_f64(x)), _p(_f64(u)), C.c_double(m), C.c_double(g), _p(xd))
    return xd


def rk4_step(x, u, dt, m=1.0, g=9.81) -> np.ndarray:
    xn = np.zeros(10)
    lib().orc_rk4_step(_p(_f64(x)), _p(_f64(u)), C.c_double(dt), C.c_double(m), C.c_double(g), _p(xn))
    return xn


def rollout(x0, U, dt, m=1.0, g=9.81) -> np.ndarray:
    U = _f64(U).reshape(-1, 4)
    T = U.shape[0]
    X = np.zeros((T + 1, 10))
    lib().orc_rollout(_p(_f64(x0)), _p(U), C.c_int(T), C.c_double(dt), C.c_double(m), C.c_double(g), _p(X))
    return X


def partition(cloud, p0, q0, P: dict) -> tuple[np.ndarray, int]:
    cloud = _f32(cloud).reshape(-1, 3)
    keys = np.zeros(P["fine_az"] * P["fine_el"], np.uint64)
    pp = params(P)
    kept = lib().orc_partition(_p(cloud), C.c_int64(len(cloud)), _p(_f32(p0)), _p(_f32(q0)),
                               C.byref(pp), _p(keys))
    return keys, int(kept)


def goal_fine_cell(goal, p0, q0, P: dict) -> int:
    pp = params(P)
    return int(lib().orc_goal_fine_cell(_p(_f32(goal)), _p(_f32(p0)), _p(_f32(q0)), C.byref(pp)))


def cell_direction(P: dict, c: int) -> np.ndarray:
    d = np.zeros(3)
    pp = params(P)
    lib().orc_cell_direction(C.byref(pp), C.c_int(c), _p(d))
    return d


def coarse(keys, P: dict) -> tuple[np.ndarray, np.ndarray]:
    nc = (P["fine_az"] // P["pool_az"]) * (P["fine_el"] // P["pool_el"])
    win = np.zeros(nc, np.int32)
    rwin = np.zeros(nc)
    pp = params(P)
    lib().orc_coarse(_p(np.ascontiguousarray(keys, np.uint64)), C.byref(pp), _p(win), _p(rwin))
    return win, rwin


def anchor_cells(goal_fine: int, P: dict) -> np.ndarray:
    cells = np.zeros(P["M_h"] * P["M_v"], np.int32)
    pp = params(P)
    lib().orc_anchor_cells(C.c_int(goal_fine), C.byref(pp), _p(cells))
    return cells


def anchor(p0, q0, d_body, ell) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_anchor(_p(_f64(p0)), _p(_f64(q0)), _p(_f64(d_body)), C.c_double(ell), _p(out))
    return out


def quintic(p_s, v_s, a_s, p_e, v_e, a_e, Tg) -> np.ndarray:
    coef = np.zeros(18)
    lib().orc_quintic(*[_p(_f64(a)) for a in (p_s, v_s, a_s, p_e, v_e, a_e)], C.c_double(Tg), _p(coef))
    return coef.reshape(3, 6)


def poly_eval(coef6, t) -> float:
    return float(lib().orc_poly_eval(_p(_f64(coef6)), C.c_double(t)))


def guide(p0, v0, pref, P: dict) -> tuple[np.ndarray, np.ndarray]:
    coef = np.zeros(18)
    g = np.zeros((P["T"], 3))
    pp = params(P)
    lib().orc_guide(_p(_f64(p0)), _p(_f64(v0)), _p(_f64(pref)), C.byref(pp), _p(coef), _p(g))
    return coef.reshape(3, 6), g


def nn_dist(p, pts) -> float:
    pts = _f64(pts).reshape(-1, 3)
    return float(lib().orc_nn_dist(_p(_f64(p)), _p(pts), C.c_int64(len(pts))))


def jcol(d: float, P: dict) -> float:
    pp = params(P)
    return float(lib().orc_jcol(C.c_double(d), C.byref(pp)))


def attitude_err(q, qg) -> float:
    return float(lib().orc_attitude_err(_p(_f64(q)), _p(_f64(qg))))


def cost_terms(X, U, guide_, goal, pts, P: dict, stage: int = 1, want_dist=False):
    """Returns {J_track, J_vnorm, J_ctrl, J_goal, J_col, S} (and d_t if asked)."""
    X = _f64(X).reshape(-1, 10)
    U = _f64(U).reshape(-1, 4)
    pts = _f64(pts).reshape(-1, 3)
    terms = np.zeros(6)
    dist = np.zeros(P["T"])
    gp = _p(_f64(guide_)) if guide_ is not None else None
    pp = params(P)
    lib().orc_cost_terms(_p(X), _p(U), gp, _p(_f64(goal)), _p(pts), C.c_int64(len(pts)),
                         C.byref(pp), C.c_int(stage), _p(terms), _p(dist))
    out = dict(zip(["J_track", "J_vnorm", "J_ctrl", "J_goal", "J_col", "S"], terms.tolist()))
    if want_dist:
        out["dist"] = dist
    return out


def cost_grad(x0, U, guide_, goal, pts, P: dict) -> tuple[float, np.ndarray]:
    """S^(1) of the noise-free rollout of U (T x 4) and dS/dU (reverse mode)."""
    U = _f64(U).reshape(-1, 4)
    pts = _f64(pts).reshape(-1, 3)
    G = np.zeros_like(U)
    pp = params(P)
    gp = _p(_f64(guide_)) if guide_ is not None else None
    L = lib()
    L.orc_cost_grad.restype = C.c_double
    S = L.orc_cost_grad(_p(_f64(x0)), _p(U), gp, _p(_f64(goal)), _p(pts), C.c_int64(len(pts)),
                        C.byref(pp), _p(G))
    return float(S), G


def refine(x0, U, guide_, goal, pts, P: dict) -> np.ndarray:
    """P["refine_steps"] clamped gradient steps of size P["refine_step"] on U."""
    U = _f64(U).reshape(-1, 4).copy()
    pts = _f64(pts).reshape(-1, 3)
    pp = params(P)
    gp = _p(_f64(guide_)) if guide_ is not None else None
    lib().orc_refine(_p(_f64(x0)), _p(U), gp, _p(_f64(goal)), _p(pts), C.c_int64(len(pts)),
                     C.byref(pp))
    return U


def accumulate(ps, p, q) -> np.ndarray:
    """World coordinates p + R(q/|q|) p_s of a frame's sensor-frame points."""
    ps = _f64(ps).reshape(-1, 3)
    out = np.zeros_like(ps)
    lib().orc_accumulate(_p(ps), C.c_int64(len(ps)), _p(_f64(p)), _p(_f64(q)), _p(out))
    return out


def project(pw, p0, q0) -> np.ndarray:
    """Body-frame coordinates R(q0/|q0|)^T (p_w - p0)."""
    pw = _f64(pw).reshape(-1, 3)
    out = np.zeros_like(pw)
    lib().orc_project(_p(pw), C.c_int64(len(pw)), _p(_f64(p0)), _p(_f64(q0)), _p(out))
    return out


def mppi_update(S, dU, lam, u_nom) -> tuple[np.ndarray, np.ndarray]:
    S = _f64(S)
    K = len(S)
    dU = _f64(dU).reshape(K, -1)
    T = dU.shape[1] // 4
    u = _f64(u_nom).copy().reshape(-1)
    eps = np.zeros(K)
    lib().orc_mppi_update(_p(S), _p(dU), C.c_int(K), C.c_int(T), C.c_double(lam), _p(u), _p(eps))
    return u.reshape(T, 4), eps


def collision_set(cloud, p0, q0, keys, P: dict) -> np.ndarray:
    cloud = _f32(cloud).reshape(-1, 3)
    cap = P["fine_az"] * P["fine_el"] if P["collision_set"] == 0 else max(len(cloud), 1)
    pts = np.zeros((cap, 3))
    pp = params(P)
    m = lib().orc_collision_set(_p(cloud), C.c_int64(len(cloud)), _p(_f32(p0)), _p(_f32(q0)),
                                _p(np.ascontiguousarray(keys, np.uint64)), C.byref(pp), _p(pts))
    return pts[:m].copy()


def plan_step(cloud, p0, q0, v0, goal, P: dict, u_nom, debug: bool = True) -> dict:
    """One full planning step.  u_nom: E x T x 4 warm start (not modified)."""
    E, K, T = P["E"], P["K"], P["T"]
    cloud = _f32(cloud).reshape(-1, 3)
    un = _f64(u_nom).copy().reshape(E, T, 4)
    u_best = np.zeros((T, 4))
    cand = np.zeros(E)
    best = np.zeros(1, np.int32)
    nc = P["fine_az"] * P["fine_el"]
    keys = np.zeros(nc, np.uint64) if debug else None
    anchors = np.zeros((E, 3)) if debug else None
    guides = np.zeros((E, T, 3)) if debug else None
    S1 = np.zeros((E, K)) if debug else None
    X2 = np.zeros((E, T + 1, 10)) if debug else None
    pp = params(P)
    opt = (lambda a: _p(a) if a is not None else None)
    lib().orc_plan_step(_p(cloud), C.c_int64(len(cloud)), _p(_f32(p0)), _p(_f32(q0)), _p(_f32(v0)),
                        _p(_f32(goal)), C.byref(pp), _p(un), _p(u_best), _p(cand), _p(best),
                        opt(keys), opt(anchors), opt(guides), opt(S1), opt(X2))
    return dict(u_nom=un, u_best=u_best, cand=cand, best=int(best[0]), keys=keys,
                anchors=anchors, guides=guides, S1=S1, X2=X2)
