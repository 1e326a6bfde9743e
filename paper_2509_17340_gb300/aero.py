"""Python binding of ``libaero_mppi.so`` (ctypes; argument marshalling only).

Every step of the planning path runs in the library's CUDA kernels; this module
only converts torch CUDA tensors and parameter dictionaries into the C ABI of
``include/aero_mppi.h``.  It raises ImportError when the library has not been
built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import library_name

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, library_name())

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2509_17340_gb300.build` (`--checked` for the checked "
                      "build; needs nvcc); there is no CPU fallback")

_lib = C.CDLL(LIB_PATH)

OK = 0
ERR_INVALID_ARG, ERR_EXCEEDS_LIMITS, ERR_CUDA, ERR_ALLOC, ERR_DEVICE_CHECK, ERR_NOT_DEVICE_PTR = (
    -1, -2, -3, -4, -5, -6)

DBG = dict(FINE_KEYS=0, COARSE_WIN=1, GOAL_CELL=2, ANCHOR_CELLS=3, ANCHORS=4, GUIDES=5,
           GRID_META=6, GRID_START=7, GRID_POINTS=8, SAMPLE_COSTS=9, STAGE2_STATES=10,
           SAMPLE_U=11, SAMPLE_X=12, SAMPLE_DIST=13, PRE_REFINE=14, POINT_COUNTS=15)

# element type of each debug buffer (float32 when not listed)
_DBG_DTYPE = {"FINE_KEYS": np.uint64, "COARSE_WIN": np.int32, "GOAL_CELL": np.int32,
              "ANCHOR_CELLS": np.int32, "GRID_START": np.int32, "POINT_COUNTS": np.int64}

STAGES = ["partition", "grid", "rollout", "update"]


class State(C.Structure):
    _fields_ = [("p", C.c_float * 3), ("q", C.c_float * 4), ("v", C.c_float * 3)]


class Limits(C.Structure):
    _fields_ = [("E_max", C.c_int32), ("K_max", C.c_int32), ("T_max", C.c_int32),
                ("fine_cells_max", C.c_int32), ("n_points_max", C.c_int64),
                ("debug_samples_max", C.c_int32), ("raw_points_max", C.c_int32)]


class Params(C.Structure):
    _fields_ = [
        ("E", C.c_int32), ("K", C.c_int32), ("T", C.c_int32), ("iters", C.c_int32),
        ("dt", C.c_float), ("lam", C.c_float), ("mass", C.c_float), ("g", C.c_float),
        ("sigma", C.c_float * 4), ("u_min", C.c_float * 4), ("u_max", C.c_float * 4),
        ("Q_track", C.c_float), ("Q_vnorm", C.c_float), ("Q_c", C.c_float), ("Q_cd", C.c_float),
        ("Q_p", C.c_float), ("Q_v", C.c_float), ("Q_q", C.c_float),
        ("C_col", C.c_float), ("a_col", C.c_float), ("d_min", C.c_float), ("d_max", C.c_float),
        ("r_max", C.c_float), ("ell", C.c_float), ("v_end", C.c_float),
        ("fine_az", C.c_int32), ("fine_el", C.c_int32), ("pool_az", C.c_int32), ("pool_el", C.c_int32),
        ("M_h", C.c_int32), ("M_v", C.c_int32),
        ("el_lo", C.c_float), ("el_hi", C.c_float),
        ("collision_set", C.c_int32),
        ("v_goal", C.c_float * 3), ("q_goal", C.c_float * 4),
        ("debug_samples", C.c_int32), ("lanes_per_sample", C.c_int32),
        ("seed", C.c_uint64), ("step_id", C.c_uint64),
        ("refine_steps", C.c_int32), ("refine_step", C.c_float),
    ]


class BatchItem(C.Structure):
    _fields_ = [("x0", State), ("cloud_xyz", C.c_void_p), ("n_points", C.c_int64),
                ("goal", C.c_float * 3), ("params", Params), ("u_nom_inout", C.c_void_p),
                ("u_best_out", C.c_void_p), ("cand_costs_out", C.c_void_p),
                ("best_idx_out", C.c_void_p)]


class BatchConfig(C.Structure):
    _fields_ = [("quad_max_samples", C.c_int32), ("rollout_ctas_per_sm", C.c_int32),
                ("dynamic_queue", C.c_int32), ("coarse_cells", C.c_int32),
                ("samples_per_cta", C.c_int32)]

    def as_dict(self) -> dict:
        return {"quad_max_samples": self.quad_max_samples,
                "rollout_ctas_per_sm": self.rollout_ctas_per_sm, "dynamic_queue": self.dynamic_queue,
                "coarse_cells": self.coarse_cells, "samples_per_cta": self.samples_per_cta}


_vp = C.c_void_p
_lib.aero_params_default.argtypes = [C.POINTER(Params)]
_lib.aero_params_default.restype = None
_lib.aero_create.argtypes = [C.POINTER(Limits), C.POINTER(_vp)]
_lib.aero_destroy.argtypes = [_vp]
_lib.aero_plan_step.argtypes = [_vp, C.POINTER(State), _vp, C.c_int64, C.POINTER(C.c_float),
                                C.POINTER(Params), _vp, _vp, _vp, _vp, _vp]
_lib.aero_plan_step_host.argtypes = _lib.aero_plan_step.argtypes
_lib.aero_plan_step_noalloc.argtypes = [C.POINTER(State), _vp, C.c_int64, C.POINTER(C.c_float),
                                        C.POINTER(Params), _vp, _vp, _vp, _vp, _vp]
_lib.aero_debug_size.argtypes = [_vp, C.c_int32]
_lib.aero_debug_size.restype = C.c_size_t
_lib.aero_get_debug.argtypes = [_vp, C.c_int32, _vp, C.c_size_t, _vp]
_lib.aero_sync_status.argtypes = [_vp, _vp]
_lib.aero_cost_grad.argtypes = [_vp, C.c_int32, _vp, C.c_int32, _vp, _vp, _vp]
_lib.aero_philox.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64, _vp, _vp]
_lib.aero_profile_enable.argtypes = [_vp, C.c_int]
_lib.aero_profile_read.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
_lib.aero_batch_create.argtypes = [C.POINTER(Limits), C.c_int32, C.POINTER(_vp)]
_lib.aero_batch_plan.argtypes = [_vp, C.POINTER(BatchItem), C.c_int32, _vp]
_lib.aero_batch_destroy.argtypes = [_vp]
_lib.aero_batch_set_config.argtypes = [_vp, C.POINTER(BatchConfig)]
_lib.aero_batch_get_config.argtypes = [_vp, C.POINTER(BatchConfig)]
_lib.aero_batch_tune.argtypes = [_vp, C.POINTER(BatchItem), C.c_int32, C.c_int32, _vp,
                                 C.POINTER(BatchConfig), C.POINTER(C.c_float)]
_lib.aero_batch_sync_status.argtypes = [_vp, C.POINTER(C.c_int32)]
_lib.aero_batch_debug_size.argtypes = [_vp, C.c_int32, C.c_int32]
_lib.aero_batch_debug_size.restype = C.c_size_t
_lib.aero_batch_get_debug.argtypes = [_vp, C.c_int32, C.c_int32, _vp, C.c_size_t, _vp]
_lib.aero_accum_create.argtypes = [C.c_int32, C.c_int64, C.POINTER(_vp)]
_lib.aero_accum_push.argtypes = [_vp, _vp, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_float), _vp]
_lib.aero_accum_view.argtypes = [_vp, C.POINTER(_vp), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
_lib.aero_accum_gather.argtypes = [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float), _vp, C.c_int64,
                                   C.POINTER(C.c_int64), _vp]
_lib.aero_accum_reset.argtypes = [_vp, _vp]
_lib.aero_accum_destroy.argtypes = [_vp]
_lib.aero_shift_nominal.argtypes = [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp]
_lib.aero_test_fail_alloc.argtypes = [C.c_int64]
_lib.aero_test_alloc_stats.argtypes = [C.POINTER(C.c_int64)]
_lib.aero_test_alloc_stats.restype = C.c_int64
_lib.aero_test_raise_check.argtypes = [C.c_int32]
_lib.aero_status_str.argtypes = [C.c_int]
_lib.aero_status_str.restype = C.c_char_p


class AeroError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {status_str(code)} ({code})")


def status_str(code: int) -> str:
    return _lib.aero_status_str(code).decode()


def _check(code: int, what: str):
    if code != OK:
        raise AeroError(code, what)


def lib() -> C.CDLL:
    return _lib


def inject_alloc_failure(n: int) -> None:
    """Make the n-th next library allocation fail once (``aero_test_fail_alloc``);
    n < 0 cancels a pending failure."""
    _lib.aero_test_fail_alloc(int(n))


def raise_check(bits: int) -> int:
    """Checked build: record `bits` as a failed index check (tests); returns the
    status code (AERO_ERR_INVALID_ARG from the product build)."""
    return int(_lib.aero_test_raise_check(int(bits)))


def alloc_stats() -> tuple[int, int]:
    """(allocations made, allocations not yet freed) by the library."""
    live = C.c_int64(0)
    total = _lib.aero_test_alloc_stats(C.byref(live))
    return int(total), int(live.value)


def default_params_struct() -> Params:
    p = Params()
    _lib.aero_params_default(C.byref(p))
    return p


def params_struct(d: dict) -> Params:
    """Marshal a parameter dictionary (``inputs.default_params`` keys)."""
    p = Params()
    for k in ("E", "K", "T", "iters", "collision_set", "debug_samples", "lanes_per_sample"):
        setattr(p, k, int(d.get(k, 0)))
    for k in ("dt", "mass", "g", "Q_track", "Q_vnorm", "Q_c", "Q_cd", "Q_p", "Q_v", "Q_q",
              "C_col", "a_col", "d_min", "d_max", "r_max", "ell", "v_end", "el_lo", "el_hi"):
        setattr(p, k, float(d[k]))
    p.lam = float(d["lam"])
    for k in ("fine_az", "fine_el", "pool_az", "pool_el", "M_h", "M_v"):
        setattr(p, k, int(d[k]))
    for k in ("sigma", "u_min", "u_max", "v_goal", "q_goal"):
        arr = getattr(p, k)
        for i, v in enumerate(d[k]):
            arr[i] = float(v)
    p.seed, p.step_id = int(d["seed"]), int(d["step_id"])
    p.refine_steps = int(d.get("refine_steps", 0))
    p.refine_step = float(d.get("refine_step", 0.05))
    return p


def state_struct(p0, q0, v0) -> State:
    s = State()
    for i in range(3):
        s.p[i] = float(p0[i])
        s.v[i] = float(v0[i])
    for i in range(4):
        s.q[i] = float(q0[i])
    return s


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class RawCloud:
    """A device cloud owned by the library (an accumulator's ring): pointer and
    point count, accepted wherever a cloud tensor is."""

    def __init__(self, ptr: int, n: int, owner=None):
        self.ptr, self.shape, self.owner = int(ptr), (int(n), 3), owner


def _dev(t, dtype, name: str) -> int:
    if isinstance(t, RawCloud) and dtype == torch.float32:
        return t.ptr
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t.data_ptr()


class Planner:
    """Owns an ``aero_planner_t`` (device workspace sized by the limits)."""

    def __init__(self, E_max=64, K_max=8192, T_max=64, fine_cells_max=512 * 64,
                 n_points_max=1 << 18, debug_samples_max=0, device=None, raw_points_max=0):
        if device is not None:
            torch.cuda.set_device(device)
        torch.cuda.init()
        lim = Limits(E_max, K_max, T_max, fine_cells_max, n_points_max, debug_samples_max,
                     raw_points_max)
        h = _vp()
        _check(_lib.aero_create(C.byref(lim), C.byref(h)), "aero_create")
        self._h = h
        self.limits = lim

    def close(self):
        if getattr(self, "_h", None):
            _lib.aero_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def plan_step(self, state: State, cloud: torch.Tensor, goal, params: Params,
                  u_nom: torch.Tensor, u_best: torch.Tensor, cand: torch.Tensor,
                  best_idx: torch.Tensor, stream=None) -> None:
        """Enqueue one planning step on device tensors (u_nom updated in place)."""
        n = cloud.shape[0] if cloud is not None else 0
        cptr = _dev(cloud, torch.float32, "cloud") if n > 0 else None
        g = (C.c_float * 3)(*[float(x) for x in goal])
        rc = _lib.aero_plan_step(self._h, C.byref(state), cptr, n, g, C.byref(params),
                                 _dev(u_nom, torch.float32, "u_nom"),
                                 _dev(u_best, torch.float32, "u_best"),
                                 _dev(cand, torch.float32, "cand"),
                                 _dev(best_idx, torch.int32, "best_idx"), _stream_ptr(stream))
        _check(rc, "aero_plan_step")

    def plan_step_host(self, state: State, cloud: torch.Tensor, goal, params: Params,
                       u_nom: torch.Tensor, u_best: torch.Tensor, cand: torch.Tensor,
                       best_idx: torch.Tensor, stream=None) -> None:
        """One planning step on CPU tensors (pinned for speed); blocks until done."""
        for name, t, dt in (("cloud", cloud, torch.float32), ("u_nom", u_nom, torch.float32),
                            ("u_best", u_best, torch.float32), ("cand", cand, torch.float32),
                            ("best_idx", best_idx, torch.int32)):
            if t.is_cuda or t.dtype != dt or not t.is_contiguous():
                raise TypeError(f"{name} must be a contiguous CPU {dt} tensor")
        n = cloud.shape[0]
        g = (C.c_float * 3)(*[float(x) for x in goal])
        rc = _lib.aero_plan_step_host(self._h, C.byref(state), cloud.data_ptr() if n else None, n, g,
                                      C.byref(params), u_nom.data_ptr(), u_best.data_ptr(),
                                      cand.data_ptr(), best_idx.data_ptr(), _stream_ptr(stream))
        _check(rc, "aero_plan_step_host")

    def debug(self, what: str, stream=None) -> np.ndarray:
        """Copy a debug buffer of the last step to the host (synchronous)."""
        wid = DBG[what]
        stream_p = _stream_ptr(stream)
        if what == "GRID_META":
            buf = np.zeros(8, np.int32)
            _check(_lib.aero_get_debug(self._h, wid, buf.ctypes.data, 32, stream_p), "aero_get_debug")
            return buf
        if what == "GRID_POINTS":
            meta = self.debug("GRID_META", stream)
            buf = np.zeros((int(meta[1]), 4), np.float32)
            _check(_lib.aero_get_debug(self._h, wid, buf.ctypes.data, buf.nbytes, stream_p),
                   "aero_get_debug")
            torch.cuda.synchronize()
            return buf
        nbytes = _lib.aero_debug_size(self._h, wid)
        dtype = _DBG_DTYPE.get(what, np.float32)
        buf = np.zeros(nbytes // np.dtype(dtype).itemsize, dtype)
        _check(_lib.aero_get_debug(self._h, wid, buf.ctypes.data, nbytes, stream_p), "aero_get_debug")
        torch.cuda.synchronize()
        return buf

    def cost_grad(self, instance: int, U: torch.Tensor, S: torch.Tensor,
                  G: torch.Tensor | None = None, stream=None) -> None:
        """S(1) of the noise-free rollouts of U (n x T x 4) for instance
        `instance` of the last step, and dS/dU into G (``aero_cost_grad``)."""
        n = U.shape[0]
        _check(_lib.aero_cost_grad(self._h, instance, _dev(U, torch.float32, "U"), n,
                                   _dev(S, torch.float32, "S"),
                                   _dev(G, torch.float32, "G") if G is not None else None,
                                   _stream_ptr(stream)), "aero_cost_grad")

    def profile(self, stages) -> None:
        """Time the given stages (names from STAGES, True = all, False = none)
        with CUDA events inside every following step."""
        if stages is True:
            mask = (1 << len(STAGES)) - 1
        elif not stages:
            mask = 0
        else:
            mask = sum(1 << STAGES.index(n) for n in stages)
        _check(_lib.aero_profile_enable(self._h, mask), "aero_profile_enable")

    def profile_read(self) -> dict:
        """{stage: (device ms summed since the last read, kernel launches)}."""
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 4)()
        _check(_lib.aero_profile_read(self._h, ms, n), "aero_profile_read")
        return {k: (ms[i], n[i]) for i, k in enumerate(STAGES)}

    def sync_status(self, stream=None) -> int:
        return _lib.aero_sync_status(self._h, _stream_ptr(stream))


def plan_step_noalloc(state: State, cloud: torch.Tensor, goal, params: Params, u_nom: torch.Tensor,
                      u_best: torch.Tensor, cand: torch.Tensor, best_idx: torch.Tensor,
                      stream=None) -> None:
    """The planning step without a planner and without allocating device memory
    (for callers that cannot allocate while running; see aero_plan_step_noalloc
    in include/aero_mppi.h for its limits).  u_nom is updated in place."""
    n = cloud.shape[0] if cloud is not None else 0
    cptr = _dev(cloud, torch.float32, "cloud") if n > 0 else None
    g = (C.c_float * 3)(*[float(x) for x in goal])
    rc = _lib.aero_plan_step_noalloc(C.byref(state), cptr, n, g, C.byref(params),
                                     _dev(u_nom, torch.float32, "u_nom"),
                                     _dev(u_best, torch.float32, "u_best"),
                                     _dev(cand, torch.float32, "cand"),
                                     _dev(best_idx, torch.int32, "best_idx"), _stream_ptr(stream))
    _check(rc, "aero_plan_step_noalloc")


def philox(seed: int, c1: int, c2: int, c3: int, n: int) -> np.ndarray:
    """out[i] = Philox4x32-10((i, c1, c2, c3), seed) computed on the GPU."""
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    _check(_lib.aero_philox(seed, c1, c2, c3, n, out.data_ptr(), _stream_ptr(None)), "aero_philox")
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def plan_step(planner: Planner, p0, q0, v0, cloud: torch.Tensor, goal, params: dict,
              u_nom: torch.Tensor, stream=None):
    """Convenience wrapper: allocate the outputs, run one step, return
    (u_best[T,4], cand[E], best_idx[1]) as CUDA tensors; u_nom is updated in place."""
    T, E = params["T"], params["E"]
    dev = u_nom.device
    u_best = torch.empty((T, 4), dtype=torch.float32, device=dev)
    cand = torch.empty((E,), dtype=torch.float32, device=dev)
    best = torch.empty((1,), dtype=torch.int32, device=dev)
    planner.plan_step(state_struct(p0, q0, v0), cloud, goal, params_struct(params), u_nom, u_best,
                      cand, best, stream)
    return u_best, cand, best


class Batch:
    """Many independent planners planned by one call (``aero_batch_plan``)."""

    def __init__(self, n_max: int, E_max=16, K_max=4096, T_max=64, fine_cells_max=128 * 64,
                 n_points_max=1 << 17, debug_samples_max=0):
        torch.cuda.init()
        lim = Limits(E_max, K_max, T_max, fine_cells_max, n_points_max, debug_samples_max, 0)
        h = _vp()
        _check(_lib.aero_batch_create(C.byref(lim), n_max, C.byref(h)), "aero_batch_create")
        self._h = h
        self.n_max = n_max

    def close(self):
        if getattr(self, "_h", None):
            _lib.aero_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def item(state: State, cloud: torch.Tensor, goal, params: Params, u_nom: torch.Tensor,
             u_best: torch.Tensor, cand: torch.Tensor, best_idx: torch.Tensor) -> BatchItem:
        it = BatchItem()
        it.x0 = state
        n = cloud.shape[0] if cloud is not None else 0
        it.cloud_xyz = _dev(cloud, torch.float32, "cloud") if n > 0 else None
        it.n_points = n
        for i in range(3):
            it.goal[i] = float(goal[i])
        it.params = params
        it.u_nom_inout = _dev(u_nom, torch.float32, "u_nom")
        it.u_best_out = _dev(u_best, torch.float32, "u_best")
        it.cand_costs_out = _dev(cand, torch.float32, "cand")
        it.best_idx_out = _dev(best_idx, torch.int32, "best_idx")
        return it

    def plan(self, items, stream=None) -> None:
        arr = (BatchItem * len(items))(*items)
        _check(_lib.aero_batch_plan(self._h, arr, len(items), _stream_ptr(stream)), "aero_batch_plan")

    def config(self) -> dict:
        c = BatchConfig()
        _check(_lib.aero_batch_get_config(self._h, C.byref(c)), "aero_batch_get_config")
        return c.as_dict()

    def set_config(self, quad_max_samples=0, rollout_ctas_per_sm=0, dynamic_queue=1,
                   coarse_cells=0, samples_per_cta=0) -> None:
        c = BatchConfig(quad_max_samples, rollout_ctas_per_sm, dynamic_queue, coarse_cells,
                        samples_per_cta)
        _check(_lib.aero_batch_set_config(self._h, C.byref(c)), "aero_batch_set_config")

    def tune(self, items, repeats=3, stream=None):
        """Time the configurations of the search space on ``items``; keeps and
        returns the fastest (dict) with its mean time in ms."""
        arr = (BatchItem * len(items))(*items)
        c, ms = BatchConfig(), C.c_float()
        _check(_lib.aero_batch_tune(self._h, arr, len(items), repeats, _stream_ptr(stream),
                                    C.byref(c), C.byref(ms)), "aero_batch_tune")
        return c.as_dict(), ms.value

    def sync_status(self) -> int:
        st = C.c_int32()
        _check(_lib.aero_batch_sync_status(self._h, C.byref(st)), "aero_batch_sync_status")
        return st.value

    def debug(self, slot: int, what: str, stream=None) -> np.ndarray:
        """Copy a debug buffer of slot `slot`'s last step to the host (synchronous)."""
        wid = DBG[what]
        stream_p = _stream_ptr(stream)
        if what == "GRID_META":
            buf = np.zeros(8, np.int32)
        elif what == "GRID_POINTS":
            meta = self.debug(slot, "GRID_META", stream)
            buf = np.zeros((int(meta[1]), 4), np.float32)
        else:
            nbytes = _lib.aero_batch_debug_size(self._h, slot, wid)
            dtype = _DBG_DTYPE.get(what, np.float32)
            buf = np.zeros(nbytes // np.dtype(dtype).itemsize, dtype)
        _check(_lib.aero_batch_get_debug(self._h, slot, wid, buf.ctypes.data, buf.nbytes, stream_p),
               "aero_batch_get_debug")
        torch.cuda.synchronize()
        return buf


def shift_nominal(u_nom: torch.Tensor, shift: int, scratch: torch.Tensor | None = None,
                  stream=None) -> None:
    """Receding-horizon warm start in place (``aero_shift_nominal``): u_nom
    (E x T x 4 CUDA tensor) advanced by `shift` steps, the last control repeated."""
    E, T = u_nom.shape[0], u_nom.shape[1]
    if scratch is None:
        scratch = torch.empty_like(u_nom)
    _check(_lib.aero_shift_nominal(_dev(u_nom, torch.float32, "u_nom"), E, T, int(shift),
                                   _dev(scratch, torch.float32, "scratch"), _stream_ptr(stream)),
           "aero_shift_nominal")


class Accumulator:
    """Ring of LiDAR frames in world coordinates on the device (``aero_accum_*``,
    Sec. IV-A.1): push sensor-frame sweeps with their capture poses; plan on
    ``view()`` (the NaN-padded ring) or on a compacted ``gather``."""

    def __init__(self, frames: int = 10, points_per_frame: int = 20000):
        torch.cuda.init()
        h = _vp()
        _check(_lib.aero_accum_create(frames, points_per_frame, C.byref(h)), "aero_accum_create")
        self._h = h
        self.frames, self.points_per_frame = frames, points_per_frame

    def close(self):
        if getattr(self, "_h", None):
            _lib.aero_accum_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, pts: torch.Tensor, p, q, stream=None) -> None:
        n = pts.shape[0]
        pp = (C.c_float * 3)(*[float(x) for x in p])
        qq = (C.c_float * 4)(*[float(x) for x in q])
        _check(_lib.aero_accum_push(self._h, _dev(pts, torch.float32, "pts") if n else None, n, pp, qq,
                                    _stream_ptr(stream)), "aero_accum_push")

    def view(self) -> tuple[RawCloud, int]:
        """The ring as a cloud (frames x points_per_frame points) and the number
        of real (non-padding) points in it."""
        ptr, n, v = _vp(), C.c_int64(), C.c_int64()
        _check(_lib.aero_accum_view(self._h, C.byref(ptr), C.byref(n), C.byref(v)), "aero_accum_view")
        return RawCloud(ptr.value, n.value, self), v.value

    def gather(self, dst: torch.Tensor, p0=None, q0=None, stream=None) -> int:
        """Live frames, oldest first, compacted into dst (world, or the body
        frame of (p0, q0)); returns the number of points written."""
        n = C.c_int64()
        pp = (C.c_float * 3)(*[float(x) for x in p0]) if p0 is not None else None
        qq = (C.c_float * 4)(*[float(x) for x in q0]) if q0 is not None else None
        _check(_lib.aero_accum_gather(self._h, pp, qq, _dev(dst, torch.float32, "dst"), dst.shape[0],
                                      C.byref(n), _stream_ptr(stream)), "aero_accum_gather")
        return n.value

    def reset(self, stream=None) -> None:
        _check(_lib.aero_accum_reset(self._h, _stream_ptr(stream)), "aero_accum_reset")


class RolloutCost(torch.autograd.Function):
    """S(1) of noise-free rollouts as a differentiable torch function:
    forward runs ``aero_cost_grad`` (cost and adjoint gradient in one kernel),
    backward scales the saved gradient.  ``RolloutCost.apply(U, planner,
    instance)`` with U an (n, T, 4) float32 CUDA tensor returns S (n,); the
    planner's last step supplies the state, guide, collision grid and weights."""

    @staticmethod
    def forward(ctx, U, planner, instance):
        U = U.detach().contiguous()
        S = torch.empty(U.shape[0], dtype=torch.float32, device=U.device)
        G = torch.empty_like(U)
        planner.cost_grad(int(instance), U, S, G, torch.cuda.current_stream(U.device))
        ctx.save_for_backward(G)
        return S

    @staticmethod
    def backward(ctx, gS):
        (G,) = ctx.saved_tensors
        return gS[:, None, None] * G, None, None
