"""ctypes binding of the MGWR C ABI (include/mgwr.h).

Argument marshalling only: every numerical step runs in the CUDA library
``libmgwr.so`` built in-tree by ``paper_1608_05400_gb300._build``.  There is
no fallback: if the library is missing or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmgwr.so")

MGWR_OK = 0
MGWR_E_INVAL = -1
MGWR_E_NOMEM = -2
MGWR_E_TOOBIG = -3
MGWR_E_NOCONV = -4
MGWR_E_NUMERIC = -5
MGWR_E_AGAIN = -6
MGWR_E_TIMEOUT = -7
MGWR_E_CUDA = -8
MGWR_E_STATE = -9

MGWR_FP64, MGWR_MIXED, MGWR_MIXED_DD, MGWR_DD, MGWR_AUTO = 0, 1, 2, 3, 4
MGWR_H64, MGWR_H32, MGWR_HDD = 64, 32, 48
MGWR_U, MGWR_F, MGWR_R = 0, 1, 2
MGWR_RED, MGWR_BLACK = 0, 1
MGWR_ORDER_TEXT, MGWR_ORDER_TABLE = 0, 1
MGWR_FAS_D_POROUS, MGWR_FAS_D_CONSTANT = 0, 1
MGWR_FAS_SMOOTHER_AUTO, MGWR_FAS_SMOOTHER_MARCH, MGWR_FAS_SMOOTHER_FIXED = 0, 1, 2
MGWR_POLICY_FIFO, MGWR_POLICY_SMALLEST = 0, 1
MGWR_SPLIT_STAGED = 16
MGWR_SPLIT_TENSOR = 32
MGWR_SPLIT_RADIX = 64


class mgwr_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("outer", C.c_int), ("relres", C.c_double),
                ("factor", C.c_double), ("seconds", C.c_double)]


class mgwr_request(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int), ("M", C.c_int), ("T", C.c_double),
                ("alpha", C.c_double), ("f", C.POINTER(C.c_double)), ("g", C.POINTER(C.c_double)),
                ("precision", C.c_int), ("order", C.c_int), ("cycle", C.c_int), ("nu1", C.c_int),
                ("nu2", C.c_int), ("tol", C.c_double), ("max_cycles", C.c_int)]


class mgwr_result(C.Structure):
    _fields_ = [("status", C.c_int), ("stats", mgwr_stats), ("queue_s", C.c_double),
                ("latency_s", C.c_double)]


class mgwr_server_info(C.Structure):
    _fields_ = [("queued", C.c_longlong), ("admitted", C.c_longlong), ("completed", C.c_longlong),
                ("in_use_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("budget_bytes", C.c_size_t), ("slots", C.c_int),
                ("max_group_members", C.c_int), ("group_launches", C.c_longlong),
                ("member_iterations", C.c_longlong), ("reused_handles", C.c_longlong),
                ("submit_copy_s", C.c_double), ("prepare_s", C.c_double),
                ("finish_s", C.c_double), ("pin_s", C.c_double),
                ("pinned_buffers", C.c_longlong)]


_h = C.c_void_p
_dp = C.POINTER(C.c_double)
_SIGS = {
    "mgwr_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(_h)]),
    "mgwr_create_batch": (C.c_int, [C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_int, C.POINTER(_h)]),
    "mgwr_batch_size": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "mgwr_set_problem": (C.c_int, [_h, _dp, _dp]),
    "mgwr_group_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "mgwr_group_destroy": (C.c_int, [C.c_void_p]),
    "mgwr_group_last_error": (C.c_char_p, [C.c_void_p]),
    "mgwr_group_add": (C.c_int, [C.c_void_p, _h, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int]),
    "mgwr_group_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "mgwr_group_collect": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int),
                                     C.POINTER(mgwr_stats)]),
    "mgwr_group_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                  C.POINTER(C.c_int)]),
    "mgwr_group_solve": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(mgwr_stats)]),
    "mgwr_instance_relres": (C.c_int, [_h, _dp]),
    "mgwr_destroy": (C.c_int, [_h]),
    "mgwr_last_error": (C.c_char_p, [_h]),
    "mgwr_status_string": (C.c_char_p, [C.c_int]),
    "mgwr_set_precision": (C.c_int, [_h, C.c_int]),
    "mgwr_set_order": (C.c_int, [_h, C.c_int]),
    "mgwr_set_stream": (C.c_int, [_h, C.c_void_p]),
    "mgwr_set_inner_cycles": (C.c_int, [_h, C.c_int]),
    "mgwr_set_outer_switch": (C.c_int, [_h, C.c_double]),
    "mgwr_set_engine_split": (C.c_int, [_h, C.c_int, C.c_int, C.c_int]),
    "mgwr_get_engine_split": (C.c_int, [_h, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "mgwr_autotune": (C.c_int, [_h]),
    "mgwr_set_graphs": (C.c_int, [_h, C.c_int]),
    "mgwr_set_device_loop": (C.c_int, [_h, C.c_int]),
    "mgwr_stage_rhs": (C.c_int, [_h, _dp]),
    "mgwr_take_rhs": (C.c_int, [_h]),
    "mgwr_stage_solution": (C.c_int, [_h, _dp]),
    "mgwr_wait_staged": (C.c_int, [_h]),
    "mgwr_set_rhs": (C.c_int, [_h, _dp, _dp]),
    "mgwr_set_rhs_dev": (C.c_int, [_h, C.c_void_p, C.c_void_p]),
    "mgwr_set_initial": (C.c_int, [_h, _dp]),
    "mgwr_solve": (C.c_int, [_h, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(mgwr_stats)]),
    "mgwr_residual": (C.c_int, [_h, _dp, _dp]),
    "mgwr_get_solution": (C.c_int, [_h, _dp]),
    "mgwr_get_solution_dev": (C.c_int, [_h, C.c_void_p]),
    "mgwr_num_levels": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "mgwr_level_n": (C.c_int, [_h, C.c_int, C.POINTER(C.c_int)]),
    "mgwr_field_set": (C.c_int, [_h, C.c_int, C.c_int, C.c_int, _dp]),
    "mgwr_field_get": (C.c_int, [_h, C.c_int, C.c_int, C.c_int, _dp]),
    "mgwr_smooth": (C.c_int, [_h, C.c_int, C.c_int, C.c_int]),
    "mgwr_defect": (C.c_int, [_h, C.c_int, C.c_int, _dp]),
    "mgwr_smooth_defect": (C.c_int, [_h, C.c_int, C.c_int, _dp]),
    "mgwr_restrict": (C.c_int, [_h, C.c_int, C.c_int]),
    "mgwr_smooth_restrict": (C.c_int, [_h, C.c_int, C.c_int]),
    "mgwr_prolong": (C.c_int, [_h, C.c_int, C.c_int]),
    "mgwr_coarsest": (C.c_int, [_h, C.c_int]),
    "mgwr_cycle": (C.c_int, [_h, C.c_int, C.c_int, C.c_int, C.c_int]),
    "mgwr_toeplitz_column": (C.c_int, [_h, _dp]),
    "mgwr_inverse_column": (C.c_int, [_h, C.c_int, _dp]),
    "mgwr_launch_count": (C.c_int, [_h, C.POINTER(C.c_longlong)]),
    "mgwr_peak_probe": (C.c_int, [_dp, _dp]),
    "mgwr_inverse_column_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "mgwr_footprint": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "mgwr_auto_precision": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "mgwr_get_precision": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "mgwr_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
    "mgwr_server_destroy": (C.c_int, [C.c_void_p]),
    "mgwr_server_set_policy": (C.c_int, [C.c_void_p, C.c_int]),
    "mgwr_submit": (C.c_int, [C.c_void_p, C.POINTER(mgwr_request), C.POINTER(C.c_uint64)]),
    "mgwr_server_buffer": (C.c_int, [C.c_void_p, C.c_size_t, C.POINTER(_dp)]),
    "mgwr_submit_buffer": (C.c_int, [C.c_void_p, C.POINTER(mgwr_request), _dp,
                                     C.POINTER(C.c_uint64)]),
    "mgwr_server_release": (C.c_int, [C.c_void_p, _dp]),
    "mgwr_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, _dp, C.POINTER(mgwr_result)]),
    "mgwr_server_stats": (C.c_int, [C.c_void_p, C.POINTER(mgwr_server_info)]),
    "mgwr_profile": (C.c_int, [_h, C.c_int]),
    "mgwr_profile_read": (C.c_int, [_h, C.c_int, C.POINTER(C.c_longlong), _dp, _dp]),
    "mgwr_fas_create": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                  C.POINTER(_h)]),
    "mgwr_fas_destroy": (C.c_int, [_h]),
    "mgwr_fas_last_error": (C.c_char_p, [_h]),
    "mgwr_fas_set_order": (C.c_int, [_h, C.c_int]),
    "mgwr_fas_set_smoother": (C.c_int, [_h, C.c_int]),
    "mgwr_fas_line_iterations": (C.c_int, [_h, C.POINTER(C.c_longlong)]),
    "mgwr_fas_reset": (C.c_int, [_h]),
    "mgwr_fas_set_stream": (C.c_int, [_h, C.c_void_p]),
    "mgwr_fas_set_rhs": (C.c_int, [_h, _dp]),
    "mgwr_fas_set_initial": (C.c_int, [_h, _dp]),
    "mgwr_fas_solve": (C.c_int, [_h, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                 C.POINTER(mgwr_stats)]),
    "mgwr_fas_cycle": (C.c_int, [_h, C.c_int, C.c_int, C.c_int]),
    "mgwr_fas_residual": (C.c_int, [_h, _dp, _dp]),
    "mgwr_fas_get_solution": (C.c_int, [_h, _dp]),
    "mgwr_fas_levels": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "mgwr_fas_smooth": (C.c_int, [_h, C.c_int, C.c_int]),
    "mgwr_fas_defect": (C.c_int, [_h, C.c_int, _dp]),
    "mgwr_fas_field_set": (C.c_int, [_h, C.c_int, C.c_int, _dp]),
    "mgwr_fas_field_get": (C.c_int, [_h, C.c_int, C.c_int, _dp]),
}

KERNEL_CLASSES = ("sweep64", "sweep32", "defect64", "defect32", "restrict", "prolong",
                  "coarsest", "refine", "defect_delta", "defect_dd", "sweep_dd")

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libmgwr.so (raises OSError / RuntimeError if it is absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_1608_05400_gb300._build)")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


class MGWRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Stats:
    cycles: int
    outer: int
    relres: float
    factor: float
    seconds: float
    status: int


class Solver:
    """MGWR problems (d, n, M) on the current CUDA device: one instance
    (T and alpha scalars) or a batch (T and alpha sequences of equal length).
    Field arrays are (N, M) for one instance and (batch, N, M) for a batch."""

    def __init__(self, d: int, n: int, M: int, T, alpha):
        self.lib = load()
        self.batched = np.ndim(alpha) > 0
        alphas = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
        Ts = np.broadcast_to(np.asarray(T, dtype=np.float64), alphas.shape).copy()
        self.d, self.n, self.M, self.T, self.alpha = d, n, M, T, alpha
        self.N = n ** d
        self.B = int(alphas.size)
        h = _h()
        st = self.lib.mgwr_create_batch(d, n, M, _ptr(Ts), _ptr(alphas), self.B, C.byref(h))
        if st != MGWR_OK:
            raise MGWRError(st, f"mgwr_create_batch({d}, {n}, {M}, batch={self.B}) failed: "
                            + self.lib.mgwr_status_string(st).decode())
        self.h = h

    def _shape(self, N=None):
        N = self.N if N is None else N
        return (self.B, N, self.M) if self.batched else (N, self.M)

    # -- plumbing --
    def _check(self, st: int, what: str, ok=(MGWR_OK,)):
        if st not in ok:
            raise MGWRError(st, f"{what}: {self.lib.mgwr_last_error(self.h).decode()}")
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.mgwr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration --
    def set_problem(self, T, alpha):
        """New final times and orders for the instances, set up in place."""
        alphas = np.atleast_1d(np.asarray(alpha, dtype=np.float64)).copy()
        Ts = np.broadcast_to(np.asarray(T, dtype=np.float64), alphas.shape).copy()
        assert alphas.size == self.B
        self._check(self.lib.mgwr_set_problem(self.h, _ptr(Ts), _ptr(alphas)), "mgwr_set_problem")
        self.T, self.alpha = T, alpha

    def set_precision(self, prec: int):
        self._check(self.lib.mgwr_set_precision(self.h, prec), "mgwr_set_precision")

    def precision(self) -> int:
        v = C.c_int()
        self._check(self.lib.mgwr_get_precision(self.h, C.byref(v)), "mgwr_get_precision")
        return v.value

    def set_order(self, order: int):
        self._check(self.lib.mgwr_set_order(self.h, order), "mgwr_set_order")

    def set_stream(self, stream_ptr: int | None):
        self._check(self.lib.mgwr_set_stream(self.h, C.c_void_p(stream_ptr or 0)), "mgwr_set_stream")

    def set_graphs(self, enable: bool):
        self._check(self.lib.mgwr_set_graphs(self.h, int(enable)), "mgwr_set_graphs")

    def set_device_loop(self, enable: bool):
        self._check(self.lib.mgwr_set_device_loop(self.h, int(enable)), "mgwr_set_device_loop")

    def set_inner_cycles(self, k: int):
        self._check(self.lib.mgwr_set_inner_cycles(self.h, k), "mgwr_set_inner_cycles")

    def set_outer_switch(self, rel: float):
        self._check(self.lib.mgwr_set_outer_switch(self.h, float(rel)), "mgwr_set_outer_switch")

    def set_engine_split(self, kernel_class: int, split: int, level: int = -1):
        """E for one level, or every level (level -1)."""
        self._check(self.lib.mgwr_set_engine_split(self.h, kernel_class, level, split),
                    "mgwr_set_engine_split")

    def engine_split(self, kernel_class: int, level: int = -1) -> int:
        """E used on one level (level -1: the finest)."""
        e = C.c_int()
        self._check(self.lib.mgwr_get_engine_split(self.h, kernel_class, level, C.byref(e)),
                    "mgwr_get_engine_split")
        return e.value

    def autotune(self) -> dict:
        """Run the launch-shape tuner; returns, per engine class, the split chosen
        on each level (coarsest first)."""
        self._check(self.lib.mgwr_autotune(self.h), "mgwr_autotune")
        return {name: [self.engine_split(k, l) for l in range(self.num_levels())]
                for k, name in enumerate(KERNEL_CLASSES)
                if name in ("sweep64", "sweep32", "defect64", "defect32", "defect_dd", "sweep_dd")}

    # -- data --
    def set_rhs(self, f: np.ndarray, g: np.ndarray | None = None):
        f = _f64(f)
        assert f.shape == self._shape(), f.shape
        g = None if g is None else _f64(g).reshape(self.B * self.N)
        self._check(self.lib.mgwr_set_rhs(self.h, _ptr(f), _ptr(g)), "mgwr_set_rhs")

    def set_rhs_dev(self, f_ptr: int, g_ptr: int | None = None):
        self._check(self.lib.mgwr_set_rhs_dev(self.h, C.c_void_p(f_ptr), C.c_void_p(g_ptr or 0)),
                    "mgwr_set_rhs_dev")

    def set_initial(self, u0: np.ndarray):
        u0 = _f64(u0)
        assert u0.shape == self._shape()
        self._check(self.lib.mgwr_set_initial(self.h, _ptr(u0)), "mgwr_set_initial")

    def solve(self, cycle=1, nu1=1, nu2=1, tol=1e-10, max_cycles=100, allow_noconv=False) -> Stats:
        st = mgwr_stats()
        ok = (MGWR_OK, MGWR_E_NOCONV) if allow_noconv else (MGWR_OK,)
        s = self._check(self.lib.mgwr_solve(self.h, cycle, nu1, nu2, tol, max_cycles, C.byref(st)),
                        "mgwr_solve", ok)
        return Stats(st.cycles, st.outer, st.relres, st.factor, st.seconds, s)

    def residual(self, want_field=False):
        rel = C.c_double()
        r = np.empty(self._shape()) if want_field else None
        self._check(self.lib.mgwr_residual(self.h, C.byref(rel), _ptr(r)), "mgwr_residual")
        return (rel.value, r) if want_field else rel.value

    def instance_relres(self) -> np.ndarray:
        out = np.empty(self.B)
        self._check(self.lib.mgwr_instance_relres(self.h, _ptr(out)), "mgwr_instance_relres")
        return out

    def solution(self) -> np.ndarray:
        u = np.empty(self._shape())
        self._check(self.lib.mgwr_get_solution(self.h, _ptr(u)), "mgwr_get_solution")
        return u

    # -- pipelined transfers (mgwr_stage_rhs ...): the caller keeps the host arrays
    #    alive and unchanged until wait_staged (pinned arrays let the copies overlap)
    def stage_rhs(self, f: np.ndarray):
        assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == self._shape()
        self._check(self.lib.mgwr_stage_rhs(self.h, _ptr(f)), "mgwr_stage_rhs")

    def take_rhs(self):
        self._check(self.lib.mgwr_take_rhs(self.h), "mgwr_take_rhs")

    def stage_solution(self, u: np.ndarray):
        assert u.dtype == np.float64 and u.flags.c_contiguous and u.shape == self._shape()
        self._check(self.lib.mgwr_stage_solution(self.h, _ptr(u)), "mgwr_stage_solution")

    def wait_staged(self):
        self._check(self.lib.mgwr_wait_staged(self.h), "mgwr_wait_staged")

    def solution_dev(self, u_ptr: int):
        self._check(self.lib.mgwr_get_solution_dev(self.h, C.c_void_p(u_ptr)), "mgwr_get_solution_dev")

    # -- components --
    def num_levels(self) -> int:
        v = C.c_int()
        self._check(self.lib.mgwr_num_levels(self.h, C.byref(v)), "mgwr_num_levels")
        return v.value

    def level_n(self, level: int) -> int:
        v = C.c_int()
        self._check(self.lib.mgwr_level_n(self.h, level, C.byref(v)), "mgwr_level_n")
        return v.value

    def field_set(self, hier: int, level: int, which: int, a: np.ndarray):
        a = _f64(a)
        nl = self.level_n(level)
        assert a.shape == self._shape(nl ** self.d), a.shape
        self._check(self.lib.mgwr_field_set(self.h, hier, level, which, _ptr(a)), "mgwr_field_set")

    def field_get(self, hier: int, level: int, which: int) -> np.ndarray:
        nl = self.level_n(level)
        a = np.empty(self._shape(nl ** self.d))
        self._check(self.lib.mgwr_field_get(self.h, hier, level, which, _ptr(a)), "mgwr_field_get")
        return a

    def smooth(self, hier: int, level: int, colour: int):
        self._check(self.lib.mgwr_smooth(self.h, hier, level, colour), "mgwr_smooth")

    def defect(self, hier: int, level: int) -> float:
        v = C.c_double()
        self._check(self.lib.mgwr_defect(self.h, hier, level, C.byref(v)), "mgwr_defect")
        return v.value

    def smooth_defect(self, hier: int, level: int) -> float:
        v = C.c_double()
        self._check(self.lib.mgwr_smooth_defect(self.h, hier, level, C.byref(v)), "mgwr_smooth_defect")
        return v.value

    def restrict(self, hier: int, level: int):
        self._check(self.lib.mgwr_restrict(self.h, hier, level), "mgwr_restrict")

    def smooth_restrict(self, hier: int, level: int):
        self._check(self.lib.mgwr_smooth_restrict(self.h, hier, level), "mgwr_smooth_restrict")

    def prolong(self, hier: int, level: int):
        self._check(self.lib.mgwr_prolong(self.h, hier, level), "mgwr_prolong")

    def coarsest(self, hier: int):
        self._check(self.lib.mgwr_coarsest(self.h, hier), "mgwr_coarsest")

    def cycle(self, hier: int, cycle=1, nu1=1, nu2=1):
        self._check(self.lib.mgwr_cycle(self.h, hier, cycle, nu1, nu2), "mgwr_cycle")

    def profile(self, enable: bool):
        self._check(self.lib.mgwr_profile(self.h, int(enable)), "mgwr_profile")

    def profile_read(self) -> dict:
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            n, ms, lines = C.c_longlong(), C.c_double(), C.c_double()
            self._check(self.lib.mgwr_profile_read(self.h, k, C.byref(n), C.byref(ms), C.byref(lines)),
                        "mgwr_profile_read")
            out[name] = dict(launches=n.value, ms=ms.value, lines=lines.value)
        return out

    def toeplitz_column(self) -> np.ndarray:
        r = np.empty((self.B, self.M) if self.batched else self.M)
        self._check(self.lib.mgwr_toeplitz_column(self.h, _ptr(r)), "mgwr_toeplitz_column")
        return r

    def inverse_column(self, level: int) -> np.ndarray:
        k = np.empty((self.B, self.M) if self.batched else self.M)
        self._check(self.lib.mgwr_inverse_column(self.h, level, _ptr(k)), "mgwr_inverse_column")
        return k


def auto_precision(d: int, n: int, M: int, precision: int = MGWR_AUTO) -> int:
    """The precision MGWR_AUTO resolves to on this grid (others unchanged)."""
    v = C.c_int()
    st = load().mgwr_auto_precision(d, n, M, precision, C.byref(v))
    if st != MGWR_OK:
        raise MGWRError(st, "mgwr_auto_precision: invalid shape or precision")
    return v.value


def footprint(d: int, n: int, M: int, batch: int = 1, precision: int = MGWR_FP64) -> int:
    v = C.c_size_t()
    st = load().mgwr_footprint(d, n, M, batch, precision, C.byref(v))
    if st != MGWR_OK:
        raise MGWRError(st, "mgwr_footprint: invalid shape")
    return v.value


@dataclass
class Result:
    status: int
    stats: Stats
    queue_s: float
    latency_s: float
    u: np.ndarray | None


class Server:
    """Request queue with HBM-budget admission and concurrent slots (mgwr_submit / mgwr_poll)."""

    def __init__(self, hbm_budget: int, slots: int = 4):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.mgwr_server_create(hbm_budget, slots, C.byref(h))
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_server_create failed")
        self.h = h
        self._shapes = {}

    def set_policy(self, policy: int):
        st = self.lib.mgwr_server_set_policy(self.h, policy)
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_server_set_policy")

    def submit(self, d, n, M, T, alpha, f, g=None, precision=MGWR_MIXED, order=MGWR_ORDER_TEXT,
               cycle=1, nu1=1, nu2=1, tol=1e-8, max_cycles=100) -> int:
        f = _f64(f)
        N = n ** d
        assert f.shape == (N, M), f.shape
        gg = None if g is None else _f64(g).reshape(N)
        rq = mgwr_request(d, n, M, T, alpha, _ptr(f), _ptr(gg), precision, order, cycle, nu1, nu2,
                          tol, max_cycles)
        t = C.c_uint64()
        st = self.lib.mgwr_submit(self.h, C.byref(rq), C.byref(t))
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_submit: " + self.lib.mgwr_status_string(st).decode())
        self._shapes[t.value] = (N, M)
        return t.value

    def buffer(self, N: int, M: int) -> np.ndarray:
        """A page-locked (N, M) float64 array lent from the server's pool
        (mgwr_server_buffer): write f into it and hand it to submit_buffer, or
        give it back with release.  The array must not be used after either."""
        p = _dp()
        st = self.lib.mgwr_server_buffer(self.h, N * M, C.byref(p))
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_server_buffer")
        return np.ctypeslib.as_array(p, shape=(N, M))

    def submit_buffer(self, d, n, M, T, alpha, buf: np.ndarray, g=None, precision=MGWR_MIXED,
                      order=MGWR_ORDER_TEXT, cycle=1, nu1=1, nu2=1, tol=1e-8,
                      max_cycles=100) -> int:
        """submit() of f held in an array from buffer(), without a copy
        (mgwr_submit_buffer); on success the server owns the array's memory."""
        N = n ** d
        assert buf.shape == (N, M) and buf.dtype == np.float64, (buf.shape, buf.dtype)
        gg = None if g is None else _f64(g).reshape(N)
        p = buf.ctypes.data_as(_dp)
        rq = mgwr_request(d, n, M, T, alpha, p, _ptr(gg), precision, order, cycle, nu1, nu2, tol,
                          max_cycles)
        t = C.c_uint64()
        st = self.lib.mgwr_submit_buffer(self.h, C.byref(rq), p, C.byref(t))
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_submit_buffer: " + self.lib.mgwr_status_string(st).decode())
        self._shapes[t.value] = (N, M)
        return t.value

    def release(self, buf: np.ndarray):
        st = self.lib.mgwr_server_release(self.h, buf.ctypes.data_as(_dp))
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_server_release")

    def poll(self, ticket: int, timeout_us: int = 0, copy_solution: bool = True) -> Result | None:
        N, M = self._shapes[ticket]
        u = np.empty((N, M)) if copy_solution else None
        res = mgwr_result()
        st = self.lib.mgwr_poll(self.h, ticket, timeout_us, _ptr(u), C.byref(res))
        if st in (MGWR_E_AGAIN, MGWR_E_TIMEOUT):
            return None
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_poll")
        del self._shapes[ticket]
        s = res.stats
        ok = res.status in (MGWR_OK, MGWR_E_NOCONV)
        return Result(res.status, Stats(s.cycles, s.outer, s.relres, s.factor, s.seconds, res.status),
                      res.queue_s, res.latency_s, u if ok and copy_solution else None)

    def info(self) -> dict:
        i = mgwr_server_info()
        self.lib.mgwr_server_stats(self.h, C.byref(i))
        return {k: getattr(i, k) for k, _ in mgwr_server_info._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.mgwr_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Solvers advancing together (mgwr_group_*): every iteration of all running
    members is one CUDA graph launch; results are bitwise those of solo solves."""

    def __init__(self):
        self.lib = load()
        g = C.c_void_p()
        st = self.lib.mgwr_group_create(C.byref(g))
        if st != MGWR_OK:
            raise MGWRError(st, "mgwr_group_create failed")
        self.g = g
        self.members = {}

    def _check(self, st: int, what: str, solver=None, ok=(MGWR_OK,)):
        if st not in ok:
            msg = (self.lib.mgwr_last_error(solver.h).decode() if solver is not None
                   else self.lib.mgwr_group_last_error(self.g).decode())
            raise MGWRError(st, f"{what}: {msg}")
        return st

    def add(self, solver: "Solver", cycle=1, nu1=1, nu2=1, tol=1e-10, max_cycles=100):
        self._check(self.lib.mgwr_group_add(self.g, solver.h, cycle, nu1, nu2, tol, max_cycles),
                    "mgwr_group_add", solver)
        self.members[solver.h.value] = solver

    def step(self) -> int:
        left = C.c_int()
        self._check(self.lib.mgwr_group_step(self.g, C.byref(left)), "mgwr_group_step")
        return left.value

    def collect(self):
        """[(solver, Stats)] of the members finished since the last call."""
        out = []
        while True:
            h, code, st = C.c_void_p(), C.c_int(), mgwr_stats()
            if self.lib.mgwr_group_collect(self.g, C.byref(h), C.byref(code), C.byref(st)) != MGWR_OK:
                return out
            solver = self.members.pop(h.value)
            out.append((solver, Stats(st.cycles, st.outer, st.relres, st.factor, st.seconds,
                                      code.value)))

    def run(self):
        """Steps until every member has finished; returns collect()'s list."""
        while self.step() > 0:
            pass
        return self.collect()

    def info(self) -> dict:
        a, b, c = C.c_longlong(), C.c_longlong(), C.c_int()
        self._check(self.lib.mgwr_group_info(self.g, C.byref(a), C.byref(b), C.byref(c)), "info")
        return {"launches": a.value, "member_iterations": b.value, "max_members": c.value}

    def close(self):
        if getattr(self, "g", None):
            self.lib.mgwr_group_destroy(self.g)
            self.g = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    v = C.c_longlong()
    load().mgwr_launch_count(None, C.byref(v))
    return v.value


def peak_probe() -> dict:
    """FP64 and FP32 FMA-chain throughput of the current device (TFLOP/s)."""
    a, b = C.c_double(), C.c_double()
    st = load().mgwr_peak_probe(C.byref(a), C.byref(b))
    if st != MGWR_OK:
        raise MGWRError(st, "mgwr_peak_probe")
    return {"fp64_tflops": a.value, "fp32_tflops": b.value}


class FAS:
    """The 1-D nonlinear problem of Sec. 7 (mgwr_fas_*): waveform relaxation FAS on
    n = 2^k - 1 interior points and M time steps; fields are (n, M) arrays."""

    def __init__(self, n: int, M: int, T: float, alpha: float, c: float = 1.0,
                 coefficient: int = MGWR_FAS_D_POROUS):
        self.lib = load()
        self.n, self.M = n, M
        h = _h()
        st = self.lib.mgwr_fas_create(n, M, T, alpha, c, coefficient, C.byref(h))
        if st != MGWR_OK:
            raise MGWRError(st, f"mgwr_fas_create({n}, {M}) failed: "
                            + self.lib.mgwr_status_string(st).decode())
        self.h = h

    def _check(self, st: int, what: str, ok=(MGWR_OK,)):
        if st not in ok:
            raise MGWRError(st, f"{what}: {self.lib.mgwr_fas_last_error(self.h).decode()}")
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.mgwr_fas_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_order(self, order: int):
        self._check(self.lib.mgwr_fas_set_order(self.h, order), "mgwr_fas_set_order")

    def set_smoother(self, smoother: int):
        self._check(self.lib.mgwr_fas_set_smoother(self.h, smoother), "mgwr_fas_set_smoother")

    def line_iterations(self) -> int:
        v = C.c_longlong()
        self._check(self.lib.mgwr_fas_line_iterations(self.h, C.byref(v)), "mgwr_fas_line_iterations")
        return v.value

    def reset(self):
        self._check(self.lib.mgwr_fas_reset(self.h), "mgwr_fas_reset")

    def set_stream(self, stream_ptr: int | None):
        self._check(self.lib.mgwr_fas_set_stream(self.h, stream_ptr), "mgwr_fas_set_stream")

    def set_rhs(self, f: np.ndarray):
        f = _f64(f)
        assert f.shape == (self.n, self.M)
        self._check(self.lib.mgwr_fas_set_rhs(self.h, _ptr(f)), "mgwr_fas_set_rhs")

    def set_initial(self, u0: np.ndarray):
        u0 = _f64(u0)
        assert u0.shape == (self.n, self.M)
        self._check(self.lib.mgwr_fas_set_initial(self.h, _ptr(u0)), "mgwr_fas_set_initial")

    def solve(self, cycle=1, nu1=0, nu2=1, tol=1e-10, max_cycles=100,
              allow_noconv=False) -> Stats:
        st = mgwr_stats()
        ok = (MGWR_OK, MGWR_E_NOCONV) if allow_noconv else (MGWR_OK,)
        s = self._check(self.lib.mgwr_fas_solve(self.h, cycle, nu1, nu2, tol, max_cycles,
                                                C.byref(st)), "mgwr_fas_solve", ok)
        return Stats(st.cycles, st.outer, st.relres, st.factor, st.seconds, s)

    def cycle(self, cycle=1, nu1=0, nu2=1):
        self._check(self.lib.mgwr_fas_cycle(self.h, cycle, nu1, nu2), "mgwr_fas_cycle")

    def residual(self, want_field=False):
        nrm = C.c_double()
        r = np.empty((self.n, self.M)) if want_field else None
        self._check(self.lib.mgwr_fas_residual(self.h, C.byref(nrm), _ptr(r)), "mgwr_fas_residual")
        return (nrm.value, r) if want_field else nrm.value

    def solution(self) -> np.ndarray:
        u = np.empty((self.n, self.M))
        self._check(self.lib.mgwr_fas_get_solution(self.h, _ptr(u)), "mgwr_fas_get_solution")
        return u

    def num_levels(self) -> int:
        v = C.c_int()
        self._check(self.lib.mgwr_fas_levels(self.h, C.byref(v)), "mgwr_fas_levels")
        return v.value

    def smooth(self, level: int, colour: int):
        self._check(self.lib.mgwr_fas_smooth(self.h, level, colour), "mgwr_fas_smooth")

    def defect(self, level: int) -> float:
        v = C.c_double()
        self._check(self.lib.mgwr_fas_defect(self.h, level, C.byref(v)), "mgwr_fas_defect")
        return v.value

    def field_set(self, level: int, which: int, a: np.ndarray):
        a = _f64(a)
        assert a.shape == ((1 << (level + 1)) - 1, self.M)
        self._check(self.lib.mgwr_fas_field_set(self.h, level, which, _ptr(a)),
                    "mgwr_fas_field_set")

    def field_get(self, level: int, which: int) -> np.ndarray:
        a = np.empty(((1 << (level + 1)) - 1, self.M))
        self._check(self.lib.mgwr_fas_field_get(self.h, level, which, _ptr(a)),
                    "mgwr_fas_field_get")
        return a
