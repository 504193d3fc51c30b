"""Python binding of the C ABI in include/dp.h (argument marshalling only).

Every function here has the name of the C call it wraps and does nothing but
convert arguments: all computation runs in libdp.so's CUDA kernels.  Host
arrays may be numpy arrays or (pinned) CPU torch tensors; they are passed by
pointer.  ``load()`` raises if the library has not been built: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import workloads as W

DP_OK, DP_EINVAL, DP_ENOMEM, DP_ECUDA, DP_ENOCONV, DP_ETIMEOUT, DP_ENONFINITE = range(7)
DP_FP64, DP_FP32 = 0, 1
DP_DYN_ORBIT, DP_DYN_UNIT_SPEED, DP_DYN_POLAR = 0, 1, 2
DP_CODE_OFF = 65535
DP_SWEEP_VI, DP_SWEEP_IMPROVE_FULL, DP_SWEEP_IMPROVE_WALK, DP_SWEEP_EVAL = 0, 1, 2, 3
DP_SWEEP_EVAL_DIAG, DP_SWEEP_VI_DIAG = 4, 5
DP_FOOT_AUTO, DP_FOOT_WORD8, DP_FOOT_PAIR = 0, 1, 2
DP_EVAL_JACOBI, DP_EVAL_GMRES, DP_EVAL_DIAG = 0, 1, 2
DP_GMRES_MAX_RESTART = 64

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdp.so")


class dp_grid_desc(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 4),
        ("lo", C.c_double * 4),
        ("hi", C.c_double * 4),
        ("dynamics", C.c_int32),
        ("mu", C.c_double),
        ("accel", C.c_double),
        ("exhaust_c", C.c_double),
        ("dt", C.c_double),
        ("beta", C.c_double),
        ("penalty_M", C.c_double),
        ("target_c", C.c_double * 4),
        ("target_w", C.c_double * 4),
        ("n_angles", C.c_int32),
        ("refine", C.c_int32),
        ("refine_tol", C.c_double),
        ("reduced", C.c_int32),
        ("energy_lo", C.c_double),
        ("energy_hi", C.c_double),
        ("precision", C.c_int32),
        ("stream", C.c_void_p),
        ("off_control", C.c_int32),
        ("cost_alpha", C.c_double),
        ("cost_beta", C.c_double),
        ("cost_gamma", C.c_double),
        ("a_bar", C.c_double),
        ("e_bar", C.c_double),
        ("omega_bar", C.c_double),
    ]


class dp_solve_opts(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("max_sweeps", C.c_int64),
        ("n_eval", C.c_int32),
        ("walk", C.c_int32),
        ("warm", C.c_int32),
        ("polish", C.c_int32),
        ("switch_tol", C.c_double),
        ("time_kernels", C.c_int32),
        ("history", C.POINTER(C.c_double)),
        ("history_capacity", C.c_int64),
        ("eval_solver", C.c_int32),
        ("gmres_restart", C.c_int32),
        ("gmres_cycles", C.c_int32),
        ("gmres_reorth", C.c_int32),
        ("gmres_rtol", C.c_double),
        ("n_eval_fp64", C.c_int32),
        ("eval_levels", C.c_int32),
    ]


class dp_solve_stats(C.Structure):
    _fields_ = [
        ("sweeps_vi", C.c_int64),
        ("sweeps_improve", C.c_int64),
        ("sweeps_eval", C.c_int64),
        ("sweeps_improve_fp64", C.c_int64),
        ("sweeps_eval_fp64", C.c_int64),
        ("residual", C.c_double),
        ("converged", C.c_int32),
        ("ms_wall", C.c_double),
        ("ms_vi", C.c_double),
        ("ms_improve", C.c_double),
        ("ms_eval", C.c_double),
        ("ms_improve_fp64", C.c_double),
        ("ms_eval_fp64", C.c_double),
        ("node_updates", C.c_int64),
        ("launches", C.c_int64),
        ("history_count", C.c_int64),
        ("switch_outer", C.c_int64),
        ("gmres_cycles", C.c_int64),
        ("gmres_matvecs", C.c_int64),
    ]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dp_grid_info(C.Structure):
    _fields_ = [
        ("n_box", C.c_int64),
        ("n_active", C.c_int64),
        ("n_target", C.c_int64),
        ("penalty_M", C.c_double),
        ("fp64_values", C.c_int32),
        ("device_bytes", C.c_int64),
    ]


class dp_mlp_train_opts(C.Structure):
    _fields_ = [
        ("epochs", C.c_int32),
        ("batch", C.c_int32),
        ("lr", C.c_double),
        ("seed", C.c_uint64),
        ("lr_final", C.c_double),
    ]


class dp_mlp_train_stats(C.Structure):
    _fields_ = [
        ("epochs", C.c_int64),
        ("steps", C.c_int64),
        ("samples", C.c_int64),
        ("first_epoch_loss", C.c_double),
        ("last_epoch_loss", C.c_double),
        ("ms", C.c_double),
        ("flops", C.c_double),
    ]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dp_batch_stats(C.Structure):
    _fields_ = [
        ("sweeps_improve", C.c_int64),
        ("sweeps_eval", C.c_int64),
        ("sweeps_improve_fp64", C.c_int64),
        ("sweeps_eval_fp64", C.c_int64),
        ("residual", C.c_double),
        ("converged", C.c_int32),
        ("nonfinite", C.c_int32),
        ("switch_outer", C.c_int64),
        ("nodes", C.c_int64),
    ]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dp error %d: %s" % (code, msg))
        self.code = code


_lib = None
_P = C.c_void_p
_dp = C.POINTER(C.c_double)


def load(path: Optional[str] = None):
    """Load libdp.so (built by paper_2407_14675_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libdp.so is not built (%s): run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    sigs = {
        "dp_grid_create": [C.POINTER(dp_grid_desc), C.POINTER(_P)],
        "dp_grid_destroy": [_P],
        "dp_grid_get_info": [_P, C.POINTER(dp_grid_info)],
        "dp_get_active_index": [_P, _P, C.c_int64],
        "dp_set_value": [_P, _P, C.c_int64],
        "dp_get_value": [_P, _P, C.c_int64],
        "dp_set_value_f32": [_P, _P, C.c_int64],
        "dp_get_value_f32": [_P, _P, C.c_int64],
        "dp_set_policy": [_P, _P, C.c_int64],
        "dp_get_policy": [_P, _P, C.c_int64],
        "dp_bellman_sweep": [_P, C.c_int32, _dp],
        "dp_value_iterate": [_P, C.POINTER(dp_solve_opts), C.POINTER(dp_solve_stats)],
        "dp_policy_iterate": [_P, C.POINTER(dp_solve_opts), C.POINTER(dp_solve_stats)],
        "dp_feedback_control": [_P, _P, C.c_int32, C.c_double, _P, _P],
        "dp_simulate_closed_loop": [_P, _P, C.c_int32, C.c_double, C.c_double, C.c_double, _P, _P],
        "dp_simulate_closed_loop_drag": [_P, _P, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, _P,
                                         _P],
        "dp_bellman_sweep_noalloc": [C.POINTER(dp_grid_desc), C.c_int32, _P, _P, _P, _dp],
        "dp_mlp_create": [_P, _P, C.c_int32, _P, C.POINTER(_P)],
        "dp_mlp_destroy": [_P],
        "dp_mlp_set_params": [_P, _P, C.c_int64],
        "dp_mlp_get_params": [_P, _P, C.c_int64],
        "dp_mlp_forward": [_P, _P, C.c_int32, _P],
        "dp_mlp_gradients": [_P, _P, _P, C.c_int32, _P, C.POINTER(C.c_float)],
        "dp_mlp_train_grid": [_P, _P, C.POINTER(dp_mlp_train_opts), C.POINTER(dp_mlp_train_stats)],
        "dp_mlp_apply_gradients": [_P, _P, C.c_int64, C.c_double],
        "dp_set_wave_wait_limit": [C.c_int64],
        "dp_set_foot_format": [_P, C.c_int32],
        "dp_mlp_set_wait_limit": [_P, C.c_int32],
        "dp_warm_start": [_P, _P, _dp],
        "dp_warm_start_from_grid": [_P, _P, _dp],
        "dp_batch_create": [_P, C.c_int32, _P, C.POINTER(_P)],
        "dp_batch_destroy": [_P],
        "dp_batch_get_info": [_P, _P, _P, _P, _P, _P, _P],
        "dp_batch_set_items": [_P, C.c_int32, C.c_int32],
        "dp_batch_autotune": [_P, _P, _P],
        "dp_policy_evaluate": [_P, C.POINTER(dp_solve_opts), C.POINTER(dp_solve_stats)],
        "dp_batch_policy_iterate": [_P, C.POINTER(dp_solve_opts), C.POINTER(dp_solve_stats), _P],
        "dp_batch_sweep": [_P, C.c_int32, _P, _dp],
        "dp_batch_set_value": [_P, C.c_int32, _P, C.c_int64],
        "dp_batch_get_value": [_P, C.c_int32, _P, C.c_int64],
        "dp_batch_set_policy": [_P, C.c_int32, _P, C.c_int64],
        "dp_batch_get_policy": [_P, C.c_int32, _P, C.c_int64],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.dp_mlp_param_count.argtypes = []
    L.dp_mlp_param_count.restype = C.c_int64
    L.dp_last_error.argtypes = []
    L.dp_last_error.restype = C.c_char_p
    _lib = L
    return L


def dp_last_error() -> str:
    return load().dp_last_error().decode()


def _check(rc: int, allow=(DP_OK,)) -> int:
    if rc not in allow:
        raise DPError(rc, dp_last_error())
    return rc


def _host_ptr(a, dtype):
    """Pointer to a contiguous host buffer (numpy array or CPU torch tensor)."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a contiguous %s array" % np.dtype(dtype))
        return C.c_void_p(a.ctypes.data)
    # torch tensor on the host
    if getattr(a, "is_cuda", False):
        raise TypeError("host buffer expected")
    if not a.is_contiguous() or a.element_size() != np.dtype(dtype).itemsize:
        raise TypeError("expected a contiguous host tensor of %d-byte elements" % np.dtype(dtype).itemsize)
    return C.c_void_p(a.data_ptr())


def current_stream() -> int:
    """The current torch CUDA stream handle (0 without CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def desc_from_problem(p: "W.Problem", stream: Optional[int] = None) -> dp_grid_desc:
    d = dp_grid_desc()
    d.n[:] = list(p.n)
    d.lo[:] = list(p.lo)
    d.hi[:] = list(p.hi)
    d.dynamics = p.dynamics
    d.mu, d.accel, d.exhaust_c = p.mu, p.accel, p.exhaust_c
    d.dt, d.beta, d.penalty_M = p.dt, p.beta, p.penalty_M
    d.target_c[:] = list(p.target_c)
    d.target_w[:] = list(p.target_w)
    d.n_angles, d.refine, d.refine_tol = p.n_angles, p.refine, p.refine_tol
    d.reduced, d.energy_lo, d.energy_hi = p.reduced, p.energy_lo, p.energy_hi
    d.precision = p.precision
    d.stream = current_stream() if stream is None else stream
    d.off_control = getattr(p, "off_control", 0)
    d.cost_alpha, d.cost_beta, d.cost_gamma = p.cost_alpha, p.cost_beta, p.cost_gamma
    d.a_bar, d.e_bar, d.omega_bar = p.a_bar, p.e_bar, p.omega_bar
    return d


def dp_grid_create(desc: dp_grid_desc) -> int:
    h = _P()
    _check(load().dp_grid_create(C.byref(desc), C.byref(h)))
    return h.value


def dp_grid_destroy(grid: int) -> None:
    _check(load().dp_grid_destroy(grid))


def dp_grid_get_info(grid: int) -> dict:
    info = dp_grid_info()
    _check(load().dp_grid_get_info(grid, C.byref(info)))
    return {k: getattr(info, k) for k, _ in info._fields_}


def dp_get_active_index(grid: int, count: int) -> np.ndarray:
    out = np.empty(count, np.int64)
    _check(load().dp_get_active_index(grid, _host_ptr(out, np.int64), count))
    return out


def dp_set_value(grid: int, V) -> None:
    _check(load().dp_set_value(grid, _host_ptr(V, np.float64), len(V)))


def dp_get_value(grid: int, count: int, out=None):
    out = np.empty(count, np.float64) if out is None else out
    _check(load().dp_get_value(grid, _host_ptr(out, np.float64), count))
    return out


def dp_set_value_f32(grid: int, V) -> None:
    _check(load().dp_set_value_f32(grid, _host_ptr(V, np.float32), len(V)))


def dp_get_value_f32(grid: int, count: int, out=None):
    out = np.empty(count, np.float32) if out is None else out
    _check(load().dp_get_value_f32(grid, _host_ptr(out, np.float32), count))
    return out


def dp_set_policy(grid: int, codes) -> None:
    _check(load().dp_set_policy(grid, _host_ptr(codes, np.uint16), len(codes)))


def dp_get_policy(grid: int, count: int, out=None) -> np.ndarray:
    out = np.empty(count, np.uint16) if out is None else out
    _check(load().dp_get_policy(grid, _host_ptr(out, np.uint16), count))
    return out


def dp_bellman_sweep(grid: int, mode: int) -> float:
    r = C.c_double(0)
    _check(load().dp_bellman_sweep(grid, mode, C.byref(r)))
    return r.value


def dp_bellman_sweep_noalloc(desc: dp_grid_desc, mode: int, V_in: int, V_out: int, codes: int = 0) -> float:
    """One sweep on caller-owned device buffers (raw device pointers); the
    library allocates nothing.  Returns the residual."""
    r = C.c_double(0)
    _check(load().dp_bellman_sweep_noalloc(C.byref(desc), mode, C.c_void_p(V_in), C.c_void_p(V_out),
                                           C.c_void_p(codes or None), C.byref(r)))
    return r.value


def make_opts(tol=1e-6, max_sweeps=100000, n_eval=20, walk=1, warm=0, polish=1, switch_tol=0.0,
              time_kernels=0, history=None, eval_solver=DP_EVAL_JACOBI, gmres_restart=0, gmres_cycles=0,
              gmres_reorth=0, gmres_rtol=0.0, n_eval_fp64=0, eval_levels=0) -> dp_solve_opts:
    """Solver options; history: optional float64 numpy array that receives the
    residual of every stopping test (kept alive by the caller).  eval_solver
    DP_EVAL_GMRES evaluates each policy by GMRES (gmres_*: 0 = default).
    eval_levels: evaluation sweeps per launch (0 = automatic, 1 = one)."""
    o = dp_solve_opts()
    o.tol, o.max_sweeps, o.n_eval, o.walk, o.warm = tol, max_sweeps, n_eval, walk, warm
    o.polish, o.switch_tol, o.time_kernels = polish, switch_tol, time_kernels
    o.eval_solver, o.gmres_restart, o.gmres_cycles = eval_solver, gmres_restart, gmres_cycles
    o.gmres_reorth, o.gmres_rtol = gmres_reorth, gmres_rtol
    o.n_eval_fp64 = n_eval_fp64
    o.eval_levels = eval_levels
    if history is not None:
        o.history = history.ctypes.data_as(C.POINTER(C.c_double))
        o.history_capacity = len(history)
    return o


def dp_value_iterate(grid: int, opts: dp_solve_opts):
    s = dp_solve_stats()
    rc = _check(load().dp_value_iterate(grid, C.byref(opts), C.byref(s)), allow=(DP_OK, DP_ENOCONV))
    return rc, s


def dp_policy_iterate(grid: int, opts: dp_solve_opts):
    s = dp_solve_stats()
    rc = _check(load().dp_policy_iterate(grid, C.byref(opts), C.byref(s)), allow=(DP_OK, DP_ENOCONV))
    return rc, s


def dp_policy_evaluate(grid: int, opts: dp_solve_opts):
    s = dp_solve_stats()
    rc = _check(load().dp_policy_evaluate(grid, C.byref(opts), C.byref(s)), allow=(DP_OK, DP_ENOCONV))
    return rc, s


def dp_feedback_control(grid: int, states, tau: float):
    st = np.ascontiguousarray(states, np.float64).reshape(-1, 4)
    n = len(st)
    alpha = np.empty(n)
    q = np.empty(n)
    _check(load().dp_feedback_control(grid, _host_ptr(st, np.float64), n, tau, _host_ptr(alpha, np.float64),
                                      _host_ptr(q, np.float64)))
    return alpha, q


def dp_simulate_closed_loop_drag(grid: int, x0, tau: float, h_rk4: float, t_max: float, drag_c: float):
    x = np.ascontiguousarray(x0, np.float64).reshape(-1, 4)
    n = len(x)
    ta = np.empty(n)
    xf = np.empty((n, 4))
    _check(load().dp_simulate_closed_loop_drag(grid, _host_ptr(x, np.float64), n, tau, h_rk4, t_max, drag_c,
                                               _host_ptr(ta, np.float64), _host_ptr(xf, np.float64)))
    return ta, xf


def dp_simulate_closed_loop(grid: int, x0, tau: float, h_rk4: float, t_max: float):
    x = np.ascontiguousarray(x0, np.float64).reshape(-1, 4)
    n = len(x)
    ta = np.empty(n)
    xf = np.empty((n, 4))
    _check(load().dp_simulate_closed_loop(grid, _host_ptr(x, np.float64), n, tau, h_rk4, t_max,
                                          _host_ptr(ta, np.float64), _host_ptr(xf, np.float64)))
    return ta, xf


class Grid:
    """Owning wrapper of a dp_grid handle (destroyed on close / exit)."""

    def __init__(self, p: "W.Problem", stream: Optional[int] = None):
        self.p = p
        self.h = dp_grid_create(desc_from_problem(p, stream))
        self.info = dp_grid_get_info(self.h)
        self.n = self.info["n_active"]

    def close(self):
        if self.h:
            dp_grid_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def active_index(self):
        return dp_get_active_index(self.h, self.n)

    def set_value(self, V):
        dp_set_value(self.h, V)

    def get_value(self):
        return dp_get_value(self.h, self.n)

    def set_policy(self, codes):
        dp_set_policy(self.h, codes)

    def get_policy(self):
        return dp_get_policy(self.h, self.n)

    def sweep(self, mode):
        return dp_bellman_sweep(self.h, mode)

    def set_foot_format(self, fmt):
        dp_set_foot_format(self.h, fmt)

    def value_iterate(self, **kw):
        return dp_value_iterate(self.h, make_opts(**kw))

    def policy_iterate(self, **kw):
        return dp_policy_iterate(self.h, make_opts(**kw))

    def policy_evaluate(self, **kw):
        return dp_policy_evaluate(self.h, make_opts(**kw))

    def feedback(self, states, tau):
        return dp_feedback_control(self.h, states, tau)

    def simulate(self, x0, tau, h_rk4, t_max, drag=0.0):
        if drag:
            return dp_simulate_closed_loop_drag(self.h, x0, tau, h_rk4, t_max, drag)
        return dp_simulate_closed_loop(self.h, x0, tau, h_rk4, t_max)


# ---- batched transfers ---------------------------------------------------------

def dp_batch_create(descs, stream: Optional[int] = 0) -> int:
    """descs: a list of dp_grid_desc; stream 0: the batch makes its own."""
    arr = (dp_grid_desc * len(descs))(*descs)
    h = _P()
    _check(load().dp_batch_create(arr, len(descs), C.c_void_p(stream or None), C.byref(h)))
    return h.value


def dp_batch_destroy(batch: int) -> None:
    _check(load().dp_batch_destroy(batch))


def dp_batch_get_info(batch: int) -> dict:
    c, ie, ii = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    n, nt, b = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _check(load().dp_batch_get_info(batch, C.byref(c), C.byref(n), C.byref(nt), C.byref(ie), C.byref(ii),
                                    C.byref(b)))
    return {"count": c.value, "nodes_total": n.value, "nodes_target": nt.value, "item_eval": ie.value,
            "item_improve": ii.value, "device_bytes": b.value}


def dp_batch_set_items(batch: int, item_eval: int, item_improve: int) -> None:
    _check(load().dp_batch_set_items(batch, item_eval, item_improve))


def dp_batch_autotune(batch: int):
    ie, ii = C.c_int32(0), C.c_int32(0)
    _check(load().dp_batch_autotune(batch, C.byref(ie), C.byref(ii)))
    return ie.value, ii.value


def dp_batch_policy_iterate(batch: int, count: int, opts: dp_solve_opts):
    s = dp_solve_stats()
    per = (dp_batch_stats * count)()
    rc = _check(load().dp_batch_policy_iterate(batch, C.byref(opts), C.byref(s), per),
                allow=(DP_OK, DP_ENOCONV))
    return rc, s, [per[i].asdict() for i in range(count)]


def dp_batch_sweep(batch: int, count: int, mode: int):
    """One sweep of every transfer; returns (per-transfer residuals, ms)."""
    r = np.empty(count, np.float64)
    ms = C.c_double(0)
    _check(load().dp_batch_sweep(batch, mode, _host_ptr(r, np.float64), C.byref(ms)))
    return r, ms.value


def dp_batch_set_value(batch: int, index: int, V) -> None:
    V = np.ascontiguousarray(V, np.float64)
    _check(load().dp_batch_set_value(batch, index, _host_ptr(V, np.float64), len(V)))


def dp_batch_get_value(batch: int, index: int, count: int) -> np.ndarray:
    out = np.empty(count, np.float64)
    _check(load().dp_batch_get_value(batch, index, _host_ptr(out, np.float64), count))
    return out


def dp_batch_set_policy(batch: int, index: int, codes) -> None:
    codes = np.ascontiguousarray(codes, np.uint16)
    _check(load().dp_batch_set_policy(batch, index, _host_ptr(codes, np.uint16), len(codes)))


def dp_batch_get_policy(batch: int, index: int, count: int) -> np.ndarray:
    out = np.empty(count, np.uint16)
    _check(load().dp_batch_get_policy(batch, index, _host_ptr(out, np.uint16), count))
    return out


class Batch:
    """Owning wrapper of a dp_batch handle over a list of workloads.Problem."""

    def __init__(self, problems, stream: Optional[int] = 0):
        self.problems = list(problems)
        self.count = len(self.problems)
        self.nodes = [int(np.prod(p.n)) for p in self.problems]
        self.h = dp_batch_create([desc_from_problem(p, 0) for p in self.problems], stream)

    def close(self):
        if self.h:
            dp_batch_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return dp_batch_get_info(self.h)

    def autotune(self):
        return dp_batch_autotune(self.h)

    def policy_iterate(self, **kw):
        return dp_batch_policy_iterate(self.h, self.count, make_opts(**kw))

    def sweep(self, mode):
        return dp_batch_sweep(self.h, self.count, mode)

    def set_value(self, i, V):
        dp_batch_set_value(self.h, i, V)

    def get_value(self, i):
        return dp_batch_get_value(self.h, i, self.nodes[i])

    def set_policy(self, i, codes):
        dp_batch_set_policy(self.h, i, codes)

    def get_policy(self, i):
        return dp_batch_get_policy(self.h, i, self.nodes[i])


# ---- learned warm start --------------------------------------------------------

def dp_mlp_param_count() -> int:
    return int(load().dp_mlp_param_count())


def dp_mlp_create(lo, hi, batch_capacity: int, stream: Optional[int] = None) -> int:
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    h = _P()
    _check(load().dp_mlp_create(_host_ptr(lo, np.float64), _host_ptr(hi, np.float64), batch_capacity,
                                current_stream() if stream is None else stream, C.byref(h)))
    return h.value


def dp_mlp_destroy(mlp: int) -> None:
    _check(load().dp_mlp_destroy(mlp))


def dp_mlp_set_params(mlp: int, params) -> None:
    p = np.ascontiguousarray(params, np.float32)
    _check(load().dp_mlp_set_params(mlp, _host_ptr(p, np.float32), len(p)))


def dp_mlp_get_params(mlp: int) -> np.ndarray:
    out = np.empty(dp_mlp_param_count(), np.float32)
    _check(load().dp_mlp_get_params(mlp, _host_ptr(out, np.float32), len(out)))
    return out


def dp_mlp_forward(mlp: int, states) -> np.ndarray:
    st = np.ascontiguousarray(states, np.float64).reshape(-1, 4)
    out = np.empty((len(st), 3), np.float32)
    _check(load().dp_mlp_forward(mlp, _host_ptr(st, np.float64), len(st), _host_ptr(out, np.float32)))
    return out


def dp_mlp_gradients(mlp: int, states, targets):
    st = np.ascontiguousarray(states, np.float64).reshape(-1, 4)
    tg = np.ascontiguousarray(targets, np.float32).reshape(-1, 3)
    g = np.empty(dp_mlp_param_count(), np.float32)
    loss = C.c_float(0)
    _check(load().dp_mlp_gradients(mlp, _host_ptr(st, np.float64), _host_ptr(tg, np.float32), len(st),
                                   _host_ptr(g, np.float32), C.byref(loss)))
    return g, loss.value


def dp_mlp_apply_gradients(mlp: int, grads, lr=1e-3):
    g = np.ascontiguousarray(grads, np.float32)
    _check(load().dp_mlp_apply_gradients(mlp, _host_ptr(g, np.float32), len(g), lr))


def dp_set_wave_wait_limit(ns: int):
    _check(load().dp_set_wave_wait_limit(ns))


def dp_set_foot_format(h, fmt: int):
    _check(load().dp_set_foot_format(h, fmt))


def dp_mlp_set_wait_limit(mlp: int, polls: int):
    _check(load().dp_mlp_set_wait_limit(mlp, polls))


def dp_mlp_train_grid(mlp: int, grid: int, epochs=4, batch=4096, lr=1e-3, seed=14675, lr_final=0.0):
    o = dp_mlp_train_opts()
    o.epochs, o.batch, o.lr, o.seed, o.lr_final = epochs, batch, lr, seed, lr_final
    s = dp_mlp_train_stats()
    _check(load().dp_mlp_train_grid(mlp, grid, C.byref(o), C.byref(s)))
    return s


def dp_warm_start(mlp: int, grid: int) -> float:
    ms = C.c_double(0)
    _check(load().dp_warm_start(mlp, grid, C.byref(ms)))
    return ms.value


def dp_warm_start_from_grid(src: int, dst: int) -> float:
    ms = C.c_double(0)
    _check(load().dp_warm_start_from_grid(src, dst, C.byref(ms)))
    return ms.value


def flatten_params(params) -> np.ndarray:
    """[[W1, b1], ..., [W4, b4]] -> the flat FP32 parameter vector of dp.h."""
    return np.concatenate([np.asarray(a, np.float64).reshape(-1) for layer in params for a in layer]).astype(np.float32)


def unflatten_params(flat, sizes=(4, 256, 256, 256, 3)):
    out, k = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(flat[k:k + fi * fo], np.float64).reshape(fo, fi)
        k += fi * fo
        b = np.asarray(flat[k:k + fo], np.float64)
        k += fo
        out.append([W, b])
    return out


class Mlp:
    """Owning wrapper of a dp_mlp handle."""

    def __init__(self, lo, hi, batch_capacity=65536, stream: Optional[int] = None):
        self.h = dp_mlp_create(lo, hi, batch_capacity, stream)

    def close(self):
        if self.h:
            dp_mlp_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
