"""FP64 CPU oracle of the semi-Lagrangian Bellman scheme (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It is a ctypes wrapper around
``dp_oracle.c``: plain double-precision loops over nodes and controls that
follow the paper's equations one step at a time (Eq. (10), (12)-(15) and the
dynamics of §3).  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Optional

import numpy as np

from .build import build_oracle

VI, IMPROVE_FULL, IMPROVE_WALK, EVAL = 0, 1, 2, 3
NCODES = 65536
CODE_OFF = 65535   # thrust off (grids with the off control)
OFF = float("nan")  # the off control as an "angle" argument

_lib = None


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int * 4),
        ("lo", C.c_double * 4),
        ("hi", C.c_double * 4),
        ("dynamics", C.c_int),
        ("mu", C.c_double),
        ("accel", C.c_double),
        ("exhaust_c", C.c_double),
        ("dt", C.c_double),
        ("beta", C.c_double),
        ("M", C.c_double),
        ("tgt_c", C.c_double * 4),
        ("tgt_w", C.c_double * 4),
        ("K", C.c_int),
        ("refine", C.c_int),
        ("refine_tol", C.c_double),
        ("reduced", C.c_int),
        ("e_lo", C.c_double),
        ("e_hi", C.c_double),
        ("off_control", C.c_int),
        ("cost_alpha", C.c_double),
        ("cost_beta", C.c_double),
        ("cost_gamma", C.c_double),
        ("a_bar", C.c_double),
        ("e_bar", C.c_double),
        ("omega_bar", C.c_double),
    ]


_dp = C.POINTER(C.c_double)
_u8 = C.POINTER(C.c_ubyte)
_u16 = C.POINTER(C.c_uint16)
_l = C.POINTER(C.c_long)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        P = C.POINTER(_Problem)
        sig = {
            "orc_node_count": (C.c_long, [P]),
            "orc_build_masks": (C.c_long, [P, _u8, _u8]),
            "orc_in_target": (C.c_int, [P, _dp]),
            "orc_energy": (C.c_double, [P, _dp]),
            "orc_elements": (None, [P, _dp, _dp, _dp, _dp]),
            "orc_running_cost": (C.c_double, [P, _dp, C.c_int]),
            "orc_dynamics": (None, [P, _dp, C.c_double, _dp]),
            "orc_heun_displacement": (None, [P, _dp, C.c_double, C.c_double, _dp]),
            "orc_rk4_step": (None, [P, _dp, C.c_double, C.c_double, _dp]),
            "orc_interp": (C.c_int, [P, _dp, _u8, _dp, _dp]),
            "orc_q_node": (C.c_double, [P, _dp, _u8, C.POINTER(C.c_int), C.c_double]),
            "orc_q_state": (C.c_double, [P, _dp, _u8, _dp, C.c_double, C.c_double]),
            "orc_foot_node": (None, [P, C.POINTER(C.c_int), C.c_double, _dp]),
            "orc_sweep": (C.c_double, [P, _dp, _dp, _u8, _u8, C.c_int, _u16, _u16, _l]),
            "orc_bellman_nodes": (None, [P, _dp, _u8, _u8, _l, C.c_long, C.c_int, _u16, _dp, _u16]),
            "orc_q_nodes": (None, [P, _dp, _u8, _l, _u16, C.c_long, _dp]),
            "orc_value_iterate": (C.c_long, [P, _dp, _u8, _u8, C.c_double, C.c_long, _dp]),
            "orc_policy_iterate": (C.c_long, [P, _dp, _u16, _u8, _u8, C.c_double, C.c_long, C.c_int,
                                              C.c_int, _l, _dp]),
            "orc_feedback": (None, [P, _dp, _u8, _dp, C.c_long, C.c_double, _u16, _dp]),
            "orc_simulate": (None, [P, _dp, _u8, _dp, C.c_long, C.c_double, C.c_double, C.c_double,
                                    _dp, _dp]),
            "orc_simulate_drag": (None, [P, _dp, _u8, _dp, C.c_long, C.c_double, C.c_double, C.c_double,
                                         C.c_double, _dp, _dp]),
            "orc_dynamics_drag": (None, [P, _dp, C.c_double, C.c_double, _dp]),
            "orc_policy_system": (None, [P, _u8, _u8, _u16, _l, _dp, _dp, C.POINTER(C.c_int)]),
            "orc_vi_diag_sweep": (C.c_double, [P, _dp, _dp, _u8, _u8]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def problem(p) -> _Problem:
    """ctypes problem from a workloads.Problem; M defaults to dt / (1 - beta)."""
    s = _Problem()
    s.n[:] = list(p.n)
    s.lo[:] = list(p.lo)
    s.hi[:] = list(p.hi)
    s.dynamics = p.dynamics
    s.mu, s.accel, s.exhaust_c = p.mu, p.accel, p.exhaust_c
    s.dt, s.beta = p.dt, p.beta
    s.M = p.penalty_M if p.penalty_M > 0 else p.dt / (1.0 - p.beta)
    s.tgt_c[:] = list(p.target_c)
    s.tgt_w[:] = list(p.target_w)
    s.K, s.refine, s.refine_tol = p.n_angles, p.refine, p.refine_tol
    s.reduced, s.e_lo, s.e_hi = p.reduced, p.energy_lo, p.energy_hi
    s.off_control = getattr(p, "off_control", 0)
    s.cost_alpha, s.cost_beta, s.cost_gamma = (getattr(p, k, 0.0) for k in ("cost_alpha", "cost_beta", "cost_gamma"))
    s.a_bar, s.e_bar, s.omega_bar = (getattr(p, k, 0.0) for k in ("a_bar", "e_bar", "omega_bar"))
    return s


class Oracle:
    """Oracle bound to one problem: masks are built once."""

    def __init__(self, p):
        self.p = p
        self.s = problem(p)
        self.N = p.nodes
        self.active = np.zeros(self.N, np.uint8)
        self.target = np.zeros(self.N, np.uint8)
        self.n_active = lib().orc_build_masks(C.byref(self.s), _ptr(self.active, _u8), _ptr(self.target, _u8))
        self.M = self.s.M

    # -- single pieces -------------------------------------------------------
    def dynamics(self, x, alpha):
        x = np.ascontiguousarray(x, np.float64)
        f = np.zeros(4)
        lib().orc_dynamics(C.byref(self.s), _ptr(x, _dp), alpha, _ptr(f, _dp))
        return f

    def heun(self, x, alpha, h):
        x = np.ascontiguousarray(x, np.float64)
        d = np.zeros(4)
        lib().orc_heun_displacement(C.byref(self.s), _ptr(x, _dp), alpha, h, _ptr(d, _dp))
        return d

    def rk4(self, x, alpha, h):
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros(4)
        lib().orc_rk4_step(C.byref(self.s), _ptr(x, _dp), alpha, h, _ptr(y, _dp))
        return y

    def energy(self, x):
        x = np.ascontiguousarray(x, np.float64)
        return lib().orc_energy(C.byref(self.s), _ptr(x, _dp))

    def elements(self, x):
        """(a, e cos omega, e sin omega) of a polar state."""
        x = np.ascontiguousarray(x, np.float64)
        a, ex, ey = C.c_double(0), C.c_double(0), C.c_double(0)
        lib().orc_elements(C.byref(self.s), _ptr(x, _dp), C.byref(a), C.byref(ex), C.byref(ey))
        return a.value, ex.value, ey.value

    def running_cost(self, x, thrust_on=True):
        x = np.ascontiguousarray(x, np.float64)
        return lib().orc_running_cost(C.byref(self.s), _ptr(x, _dp), int(thrust_on))

    def in_target(self, x):
        x = np.ascontiguousarray(x, np.float64)
        return bool(lib().orc_in_target(C.byref(self.s), _ptr(x, _dp)))

    def interp(self, V, s, use_active=True):
        V = np.ascontiguousarray(V, np.float64)
        s = np.ascontiguousarray(s, np.float64)
        out = C.c_double(0)
        ok = lib().orc_interp(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8) if use_active else None,
                              _ptr(s, _dp), C.byref(out))
        return out.value if ok else None

    def q_node(self, V, idx, alpha):
        V = np.ascontiguousarray(V, np.float64)
        i = (C.c_int * 4)(*idx)
        return lib().orc_q_node(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8), i, alpha)

    def foot_node(self, idx, alpha):
        """Foot of the Heun step from node idx, in grid units."""
        i = (C.c_int * 4)(*[int(v) for v in idx])
        s = np.zeros(4)
        lib().orc_foot_node(C.byref(self.s), i, alpha, _ptr(s, _dp))
        return s

    def q_state(self, V, y, alpha, tau):
        V = np.ascontiguousarray(V, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        return lib().orc_q_state(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8), _ptr(y, _dp), alpha, tau)

    # -- sweeps --------------------------------------------------------------
    def sweep(self, V, mode=VI, codes=None):
        """One Jacobi sweep: returns (V_out, codes_out, residual, evaluations)."""
        V = np.ascontiguousarray(V, np.float64)
        W = np.empty(self.N)
        ci = None if codes is None else np.ascontiguousarray(codes, np.uint16)
        co = np.zeros(self.N, np.uint16) if mode != VI else None
        ev = C.c_long(0)
        r = lib().orc_sweep(C.byref(self.s), _ptr(V, _dp), _ptr(W, _dp), _ptr(self.active, _u8),
                            _ptr(self.target, _u8), mode, _ptr(ci, _u16), _ptr(co, _u16), C.byref(ev))
        return W, co, r, ev.value

    def bellman_nodes(self, V, nodes, mode=VI, codes=None):
        """The update at selected nodes: returns (values, codes)."""
        V = np.ascontiguousarray(V, np.float64)
        nodes = np.ascontiguousarray(nodes, np.int64)
        n = len(nodes)
        out = np.empty(n)
        co = np.zeros(n, np.uint16)
        ci = None if codes is None else np.ascontiguousarray(codes, np.uint16)
        lib().orc_bellman_nodes(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8), _ptr(self.target, _u8),
                                nodes.ctypes.data_as(_l), n, mode, _ptr(ci, _u16), _ptr(out, _dp), _ptr(co, _u16))
        return out, co

    def q_nodes(self, V, nodes, codes):
        V = np.ascontiguousarray(V, np.float64)
        nodes = np.ascontiguousarray(nodes, np.int64)
        codes = np.ascontiguousarray(codes, np.uint16)
        out = np.empty(len(nodes))
        lib().orc_q_nodes(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8), nodes.ctypes.data_as(_l),
                          _ptr(codes, _u16), len(nodes), _ptr(out, _dp))
        return out

    def policy_system(self, codes):
        """Eq. (13) at a frozen policy as the affine map V -> b + beta W V:
        returns (W, b) with W a scipy CSR matrix of the Q1 foot weights (rows
        of target, inactive and outside nodes are empty)."""
        import scipy.sparse as sp
        codes = np.ascontiguousarray(codes, np.uint16)
        idx = np.zeros((self.N, 16), np.int64)
        w = np.zeros((self.N, 16))
        b = np.zeros(self.N)
        cnt = np.zeros(self.N, np.int32)
        lib().orc_policy_system(C.byref(self.s), _ptr(self.active, _u8), _ptr(self.target, _u8), _ptr(codes, _u16),
                                idx.ctypes.data_as(_l), _ptr(w, _dp), _ptr(b, _dp),
                                cnt.ctypes.data_as(C.POINTER(C.c_int)))
        rows = np.repeat(np.arange(self.N), 16).reshape(self.N, 16)
        used = cnt[:, None] > np.arange(16)[None, :]
        W = sp.csr_matrix((w[used], (rows[used], idx[used])), shape=(self.N, self.N))
        return W, b

    def evaluate_exact(self, codes):
        """Exact policy evaluation: the solution of (I - beta W) V = b, the
        linear system of Eq. (13) at a frozen policy, by a sparse direct solve."""
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        W, b = self.policy_system(codes)
        A = (sp.identity(self.N, format="csr") - self.s.beta * W).tocsc()
        return spla.spsolve(A, b)

    def vi_diag_sweep(self, V):
        """One value-iteration sweep (Eq. (12)) with each node's own coefficient
        solved: V'_j = min_a (c_a + beta R_a) / (1 - beta w_jj^a).  Minimum time
        only.  Returns (V', max |V' - V| over the node set)."""
        V = np.ascontiguousarray(V, np.float64)
        W = np.empty(self.N)
        r = lib().orc_vi_diag_sweep(C.byref(self.s), _ptr(V, _dp), _ptr(W, _dp), _ptr(self.active, _u8),
                                    _ptr(self.target, _u8))
        return W, r

    def eval_diag_sweep(self, V, codes):
        """One Jacobi iteration on the policy-evaluation system (I - beta W) V = b
        (Eq. (13) at a frozen policy) with each node's own coefficient solved:
            V'_j = (b_j + beta sum_{c != j} W_jc V_c) / (1 - beta W_jj).
        The evaluation sweep V' = b + beta W V has the same fixed point.
        Returns (V', max |V' - V| over the node set)."""
        Wm, b = self.policy_system(codes)
        V = np.asarray(V, np.float64)
        d = Wm.diagonal()
        beta = self.s.beta
        Vn = (b + beta * (Wm @ V - d * V)) / (1.0 - beta * d)
        act = self.active.astype(bool)
        return Vn, float(np.abs(Vn - V)[act].max())

    def value_iterate(self, V0=None, tol=None, max_sweeps=100000):
        V = np.zeros(self.N) if V0 is None else np.array(V0, np.float64)
        res = C.c_double(0)
        tol = self.p.tol if tol is None else tol
        s = lib().orc_value_iterate(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8), _ptr(self.target, _u8),
                                    tol, max_sweeps, C.byref(res))
        return V, s, res.value

    def policy_iterate(self, V0=None, codes0=None, tol=None, max_outer=100000, n_eval=None, walk=True):
        V = np.zeros(self.N) if V0 is None else np.array(V0, np.float64)
        codes = np.zeros(self.N, np.uint16) if codes0 is None else np.array(codes0, np.uint16)
        res = C.c_double(0)
        ev = C.c_long(0)
        tol = self.p.tol if tol is None else tol
        n_eval = self.p.n_eval if n_eval is None else n_eval
        outer = lib().orc_policy_iterate(C.byref(self.s), _ptr(V, _dp), _ptr(codes, _u16), _ptr(self.active, _u8),
                                         _ptr(self.target, _u8), tol, max_outer, n_eval, int(walk),
                                         C.byref(ev), C.byref(res))
        return V, codes, outer, ev.value, res.value

    def feedback(self, V, states, tau=None):
        V = np.ascontiguousarray(V, np.float64)
        st = np.ascontiguousarray(states, np.float64).reshape(-1, 4)
        n = len(st)
        codes = np.zeros(n, np.uint16)
        q = np.zeros(n)
        tau = self.p.dt if tau is None else tau
        lib().orc_feedback(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8), _ptr(st, _dp), n, tau,
                           _ptr(codes, _u16), _ptr(q, _dp))
        return codes, q

    def simulate(self, V, x0, tau=None, h=None, t_max=200.0, drag=0.0):
        V = np.ascontiguousarray(V, np.float64)
        x0 = np.ascontiguousarray(x0, np.float64).reshape(-1, 4)
        n = len(x0)
        tau = self.p.dt if tau is None else tau
        h = tau if h is None else h
        ta = np.zeros(n)
        xf = np.zeros((n, 4))
        lib().orc_simulate_drag(C.byref(self.s), _ptr(V, _dp), _ptr(self.active, _u8), _ptr(x0, _dp), n, tau, h,
                                t_max, drag, _ptr(ta, _dp), _ptr(xf, _dp))
        return ta, xf

    def dynamics_drag(self, x, alpha, drag):
        x = np.ascontiguousarray(x, np.float64)
        f = np.zeros(4)
        lib().orc_dynamics_drag(C.byref(self.s), _ptr(x, _dp), alpha, drag, _ptr(f, _dp))
        return f


def code_angle(code):
    return 2.0 * math.pi * (np.asarray(code, np.float64) % NCODES) / NCODES
