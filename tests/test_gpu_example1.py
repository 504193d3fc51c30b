"""The paper's Example 1 (§4) on the GPU: polar dynamics with the periodic
orbital angle, the running cost of Eq. (11) and the thrust-off control.

FP64 throughout, so the tolerances are those of the FP64 grids: values within
1e-9 max|V|, decisions equal or ties (the oracle's q at the GPU's code within
1e-12 of the value scale of its q at its own code).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W
from test_gpu_parity import TOL64, _check_codes, _check_values, _lockstep

pytestmark = pytest.mark.gpu


def _small():
    return W.example1(n=(12, 7, 7, 8))


def test_example1_sweeps_match_oracle(dp):
    p = _small()
    o = oracle.Oracle(p)
    V = W.smooth_value(p, 5) * 1e-2      # values of the size of the discounted cost
    with dp.Grid(p) as g:
        g.set_value(V)
        tie = 1e-12 * np.abs(V).max()
        _lockstep(dp, g, o, [dp.DP_SWEEP_VI, dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_EVAL, dp.DP_SWEEP_EVAL,
                             dp.DP_SWEEP_IMPROVE_WALK, dp.DP_SWEEP_EVAL, dp.DP_SWEEP_IMPROVE_WALK], TOL64, tie)
        codes = g.get_policy()
    # both thrust and thrust-off decisions occur
    assert (codes == dp.DP_CODE_OFF).any() and (codes != dp.DP_CODE_OFF).any()


def test_example1_off_policy_evaluates_without_thrust(dp):
    # every node off: one evaluation sweep is dt l(x, off) + beta I[V](drift foot)
    p = _small()
    o = oracle.Oracle(p)
    V = W.smooth_value(p, 6) * 1e-2
    codes = np.full(p.nodes, dp.DP_CODE_OFF, np.uint16)
    with dp.Grid(p) as g:
        g.set_value(V)
        g.set_policy(codes)
        g.sweep(dp.DP_SWEEP_EVAL)
        v_g = g.get_value()
    v_o, _, _, _ = o.sweep(V, mode=oracle.EVAL, codes=codes)
    _check_values(v_g, v_o, TOL64, "off evaluation")


def test_example1_feedback_matches_oracle(dp):
    p = _small()
    o = oracle.Oracle(p)
    rng = np.random.default_rng(8)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=400, n_eval=20, polish=0)
        V = g.get_value()
        lo, hi = np.array(p.lo), np.array(p.hi)
        y = lo + (hi - lo) * rng.uniform(0.05, 0.95, size=(64, 4))
        y[:, 3] = rng.uniform(0, 2 * math.pi, 64) + 2 * math.pi * rng.integers(-3, 40, 64)   # angle wraps
        alpha, q = g.feedback(y, p.dt)
    codes, q_o = o.feedback(V, y, tau=p.dt)
    off_o = codes == oracle.CODE_OFF
    assert (np.isnan(alpha) == off_o).mean() >= 0.95
    assert np.abs(q - q_o).max() <= 1e-9 * np.abs(q_o).max()
    both = ~off_o & ~np.isnan(alpha)
    d = np.abs((alpha[both] - oracle.code_angle(codes[both]) + math.pi) % (2 * math.pi) - math.pi)
    # equal angles, or ties in q (checked above at 1e-9 of the scale)
    assert (d < 1e-3).mean() >= 0.9


def test_example1_closed_loop_raises_the_orbit(dp):
    # an 80 x 22 x 22 x 24 grid solved to 1e-7, then the closed loop from the
    # paper's circular start at 6978 km: the semi-major axis comes within 1 km
    # of 7000 km (the paper: the target neighbourhood after about 1e5 s) and
    # stays there (qualitative, as in §4; the oracle's elements give a)
    p = W.example1(n=(80, 22, 22, 24))
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=p.tol, max_sweeps=3000, n_eval=20, polish=0)
        assert st.converged, st.asdict()
        y = W.example1_start(6978.0)[None, :]
        a0 = o.elements(y[0])[0]
        t, t_near, a_hist = 0.0, None, []
        while t < 4e5:
            ta, y = g.simulate(y, p.dt, p.dt, 5000.0)
            t += 5000.0
            a = o.elements(y[0])[0]
            a_hist.append(a)
            if t_near is None and abs(a - p.a_bar) < 1.0:
                t_near = t
    assert abs(a0 - p.a_bar) == pytest.approx(22.0, abs=0.5)
    assert t_near is not None and t_near <= 1.5e5
    assert max(abs(a - p.a_bar) for a in a_hist[-20:]) < 1.0


def test_example2_drag_closed_loop_matches_oracle(dp):
    # the feedback of the drag-free model flown on a system with drag (§4
    # Example 2); C exaggerated so that the drag changes the trajectory
    p = _small()
    o = oracle.Oracle(p)
    C = 1e-8
    rng = np.random.default_rng(9)
    with dp.Grid(p) as g:
        g.policy_iterate(tol=1e-6, max_sweeps=400, n_eval=20, polish=0)
        V = g.get_value()
        lo, hi = np.array(p.lo), np.array(p.hi)
        x0 = lo + (hi - lo) * rng.uniform(0.3, 0.7, size=(6, 4))
        ta, xg = g.simulate(x0, p.dt, p.dt, 300.0, drag=C)
        ta0, xg0 = g.simulate(x0, p.dt, p.dt, 300.0)
    _, xo = o.simulate(V, x0, tau=p.dt, h=p.dt, t_max=300.0, drag=C)
    agree = np.abs(xg - xo).max(axis=1) <= 1e-9 * np.abs(xo).max(axis=1)
    assert agree.sum() >= 5, np.abs(xg - xo).max(axis=1)
    assert np.abs(xg[:, 2] - xg0[:, 2]).max() > 1e-6     # the drag acts


def test_example2_feedback_holds_the_orbit_with_drag(dp):
    # the paper's drag (C_D 2.2, S 2.25 m^2, m 350 kg, rho_D 8.09e-14 kg/m^3):
    # the drag-free feedback still brings a within 1 km of 7000 km and keeps it
    p = W.example1(n=(80, 22, 22, 24))
    o = oracle.Oracle(p)
    C = W.example2_drag()
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=p.tol, max_sweeps=3000, n_eval=20, polish=0)
        y = W.example1_start(6978.0)[None, :]
        t, a_hist = 0.0, []
        while t < 4e5:
            ta, y = g.simulate(y, p.dt, p.dt, 5000.0, drag=C)
            t += 5000.0
            a_hist.append(o.elements(y[0])[0])
    assert max(abs(a - p.a_bar) for a in a_hist[-20:]) < 1.0
