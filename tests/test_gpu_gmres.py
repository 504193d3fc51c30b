"""Policy evaluation by GMRES on the GPU (§3 after Eq. (14): with the control
frozen, Eq. (13) is a sparse linear system, solved by GMRES).

The oracle's exact evaluation is a sparse direct solve of the same system
(oracle.Oracle.evaluate_exact, pinned by the CPU tests).  FP64 grids compare
element by element at 1e-9 of the value scale.  FP32 grids compare against
closed forms where the geometry is exact, and elsewhere within the bound of
FP32 rounding carried through the discounted sum, eps_32 M / (1 - beta).
"""
import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W
from test_gpu_parity import TOL32, _check_values

pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)


def _evaluate(dp, p, V0, codes, **kw):
    with dp.Grid(p) as g:
        g.set_value(V0)
        g.set_policy(codes)
        rc, st = g.policy_evaluate(**kw)
        return rc, st, g.get_value()


@pytest.mark.parametrize("name", ["config1_11x9x9x9", "example1_12x7x7x8", "band_13x4"])
def test_policy_evaluate_fp64_matches_exact_solution(dp, name):
    if name == "config1_11x9x9x9":
        p = W.config1(13).replace(n=(11, 9, 9, 9), precision=W.FP64)
    elif name == "example1_12x7x7x8":
        p = W.example1(n=(12, 7, 7, 8))
    else:
        p = W.config2(13).replace(precision=W.FP64)
    o = oracle.Oracle(p)
    codes = W.random_codes(p, 21)
    if p.off_control:
        codes[::7] = oracle.CODE_OFF
    exact = o.evaluate_exact(codes)
    V0 = W.smooth_value(p, 22) * (np.abs(exact).max() / o.M)
    idx = np.flatnonzero(o.active)
    rc, st, v = _evaluate(dp, p, V0[idx], codes[idx], tol=1e-13 * np.abs(exact).max(), max_sweeps=200,
                          gmres_restart=30)
    assert rc == dp.DP_OK and st.converged, st.asdict()
    assert st.gmres_cycles >= 1 and st.gmres_matvecs >= st.gmres_cycles
    _check_values(v, exact[idx], 1e-9, name)


def test_policy_evaluate_fp32_closed_form_1d(dp):
    # feet land on nodes, so FP32 geometry is exact: discounted time to go on
    # the left of the target, penalty M after leaving the box on the right
    M = 3.0
    p = W.unit_speed_1d().replace(penalty_M=M, precision=W.FP32)
    o = oracle.Oracle(p)
    exact = o.evaluate_exact(np.zeros(p.nodes, np.uint16))
    rc, st, v = _evaluate(dp, p, np.zeros(p.nodes), np.zeros(p.nodes, np.uint16), tol=1e-6, max_sweeps=50,
                          gmres_restart=20)
    assert rc == dp.DP_OK and st.converged, st.asdict()
    assert np.abs(v - exact).max() <= 4 * EPS32 * M / (1 - p.beta)


def test_policy_evaluate_fp32_config1(dp):
    p = W.config1(13).replace(n=(11, 9, 9, 9))
    o = oracle.Oracle(p)
    codes = W.random_codes(p, 23)
    exact = o.evaluate_exact(codes)
    rc, st, v = _evaluate(dp, p, W.smooth_value(p, 24), codes, tol=5e-6, max_sweeps=100, gmres_restart=30)
    assert st.converged, st.asdict()
    bound = EPS32 * o.M / (1 - p.beta)
    err = np.abs(v - exact)
    # FP32 geometry may put a foot that lies within ~1e-6 cells of a cell face
    # on the other side; the few nodes it reaches are counted and bounded
    assert np.mean(err > bound) <= 0.01, (err.max(), np.mean(err > bound))
    assert np.median(err) <= 0.1 * bound


def test_policy_evaluate_is_deterministic_and_stops_at_a_fixed_point(dp):
    p = W.config1(13).replace(n=(11, 9, 9, 9), precision=W.FP64)
    codes = W.random_codes(p, 25)
    V0 = W.smooth_value(p, 26)
    outs = []
    for _ in range(2):
        with dp.Grid(p) as g:
            g.set_value(V0)
            g.set_policy(codes)
            rc, st = g.policy_evaluate(tol=1e-12, max_sweeps=200, gmres_restart=25, gmres_reorth=1)
            assert st.converged
            outs.append(g.get_value())
            rc, st2 = g.policy_evaluate(tol=1e-10, max_sweeps=200)
            assert st2.converged and st2.gmres_cycles == 0 and st2.sweeps_eval == 1
    # the block sums are reduced in a fixed order: bit-identical runs
    assert np.array_equal(outs[0], outs[1])


def test_gmres_policy_iteration_fp32_with_polish_matches_oracle(dp):
    # the problem of the Jacobi polish test: the fixed point does not depend
    # on how each policy is evaluated
    p = W.config1(n=9).replace(beta=0.995, dt=0.1)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=500, polish=1, eval_solver=dp.DP_EVAL_GMRES,
                                  gmres_restart=20)
        assert rc == dp.DP_OK and st.converged and st.residual < 1e-6, st.asdict()
        assert st.sweeps_improve_fp64 > 0 and st.gmres_matvecs > 0
        v_gpu = g.get_value()
    V, codes, outer, ev, res = o.policy_iterate(tol=1e-9, max_outer=20000, n_eval=20)
    _check_values(v_gpu, V, TOL32, "GMRES policy iteration, FP32 + polish")


def test_gmres_policy_iteration_fp64_matches_oracle(dp):
    p = W.config1(n=9).replace(beta=0.995, dt=0.1, precision=W.FP64)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=1e-10, max_sweeps=500, eval_solver=dp.DP_EVAL_GMRES, gmres_restart=30,
                                  gmres_cycles=2)
        assert rc == dp.DP_OK and st.converged, st.asdict()
        assert st.sweeps_eval > 0          # the second cycle of each evaluation
        v_gpu = g.get_value()
    V, codes, outer, ev, res = o.policy_iterate(tol=1e-12, max_outer=20000, n_eval=20)
    # both are within tol / (1 - beta) of the scheme's fixed point
    _check_values(v_gpu, V, 1e-7, "GMRES policy iteration, FP64")


def test_gmres_policy_iteration_example1_matches_jacobi(dp):
    p = W.example1(n=(12, 7, 7, 8))
    o = oracle.Oracle(p)
    out = {}
    for solver in (dp.DP_EVAL_JACOBI, dp.DP_EVAL_GMRES):
        with dp.Grid(p) as g:
            rc, st = g.policy_iterate(tol=1e-7, max_sweeps=2000, n_eval=20, polish=0, eval_solver=solver,
                                      gmres_restart=30)
            assert rc == dp.DP_OK and st.converged, st.asdict()
            out[solver] = (g.get_value(), st)
    v_j, st_j = out[dp.DP_EVAL_JACOBI]
    v_g, st_g = out[dp.DP_EVAL_GMRES]
    assert st_g.sweeps_improve < st_j.sweeps_improve
    scale = np.abs(v_j).max()
    assert np.abs(v_g - v_j).max() <= 2e-7 / (1 - p.beta) + 1e-12 * scale
    # the GMRES solution is a fixed point of the oracle's Bellman operator
    v1, _, r, _ = o.sweep(v_g, mode=oracle.IMPROVE_FULL)
    assert r <= 1e-6 * scale


def test_gmres_options_are_checked(dp):
    p = W.config1(n=9)
    with dp.Grid(p) as g:
        for kw in ({"gmres_restart": dp.DP_GMRES_MAX_RESTART + 1}, {"gmres_rtol": 1.5}, {"gmres_reorth": 2},
                   {"gmres_cycles": -1}, {"eval_solver": 7}):
            with pytest.raises(dp.DPError) as e:
                g.policy_iterate(tol=1e-6, max_sweeps=5, eval_solver=kw.pop("eval_solver", dp.DP_EVAL_GMRES),
                                 **kw)
            assert e.value.code == dp.DP_EINVAL
    b = dp.Batch([W.config1(n=9)])
    try:
        with pytest.raises(dp.DPError) as e:
            b.policy_iterate(tol=1e-6, max_sweeps=5, eval_solver=dp.DP_EVAL_GMRES)
        assert e.value.code == dp.DP_EINVAL
    finally:
        b.close()


def test_gmres_restart_one_and_ragged_sizes(dp):
    # GMRES(1) (one Arnoldi step per cycle) and node counts that are not a
    # multiple of the 1024-node tile
    p = W.config1(13).replace(n=(7, 5, 6, 7), precision=W.FP64)
    o = oracle.Oracle(p)
    codes = W.random_codes(p, 27)
    exact = o.evaluate_exact(codes)
    rc, st, v = _evaluate(dp, p, np.zeros(p.nodes), codes, tol=1e-12, max_sweeps=20000, gmres_restart=1)
    assert st.converged, st.asdict()
    assert st.gmres_matvecs == st.gmres_cycles
    _check_values(v, exact, 1e-9, "GMRES(1)")
