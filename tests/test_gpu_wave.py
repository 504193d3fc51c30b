"""Multi-level evaluation (several Jacobi evaluation sweeps of Eq. (13) per
launch, as a wavefront over node chunks): the values, policies and residuals
of policy iteration must equal those of one evaluation sweep per launch bit
for bit, whatever the number of levels, on the full box and on the reduced
grid, for plain and diagonal-solved evaluation, and for the FP32 increments of
the FP64-value phase.  One sweep per launch is checked against the oracle by
the other GPU tests.
"""
import numpy as np
import pytest

from paper_2407_14675_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _solve(dp, p, levels, **kw):
    hist = np.zeros(64)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=0.0, warm=0, eval_levels=levels, history=hist, **kw)
        return g.get_value(), g.get_policy(), hist[:st.history_count].copy(), st


def _same(a, b, what):
    va, ca, ha, sa = a
    vb, cb, hb, sb = b
    assert np.array_equal(va, vb), (what, float(np.abs(va - vb).max()), int((va != vb).sum()))
    assert np.array_equal(ca, cb), (what, int((ca != cb).sum()))
    assert np.array_equal(ha, hb), (what, ha, hb)
    assert (sa.sweeps_eval, sa.sweeps_eval_fp64) == (sb.sweeps_eval, sb.sweeps_eval_fp64)


@pytest.mark.parametrize("name,p", [
    ("box_41x4", W.config1(n=41)),
    ("band_61x4", W.config2(n=61)),
    ("box_17x4", W.config1(n=17)),          # fewer chunks than the reach: levels serialise
])
def test_multi_level_evaluation_equals_one_sweep_per_launch(dp, name, p):
    ref = _solve(dp, p, 1, max_sweeps=3, n_eval=20, polish=0)
    for levels in (2, 5, 20):
        _same(ref, _solve(dp, p, levels, max_sweeps=3, n_eval=20, polish=0), (name, levels))


@pytest.mark.parametrize("name,p", [("box_41x4", W.config1(n=41)), ("band_61x4", W.config2(n=61))])
def test_multi_level_diagonal_solved_evaluation(dp, name, p):
    kw = dict(max_sweeps=3, n_eval=12, polish=0, eval_solver=dp.DP_EVAL_DIAG)
    ref = _solve(dp, p, 1, **kw)
    for levels in (3, 12):
        _same(ref, _solve(dp, p, levels, **kw), (name, levels))


@pytest.mark.parametrize("solver", ["jacobi", "diag"])
def test_multi_level_increments_of_the_fp64_value_phase(dp, solver):
    """FP32 grid switched to FP64 values after the first improvement (switch
    tolerance 100, above the first residual, M = 20): the evaluation then runs
    on FP32 increments summed into the FP64 value."""
    p = W.config2(n=61)
    es = dp.DP_EVAL_DIAG if solver == "diag" else dp.DP_EVAL_JACOBI
    kw = dict(max_sweeps=4, n_eval=10, n_eval_fp64=16, polish=1, switch_tol=100.0, eval_solver=es)
    ref = _solve(dp, p, 1, **kw)
    assert ref[3].switch_outer >= 0 and ref[3].sweeps_eval_fp64 > 0
    for levels in (4, 16):
        _same(ref, _solve(dp, p, levels, **kw), (solver, levels))


def test_multi_level_solve_to_tolerance_matches(dp):
    """A whole FP32 + polish solve to 1e-6 with the automatic level count
    ends where the one-sweep-per-launch solve ends."""
    p = W.config1(n=41)
    hist = np.zeros(4000)
    out = []
    for levels in (1, 0):
        with dp.Grid(p) as g:
            rc, st = g.policy_iterate(tol=1e-6, max_sweeps=3000, n_eval=20, polish=1, warm=0,
                                      eval_levels=levels, history=hist)
            out.append((g.get_value(), g.get_policy(), st.converged, st.sweeps_improve, st.sweeps_improve_fp64))
    assert out[0][2] and out[1][2]
    assert out[0][3:] == out[1][3:]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_multi_level_wait_limit_gives_up_cleanly(dp):
    """Test hook: with a wait limit of 0 the first unmet dependency makes the
    launch give up (on 17^4 every chunk of a level depends on every chunk of
    the previous one, and the blocks waiting for level 1 start while level 0
    runs): the call returns DP_ETIMEOUT, no block hangs, and with the default
    limit restored the next solve is bit-identical to one sweep per launch."""
    p = W.config1(n=17)
    dp.dp_set_wave_wait_limit(0)
    try:
        with dp.Grid(p) as g:
            with pytest.raises(dp.DPError) as e:
                g.policy_iterate(tol=0.0, max_sweeps=2, n_eval=20, polish=0, warm=0, eval_levels=20)
            assert e.value.code == dp.DP_ETIMEOUT
    finally:
        dp.dp_set_wave_wait_limit(-1)
    ref = _solve(dp, p, 1, max_sweeps=3, n_eval=20, polish=0)
    _same(ref, _solve(dp, p, 20, max_sweeps=3, n_eval=20, polish=0), "after a timeout")


def test_multi_level_with_each_foot_format(dp):
    """dp_set_foot_format: with 8-byte feet forced, the diagonal-solved
    evaluation recomputes the feet one sweep per launch (whatever
    eval_levels asks), with word pairs forced the plain evaluation's levels
    read the pairs; each equals the same solve one sweep per launch."""
    p = W.config2(n=41)
    for fmt, solver in ((dp.DP_FOOT_WORD8, dp.DP_EVAL_DIAG), (dp.DP_FOOT_PAIR, dp.DP_EVAL_JACOBI)):
        out = []
        for levels in (1, 6):
            hist = np.zeros(64)
            with dp.Grid(p) as g:
                g.set_foot_format(fmt)
                rc, st = g.policy_iterate(tol=0.0, max_sweeps=3, n_eval=12, polish=0, warm=0, eval_levels=levels,
                                          eval_solver=solver, history=hist)
                out.append((g.get_value(), g.get_policy(), hist[:st.history_count].copy(), st))
        _same(out[0], out[1], (fmt, solver))
