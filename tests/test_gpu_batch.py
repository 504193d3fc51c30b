"""Batched transfers through the C ABI (dp_batch_*).

Three kinds of evidence:
  * one-operator parity of every transfer of a heterogeneous batch with the
    FP64 oracle (the tolerances of the single-grid parity tests);
  * the batched solve reproduces, transfer by transfer, the solve of a grid
    of its own (same sweep sequence, same per-node arithmetic);
  * unit-speed batches against the closed-form minimum-time value.
"""
import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W
from test_gpu_parity import TOL32, _check_codes, _check_values

pytestmark = pytest.mark.gpu


def _oracle_mode(dp, mode):
    return {dp.DP_SWEEP_IMPROVE_FULL: oracle.IMPROVE_FULL, dp.DP_SWEEP_IMPROVE_WALK: oracle.IMPROVE_WALK,
            dp.DP_SWEEP_EVAL: oracle.EVAL}[mode]


def test_batch_sweeps_match_oracle_per_transfer(dp):
    # uneven sizes (ragged item tails), different thrust, targets and boxes
    probs = W.batch_transfers(count=4, seed=5, sizes=(9, 11, 13))
    ors = [oracle.Oracle(p) for p in probs]
    with dp.Batch(probs) as b:
        dp.dp_batch_set_items(b.h, 256, 512)
        for i, p in enumerate(probs):
            b.set_value(i, W.smooth_value(p, 30 + i))
        for mode in (dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_EVAL, dp.DP_SWEEP_IMPROVE_WALK, dp.DP_SWEEP_EVAL):
            before = [(b.get_value(i), b.get_policy(i)) for i in range(b.count)]
            res, ms = b.sweep(mode)
            for i, (p, o) in enumerate(zip(probs, ors)):
                V, codes = before[i]
                v_o, c_o, r_o, _ = o.sweep(V, mode=_oracle_mode(dp, mode), codes=codes)
                v_g = b.get_value(i)
                idx = np.arange(p.nodes)
                if mode == dp.DP_SWEEP_EVAL:
                    _check_values(v_g, v_o, TOL32, "transfer %d mode %d" % (i, mode), o=o, nodes=idx, codes=codes)
                else:
                    _check_values(v_g, v_o, TOL32, "transfer %d mode %d" % (i, mode))
                    free = np.flatnonzero(~o.target.astype(bool))
                    _check_codes(o, V, free, b.get_policy(i)[free], c_o[free], 1e-5 * o.M)
                assert res[i] == pytest.approx(np.abs(v_g - V).max(), rel=1e-6, abs=1e-12)


@pytest.mark.parametrize("solver", ["sweeps", "diag"])
def test_batch_solve_reproduces_single_grid_solves(dp, solver):
    probs = W.batch_transfers(count=6, seed=11, sizes=(9, 11, 13))
    opts = dict(tol=1e-6, max_sweeps=4000, n_eval=20, polish=1,
                eval_solver=dp.DP_EVAL_DIAG if solver == "diag" else dp.DP_EVAL_JACOBI)
    with dp.Batch(probs) as b:
        dp.dp_batch_set_items(b.h, 512, 256)
        rc, tot, per = b.policy_iterate(**opts)
        assert rc == dp.DP_OK and tot.converged
        got = [(b.get_value(i), b.get_policy(i)) for i in range(b.count)]
    assert tot.node_updates > 0 and tot.launches > 0
    for i, p in enumerate(probs):
        with dp.Grid(p) as g:
            # a batch evaluates n_eval sweeps per improvement in both precision
            # phases: the single grid is given the same FP64-phase count
            rc, st = g.policy_iterate(n_eval_fp64=opts["n_eval"], **opts)
            assert st.converged
            V, C = g.get_value(), g.get_policy()
        s = per[i]
        assert s["converged"] == 1 and s["nodes"] == p.nodes
        assert (s["sweeps_improve"], s["sweeps_eval"], s["sweeps_improve_fp64"], s["sweeps_eval_fp64"]) == \
            (st.sweeps_improve, st.sweeps_eval, st.sweeps_improve_fp64, st.sweeps_eval_fp64), (i, s, st.asdict())
        assert s["switch_outer"] == st.switch_outer
        assert s["residual"] == st.residual
        np.testing.assert_array_equal(got[i][0], V)
        np.testing.assert_array_equal(got[i][1], C)


def test_batch_unit_speed_closed_form(dp):
    # x' = cos a with dt = h: feet on nodes, V = dt (1 - beta^n) / (1 - beta)
    cases = [(17, 0.9, 8), (21, 0.95, 3), (9, 0.8, 0), (33, 0.97, 20)]
    probs = [W.unit_speed_1d(n=n, beta=beta, target_node=t).replace(precision=W.FP32) for n, beta, t in cases]
    with dp.Batch(probs) as b:
        rc, tot, per = b.policy_iterate(tol=1e-7, max_sweeps=200, n_eval=3, polish=1)
        assert tot.converged
        for i, (n, beta, t) in enumerate(cases):
            p = probs[i]
            steps = np.abs(np.arange(n) - t)
            exact = p.dt * (1 - beta ** steps) / (1 - beta)
            V = b.get_value(i).reshape(p.n)
            for k in range(2):
                assert np.abs(V[:, k, k, k] - exact).max() < 1e-6 * exact.max() + 1e-7
            c = b.get_policy(i).reshape(p.n)[:, 0, 0, 0]
            assert (c[:t] == 0).all() and (c[t + 1:] == 32768).all()


def test_batch_warm_start_from_a_solved_value(dp):
    # a warm start from the converged value and policy stops after the
    # confirming improvements
    probs = W.batch_transfers(count=3, seed=12, sizes=(9, 11))
    with dp.Batch(probs) as b:
        rc, tot, per = b.policy_iterate(tol=1e-6, max_sweeps=4000, n_eval=20, polish=1)
        assert tot.converged
        V0 = [b.get_value(i) for i in range(3)]
        C0 = [b.get_policy(i) for i in range(3)]
        for i in range(3):
            b.set_value(i, V0[i])
            b.set_policy(i, C0[i])
        rc, tot2, per2 = b.policy_iterate(tol=1e-6, max_sweeps=4000, n_eval=20, polish=1, warm=1)
        assert tot2.converged
        imp = tot2.sweeps_improve + tot2.sweeps_improve_fp64
        assert imp < (tot.sweeps_improve + tot.sweeps_improve_fp64) / 5
        for i in range(3):
            M = probs[i].M()
            assert np.abs(b.get_value(i) - V0[i]).max() <= 1e-4 * M


def test_batch_autotune_and_errors(dp):
    probs = W.batch_transfers(count=3, seed=13, sizes=(9, 11))
    with dp.Batch(probs) as b:
        ie, ii = b.autotune()
        cands = (512, 1024, 2048, 4096, 8192, 16384, 32768)
        assert ie in cands and ii in cands
        info = b.info()
        assert (info["item_eval"], info["item_improve"]) == (ie, ii)
        assert info["nodes_total"] == sum(p.nodes for p in probs)
        assert (b.get_value(0) == 0).all()
        with pytest.raises(dp.DPError) as e:
            dp.dp_batch_set_items(b.h, 300, 256)
        assert e.value.code == dp.DP_EINVAL
        with pytest.raises(dp.DPError):
            dp.dp_batch_get_value(b.h, 3, probs[0].nodes)
        with pytest.raises(dp.DPError):
            dp.dp_batch_get_value(b.h, 0, probs[0].nodes + 1)
        bad = W.random_value(probs[1], 1)
        bad[5] = np.nan
        with pytest.raises(dp.DPError) as e:
            b.set_value(1, bad)
        assert e.value.code == dp.DP_ENONFINITE
    for bad_p in (probs[0].replace(precision=W.FP64), W.config2(n=21).replace(precision=W.FP32),
                  W.unit_speed_1d().replace(precision=W.FP32)):
        with pytest.raises(dp.DPError) as e:
            dp.Batch([probs[1], bad_p])
        assert e.value.code == dp.DP_EINVAL and "transfer 1" in str(e.value)


@pytest.mark.parametrize("solver,polish", [("diag", 0), ("sweeps", 1)])
def test_batch_standalone_evaluation_after_a_solve(dp, solver, polish):
    # the frozen feet a batched solve leaves behind: word pairs after a
    # diagonal-solved solve (FP32 values), word pairs of the FP64-value phase
    # after a polished one (switch at the first improvement); a stand-alone
    # evaluation sweep afterwards reads or recomputes them and matches the
    # oracle transfer by transfer
    probs = W.batch_transfers(count=3, seed=7, sizes=(9, 11))
    ors = [oracle.Oracle(p) for p in probs]
    kw = dict(tol=1e-6, max_sweeps=40, n_eval=10, polish=polish)
    if solver == "diag":
        kw["eval_solver"] = dp.DP_EVAL_DIAG
    if polish:
        kw["switch_tol"] = 100.0
    with dp.Batch(probs) as b:
        rc, tot, per = b.policy_iterate(**kw)
        if polish:
            assert all(s["switch_outer"] >= 0 for s in per)
        before = [(b.get_value(i), b.get_policy(i)) for i in range(b.count)]
        b.sweep(dp.DP_SWEEP_EVAL)
        for i, (p, o) in enumerate(zip(probs, ors)):
            V, codes = before[i]
            v_o = o.sweep(V, mode=oracle.EVAL, codes=codes)[0]
            _check_values(b.get_value(i), v_o, TOL32, "transfer %d" % i, o=o, nodes=np.arange(p.nodes),
                          codes=codes)
