"""The evaluation as the Jacobi method proper on the linear system of Eq. (13):
each node's own coefficient solved (DP_SWEEP_EVAL_DIAG, DP_EVAL_DIAG), against
the oracle's eval_diag_sweep (pinned by the CPU tests) and, for whole solves,
against the oracle's fixed point, which this iteration shares with the plain
evaluation sweep.
"""
import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W
from test_gpu_parity import TOL32, TOL64, _check_values

pytestmark = pytest.mark.gpu


def _problem(name):
    if name == "config1_11x9x9x9_fp64":
        return W.config1(13).replace(n=(11, 9, 9, 9), precision=W.FP64)
    if name == "example1_12x7x7x8":
        return W.example1(n=(12, 7, 7, 8))
    if name == "band_13x4_fp64":
        return W.config2(13).replace(precision=W.FP64)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["config1_11x9x9x9_fp64", "example1_12x7x7x8", "band_13x4_fp64"])
def test_eval_diag_sweep_matches_oracle_fp64(dp, name):
    p = _problem(name)
    o = oracle.Oracle(p)
    codes = W.random_codes(p, 41)
    if p.off_control:
        codes[::6] = oracle.CODE_OFF
    scale = 1.0 if not p.off_control else 1e-2
    V = W.smooth_value(p, 42) * scale
    V[o.target.astype(bool)] = 0.0
    idx = np.flatnonzero(o.active)
    want, r_o = o.eval_diag_sweep(V, codes)
    with dp.Grid(p) as g:
        g.set_value(V[idx])
        g.set_policy(codes[idx])
        r = g.sweep(dp.DP_SWEEP_EVAL_DIAG)
        v = g.get_value()
    _check_values(v, want[idx], TOL64, name)
    assert abs(r - r_o) <= TOL64 * np.abs(want).max()


def test_eval_diag_sweep_fp32_frozen_feet_and_recomputed(dp):
    p = W.config1(n=17)
    o = oracle.Oracle(p)
    V0 = W.smooth_value(p, 43)
    V0[o.target.astype(bool)] = 0.0
    with dp.Grid(p) as g:
        # the diagonal-solved evaluation reads the 24-bit word pairs
        g.set_foot_format(dp.DP_FOOT_PAIR)
        # recomputed feet: a policy set from the host has no frozen feet
        codes = W.random_codes(p, 44)
        g.set_value(V0)
        g.set_policy(codes)
        g.sweep(dp.DP_SWEEP_EVAL_DIAG)
        v_rec = g.get_value()
        want, _ = o.eval_diag_sweep(V0, codes)
        _check_values(v_rec, want, TOL32, "recomputed", o=o, nodes=np.arange(p.nodes), codes=codes)
        # frozen feet: stored by the improvement sweep
        g.set_value(V0)
        g.sweep(dp.DP_SWEEP_IMPROVE_FULL)
        V1, c1 = g.get_value(), g.get_policy()
        g.sweep(dp.DP_SWEEP_EVAL_DIAG)
        v_feet = g.get_value()
    want, _ = o.eval_diag_sweep(V1, c1)
    _check_values(v_feet, want, TOL32, "frozen feet", o=o, nodes=np.arange(p.nodes), codes=c1)


def test_diag_policy_iteration_fp32_with_polish_matches_oracle(dp):
    # the problem of the Jacobi polish test; the FP64-value phase runs the
    # diagonal-solved increments
    p = W.config1(n=9).replace(beta=0.995, dt=0.1)
    o = oracle.Oracle(p)
    out = {}
    for solver in (dp.DP_EVAL_JACOBI, dp.DP_EVAL_DIAG):
        with dp.Grid(p) as g:
            rc, st = g.policy_iterate(tol=1e-6, max_sweeps=5000, n_eval=20, polish=1, eval_solver=solver)
            assert rc == dp.DP_OK and st.converged and st.residual < 1e-6, st.asdict()
            out[solver] = (g.get_value(), st)
    v_gpu, st = out[dp.DP_EVAL_DIAG]
    assert st.sweeps_improve_fp64 > 0
    st_j = out[dp.DP_EVAL_JACOBI][1]
    assert st.sweeps_improve + st.sweeps_improve_fp64 < st_j.sweeps_improve + st_j.sweeps_improve_fp64
    V, codes, outer, ev, res = o.policy_iterate(tol=1e-9, max_outer=20000, n_eval=20)
    _check_values(v_gpu, V, TOL32, "diagonal-solved policy iteration, FP32 + polish")


def test_diag_policy_iteration_fp64_matches_oracle(dp):
    p = W.config1(n=9).replace(beta=0.995, dt=0.1, precision=W.FP64)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=1e-10, max_sweeps=5000, n_eval=20, eval_solver=dp.DP_EVAL_DIAG)
        assert rc == dp.DP_OK and st.converged, st.asdict()
        v_gpu = g.get_value()
    V, codes, outer, ev, res = o.policy_iterate(tol=1e-12, max_outer=20000, n_eval=20)
    _check_values(v_gpu, V, 1e-7, "diagonal-solved policy iteration, FP64")


def test_diag_policy_iteration_example1_matches_jacobi(dp):
    p = W.example1(n=(12, 7, 7, 8))
    o = oracle.Oracle(p)
    out = {}
    for solver in (dp.DP_EVAL_JACOBI, dp.DP_EVAL_DIAG):
        with dp.Grid(p) as g:
            rc, st = g.policy_iterate(tol=1e-7, max_sweeps=2000, n_eval=20, polish=0, eval_solver=solver)
            assert rc == dp.DP_OK and st.converged, st.asdict()
            out[solver] = (g.get_value(), st)
    v_j, st_j = out[dp.DP_EVAL_JACOBI]
    v_d, st_d = out[dp.DP_EVAL_DIAG]
    assert st_d.sweeps_improve <= st_j.sweeps_improve
    scale = np.abs(v_j).max()
    assert np.abs(v_d - v_j).max() <= 2e-7 / (1 - p.beta) + 1e-12 * scale
    v1, _, r, _ = o.sweep(v_d, mode=oracle.IMPROVE_FULL)
    assert r <= 1e-6 * scale


def test_diag_modes_are_rejected_where_unsupported(dp):
    import torch
    p = W.config1(n=9)
    a = torch.zeros(p.nodes, device="cuda", dtype=torch.float32)
    b = torch.zeros(p.nodes, device="cuda", dtype=torch.float32)
    c = torch.zeros(p.nodes, device="cuda", dtype=torch.int16)
    desc = dp.desc_from_problem(p, stream=int(torch.cuda.current_stream().cuda_stream))
    with pytest.raises(dp.DPError) as e:
        dp.dp_bellman_sweep_noalloc(desc, dp.DP_SWEEP_EVAL_DIAG, a.data_ptr(), b.data_ptr(), c.data_ptr())
    assert e.value.code == dp.DP_EINVAL
    with dp.Grid(p) as g:
        with pytest.raises(dp.DPError) as e:
            g.sweep(6)
        assert e.value.code == dp.DP_EINVAL


@pytest.mark.parametrize("name", ["config0_17x4", "unit_speed_2d"])
def test_vi_diag_sweeps_match_oracle_fp64(dp, name):
    p = W.config0() if name == "config0_17x4" else W.unit_speed_2d(n=13, n_angles=8)
    o = oracle.Oracle(p)
    V = W.smooth_value(p, 45)
    V[o.target.astype(bool)] = 0.0
    with dp.Grid(p) as g:
        g.set_value(V)
        for k in range(3):
            want, r_o = o.vi_diag_sweep(V)
            r = g.sweep(dp.DP_SWEEP_VI_DIAG)
            v = g.get_value()
            _check_values(v, want, TOL64, "%s sweep %d" % (name, k))
            assert abs(r - r_o) <= TOL64 * np.abs(want).max()
            V = want


def test_vi_diag_reaches_the_value_iteration_fixed_point(dp):
    p = W.config0()
    out = {}
    for solver in (dp.DP_EVAL_JACOBI, dp.DP_EVAL_DIAG):
        with dp.Grid(p) as g:
            rc, st = g.value_iterate(tol=1e-10, max_sweeps=60000, eval_solver=solver)
            assert rc == dp.DP_OK and st.converged, st.asdict()
            out[solver] = (g.get_value(), st.sweeps_vi)
    (v_p, n_p), (v_d, n_d) = out[dp.DP_EVAL_JACOBI], out[dp.DP_EVAL_DIAG]
    assert n_d < n_p / 3
    # both within tol / (1 - beta) of the fixed point
    assert np.abs(v_d - v_p).max() <= 2e-10 / (1 - p.beta)
    with dp.Grid(W.example1(n=(12, 7, 7, 8))) as g:
        with pytest.raises(dp.DPError) as e:
            g.value_iterate(tol=1e-6, max_sweeps=5, eval_solver=dp.DP_EVAL_DIAG)
        assert e.value.code == dp.DP_EINVAL
        with pytest.raises(dp.DPError) as e:
            g.sweep(dp.DP_SWEEP_VI_DIAG)
        assert e.value.code == dp.DP_EINVAL


@pytest.mark.parametrize("name", ["config1_11x9x9x9_fp64", "example1_12x7x7x8", "band_13x4_fp64"])
def test_fp64_frozen_feet_evaluate_as_recomputing(dp, name):
    # FP64 grids store the foot of the chosen control in their improvement
    # sweeps; evaluation from it must equal the recomputing evaluation (a
    # policy set from the host has no stored feet), bit for bit for the
    # minimum-time dynamics
    p = _problem(name)
    o = oracle.Oracle(p)
    scale = 1.0 if not p.off_control else 1e-2
    V = W.smooth_value(p, 47) * scale
    V[o.target.astype(bool)] = 0.0
    idx = np.flatnonzero(o.active)
    with dp.Grid(p) as g:
        for mode in (dp.DP_SWEEP_EVAL, dp.DP_SWEEP_EVAL_DIAG):
            g.set_value(V[idx])
            g.sweep(dp.DP_SWEEP_IMPROVE_FULL)
            V1, c1 = g.get_value(), g.get_policy()
            g.sweep(mode)
            v_feet = g.get_value()
            g.set_value(V1)
            g.set_policy(c1)
            g.sweep(mode)
            v_rec = g.get_value()
            if p.off_control:
                # the running cost of Eq. (11) is computed by the improvement
                # kernel for the stored feet and by the evaluation kernel when
                # recomputing: their FMA contractions may differ by an ulp,
                # which the diagonal step's cancellation can enlarge a little
                np.testing.assert_allclose(v_feet, v_rec, rtol=1e-13, atol=0)
                assert (c1 == dp.DP_CODE_OFF).any()
            else:
                np.testing.assert_array_equal(v_feet, v_rec)


def test_solvers_agree_on_the_fp32_band_grid(dp):
    # the energy-band (reduced) grid in FP32 with the FP64 polish: plain,
    # diagonal-solved and GMRES evaluation reach the same fixed point
    p = W.config2(25)
    out = {}
    for name, kw in (("sweeps", dict(n_eval=20)), ("diag", dict(n_eval=20, eval_solver=dp.DP_EVAL_DIAG)),
                     ("gmres", dict(eval_solver=dp.DP_EVAL_GMRES, gmres_restart=20))):
        with dp.Grid(p) as g:
            rc, st = g.policy_iterate(tol=1e-6, max_sweeps=3000, polish=1, **kw)
            assert rc == dp.DP_OK and st.converged, (name, st.asdict())
            out[name] = (g.get_value(), st.sweeps_improve + st.sweeps_improve_fp64)
    v0 = out["sweeps"][0]
    for name in ("diag", "gmres"):
        # each is within tol / (1 - beta) of the scheme's fixed point
        assert np.abs(out[name][0] - v0).max() <= 2e-6 / (1 - p.beta), name
    assert out["diag"][1] < out["sweeps"][1]


def test_fp64_phase_evaluation_count(dp):
    # n_eval_fp64 sets the evaluation sweeps per improvement once the values
    # are FP64; every count reaches the same fixed point
    p = W.config1(n=9).replace(beta=0.995, dt=0.1)
    out = {}
    for ne64 in (0, 7, 120):
        with dp.Grid(p) as g:
            rc, st = g.policy_iterate(tol=1e-6, max_sweeps=5000, n_eval=20, polish=1,
                                      eval_solver=dp.DP_EVAL_DIAG, n_eval_fp64=ne64)
            assert rc == dp.DP_OK and st.converged and st.sweeps_improve_fp64 > 0, st.asdict()
            out[ne64] = (g.get_value(), st)
    for ne64 in (7, 120):
        st = out[ne64][1]
        # the device stops the queue at the first converged improvement: the
        # converged walk and the full tabulation that confirms it run no
        # evaluation sweeps
        assert st.sweeps_eval_fp64 <= ne64 * st.sweeps_improve_fp64
        assert st.sweeps_eval_fp64 >= ne64 * (st.sweeps_improve_fp64 - 2)
        assert np.abs(out[ne64][0] - out[0][0]).max() <= 2e-6 / (1 - p.beta)
    st0 = out[0][1]
    assert st0.sweeps_eval_fp64 >= 80 * (st0.sweeps_improve_fp64 - 2)   # automatic: at least 80 (diagonal-solved)
    with dp.Grid(p) as g:
        with pytest.raises(dp.DPError) as e:
            g.policy_iterate(tol=1e-6, max_sweeps=5, n_eval=20, n_eval_fp64=-1)
        assert e.value.code == dp.DP_EINVAL


@pytest.mark.parametrize("fmt", ["word8", "pair"])
def test_large_grid_block_layout_sweeps_match_oracle(dp, fmt):
    # a reduced grid large enough for the large-block layout of the frozen-feet
    # sweeps (384,580 stored nodes: every SM gets a 1024- or 768-thread
    # block): one plain and one diagonal-solved evaluation sweep at the feet
    # an improvement stored (8-byte words: the plain sweep reads them, the
    # diagonal-solved one recomputes; word pairs: both read them), against
    # the oracle
    p = W.config2(n=35)
    o = oracle.Oracle(p)
    idx = np.flatnonzero(o.active)
    V = W.smooth_value(p, 48)
    V[o.target.astype(bool)] = 0.0
    with dp.Grid(p) as g:
        g.set_foot_format(dp.DP_FOOT_WORD8 if fmt == "word8" else dp.DP_FOOT_PAIR)
        g.set_value(V[idx])
        g.sweep(dp.DP_SWEEP_IMPROVE_FULL)
        V1, c1 = g.get_value(), g.get_policy()
        g.sweep(dp.DP_SWEEP_EVAL)
        v_plain = g.get_value()
        g.set_value(V1)                      # the stored feet stay valid
        g.sweep(dp.DP_SWEEP_EVAL_DIAG)
        v_diag = g.get_value()
    Vf = np.zeros(p.nodes)
    Vf[idx] = V1
    cf = np.zeros(p.nodes, np.uint16)
    cf[idx] = c1
    want_plain = o.sweep(Vf, mode=oracle.EVAL, codes=cf)[0][idx]
    want_diag = o.eval_diag_sweep(Vf, cf)[0][idx]
    _check_values(v_plain, want_plain, TOL32, "plain evaluation", o=o, nodes=idx, codes=c1)
    _check_values(v_diag, want_diag, TOL32, "diagonal-solved evaluation", o=o, nodes=idx, codes=c1)


def test_large_grid_solvers_agree_with_polish(dp):
    # 25^4 (390,625 nodes): the large-block evaluation and increment sweeps
    # in both precision phases; plain and diagonal-solved evaluation reach the
    # same fixed point
    p = W.config1(n=25)
    out = {}
    for name, kw in (("sweeps", dict(n_eval=20)), ("diag", dict(n_eval=20, eval_solver=dp.DP_EVAL_DIAG))):
        with dp.Grid(p) as g:
            rc, st = g.policy_iterate(tol=1e-6, max_sweeps=3000, polish=1, **kw)
            assert rc == dp.DP_OK and st.converged and st.sweeps_improve_fp64 > 0, (name, st.asdict())
            out[name] = g.get_value()
    assert np.abs(out["diag"] - out["sweeps"]).max() <= 2e-6 / (1 - p.beta)
