"""Warm start of a grid from another grid's solution (dp_warm_start_from_grid):
Q1 interpolation of the source value at the destination nodes, checked in
FP64 against the oracle's own interpolation, and a solve started from it."""
import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dst_reduced", [False, True])
def test_interpolated_value_and_nearest_policy_match_the_oracle(dp, dst_reduced):
    src_p = W.config1(n=13).replace(precision=W.FP64)
    dst_p = (W.config2(n=21) if dst_reduced else W.config1(n=21)).replace(precision=W.FP64)
    o_src = oracle.Oracle(src_p)
    o_dst = oracle.Oracle(dst_p)
    V = W.smooth_value(src_p, 3)
    V[o_src.target.astype(bool)] = 0.0
    codes = W.random_codes(src_p, 4)
    with dp.Grid(src_p) as s, dp.Grid(dst_p) as d:
        s.set_value(V)
        s.set_policy(codes)
        dp.dp_warm_start_from_grid(s.h, d.h)
        got_v, got_c, idx = d.get_value(), d.get_policy(), d.active_index()
    lo_s, hi_s = np.array(src_p.lo), np.array(src_p.hi)
    h_s = (hi_s - lo_s) / (np.array(src_p.n) - 1)
    h_d = (np.array(dst_p.hi) - np.array(dst_p.lo)) / (np.array(dst_p.n) - 1)
    for k in range(0, len(idx), 7):
        i = np.array(np.unravel_index(idx[k], dst_p.n))
        x = np.array(dst_p.lo) + i * h_d
        if o_dst.target[idx[k]]:
            assert got_v[k] == 0.0
            continue
        s = (x - lo_s) / h_s
        ref = o_src.interp(V, s)
        ref = o_dst.M if ref is None else ref
        assert got_v[k] == pytest.approx(ref, rel=1e-13, abs=1e-12)
        nn = np.clip(np.floor(s + 0.5).astype(int), 0, np.array(src_p.n) - 1)
        assert got_c[k] == codes[np.ravel_multi_index(nn, src_p.n)]


def test_solve_from_a_coarse_solution_reaches_the_cold_fixed_point(dp):
    coarse, fine = W.config1(n=13), W.config1(n=21)
    opts = dict(tol=1e-6, max_sweeps=4000, n_eval=20, polish=1)
    with dp.Grid(coarse) as c, dp.Grid(fine) as f:
        rc, sc = c.policy_iterate(**opts)
        assert sc.converged
        rc, s_cold = f.policy_iterate(**opts)
        V_cold = f.get_value()
        dp.dp_warm_start_from_grid(c.h, f.h)
        rc, s_warm = f.policy_iterate(warm=1, **opts)
        assert s_warm.converged
        V_warm = f.get_value()
        M = f.info["penalty_M"]
    assert np.abs(V_warm - V_cold).max() <= 1e-4 * M
    assert s_warm.sweeps_improve + s_warm.sweeps_improve_fp64 < s_cold.sweeps_improve + s_cold.sweeps_improve_fp64
