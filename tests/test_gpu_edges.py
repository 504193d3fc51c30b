"""Edge cases of the sweep through the C ABI, against the oracle: the
smallest grids (two nodes per coordinate, so every node is a box corner and
every cell a boundary cell; and an uneven 3 x 2 x 5 x 2 grid), a target that
covers the whole box (every node on the target: V = 0 and a zero residual),
a box with no target node, and an energy band that holds no node (refused
when the grid is created).
"""
import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W
from test_gpu_parity import TOL32, TOL64, _check_codes, _check_values

pytestmark = pytest.mark.gpu


def _oracle_mode(dp, mode):
    return {dp.DP_SWEEP_VI: oracle.VI, dp.DP_SWEEP_IMPROVE_FULL: oracle.IMPROVE_FULL,
            dp.DP_SWEEP_EVAL: oracle.EVAL}[mode]


def _one_sweep_each(dp, p, seed):
    """VI, full-table improvement and evaluation sweeps from the same value
    and policy, each against the oracle's sweep of the GPU's own input."""
    o = oracle.Oracle(p)
    tol = TOL64 if p.precision == W.FP64 else TOL32
    V = W.smooth_value(p, seed)
    codes = W.random_codes(p, seed + 1)
    nodes = np.arange(o.N)
    free = np.flatnonzero(~o.target.astype(bool))
    with dp.Grid(p) as g:
        for mode in (dp.DP_SWEEP_VI, dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_EVAL):
            g.set_value(V)
            g.set_policy(codes)
            V_in = g.get_value()               # storage-rounded, target zeroed
            r = g.sweep(mode)
            v_gpu, c_gpu = g.get_value(), g.get_policy()
            want, c_or, r_or, _ = o.sweep(V_in, mode=_oracle_mode(dp, mode), codes=codes)
            if mode == dp.DP_SWEEP_EVAL:
                _check_values(v_gpu, want, tol, "eval %s" % (p.n,), o=o, nodes=nodes, codes=codes)
            else:
                _check_values(v_gpu, want, tol, "mode %d %s" % (mode, p.n))
            if mode == dp.DP_SWEEP_IMPROVE_FULL and free.size:
                _check_codes(o, V_in, free, c_gpu[free], c_or[free], tie=1e-5 * o.M)
            assert abs(r - r_or) <= tol * max(np.abs(want).max(), 1e-300)


@pytest.mark.parametrize("prec", [W.FP64, W.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("n", [(2, 2, 2, 2), (3, 2, 5, 2)], ids=["2x2x2x2", "3x2x5x2"])
def test_smallest_grids_match_oracle(dp, n, prec):
    # a larger thrust and step than config 0 so that the feet move across
    # the single cells: the penalty and the interior blend both occur
    p = W.config0().replace(n=n, precision=prec, accel=2e-2, dt=0.5, refine=1 if prec == W.FP32 else 0)
    _one_sweep_each(dp, p, 11)


def test_target_covering_the_whole_box(dp):
    p = W.config0().replace(n=(5, 5, 5, 5), target_c=(1.05, 0.0, 0.975, 0.95), target_w=(1.0, 1.0, 1.0, 1.0))
    o = oracle.Oracle(p)
    assert o.target.all()
    with dp.Grid(p) as g:
        assert g.info["n_target"] == g.info["n_active"] == p.nodes
        g.set_value(W.smooth_value(p, 3))
        assert np.all(g.get_value() == 0.0)   # target nodes hold V = 0
        assert g.sweep(dp.DP_SWEEP_VI) == 0.0
        assert np.all(g.get_value() == 0.0)
        rc, st = g.policy_iterate(tol=1e-9, max_sweeps=5, n_eval=3, polish=0)
        assert st.converged and st.residual == 0.0
        assert np.all(g.get_value() == 0.0)


@pytest.mark.parametrize("prec", [W.FP64, W.FP32], ids=["fp64", "fp32"])
def test_box_without_target(dp, prec):
    # target outside the box: no node is on it, every node's value comes
    # from the blend or the penalty alone
    p = W.config0().replace(n=(9, 7, 9, 5), target_c=(5.0, 0.0, 1.0, 0.95), precision=prec)
    o = oracle.Oracle(p)
    assert not o.target.any()
    _one_sweep_each(dp, p, 21)


def test_energy_band_without_nodes_is_refused(dp):
    # a band below every node's specific energy: no stored node
    p = W.config2(n=21).replace(energy_lo=-9.0, energy_hi=-8.0)
    with pytest.raises(dp.DPError) as e:
        dp.Grid(p)
    assert e.value.code == dp.DP_EINVAL
