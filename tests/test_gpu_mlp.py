"""Warm-start network on the GPU (tcgen05 BF16 GEMMs) vs the FP64 reference.

Tolerances come from BF16 operands (8-bit mantissa) with FP32 accumulation:
outputs within 3 % of their scale, gradients within 5 % in relative L2 norm
per parameter tensor, the loss within 2 %.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2407_14675_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _states(p, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = np.array(p.lo), np.array(p.hi)
    return lo + (hi - lo) * rng.uniform(size=(n, 4))


def test_forward_matches_fp64_reference(dp):
    p = W.config1()
    params = W.mlp_init_params(seed=3)
    X = _states(p, 1000, 4)                  # not a multiple of the 128-row tile
    flat = dp.flatten_params(params)
    with dp.Mlp(p.lo, p.hi, batch_capacity=4096) as net:
        dp.dp_mlp_set_params(net.h, flat)
        assert (dp.dp_mlp_get_params(net.h) == flat).all()
        Y = dp.dp_mlp_forward(net.h, X)
    Yref = mlp.forward(params, mlp.normalise_states(X, p.lo, p.hi))[0]
    scale = np.abs(Yref).max()
    assert np.abs(Y - Yref).max() <= 3e-2 * scale + 1e-3


def test_large_batch_forward_equals_small_batches(dp):
    # 40,000 rows in one call take the persistent large-batch GEMM; 4,096-row
    # calls the per-tile one.  Same staging layout, MMA order and epilogue:
    # the outputs are bit-identical, and within the BF16 tolerance of the
    # FP64 reference
    p = W.config1()
    params = W.mlp_init_params(seed=5)
    X = _states(p, 40000, 6)
    flat = dp.flatten_params(params)
    with dp.Mlp(p.lo, p.hi, batch_capacity=65536) as big, dp.Mlp(p.lo, p.hi, batch_capacity=4096) as small:
        dp.dp_mlp_set_params(big.h, flat)
        dp.dp_mlp_set_params(small.h, flat)
        Yb = dp.dp_mlp_forward(big.h, X)
        Yb2 = dp.dp_mlp_forward(big.h, X)
        Ys = dp.dp_mlp_forward(small.h, X)
    np.testing.assert_array_equal(Yb, Ys)
    np.testing.assert_array_equal(Yb, Yb2)
    Yref = mlp.forward(params, mlp.normalise_states(X[:2000], p.lo, p.hi))[0]
    assert np.abs(Yb[:2000] - Yref).max() <= 3e-2 * np.abs(Yref).max() + 1e-3


def test_gradients_match_fp64_reference(dp):
    p = W.config1()
    params = W.mlp_init_params(seed=5)
    X = _states(p, 1024, 6)
    rng = np.random.default_rng(7)
    T = rng.uniform(-1, 1, size=(1024, 3))
    with dp.Mlp(p.lo, p.hi, batch_capacity=4096) as net:
        dp.dp_mlp_set_params(net.h, dp.flatten_params(params))
        g, loss = dp.dp_mlp_gradients(net.h, X, T)
    Yref, cache = mlp.forward(params, mlp.normalise_states(X, p.lo, p.hi))
    gref = mlp.backward(params, cache, Yref, T)
    assert loss == pytest.approx(mlp.loss(Yref, T), rel=2e-2)
    got = dp.unflatten_params(g)
    for li in range(4):
        for pi in range(2):
            a, b = got[li][pi], gref[li][pi]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel < 5e-2, (li, pi, rel)


def test_training_fits_a_solved_grid_and_warm_starts_policy_iteration(dp):
    # Solve a 21^4 grid with the config-1 physics, train on its nodes, then
    # start policy iteration on a fresh grid from the network's V and policy:
    # it must reach the same fixed point (FP32 tolerance) as the cold solve.
    p = W.config1(n=21)
    with dp.Grid(p) as cold:
        rc, st_cold = cold.policy_iterate(tol=1e-6, max_sweeps=4000, n_eval=20, polish=1)
        assert st_cold.converged
        V_cold = cold.get_value()
        M = cold.info["penalty_M"]
        with dp.Mlp(p.lo, p.hi, batch_capacity=4096) as net:
            dp.dp_mlp_set_params(net.h, dp.flatten_params(W.mlp_init_params(seed=11)))
            st = dp.dp_mlp_train_grid(net.h, cold.h, epochs=8, batch=4096, lr=1e-3)
            assert st.last_epoch_loss < st.first_epoch_loss / 3, st.asdict()
            with dp.Grid(p) as warm:
                dp.dp_warm_start(net.h, warm.h)
                V0 = warm.get_value()
                C0 = warm.get_policy()
                fit = np.abs(V0 - V_cold).max() / M
                rc, st_warm = warm.policy_iterate(tol=1e-6, max_sweeps=4000, n_eval=20, polish=1, warm=1)
                assert st_warm.converged
                V_warm = warm.get_value()
            # the cold grid holds FP64 values after its polished solve: a warm
            # start into it writes the same FP32 values as into a fresh grid
            assert st_cold.switch_outer >= 0
            dp.dp_warm_start(net.h, cold.h)
            assert cold.info["n_active"] == len(V0)
            np.testing.assert_array_equal(cold.get_value(), V0)
            np.testing.assert_array_equal(cold.get_policy(), C0)
    assert np.isfinite(V0).all() and V0.min() >= 0 and V0.max() <= float(np.float32(M))   # FP32 storage
    assert np.abs(V_warm - V_cold).max() <= 1e-4 * M
    print("fit %.3g, improvements cold %d warm %d" % (
        fit, st_cold.sweeps_improve + st_cold.sweeps_improve_fp64,
        st_warm.sweeps_improve + st_warm.sweeps_improve_fp64))
