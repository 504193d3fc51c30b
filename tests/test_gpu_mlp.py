"""Warm-start network on the GPU (tcgen05 BF16 GEMMs) vs the references.

The reference for element-wise checks is the FP64 network with BF16 rounding
where the tensor-core path rounds (oracle.mlp.forward_bf16 / backward_bf16:
hidden activations, the weights of the two 256 x 256 layers, the
back-propagated pre-activation gradients).  What remains between the two is
FP32 accumulation over 256 terms (~1e-6 of the terms' magnitude) and isolated
one-unit BF16 rounding flips where the FP32 and FP64 pre-activations straddle
a rounding boundary (each moves the next layer by about |w| 2^-8 |h| ~ 1e-4).
Bounds: outputs element by element within 2e-3 of their scale; gradients
within 1e-2 in relative L2 norm per tensor.  Each test also checks that a
planted mistake in the reference (a layer's bias dropped, a GELU or GELU'
skipped) lies far outside its bound.  Against the unrounded FP64 network the
BF16 rounding itself is a few per cent.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2407_14675_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_Y = 2e-3        # outputs, element-wise, relative to the output scale
TOL_G = 1e-2        # gradients, relative L2 per tensor


def _states(p, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = np.array(p.lo), np.array(p.hi)
    return lo + (hi - lo) * rng.uniform(size=(n, 4))


def _planted_forward(params, Xn, what):
    """The BF16 reference with one mistake planted (CPU only)."""
    pr = [[Wt.copy(), bv.copy()] for Wt, bv in params]
    if what == "bias2":
        pr[1][1][:] = 0.0
        return mlp.forward_bf16(pr, Xn)[0]
    if what == "gelu3":
        a = np.asarray(Xn, np.float32).astype(np.float64)
        for li, (Wt, bv) in enumerate(pr):
            Wt = np.asarray(Wt, np.float32).astype(np.float64)
            if 0 < li < 3:
                Wt = mlp.bf16(Wt)
            z = a @ Wt.T + np.asarray(bv, np.float32)
            a = z if li in (2, 3) else mlp.bf16(mlp.gelu(z))
            if li == 2:
                a = mlp.bf16(a)
        return a
    raise KeyError(what)


def _check_forward(Y, params, X, p):
    Xn = mlp.normalise_states(X, p.lo, p.hi)
    Yref = mlp.forward_bf16(params, Xn)[0]
    scale = np.abs(Yref).max()
    err = np.abs(Y - Yref)
    assert err.max() <= TOL_Y * scale, (err.max(), scale)
    for what in ("bias2", "gelu3"):
        assert np.abs(Y - _planted_forward(params, Xn, what)).max() > 10 * TOL_Y * scale, what
    # the BF16 operands move the outputs by ~1e-2 of scale from the FP64 network
    Y64 = mlp.forward(params, Xn)[0]
    assert np.abs(Y - Y64).max() <= 3e-2 * scale
    return err.max() / scale


def test_forward_matches_bf16_reference_element_wise(dp):
    p = W.config1()
    params = W.mlp_init_params(seed=3)
    X = _states(p, 1000, 4)                  # not a multiple of the 128-row tile
    flat = dp.flatten_params(params)
    with dp.Mlp(p.lo, p.hi, batch_capacity=4096) as net:
        dp.dp_mlp_set_params(net.h, flat)
        assert (dp.dp_mlp_get_params(net.h) == flat).all()
        Y = dp.dp_mlp_forward(net.h, X)
    _check_forward(Y, dp.unflatten_params(flat), X, p)


def test_large_batch_forward_equals_small_batches(dp):
    # 40,000 rows in one call take the persistent large-batch GEMM; 4,096-row
    # calls the per-tile one.  Same staging layout, MMA order and epilogue:
    # the outputs are bit-identical, and element-wise within the bound of the
    # BF16 reference
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
    _check_forward(Yb[:4000], dp.unflatten_params(flat), X[:4000], p)


@pytest.mark.parametrize("n", [1024, 16384])
def test_gradients_match_bf16_reference(dp, n):
    # 16,384 rows: the hidden layers' GEMMs run the persistent, pipelined
    # kernel of large batches (forward with the saved pre-activations, and
    # the GELU' backward), 1,024 rows the one-tile-per-CTA kernel
    p = W.config1()
    params = W.mlp_init_params(seed=5)
    X = _states(p, n, 6)
    rng = np.random.default_rng(7)
    T = rng.uniform(-1, 1, size=(n, 3))
    flat = dp.flatten_params(params)
    with dp.Mlp(p.lo, p.hi, batch_capacity=max(4096, n)) as net:
        dp.dp_mlp_set_params(net.h, flat)
        g, loss = dp.dp_mlp_gradients(net.h, X, T)
    pr = dp.unflatten_params(flat)
    Xn = mlp.normalise_states(X, p.lo, p.hi)
    T32 = T.astype(np.float32).astype(np.float64)
    Yb, cache = mlp.forward_bf16(pr, Xn)
    gref = mlp.backward_bf16(pr, cache, Yb, T32)
    assert loss == pytest.approx(mlp.loss(Yb, T32), rel=1e-3)
    got = dp.unflatten_params(g)
    # planted: GELU' of layer 2 skipped (the first layer's gradients change)
    n_out = Yb.size
    d = 2.0 * (Yb - T32) / n_out
    wrong = None
    for li in range(3, -1, -1):
        a_in, z = cache[li]
        if li < 3:
            d = mlp.bf16(d * (mlp.gelu_grad(z) if li != 1 else 1.0))
        Wt = np.asarray(pr[li][0], np.float32).astype(np.float64)
        if 0 < li < 3:
            Wt = mlp.bf16(Wt)
        if li == 1:
            wrong = [d.T @ a_in, d.sum(axis=0)]
        d = d @ Wt
    for li in range(4):
        for pi in range(2):
            a, b = got[li][pi], gref[li][pi]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel < TOL_G, (li, pi, rel)
    for pi in range(2):
        assert np.linalg.norm(wrong[pi] - gref[1][pi]) / np.linalg.norm(gref[1][pi]) > 10 * TOL_G
    # weight gradients element by element: dW = dz^T a summed in FP32 over BF16
    # operands, so each entry is within 2^-6 sum_s |dz_si| |a_sj| of the
    # reference (a BF16 rounding flip of either operand is 2^-8 of its term);
    # a transposed or misplaced operand lies orders of magnitude outside
    d = 2.0 * (Yb - T32) / n_out
    for li in range(3, -1, -1):
        a_in, z = cache[li]
        if li < 3:
            d = mlp.bf16(d * mlp.gelu_grad(z))
        E = np.abs(d).T @ np.abs(a_in)
        ratio = np.abs(got[li][0] - gref[li][0]) / (E + 1e-30)
        assert ratio.max() <= 2.0 ** -6, (li, float(ratio.max()))
        if li in (1, 2):
            # planted: the 256 x 256 gradient transposed fails the same bound
            assert (np.abs(got[li][0].T - gref[li][0]) / (E + 1e-30)).max() > 1.0
        Wt = np.asarray(pr[li][0], np.float32).astype(np.float64)
        if 0 < li < 3:
            Wt = mlp.bf16(Wt)
        d = d @ Wt


def test_adam_matches_fp64_reference_from_the_same_gradients(dp):
    # three Adam steps from the same gradients on the GPU (FP32 master weights,
    # moments and hyperparameters) and in FP64 (oracle.mlp.adam_step): every
    # parameter within 4 FP32 units of itself plus 3e-5 of the steps taken.
    # The second term is the FP32 rounding of beta1 = 0.9 and beta2 = 0.999
    # (2.4e-8 and 1.3e-8) and of the bias corrections 1 - beta^t (powf, one
    # unit): relative to 1 - beta2^t ~ t 1e-3 these are up to ~3e-5 of the
    # step size in the first steps
    p = W.config1()
    params = W.mlp_init_params(seed=8)
    flat = dp.flatten_params(params)
    rng = np.random.default_rng(9)
    grads = []
    for k in range(3):
        g = (rng.normal(size=flat.size) * 10.0 ** rng.uniform(-6, 0, flat.size)).astype(np.float32)
        g[k::7] = 0.0
        grads.append(g)
    ref = dp.unflatten_params(flat.astype(np.float64))
    state = {}
    lr_sum = 0.0
    with dp.Mlp(p.lo, p.hi, batch_capacity=4096) as net:
        dp.dp_mlp_set_params(net.h, flat)
        for k, g in enumerate(grads):
            lr = 1e-3 * (k + 1)
            lr_sum += lr
            dp.dp_mlp_apply_gradients(net.h, g, lr=lr)
            mlp.adam_step(ref, dp.unflatten_params(g.astype(np.float64)), state, lr=lr)
            got = dp.dp_mlp_get_params(net.h).astype(np.float64)
            want = np.concatenate([a.reshape(-1) for layer in ref for a in layer])
            ulp = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
            err = np.abs(got - want)
            bound = 4 * ulp + 3e-5 * lr_sum
            assert (err <= bound).all(), (k, float((err / bound).max()))
            # the step itself is lr-sized where the gradient is non-zero
            assert np.abs(got - flat).max() > 0.5e-3


def test_bounded_wait_gives_up_cleanly_and_the_next_call_runs(dp):
    # test hook: the tensor-core GEMMs give up their first wait at once; the
    # call reports DP_ETIMEOUT (each GEMM still drained its committed MMAs and
    # freed its TMEM), and after the default limit is restored the same call
    # gives the normal result, for the per-tile and the persistent GEMM
    p = W.config1()
    params = W.mlp_init_params(seed=10)
    flat = dp.flatten_params(params)
    for n, cap in ((1000, 4096), (40000, 65536)):
        X = _states(p, n, 11)
        with dp.Mlp(p.lo, p.hi, batch_capacity=cap) as net:
            dp.dp_mlp_set_params(net.h, flat)
            Y0 = dp.dp_mlp_forward(net.h, X)
            dp.dp_mlp_set_wait_limit(net.h, 0)
            with pytest.raises(dp.DPError) as e:
                dp.dp_mlp_forward(net.h, X)
            assert e.value.code == dp.DP_ETIMEOUT
            dp.dp_mlp_set_wait_limit(net.h, -1)
            Y1 = dp.dp_mlp_forward(net.h, X)
        np.testing.assert_array_equal(Y0, Y1)


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
    # what the trained network gains over the method without it: the solve
    # started from its V and policy needs fewer improvement sweeps (and fewer
    # sweeps in all) than the cold start
    imp_cold = st_cold.sweeps_improve + st_cold.sweeps_improve_fp64
    imp_warm = st_warm.sweeps_improve + st_warm.sweeps_improve_fp64
    all_cold = imp_cold + st_cold.sweeps_eval + st_cold.sweeps_eval_fp64
    all_warm = imp_warm + st_warm.sweeps_eval + st_warm.sweeps_eval_fp64
    print("fit %.3g, improvements cold %d warm %d, sweeps cold %d warm %d" % (
        fit, imp_cold, imp_warm, all_cold, all_warm))
    assert imp_warm < imp_cold and all_warm < all_cold


def test_training_and_gradients_are_reproducible(dp):
    # every gradient sum is reduced through per-block partial sums in a fixed
    # order (no float atomics): the same gradients twice, and two trainings
    # from the same parameters on the same grid end with bit-identical
    # parameters and losses
    p = W.config1(n=13)
    X = _states(p, 16384, 8)
    T = np.random.default_rng(9).uniform(-1, 1, size=(16384, 3))
    with dp.Mlp(p.lo, p.hi, batch_capacity=16384) as net:
        dp.dp_mlp_set_params(net.h, dp.flatten_params(W.mlp_init_params(seed=3)))
        g1, l1 = dp.dp_mlp_gradients(net.h, X, T)
        g2, l2 = dp.dp_mlp_gradients(net.h, X, T)
    assert np.array_equal(g1, g2) and l1 == l2
    with dp.Grid(p) as g:
        g.policy_iterate(tol=1e-5, max_sweeps=2000, n_eval=20, polish=0)
        outs = []
        for _ in range(2):
            with dp.Mlp(p.lo, p.hi, batch_capacity=16384) as net:
                dp.dp_mlp_set_params(net.h, dp.flatten_params(W.mlp_init_params()))
                st = dp.dp_mlp_train_grid(net.h, g.h, epochs=2, batch=4096, lr=1e-3)
                outs.append((dp.dp_mlp_get_params(net.h), st.last_epoch_loss))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_gradients_of_a_large_batch_are_the_mean_of_its_slices(dp):
    # 131,072 rows: the feature reductions take 512 rows per block in
    # 256-row slices and the weight gradients 32 splits of 4,096 rows; the
    # gradient of the mean squared error is the mean of the eight 16,384-row
    # slices' gradients up to FP32 rounding
    p = W.config1()
    n, k = 131072, 8
    X = _states(p, n, 12)
    T = np.random.default_rng(13).uniform(-1, 1, size=(n, 3))
    with dp.Mlp(p.lo, p.hi, batch_capacity=n) as net:
        dp.dp_mlp_set_params(net.h, dp.flatten_params(W.mlp_init_params(seed=4)))
        g_all, l_all = dp.dp_mlp_gradients(net.h, X, T)
        m = n // k
        parts = [dp.dp_mlp_gradients(net.h, X[i * m:(i + 1) * m], T[i * m:(i + 1) * m]) for i in range(k)]
    g_mean = np.mean([g for g, _ in parts], axis=0)
    l_mean = np.mean([l for _, l in parts])
    assert np.linalg.norm(g_all - g_mean) <= 1e-5 * np.linalg.norm(g_mean)
    assert abs(l_all - l_mean) <= 1e-5 * l_mean
