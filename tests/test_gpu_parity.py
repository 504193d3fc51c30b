"""CUDA path vs the FP64 oracle, through the C ABI, on the same seeded inputs.

Tolerances (element by element, over the stored nodes):
  FP64 grids  max|dV| <= 1e-9 max|V|
  FP32 grids  max|dV| <= 1e-4 max|V|
Decisions (policy codes) must agree, or be ties: the oracle's own q at the
GPU's code is within tol_tie of its q at its code (1e-12 M in FP64, 1e-5 M in
FP32), and >= 99.9 % of nodes must agree exactly unless stated otherwise.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 1e-4


def _full(grid, o, v_compact, fill=None):
    """Scatter compact values into a full-box array (inactive nodes: M)."""
    V = np.full(o.N, o.M if fill is None else fill)
    V[grid.active_index()] = v_compact
    return V


def _check_values(v_gpu, v_or, tol, what="", o=None, nodes=None, codes=None, max_face=0.005):
    """max|dV| <= tol max|V|.  With (o, nodes, codes) given (evaluation at a
    frozen policy), nodes whose foot lies within 1e-4 cells of a cell face may
    differ by the penalty jump: FP32 geometry puts such a foot on the other
    side of the face.  They are counted and bounded, and excluded."""
    scale = np.abs(v_or).max()
    bad = np.abs(v_gpu - v_or) > tol * scale
    if bad.any() and o is not None:
        for k in np.flatnonzero(bad):
            s = o.foot_node(np.unravel_index(nodes[k], o.p.n), oracle.code_angle(codes[k]))
            if np.abs(s - np.round(s)).min() < 1e-4:
                bad[k] = False
        assert (np.abs(v_gpu - v_or) > tol * scale).mean() <= max_face
    err = np.abs(v_gpu - v_or)[~bad].max() if (~bad).any() else 0.0
    assert not bad.any(), "%s max|dV| = %.3g > %.1g * %.3g at %d nodes" % (
        what, np.abs(v_gpu - v_or).max(), tol, scale, bad.sum())
    return err


def _check_codes(o, V_full, nodes, c_gpu, c_or, tie, min_agree=0.999, max_face=0.005):
    """Decisions agree when the codes are equal or the oracle's q at the GPU's
    code is within `tie` of its q at its own code.  A larger gap is accepted
    only where the GPU's foot lies within 1e-4 cells of a cell face: q jumps to
    the penalty M there, and FP32 geometry moves that jump by ~1e-6 cells (a
    few lattice codes).  Such face decisions are counted and bounded."""
    agree = c_gpu == c_or
    face = np.zeros(len(nodes), bool)
    diff = np.flatnonzero(~agree)
    if len(diff):
        q_g = o.q_nodes(V_full, nodes[diff], c_gpu[diff])
        q_o = o.q_nodes(V_full, nodes[diff], c_or[diff])
        gap = np.abs(q_g - q_o)
        agree[diff[gap <= tie]] = True
        for k in diff[gap > tie]:
            s = o.foot_node(np.unravel_index(nodes[k], o.p.n), oracle.code_angle(c_gpu[k]))
            dist = np.abs(s - np.round(s)).min()
            assert dist < 1e-4, "non-tie decision at node %d: gap %.3g, foot %s" % (
                nodes[k], gap[list(diff).index(k)], s)
            face[k] = True
    assert face.mean() <= max_face, "face decisions at %.4f of nodes" % face.mean()
    assert (agree | face).mean() >= min_agree
    return agree.mean(), face.mean()


def _lockstep(dp, g, o, schedule, tol, tie):
    """Run the sweeps of `schedule` on the GPU one at a time; before each, the
    oracle applies the same operator to the GPU's current value and policy.
    Values and decisions are compared after every sweep (ties on plateaus make
    two valid runs drift apart, so the comparison is per operator)."""
    idx = g.active_index()
    for mode in schedule:
        V = np.full(o.N, o.M)
        V[idx] = g.get_value()
        codes = np.zeros(o.N, np.uint16)
        codes[idx] = g.get_policy()
        r_gpu = g.sweep(mode)
        v_g = g.get_value()
        v_o, c_o, r_o, _ = o.sweep(V, mode={dp.DP_SWEEP_VI: oracle.VI, dp.DP_SWEEP_IMPROVE_FULL: oracle.IMPROVE_FULL,
                                            dp.DP_SWEEP_IMPROVE_WALK: oracle.IMPROVE_WALK,
                                            dp.DP_SWEEP_EVAL: oracle.EVAL}[mode], codes=codes)
        if mode == dp.DP_SWEEP_EVAL and tol > TOL64:
            _check_values(v_g, v_o[idx], tol, "mode %d" % mode, o=o, nodes=idx, codes=codes[idx])
        else:
            _check_values(v_g, v_o[idx], tol, "mode %d" % mode)
        if mode in (dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_IMPROVE_WALK):
            free = np.flatnonzero(~o.target[idx].astype(bool))
            _check_codes(o, V, idx[free], g.get_policy()[free], c_o[idx][free], tie)


# ------------------------------------------------------------ grid set-up --

def test_grid_info_matches_oracle(dp):
    for p in (W.config0(), W.config2(n=41)):
        o = oracle.Oracle(p)
        with dp.Grid(p) as g:
            assert g.info["n_box"] == p.nodes
            assert g.info["n_active"] == o.n_active
            assert g.info["n_target"] == int(o.target.sum())
            assert (g.active_index() == np.flatnonzero(o.active)).all()
            assert g.info["penalty_M"] == pytest.approx(o.M, rel=1e-15)


def test_set_get_roundtrip_and_target_zero(dp):
    p = W.config0()
    o = oracle.Oracle(p)
    V = W.random_value(p, 1)
    with dp.Grid(p) as g:
        g.set_value(V)
        back = g.get_value()
    t = o.target.astype(bool)
    assert (back[t] == 0).all()
    assert (back[~t] == V[~t]).all()


@pytest.mark.parametrize("prec", [W.FP32, W.FP64], ids=["fp32", "fp64"])
def test_fp32_value_transfers(dp, prec):
    # dp_set_value_f32 / dp_get_value_f32: the stored FP32 values exactly on
    # FP32 grids, widened / rounded on FP64 grids; targets forced to 0,
    # non-finite input refused with the resident V unchanged
    p = W.config2(n=21).replace(precision=prec)
    with dp.Grid(p) as g:
        idx = g.active_index()
        o = oracle.Oracle(p)
        t = o.target.astype(bool)[idx]
        V = W.random_value(p, 2)[idx].astype(np.float32)
        dp.dp_set_value_f32(g.h, V)
        back64 = g.get_value()
        back32 = dp.dp_get_value_f32(g.h, g.n)
        assert (back64[t] == 0).all() and (back32[t] == 0).all()
        assert np.array_equal(back64[~t], V[~t].astype(np.float64))
        assert np.array_equal(back32[~t], V[~t])
        # the FP64 call and the FP32 call agree on what the grid holds
        g.set_value(W.random_value(p, 3)[idx])
        assert np.array_equal(dp.dp_get_value_f32(g.h, g.n), g.get_value().astype(np.float32))
        before = g.get_value()
        bad = V.copy()
        bad[len(bad) // 2] = np.nan
        with pytest.raises(dp.DPError) as e:
            dp.dp_set_value_f32(g.h, bad)
        assert e.value.code == dp.DP_ENONFINITE
        assert np.array_equal(g.get_value(), before)
        with pytest.raises(TypeError):
            dp.dp_set_value_f32(g.h, V.astype(np.float64))


def test_fp32_value_transfer_after_the_fp64_phase(dp):
    # after a polish the values are FP64: dp_get_value_f32 rounds them
    p = W.config1(n=17)
    with dp.Grid(p) as g:
        g.policy_iterate(tol=1e-6, max_sweeps=400, n_eval=20, polish=1, switch_tol=100.0)
        assert dp.dp_grid_get_info(g.h)["fp64_values"]
        assert np.array_equal(dp.dp_get_value_f32(g.h, g.n), g.get_value().astype(np.float32))


# -------------------------------------------------- closed-form dynamics --

@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_1d_closed_form(dp, precision):
    p = W.unit_speed_1d(beta=0.9).replace(precision=precision)
    n = np.abs(np.arange(p.n[0]) - 8)
    exact = p.dt * (1 - p.beta ** n) / (1 - p.beta)
    with dp.Grid(p) as g:
        rc, st = g.value_iterate(tol=1e-13 if precision == W.FP64 else 0.0, max_sweeps=40)
        V = g.get_value().reshape(p.n)
    tol = 1e-14 if precision == W.FP64 else 4e-7
    for k in range(2):
        assert np.abs(V[:, k, k, k] - exact).max() < tol


def test_2d_manhattan(dp):
    p = W.unit_speed_2d()
    with dp.Grid(p) as g:
        rc, st = g.value_iterate(tol=1e-13, max_sweeps=200)
        assert rc == dp.DP_OK and st.converged
        V = g.get_value().reshape(p.n)
    i, j = np.meshgrid(np.arange(p.n[0]), np.arange(p.n[1]), indexing="ij")
    d = np.abs(i - 6) + np.abs(j - 4)
    exact = p.dt * (1 - p.beta ** d) / (1 - p.beta)
    assert np.abs(V[:, :, 0, 0] - exact).max() < 1e-14


# --------------------------------------------------------- FP64 (config 0) --

def test_vi_sweep_parity_fp64_config0(dp):
    p = W.config0()
    o = oracle.Oracle(p)
    V = W.smooth_value(p, 21)
    with dp.Grid(p) as g:
        g.set_value(V)
        r_gpu = g.sweep(dp.DP_SWEEP_VI)
        v_gpu = g.get_value()
    V[o.target.astype(bool)] = 0
    W1, _, r_or, _ = o.sweep(V)
    _check_values(v_gpu, W1, TOL64, "VI sweep")
    assert r_gpu == pytest.approx(r_or, rel=1e-12)


def test_vi_many_sweeps_parity_fp64_config0(dp):
    p = W.config0()
    o = oracle.Oracle(p)
    n = 25
    with dp.Grid(p) as g:
        rc, st = g.value_iterate(tol=0.0, max_sweeps=n)
        assert rc == dp.DP_ENOCONV and st.sweeps_vi == n
        v_gpu = g.get_value()
    V = np.zeros(p.nodes)
    for _ in range(n):
        V, _, r, _ = o.sweep(V)
    _check_values(v_gpu, V, TOL64, "VI x%d" % n)
    assert st.residual == pytest.approx(r, rel=1e-9)


def test_vi_converges_and_stops_at_tolerance(dp):
    # 9^4 FP64 with the config-0 physics, VI to 1e-8: the reported sweep count
    # is the first sweep whose residual is below tol, and the value there
    # matches the oracle after the same number of sweeps.
    p = W.config0().replace(n=(7, 7, 7, 7), beta=0.99)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        rc, st = g.value_iterate(tol=1e-8, max_sweeps=100000)
        assert rc == dp.DP_OK and st.converged and st.residual < 1e-8
        v_gpu = g.get_value()
    V, s, r = o.value_iterate(tol=1e-8)
    assert st.sweeps_vi == s
    _check_values(v_gpu, V, TOL64, "VI converged")


def test_policy_iteration_parity_fp64(dp):
    p = W.config0().replace(n=(9, 9, 9, 9), refine=1, n_angles=16)
    o = oracle.Oracle(p)
    sched = [dp.DP_SWEEP_IMPROVE_FULL] + [dp.DP_SWEEP_EVAL] * 4 + [dp.DP_SWEEP_IMPROVE_WALK] + \
        [dp.DP_SWEEP_EVAL] * 4 + [dp.DP_SWEEP_IMPROVE_WALK]
    with dp.Grid(p) as g:
        _lockstep(dp, g, o, sched, TOL64, tie=1e-12 * o.M)


def test_policy_iteration_driver_fp64(dp):
    # the driver's sweep schedule (improvement + n_eval evaluations) gives the
    # same values as the same schedule issued one sweep at a time
    p = W.config0().replace(n=(9, 9, 9, 9), refine=1, n_angles=16)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=0.0, max_sweeps=3, n_eval=4, polish=0)
        assert (st.sweeps_improve, st.sweeps_eval) == (3, 12)
        v1, c1 = g.get_value(), g.get_policy()
    with dp.Grid(p) as g:
        for k in range(3):
            g.sweep(dp.DP_SWEEP_IMPROVE_FULL if k == 0 else dp.DP_SWEEP_IMPROVE_WALK)
            for e in range(4):
                g.sweep(dp.DP_SWEEP_EVAL)
        v2, c2 = g.get_value(), g.get_policy()
    assert (v1 == v2).all() and (c1 == c2).all()


# ------------------------------------------------ FP32 (config-1 physics) --

@pytest.fixture(scope="module")
def small1():
    p = W.config1(n=17)
    return p, oracle.Oracle(p)


def test_improve_full_parity_fp32(dp, small1):
    p, o = small1
    V = W.smooth_value(p, 31)
    with dp.Grid(p) as g:
        g.set_value(V)
        g.sweep(dp.DP_SWEEP_IMPROVE_FULL)
        v_gpu, c_gpu = g.get_value(), g.get_policy()
    V32 = V.astype(np.float32).astype(np.float64)
    V32[o.target.astype(bool)] = 0
    W1, c_or, _, _ = o.sweep(V32, mode=oracle.IMPROVE_FULL)
    _check_values(v_gpu, W1, TOL32, "improve fp32")
    nodes = np.flatnonzero(~o.target.astype(bool))
    _check_codes(o, V32, nodes, c_gpu[nodes], c_or[nodes], tie=1e-5 * o.M)


def test_eval_parity_fp32(dp, small1):
    p, o = small1
    V = W.smooth_value(p, 32)
    codes = W.random_codes(p, 33)
    with dp.Grid(p) as g:
        g.set_value(V)
        g.set_policy(codes)
        g.sweep(dp.DP_SWEEP_EVAL)
        v_gpu = g.get_value()
    V32 = V.astype(np.float32).astype(np.float64)
    V32[o.target.astype(bool)] = 0
    W1 = o.sweep(V32, mode=oracle.EVAL, codes=codes)[0]
    _check_values(v_gpu, W1, TOL32, "eval fp32", o=o, nodes=np.arange(o.N), codes=codes)


def test_walk_parity_fp32(dp, small1):
    p, o = small1
    V = W.smooth_value(p, 34)
    start = W.random_codes(p, 35)
    with dp.Grid(p) as g:
        g.set_value(V)
        g.set_policy(start)
        g.sweep(dp.DP_SWEEP_IMPROVE_WALK)
        v_gpu, c_gpu = g.get_value(), g.get_policy()
    V32 = V.astype(np.float32).astype(np.float64)
    V32[o.target.astype(bool)] = 0
    W1, c_or, _, _ = o.sweep(V32, mode=oracle.IMPROVE_WALK, codes=start)
    _check_values(v_gpu, W1, TOL32, "walk fp32")
    nodes = np.flatnonzero(~o.target.astype(bool))
    _check_codes(o, V32, nodes, c_gpu[nodes], c_or[nodes], tie=1e-5 * o.M)


def test_policy_iteration_parity_fp32(dp, small1):
    p, o = small1
    sched = ([dp.DP_SWEEP_IMPROVE_FULL] + [dp.DP_SWEEP_EVAL] * 3 + [dp.DP_SWEEP_IMPROVE_WALK] +
             [dp.DP_SWEEP_EVAL] * 3 + [dp.DP_SWEEP_IMPROVE_WALK])
    with dp.Grid(p) as g:
        _lockstep(dp, g, o, sched, TOL32, tie=1e-5 * o.M)


def _sampled_pi_parity(dp, p, seed, n_sample=1500):
    """The operators of the benchmark step in its launch configuration on a
    full-size grid: a full-tabulation improvement, an evaluation sweep at the
    frozen feet and a walk + golden improvement, each checked at sampled
    stored nodes that the oracle computes one by one from the GPU's input."""
    o = oracle.Oracle(p)
    V = W.smooth_value(p, seed)
    V[o.target.astype(bool)] = 0
    rng = np.random.default_rng(seed + 1)
    nodes = np.sort(rng.choice(np.flatnonzero((o.active & ~o.target).astype(bool)), n_sample, replace=False))
    with dp.Grid(p) as g:
        idx = g.active_index()
        pos = np.searchsorted(idx, nodes)            # compact position of each sampled node
        g.set_value(V[idx])
        v0 = g.get_value()
        g.sweep(dp.DP_SWEEP_IMPROVE_FULL)
        v1, c1 = g.get_value(), g.get_policy()
        g.sweep(dp.DP_SWEEP_EVAL)
        v2 = g.get_value()
        g.sweep(dp.DP_SWEEP_IMPROVE_WALK)
        v3, c3 = g.get_value(), g.get_policy()
    Vg = np.full(o.N, o.M)
    Vg[idx] = v0                                     # the FP32-rounded start
    ov1, oc1 = o.bellman_nodes(Vg, nodes, mode=oracle.IMPROVE_FULL)
    _check_values(v1[pos], ov1, TOL32, "improve")
    _check_codes(o, Vg, nodes, c1[pos], oc1, tie=1e-5 * o.M)
    Vg[idx] = v1
    ov2, _ = o.bellman_nodes(Vg, nodes, mode=oracle.EVAL, codes=c1[pos])
    _check_values(v2[pos], ov2, TOL32, "eval", o=o, nodes=nodes, codes=c1[pos])
    Vg[idx] = v2
    ov3, oc3 = o.bellman_nodes(Vg, nodes, mode=oracle.IMPROVE_WALK, codes=c1[pos])
    _check_values(v3[pos], ov3, TOL32, "walk")
    _check_codes(o, Vg, nodes, c3[pos], oc3, tie=1e-5 * o.M)


def test_full_size_config1_sampled_parity(dp):
    # 61^4 (13.8M nodes) in the launch configuration of the benchmark
    _sampled_pi_parity(dp, W.config1(), 41)


def test_full_size_band_sampled_parity(dp):
    # the benchmark's grid: 121^4 box reduced to the energy band (56M stored
    # nodes), the same operators in the benchmark's launch configuration
    _sampled_pi_parity(dp, W.config2(), 43)


# ------------------------------------------------------------ reduced grid --

def test_reduced_grid_parity(dp):
    p = W.config2(n=31)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        assert (g.active_index() == np.flatnonzero(o.active)).all()
        sched = [dp.DP_SWEEP_IMPROVE_FULL] + [dp.DP_SWEEP_EVAL] * 3 + [dp.DP_SWEEP_IMPROVE_WALK]
        _lockstep(dp, g, o, sched, TOL32, tie=1e-5 * o.M)


def test_reduced_grid_fp64_sweep_parity(dp):
    p = W.config2(n=25).replace(precision=W.FP64, refine=0, n_angles=16)
    o = oracle.Oracle(p)
    V = W.smooth_value(p, 51)
    with dp.Grid(p) as g:
        idx = g.active_index()
        g.set_value(V[idx])
        g.sweep(dp.DP_SWEEP_VI)
        v_gpu = g.get_value()
    V[o.target.astype(bool)] = 0
    W1 = o.sweep(V)[0]
    _check_values(v_gpu, W1[idx], TOL64, "reduced VI fp64")


# ----------------------------------------------------- feedback and loop --

def _check_feedback_codes(o, V, states, tau, c_gpu, c_or, tie, min_agree=0.999):
    """Feedback decisions agree when the codes are equal or the oracle's q of
    Eq. (15) at the GPU's code is within `tie` of its q at its own code."""
    agree = c_gpu == c_or
    for k in np.flatnonzero(~agree):
        q_g = o.q_state(V, states[k], float(oracle.code_angle(c_gpu[k])), tau)
        q_o = o.q_state(V, states[k], float(oracle.code_angle(c_or[k])), tau)
        agree[k] = abs(q_g - q_o) <= tie
    assert agree.mean() >= min_agree, "feedback decisions agree at %.4f" % agree.mean()
    return agree.mean()


@pytest.mark.parametrize("k_tau", [1, 2, 3])
def test_feedback_parity(dp, k_tau):
    # Eq. (15) with the feedback's own step tau = k dt at off-grid states
    p = W.config0().replace(n=(9, 9, 9, 9), refine=1, accel=0.02, dt=0.05)
    o = oracle.Oracle(p)
    V = W.smooth_value(p, 61)
    V[o.target.astype(bool)] = 0
    states = W.closed_loop_states(p, 256, seed=62)
    tau = k_tau * p.dt
    codes_or, q_or = o.feedback(V, states, tau=tau)
    with dp.Grid(p) as g:
        g.set_value(V)
        alpha, q = g.feedback(states, tau)
    assert np.abs(q - q_or).max() <= 1e-12 * o.M
    codes = np.round(alpha * 65536 / (2 * np.pi)).astype(np.int64) % 65536
    _check_feedback_codes(o, V, states, tau, codes, codes_or.astype(np.int64), tie=1e-12 * o.M)


@pytest.mark.parametrize("k_tau,h_div", [(1, 1), (2, 2), (3, 3), (1, 4)])
def test_closed_loop_1d_arrival(dp, k_tau, h_div):
    # feedback step tau = k dt, RK4 step h = dt / h_div: the closed form holds
    # for every pair (unit speed, h divides dt)
    p = W.unit_speed_1d()
    with dp.Grid(p) as g:
        g.value_iterate(tol=1e-13, max_sweeps=100)
        x0 = np.array([[1.0, 1.0, 1.0, 1.0], [2.0, 1.5, 1.0, 1.0], [1.0 + 3 * p.dt, 1.0, 1.0, 1.0]])
        ta, xf = g.simulate(x0, k_tau * p.dt, p.dt / h_div, 2.0)
    assert ta == pytest.approx([8 * p.dt, 8 * p.dt, 5 * p.dt], abs=1e-12)
    assert xf[:, 0] == pytest.approx([1.5, 1.5, 1.5], abs=1e-12)


def _edelbaum_time(r0, rT, a, c, m0=1.0):
    dv = abs(1 / math.sqrt(r0) - 1 / math.sqrt(rT))
    return (1 - math.exp(-dv / c)) * c * m0 / a


@pytest.fixture(scope="module")
def config0_solved(dp):
    p = W.config0()
    with dp.Grid(p) as g:
        rc, st = g.value_iterate(tol=1e-8, max_sweeps=100000)
        assert rc == dp.DP_OK and st.converged, st.asdict()
        return p, g.get_value()


@pytest.mark.parametrize("k_tau,h_div", [(1, 1), (2, 2), (2, 1)])
def test_config0_converged_closed_loop(dp, config0_solved, k_tau, h_div):
    # Config 0 to 1e-8 on the GPU, then the closed loop from circular orbits
    # at r = 1 (GPU, and the oracle on the GPU's value function) with
    # feedback step tau = k dt and RK4 step h = dt / h_div: each transfer time
    # agrees with the oracle's within 0.5 % of itself, and is no shorter than
    # the Edelbaum (impulse-free, circle-to-circle) bound.
    p, V = config0_solved
    o = oracle.Oracle(p)
    tau, h = k_tau * p.dt, p.dt / h_div
    x0 = np.array([W.transfer_start(1.0, m) for m in (1.0, 0.98, 0.96)] +
                  [[1.0, 0.01, 1.0, 1.0], [0.98, 0.0, 1.0 / math.sqrt(0.98), 0.99]])
    with dp.Grid(p) as g:
        g.set_value(V)
        ta, xf = g.simulate(x0, tau, h, 200.0)
    ta_or, xf_or = o.simulate(V, x0, tau=tau, h=h, t_max=200.0)
    assert (ta > 0).all() and (ta_or > 0).all()
    assert (np.abs(ta - ta_or) <= 0.005 * ta_or).all(), (ta, ta_or)
    tE = _edelbaum_time(1.0, 1.05, p.accel, p.exhaust_c)
    assert ta[0] >= 0.9 * tE and ta[0] <= 2.0 * tE


# ------------------------------------------------------------------ polish --

def _oracle_fixed_point(o, n_eval, tol=1e-9):
    """The oracle's fixed point of Eq. (12): policy iteration with the local
    walk (§3 "Efficient computation of the minimum"), then continued with full
    tabulation in every improvement until that also moves V by less than tol.
    The walk alone can stop in a local minimum of the tabulated angles; the
    GPU solver confirms a converged walk with a full tabulation in the same
    way."""
    V, codes, outer, ev, res = o.policy_iterate(tol=tol, max_outer=20000, n_eval=n_eval)
    V, codes, outer, ev, res = o.policy_iterate(V0=V, codes0=codes, tol=tol, max_outer=20000, n_eval=n_eval,
                                                walk=False)
    assert res < tol
    return V

def test_fp32_policy_iteration_with_fp64_polish_reaches_1e6(dp):
    # M = dt / (1 - beta) = 20: one FP32 ulp of V (1.9e-6) exceeds the
    # tolerance, so the solve must finish with FP64 values.
    p = W.config1(n=9).replace(beta=0.995, dt=0.1)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=5000, n_eval=20, polish=1)
        assert rc == dp.DP_OK and st.converged and st.residual < 1e-6, st.asdict()
        assert st.sweeps_improve_fp64 > 0
        info = dp.dp_grid_get_info(g.h)
        assert info["fp64_values"] == 1
        v_gpu = g.get_value()
    _check_values(v_gpu, _oracle_fixed_point(o, n_eval=20), TOL32, "converged FP32+polish")


def test_fp32_polish_solve_matches_converged_oracle_17x4(dp):
    # the same on the 17^4 grid (83,521 nodes; beta = 0.99 keeps the oracle's
    # converged solve under a minute): the FP32 + FP64-polish solve to 1e-6 is
    # within the FP32 tolerance of the oracle's fixed point (its distance to
    # the fixed point is at most 1e-6 beta / (1 - beta) ~ 1e-4, 1e-5 of M)
    p = W.config1(n=17).replace(beta=0.99, dt=0.1)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=5000, n_eval=100, polish=1)
        assert rc == dp.DP_OK and st.converged and st.residual < 1e-6, st.asdict()
        assert st.sweeps_improve_fp64 > 0
        v_gpu = g.get_value()
    _check_values(v_gpu, _oracle_fixed_point(o, n_eval=100), TOL32, "converged FP32+polish 17^4")


# ------------------------------------------------------------------ errors --

def test_errors(dp):
    p = W.config0().replace(n=(5, 5, 5, 5))
    with dp.Grid(p) as g:
        V = np.zeros(g.n)
        V[3] = np.nan
        with pytest.raises(dp.DPError) as e:
            g.set_value(V)
        assert e.value.code == dp.DP_ENONFINITE
        with pytest.raises(dp.DPError) as e:
            dp.dp_set_value(g.h, np.zeros(g.n - 1))
        assert e.value.code == dp.DP_EINVAL
        with pytest.raises(dp.DPError) as e:
            g.sweep(7)
        assert e.value.code == dp.DP_EINVAL
        rc, st = g.value_iterate(tol=0.0, max_sweeps=3)
        assert rc == dp.DP_ENOCONV and st.sweeps_vi == 3
    with pytest.raises(dp.DPError) as e:
        dp.Grid(W.config2(n=9).replace(lo=(0.95, -0.1, -0.2, 0.9)))
    assert e.value.code == dp.DP_EINVAL


# ------------------------------------------------------------ frozen feet --

@pytest.mark.parametrize("fmt", ["word8", "pair"])
@pytest.mark.parametrize("p", [W.config1(n=25), W.config2(n=31)], ids=["full", "reduced"])
def test_frozen_feet_match_recomputed_evaluation(dp, p, fmt):
    # After an improvement sweep the evaluation sweeps read each node's stored
    # foot (an 8-byte word with 18-bit cell fractions, or the word pair with
    # 24-bit ones) instead of recomputing the Heun step; the result must match
    # the recomputing sweep (the same codes set again, which invalidates the
    # stored feet) to the fraction quantisation: at most 3 * 2^-19 of a cell's
    # value spread per sweep, far below 1e-5 M.
    # GPU against GPU: both forms are checked against the oracle elsewhere.
    V = W.smooth_value(p, 81)
    o = oracle.Oracle(p)
    with dp.Grid(p) as g:
        g.set_foot_format(dp.DP_FOOT_WORD8 if fmt == "word8" else dp.DP_FOOT_PAIR)
        idx = g.active_index()
        g.set_value(V[idx])
        g.sweep(dp.DP_SWEEP_IMPROVE_FULL)
        v1, codes = g.get_value(), g.get_policy()
        g.sweep(dp.DP_SWEEP_EVAL)                 # frozen feet
        v_feet = g.get_value()
        g.set_value(v1)
        g.set_policy(codes)                       # same policy, feet invalidated
        g.sweep(dp.DP_SWEEP_EVAL)                 # recomputed
        v_full = g.get_value()
    assert np.abs(v_feet - v_full).max() <= 1e-5 * o.M


def test_feet_of_the_fp64_value_phase_are_not_read_as_fp32_feet(dp, small1):
    # An FP64-value improvement stores each foot as the 24-bit word pair, an
    # FP32-value improvement of a plain-evaluation solve as one 8-byte word.
    # A grid returned to FP32 values after the FP64 phase (set_value) still
    # holds the word pairs: its evaluation sweep must read them as pairs, and
    # after the next FP32 improvement read the 8-byte words; both against the
    # oracle.  An unknown format is refused.
    p, o = small1
    with dp.Grid(p) as g:
        with pytest.raises(dp.DPError) as e:
            g.set_foot_format(3)
        assert e.value.code == dp.DP_EINVAL
        rc, st = g.policy_iterate(tol=0.0, max_sweeps=3, n_eval=5, n_eval_fp64=5, polish=1, switch_tol=100.0,
                                  warm=0)
        assert st.switch_outer >= 0 and dp.dp_grid_get_info(g.h)["fp64_values"]
        V, codes = g.get_value(), g.get_policy()
        g.set_value(V)                            # FP32 values, the word pairs still stored
        g.sweep(dp.DP_SWEEP_EVAL)
        v_eval = g.get_value()
        g.set_value(V)
        g.sweep(dp.DP_SWEEP_IMPROVE_WALK)         # stores 8-byte feet
        V1, c1 = g.get_value(), g.get_policy()
        g.sweep(dp.DP_SWEEP_EVAL)
        v_eval1 = g.get_value()
    V32 = V.astype(np.float32).astype(np.float64)
    V32[o.target.astype(bool)] = 0
    want = o.sweep(V32, mode=oracle.EVAL, codes=codes)[0]
    _check_values(v_eval, want, TOL32, "evaluation after the FP64 phase", o=o, nodes=np.arange(o.N), codes=codes)
    want1 = o.sweep(V1, mode=oracle.EVAL, codes=c1)[0]
    _check_values(v_eval1, want1, TOL32, "evaluation at 8-byte feet", o=o, nodes=np.arange(o.N), codes=c1)
