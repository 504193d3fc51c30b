"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test targets a plausible mistake: a dropped or sign-flipped term of the
dynamics, a wrong RK order, a transposed interpolation weight, a broken
minimisation, a wrong discount or penalty.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2407_14675_gb300 import workloads as W


# --------------------------------------------------------------- Q1 weights --

def _multilinear(coef, s):
    """sum_e coef[e] prod_d s_d^e_d (grid units)."""
    out = 0.0
    for e in range(16):
        term = coef[e]
        for d in range(4):
            if (e >> (3 - d)) & 1:
                term *= s[d]
        out += term
    return out


def test_q1_exact_on_multilinear_functions():
    # Q1 reproduces every multilinear function exactly (§3 after Eq. (10)).
    p = W.Problem(n=(5, 4, 6, 3), lo=(0, 0, 0, 0), hi=(4, 3, 5, 2))  # h = 1: grid units = coordinates
    o = oracle.Oracle(p)
    rng = np.random.default_rng(1)
    for trial in range(20):
        coef = rng.normal(size=16)
        idx = np.stack(np.meshgrid(*[np.arange(k) for k in p.n], indexing="ij"), -1).reshape(-1, 4)
        V = np.array([_multilinear(coef, x) for x in idx])
        for _ in range(10):
            s = rng.uniform(0, 1, 4) * (np.array(p.n) - 1)
            got = o.interp(V, s, use_active=False)
            assert got == pytest.approx(_multilinear(coef, s), rel=1e-12, abs=1e-12)


def test_q1_weights_convex_and_local():
    # I[V] is a convex combination of the 16 corner values (§3 after Eq. (13)).
    p = W.Problem(n=(4, 4, 4, 4), lo=(0, 0, 0, 0), hi=(3, 3, 3, 3))
    o = oracle.Oracle(p)
    rng = np.random.default_rng(2)
    s = np.array([1.3, 0.2, 2.7, 1.5])
    weights = np.zeros(p.nodes)
    for j in range(p.nodes):
        e = np.zeros(p.nodes)
        e[j] = 1.0
        weights[j] = o.interp(e, s, use_active=False)
    assert weights.min() >= 0.0
    assert weights.sum() == pytest.approx(1.0, abs=1e-14)
    assert np.count_nonzero(weights) == 16
    nz = np.argwhere(weights.reshape(p.n) > 0)
    assert (nz.min(0) == np.floor(s)).all() and (nz.max(0) == np.floor(s) + 1).all()
    # explicit value of one weight: corner (1,0,2,1) gets (1-.3)(1-.2)(1-.7)(1-.5)
    assert weights.reshape(p.n)[1, 0, 2, 1] == pytest.approx(0.7 * 0.8 * 0.3 * 0.5, abs=1e-15)
    V = rng.uniform(0, 1, p.nodes)
    assert o.interp(V, s, use_active=False) == pytest.approx(weights @ V, abs=1e-14)


def test_interp_box_edges():
    p = W.Problem(n=(3, 3, 3, 3), lo=(0, 0, 0, 0), hi=(2, 2, 2, 2))
    o = oracle.Oracle(p)
    V = np.arange(p.nodes, dtype=float)
    assert o.interp(V, np.array([2.0, 2.0, 2.0, 2.0]), use_active=False) == V[-1]
    assert o.interp(V, np.array([0.0, 0.0, 0.0, 0.0]), use_active=False) == V[0]
    assert o.interp(V, np.array([2.0 + 1e-12, 1, 1, 1]), use_active=False) is None
    assert o.interp(V, np.array([1, -1e-12, 1, 1]), use_active=False) is None
    assert o.interp(V, np.array([1, 1, np.nan, 1]), use_active=False) is None


# ---------------------------------------------------------------- dynamics --

def test_circular_orbit_is_equilibrium_of_drift():
    # With the thrust off, the circular orbit v_r = 0, v_t = sqrt(mu/r) is a
    # rest point of (r, v_r, v_t); with the printed minus sign on v_t^2/r it
    # would accelerate inwards at -2 mu / r^2.
    for r in (0.95, 1.0, 1.05, 1.13):
        o = oracle.Oracle(W.config0().replace(accel=0.0))
        f = o.dynamics([r, 0.0, math.sqrt(1.0 / r), 0.95], 0.7)
        assert np.abs(f[:3]).max() < 1e-15


def test_dynamics_energy_and_momentum_rates():
    # d/dt (v^2/2 - mu/r) = (a/m)(v_r sin a + v_t cos a)   (thrust power)
    # d/dt (r v_t)        = r (a/m) cos a                   (thrust torque)
    # d/dt m              = -a/c
    # These fix every term and sign of the polar dynamics, and the angle
    # convention (sin -> radial, cos -> tangential).
    p = W.config0().replace(accel=3e-3, exhaust_c=2.0)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(3)
    for _ in range(50):
        x = np.array([rng.uniform(0.9, 1.2), rng.uniform(-0.1, 0.1), rng.uniform(0.8, 1.1), rng.uniform(0.9, 1)])
        a = rng.uniform(0, 2 * np.pi)
        f = o.dynamics(x, a)
        r, vr, vt, m = x
        dE = vr * f[1] + vt * f[2] + p.mu / r ** 2 * f[0]
        dh = f[0] * vt + r * f[2]
        am = p.accel / m
        assert dE == pytest.approx(am * (vr * math.sin(a) + vt * math.cos(a)), abs=1e-15)
        assert dh == pytest.approx(r * am * math.cos(a), abs=1e-15)
        assert f[3] == -p.accel / p.exhaust_c
        assert f[0] == vr


def _two_body_invariants(x):
    r, vr, vt, _ = x
    return 0.5 * (vr * vr + vt * vt) - 1.0 / r, r * vt


def test_rk4_fourth_order_and_conservation():
    # With the thrust off, energy and angular momentum are invariants; RK4's
    # global error over a fixed time falls by 2^4 when the step halves.
    p = W.config0().replace(accel=0.0)
    o = oracle.Oracle(p)
    x0 = np.array([1.0, 0.05, 1.08, 1.0])  # eccentric orbit
    E0, h0 = _two_body_invariants(x0)
    errs = []
    for h in (0.2, 0.1, 0.05):
        x = x0.copy()
        for _ in range(int(round(6.0 / h))):
            x = o.rk4(x, 0.0, h)
        E, hh = _two_body_invariants(x)
        errs.append(abs(E - E0) + abs(hh - h0))
    assert errs[2] < 1e-7
    for a, b in zip(errs, errs[1:]):
        assert 10.0 < a / b < 24.0


def test_heun_is_second_order():
    # Local error of the Heun step against a converged RK4 reference is O(h^3).
    p = W.config0().replace(accel=2e-2)
    o = oracle.Oracle(p)
    x = np.array([1.02, 0.04, 0.93, 0.95])
    alpha = 1.1
    errs = []
    for h in (0.2, 0.1, 0.05):
        ref = x.copy()
        for _ in range(200):
            ref = o.rk4(ref, alpha, h / 200)
        errs.append(np.abs(x + o.heun(x, alpha, h) - ref).max())
    for a, b in zip(errs, errs[1:]):
        assert 6.5 < a / b < 9.5
    # constant rates are integrated exactly (the mass)
    assert o.heun(x, alpha, 0.1)[3] == pytest.approx(-0.1 * p.accel / p.exhaust_c, rel=1e-15)


# --------------------------------------------------------- Bellman operator --

def _small_orbit(n=7, **kw):
    p = W.config0().replace(n=(n, n, n, n), n_angles=8, accel=5e-3, **kw)
    return p, oracle.Oracle(p)


def test_bellman_operator_monotone_and_contractive():
    # Q1 makes the scheme monotone (§3 after Eq. (10)); the fixed-point map
    # is a contraction with constant beta (§3, Eq. (12)).
    p, o = _small_orbit()
    rng = np.random.default_rng(4)
    for trial in range(4):
        V = W.random_value(p, seed=10 + trial)
        U = V + rng.uniform(0, 3, p.nodes)
        TV = o.sweep(V)[0]
        TU = o.sweep(U)[0]
        act = o.active.astype(bool)
        assert (TU[act] >= TV[act] - 1e-12).all()
        Z = W.random_value(p, seed=100 + trial)
        TZ = o.sweep(Z)[0]
        assert np.abs(TZ - TV)[act].max() <= p.beta * np.abs(Z - V).max() + 1e-12


def test_constant_field_and_penalty():
    # V = M everywhere is the fixed point off the target: dt + beta M = M
    # for M = dt / (1 - beta); target nodes are pinned to 0.
    p, o = _small_orbit()
    V = np.full(p.nodes, o.M)
    TV = o.sweep(V)[0]
    t = o.target.astype(bool)
    assert t.sum() >= 1
    assert np.abs(TV[~t] - o.M).max() < 1e-12
    assert (TV[t] == 0).all()
    # a different M changes only the out-of-box charge
    p2, o2 = _small_orbit(penalty_M=123.0)
    V = np.zeros(p.nodes)
    TV2 = o2.sweep(V)[0]
    assert TV2.max() == pytest.approx(p.dt + p.beta * 123.0)


def test_1d_minimum_time_closed_form():
    # x' = cos a, a in {0, pi}, dt = h: the foot lands on a node, and the
    # value is dt (1 - beta^n)/(1 - beta) with n the grid distance to target.
    for beta in (0.9, 0.999):
        p = W.unit_speed_1d(beta=beta)
        o = oracle.Oracle(p)
        V, sweeps, res = o.value_iterate(tol=1e-13, max_sweeps=100)
        n = np.abs(np.arange(p.n[0]) - 8)
        exact = p.dt * (1 - beta ** n) / (1 - beta)
        got = V.reshape(p.n)
        for k in range(2):
            assert np.abs(got[:, k, k, k] - exact).max() < 1e-14
        Vp, codes, outer, evals, res = o.policy_iterate(tol=1e-13, max_outer=50, n_eval=3)
        assert np.abs(Vp.reshape(p.n)[:, 0, 0, 0] - exact).max() < 1e-14
        c = codes.reshape(p.n)[:, 0, 0, 0]
        assert (c[:8] == 0).all() and (c[9:] == 32768).all()   # move towards the target


def test_2d_minimum_time_manhattan():
    # x' = (cos a, sin a), 4 axis directions, dt = h: the value is the
    # discounted Manhattan step count to the target node.
    p = W.unit_speed_2d()
    o = oracle.Oracle(p)
    V, s, res = o.value_iterate(tol=1e-13, max_sweeps=200)
    i, j = np.meshgrid(np.arange(p.n[0]), np.arange(p.n[1]), indexing="ij")
    d = np.abs(i - 6) + np.abs(j - 4)
    exact = p.dt * (1 - p.beta ** d) / (1 - p.beta)
    assert np.abs(V.reshape(p.n)[:, :, 0, 0] - exact).max() < 1e-14
    assert np.abs(V.reshape(p.n)[:, :, 1, 1] - exact).max() < 1e-14


def test_2d_euclidean_limit():
    # With many directions the discrete value approaches the discounted
    # Euclidean arrival time; the error shrinks as the grid is refined.
    errs = []
    for n in (9, 17, 33):
        p = W.unit_speed_2d(n=n, beta=0.9, target=((n - 1) // 2, (n - 1) // 2), n_angles=32)
        p = p.replace(target_w=(0.26, 0.26, 0.0, 0.0))
        o = oracle.Oracle(p)
        V, s, res = o.value_iterate(tol=1e-12, max_sweeps=2000)
        g = np.linspace(1, 2, n)
        X, Y = np.meshgrid(g, g, indexing="ij")
        # distance to the target square |x - c| < 0.26 (max-norm box)
        dx = np.maximum(np.abs(X - 1.5) - 0.26, 0)
        dy = np.maximum(np.abs(Y - 1.5) - 0.26, 0)
        T = np.hypot(dx, dy)
        lam = -math.log(p.beta) / p.dt
        exact = (1 - np.exp(-lam * T)) / lam
        errs.append(np.abs(V.reshape(p.n)[:, :, 0, 0] - exact).max())
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.1


def test_ties_keep_the_lowest_tabulated_angle():
    # V = 0 on an interior where every foot stays inside: every control gives
    # q = dt exactly.  The enumeration keeps the lowest index (code 0), the
    # refinement keeps the tabulated point when nothing is strictly lower, and
    # the value is dt.
    for refine in (0, 1):
        p = W.unit_speed_2d(n=9, n_angles=8).replace(refine=refine, refine_tol=1e-4)
        o = oracle.Oracle(p)
        V = np.zeros(o.N)
        Vn, codes, res, ev = o.sweep(V, mode=oracle.IMPROVE_FULL, codes=np.full(o.N, 999, np.uint16))
        idx = np.array(np.unravel_index(np.arange(o.N), p.n)).T
        inner = (idx[:, 0] > 0) & (idx[:, 0] < p.n[0] - 1) & (idx[:, 1] > 0) & (idx[:, 1] < p.n[1] - 1)
        inner &= ~o.target.astype(bool)
        assert inner.sum() > 20
        assert (codes[inner] == 0).all(), refine
        assert np.allclose(Vn[inner], p.dt, rtol=0, atol=1e-15)


def test_walk_starts_at_the_nearest_tabulated_angle():
    # with q flat (V = 0, every foot inside) the walk never moves, so it
    # returns its starting index: the table index nearest to the previous
    # code, also for codes just below or just above a table point
    p = W.unit_speed_2d(n=9, n_angles=8).replace(refine=0)
    o = oracle.Oracle(p)
    step = 65536 // 8
    idx = np.array(np.unravel_index(np.arange(o.N), p.n)).T
    inner = (idx[:, 0] > 0) & (idx[:, 0] < p.n[0] - 1) & (idx[:, 1] > 0) & (idx[:, 1] < p.n[1] - 1)
    inner &= ~o.target.astype(bool)
    for prev, want in ((3 * step - 1, 3), (3 * step - step // 2 + 1, 3), (3 * step + step // 2 - 1, 3),
                       (5 * step + 7, 5), (65535 - 3, 0)):
        _, codes, _, _ = o.sweep(np.zeros(o.N), mode=oracle.IMPROVE_WALK, codes=np.full(o.N, prev, np.uint16))
        assert (codes[inner] == want * step).all(), (prev, want)


def test_sweep_residual_is_the_sup_norm_of_the_change():
    # from a value above the fixed point the sweep lowers V: the residual is
    # still max |V' - V| over the node set, not a signed difference
    for p in (W.unit_speed_2d(), W.config0().replace(n=(7, 7, 7, 7))):
        o = oracle.Oracle(p)
        act = o.active.astype(bool)
        for V in (np.full(o.N, 0.9 * p.penalty_M if p.penalty_M > 0 else 0.9 * p.dt / (1 - p.beta)),
                  W.random_value(p, 5)):
            Vn, _, r, _ = o.sweep(V, mode=oracle.VI)
            assert r == np.abs(Vn - V)[act].max()
            assert r > 0


def test_policy_iteration_starts_with_a_full_tabulation():
    # the first improvement of policy iteration enumerates every tabulated
    # control (the walk only follows); from a random policy it equals the
    # full-table improvement sweep, not the walk from that policy
    p = W.config0().replace(n=(9, 9, 9, 9), refine=1)
    o = oracle.Oracle(p)
    V0 = W.random_value(p, 8)
    codes0 = W.random_codes(p, 9)
    V1, c1, outer, ev, res = o.policy_iterate(V0=V0, codes0=codes0, max_outer=1, n_eval=0, walk=True)
    Vf, cf, _, _ = o.sweep(V0, mode=oracle.IMPROVE_FULL, codes=codes0)
    Vw, cw, _, _ = o.sweep(V0, mode=oracle.IMPROVE_WALK, codes=codes0)
    assert outer == 1
    assert (c1 == cf).all() and (V1 == Vf).all()
    assert (cw != cf).any()      # the walk from a random policy differs


def test_tabulated_angles_are_the_nearest_lattice_codes():
    # alpha_k = 2 pi k / K on the 16-bit lattice, rounded to the nearest code:
    # with K = 72 (the paper's 5 degree table) 910.22 codes per step, so
    # rounding and truncation differ for four k of every nine
    p = W.example1(n=(8, 6, 6, 9)).replace(refine=0)
    o = oracle.Oracle(p)
    V = W.random_value(p, 4, hi=p.penalty_M)
    _, codes, _, _ = o.sweep(V, mode=oracle.IMPROVE_FULL, codes=np.zeros(o.N, np.uint16))
    act = o.active.astype(bool) & ~o.target.astype(bool)
    on = codes[act][codes[act] != oracle.CODE_OFF].astype(np.int64)
    assert on.size > 50
    k = np.rint(on * p.n_angles / 65536.0).astype(np.int64) % p.n_angles
    nearest = (k * 65536 + p.n_angles // 2) // p.n_angles
    assert (on == nearest).all()
    assert (np.abs(on - k * 65536.0 / p.n_angles) <= 0.5).all()
    # the sample reaches indices where the two roundings differ
    assert np.isin(k % 9, (3, 4, 7, 8)).any()


@pytest.mark.slow
def test_vi_and_pi_reach_the_same_fixed_point():
    # Eq. (12) and Eq. (13)-(14) solve the same fixed-point problem; the
    # sup-norm stop bounds the distance by tol beta/(1-beta) each.
    p, o = _small_orbit(n=6, beta=0.95, dt=0.2, refine=0)
    tol = 1e-11
    Vv, sv, rv = o.value_iterate(tol=tol, max_sweeps=5000)
    Vp, codes, outer, ev, rp = o.policy_iterate(tol=tol, max_outer=500, n_eval=10)
    assert rv < tol and rp < tol
    assert np.abs(Vv - Vp).max() <= 2 * tol * p.beta / (1 - p.beta) + 1e-12
    assert outer < sv


# ------------------------------------------------------------ minimisation --

def _brute_force_codes(o, V, j, codes):
    return o.q_nodes(V, np.full(len(codes), j), codes)


def test_golden_refinement_against_brute_force():
    # The refined control is the brute-force minimiser over the lattice
    # bracket (to one lattice step) where q is unimodal there, and never worse
    # than the tabulated minimiser (§3 "Efficient computation of the minimum").
    p = W.config0().replace(n=(7, 7, 7, 7), n_angles=16, refine=1, accel=0.05, dt=0.1)
    o = oracle.Oracle(p)
    V = W.smooth_value(p, seed=5)
    rng = np.random.default_rng(6)
    nodes = rng.choice(np.flatnonzero(o.active & ~o.target), 40, replace=False)
    v_ref, c_ref = o.bellman_nodes(V, nodes, mode=oracle.IMPROVE_FULL)
    p_tab = p.replace(refine=0)
    o_tab = oracle.Oracle(p_tab)
    v_tab, c_tab = o_tab.bellman_nodes(V, nodes, mode=oracle.IMPROVE_FULL)
    checked = 0
    S = 65536 // p.n_angles
    for i, j in enumerate(nodes):
        assert v_ref[i] <= v_tab[i]
        codes = (int(c_tab[i]) + np.arange(-S + 1, S)) % 65536
        q = _brute_force_codes(o, V, j, codes.astype(np.uint16))
        if np.ptp(q) < 1e-9:
            continue   # flat (every foot out of the box)
        k = int(np.argmin(q))
        unimodal = (np.diff(q[: k + 1]) <= 1e-15).all() and (np.diff(q[k:]) >= -1e-15).all()
        if not unimodal:
            continue
        checked += 1
        assert v_ref[i] <= q[k] + 1e-12 * max(1, abs(q[k])) + (q.max() - q.min()) * 1e-6
        dist = abs(int(c_ref[i]) - int(codes[k]))
        dist = min(dist, 65536 - dist)
        assert dist <= 2
        assert dist * 2 * math.pi / 65536 <= p.refine_tol * 2
    assert checked >= 20


def test_walk_finds_the_tabulated_minimum_where_q_is_unimodal():
    # The local walk from any start reaches the full-enumeration minimiser at
    # every node whose tabulated q has a single strict local minimum over the
    # circle of angles (§3 "Efficient computation of the minimum"); elsewhere
    # it stops at a local minimum of the table.
    K = 32
    p = W.config0().replace(n=(7, 7, 7, 7), n_angles=K, refine=0, accel=0.05, dt=0.1)
    o = oracle.Oracle(p)
    V = W.smooth_value(p, seed=7)
    v_full, c_full = o.sweep(V, mode=oracle.IMPROVE_FULL)[:2]
    rng = np.random.default_rng(8)
    start = ((c_full.astype(np.int64) + rng.integers(-8, 9, p.nodes) * (65536 // K)) % 65536).astype(np.uint16)
    v_walk, c_walk = o.sweep(V, mode=oracle.IMPROVE_WALK, codes=start)[:2]
    table = (np.arange(K) * 65536 // K).astype(np.uint16)
    nodes = np.flatnonzero((o.active & ~o.target).astype(bool))
    unimodal = 0
    for j in nodes:
        q = o.q_nodes(V, np.full(K, j), table)
        left, right = np.roll(q, 1), np.roll(q, -1)
        strict_min = (q < left) & (q < right)
        local_min = (q <= left) & (q <= right)
        k = int(np.flatnonzero(c_walk[j] == table)[0])
        assert local_min[k], "walk must stop at a local minimum of the table"
        if strict_min.sum() == 1 and local_min.sum() == 1:
            unimodal += 1
            assert c_walk[j] == c_full[j] and v_walk[j] == v_full[j]
    assert unimodal > 0.3 * len(nodes)


def test_eval_mode_uses_frozen_policy():
    p, o = _small_orbit()
    V = W.random_value(p, 11)
    codes = W.random_codes(p, 12)
    TV, _, _, _ = o.sweep(V, mode=oracle.EVAL, codes=codes)
    rng = np.random.default_rng(13)
    for j in rng.choice(np.flatnonzero(~o.target.astype(bool)), 20, replace=False):
        idx = np.unravel_index(j, p.n)
        assert TV[j] == o.q_node(V, idx, oracle.code_angle(codes[j]))
    # the improvement over the table never does worse than a frozen policy
    # that picks tabulated angles
    tab = (rng.integers(0, p.n_angles, p.nodes) * (65536 // p.n_angles)).astype(np.uint16)
    TT = o.sweep(V, mode=oracle.EVAL, codes=tab)[0]
    TI = o.sweep(V, mode=oracle.IMPROVE_FULL)[0]
    assert (TI <= TT).all() and (TI < TT).any()


# ------------------------------------------------------------ reduced grid --

def test_reduced_grid_rows_are_contiguous_in_vt():
    # For v_t > 0 the energy rises with v_t, so each (r, v_r) row keeps one
    # contiguous run of v_t nodes (all masses).
    p = W.config2(n=41)
    o = oracle.Oracle(p)
    a = o.active.reshape(p.n)
    assert (a == a[..., :1]).all()     # independent of m
    rows = a[..., 0]
    for ir in range(p.n[0]):
        for iv in range(p.n[1]):
            k = np.flatnonzero(rows[ir, iv])
            if len(k):
                assert k[-1] - k[0] + 1 == len(k)
    frac = o.n_active / p.nodes
    assert 0.15 < frac < 0.4
    assert (o.target <= o.active).all() and o.target.sum() > 0


def test_reduced_grid_cells_leaving_the_band_are_penalised():
    p = W.config2(n=21).replace(accel=2e-3, dt=0.05)
    o = oracle.Oracle(p)
    V = np.zeros(p.nodes)
    TV = o.sweep(V)[0]
    act = o.active.astype(bool)
    # with V = 0 the update is dt (foot inside the set) or dt + beta M
    vals = np.unique(np.round(TV[act & ~o.target.astype(bool)], 12))
    assert set(vals) <= {round(p.dt, 12), round(p.dt + p.beta * o.M, 12)}
    assert len(vals) == 2
    # compare with the full box: a node whose foot stays in a fully active cell
    # sees the same value on both grids
    pf = p.replace(reduced=0)
    of = oracle.Oracle(pf)
    TVf = of.sweep(V)[0]
    same = TV[act] == TVf[act]
    assert same.mean() > 0.5


# -------------------------------------------------- feedback / closed loop --

def test_feedback_at_nodes_matches_improvement():
    # Eq. (15) with tau = dt at a grid node is the minimisation of Eq. (14).
    p = W.config0().replace(n=(7, 7, 7, 7), n_angles=16, refine=1, accel=0.05, dt=0.1)
    o = oracle.Oracle(p)
    V = W.smooth_value(p, seed=9)
    rng = np.random.default_rng(10)
    nodes = rng.choice(np.flatnonzero(~o.target.astype(bool)), 30, replace=False)
    v, c = o.bellman_nodes(V, nodes, mode=oracle.IMPROVE_FULL)
    idx = np.stack(np.unravel_index(nodes, p.n), -1)
    h = (np.array(p.hi) - np.array(p.lo)) / (np.array(p.n) - 1)
    states = np.array(p.lo) + idx * h
    cf, qf = o.feedback(V, states, tau=p.dt)
    assert np.abs(qf - v).max() < 1e-12
    assert np.mean(cf == c) > 0.9


def test_closed_loop_1d_arrival_time():
    # Unit speed towards the target from the left end: arrival after exactly
    # the grid distance (8 steps of h).
    p = W.unit_speed_1d()
    o = oracle.Oracle(p)
    V, s, r = o.value_iterate(tol=1e-13)
    x0 = np.array([[1.0, 1.0, 1.0, 1.0], [2.0, 1.5, 1.0, 1.0], [1.0 + 3 * p.dt, 1.0, 1.0, 1.0]])
    ta, xf = o.simulate(V, x0, tau=p.dt, h=p.dt, t_max=2.0)
    assert ta == pytest.approx([8 * p.dt, 8 * p.dt, 5 * p.dt], abs=1e-12)
    assert xf[:, 0] == pytest.approx([1.5, 1.5, 1.5], abs=1e-12)


def _unit_1d_closed_form(p, target_node=8):
    """V of the 1-D unit-speed problem on the full box: dt (1 - beta^n) /
    (1 - beta), n the grid distance to the target node (dt = h)."""
    n = np.abs(np.arange(p.n[0]) - target_node)
    exact = p.dt * (1 - p.beta ** n) / (1 - p.beta)
    return np.repeat(exact, np.prod(p.n[1:])), n


def test_feedback_with_its_own_step_tau_closed_form():
    # Eq. (15) with a feedback step tau = k dt (the paper takes dt = o(tau)).
    # In the 1-D unit-speed problem the foot of a node moves k cells, so
    # towards the target q = tau * 1 + beta^(tau / dt) V(n - k), with V the
    # closed form.  A discount of beta instead of beta^(tau / dt), or a running
    # cost dt instead of tau, misses it by O(dt).
    p = W.unit_speed_1d(beta=0.95)
    o = oracle.Oracle(p)
    V, n = _unit_1d_closed_form(p)
    for k in (2, 3):
        tau = k * p.dt
        idx = np.flatnonzero(n >= k)
        states = np.zeros((len(idx), 4)) + 1.0
        states[:, 0] = 1.0 + idx * p.dt
        codes, q = o.feedback(V, states, tau=tau)
        d = np.abs(idx - 8) - k                       # grid distance after the step
        v_after = p.dt * (1 - p.beta ** d) / (1 - p.beta)
        want = tau + p.beta ** k * v_after
        assert np.abs(q - want).max() < 1e-13, (k, np.abs(q - want).max())
        assert (codes[idx < 8] == 0).all() and (codes[idx > 8] == 32768).all()
        # neither the discount of one grid step nor the running cost of one
        # would do (where the foot is not in the target, V > 0 there)
        far = d > 0
        assert np.abs(tau + p.beta * v_after - want)[far].min() > 1e-4
        assert np.abs(p.dt + p.beta ** k * v_after - want).min() > 1e-4


def test_closed_loop_1d_with_unequal_feedback_and_rk4_steps():
    # The closed loop re-decides the control every RK4 step h and looks ahead
    # by tau; unit speed is integrated exactly by RK4, so from grid distance n
    # the state reaches the target after n dt whatever tau and h (h dividing
    # dt), and the arrival time is counted in steps of h.
    p = W.unit_speed_1d()
    o = oracle.Oracle(p)
    V, _ = _unit_1d_closed_form(p)
    x0 = np.array([[1.0, 1.0, 1.0, 1.0], [2.0, 1.5, 1.0, 1.0], [1.0 + 3 * p.dt, 1.0, 1.0, 1.0]])
    for tau, h in ((2 * p.dt, p.dt / 2), (3 * p.dt, p.dt / 3), (p.dt, p.dt / 4), (2 * p.dt, p.dt)):
        ta, xf = o.simulate(V, x0, tau=tau, h=h, t_max=2.0)
        assert ta == pytest.approx([8 * p.dt, 8 * p.dt, 5 * p.dt], abs=1e-12), (tau, h, ta)
        assert xf[:, 0] == pytest.approx([1.5, 1.5, 1.5], abs=1e-12)


# ------------------------------------------ the paper's Example 1 (§4) --

def _ellipse_state(mu, a, e, omega, nu):
    """Textbook Kepler orbit: state at true anomaly nu of the orbit (a, e,
    argument of perigee omega), in the polar form (rho, v_rho, v_theta, theta)."""
    p_ = a * (1.0 - e * e)
    rho = p_ / (1.0 + e * math.cos(nu))
    k = math.sqrt(mu / p_)
    return np.array([rho, k * e * math.sin(nu), k * (1.0 + e * math.cos(nu)), omega + nu])


def test_example1_orbital_elements_match_kepler_orbits():
    p = W.example1(n=(5, 3, 3, 4))
    o = oracle.Oracle(p)
    for a, e, w in ((7000.0, 0.0, 0.0), (7000.0, 0.001, 0.0), (6990.0, 0.004, 1.3), (7040.0, 0.02, -2.5)):
        for nu in (0.0, 0.7, 2.0, math.pi, 4.4):
            x = _ellipse_state(W.MU_EARTH, a, e, w, nu)
            ga, ex, ey = o.elements(x)
            assert ga == pytest.approx(a, rel=1e-12)
            assert ex == pytest.approx(e * math.cos(w), abs=1e-12)
            assert ey == pytest.approx(e * math.sin(w), abs=1e-12)


def test_example1_cost_vanishes_on_the_target_orbit():
    # Eq. (11): on the target orbit only the control term remains
    p = W.example1(n=(5, 3, 3, 4))
    o = oracle.Oracle(p)
    for nu in np.linspace(0.0, 2 * math.pi, 9):
        x = _ellipse_state(W.MU_EARTH, p.a_bar, p.e_bar, p.omega_bar, nu)
        assert abs(o.running_cost(x, thrust_on=False)) < 1e-12
        assert o.running_cost(x, thrust_on=True) == pytest.approx(p.cost_alpha * p.accel, abs=1e-12)
    # off the target: beta (a - a_bar)^2 + gamma e^2 on a circular orbit
    x = W.example1_start(6980.0)
    assert o.running_cost(x, False) == pytest.approx(p.cost_beta * 20.0 ** 2 + p.cost_gamma * p.e_bar ** 2,
                                                     rel=1e-9)


def test_example1_cost_eccentricity_vector_term():
    # Eq. (11) with a = a_bar: only gamma |e_vec - e_bar_vec|^2 remains (thrust
    # off), where e_vec = e (cos omega, sin omega).  Orbits of the same
    # eccentricity but another argument of perigee cost more than the target's
    # own, which a scalar (e - e_bar)^2 would miss.
    p = W.example1(n=(5, 3, 3, 4))
    o = oracle.Oracle(p)
    ebx, eby = p.e_bar * math.cos(p.omega_bar), p.e_bar * math.sin(p.omega_bar)
    for e, w in ((0.003, 1.0), (0.001, math.pi / 2), (0.001, math.pi), (0.0025, -2.2)):
        want = p.cost_gamma * ((e * math.cos(w) - ebx) ** 2 + (e * math.sin(w) - eby) ** 2)
        for nu in (0.3, 2.5, 5.1):
            x = _ellipse_state(W.MU_EARTH, p.a_bar, e, w, nu)
            assert o.running_cost(x, thrust_on=False) == pytest.approx(want, rel=1e-7, abs=1e-18)
    # same eccentricity as the target, perigee turned by pi: |e_vec - e_bar_vec| = 2 e_bar
    x = _ellipse_state(W.MU_EARTH, p.a_bar, p.e_bar, p.omega_bar + math.pi, 1.1)
    assert o.running_cost(x, thrust_on=False) == pytest.approx(p.cost_gamma * (2 * p.e_bar) ** 2, rel=1e-7)


def test_energy_is_the_vis_viva_energy_on_kepler_orbits():
    # the specific energy v^2/2 - mu/r that selects the band (§3) equals
    # -mu / (2a) everywhere on a Kepler ellipse, radial speed included
    p = W.config2(n=9)
    o = oracle.Oracle(p)
    for a, e in ((1.0, 0.0), (1.02, 0.05), (0.97, 0.2)):
        for nu in (0.4, 1.9, 3.6, 5.5):
            x = _ellipse_state(1.0, a, e, 0.0, nu)
            assert o.energy(np.array([x[0], x[1], x[2], 1.0])) == pytest.approx(-1.0 / (2.0 * a), rel=1e-13)


def test_example1_dynamics_identities():
    p = W.example1(n=(5, 3, 3, 4))
    o = oracle.Oracle(p)
    x = W.example1_start(7000.0)
    f = o.dynamics(x, oracle.OFF)   # circular orbit, thrust off: at rest but the angle
    assert np.abs(f[:3]).max() < 1e-15 and f[3] == pytest.approx(x[2] / x[0], rel=1e-15)
    y = np.array([6990.0, 0.004, 7.55, 1.1])
    for alpha in (0.0, 0.9, 2.5, 4.0):
        f = o.dynamics(y, alpha)
        u = p.accel
        dE = y[1] * f[1] + y[2] * f[2] + W.MU_EARTH / y[0] ** 2 * f[0]   # d/dt (v^2/2 - mu/rho)
        assert dE == pytest.approx(u * (y[1] * math.sin(alpha) + y[2] * math.cos(alpha)), rel=1e-9, abs=1e-18)
        dh = f[0] * y[2] + y[0] * f[2]                                  # d/dt (rho v_theta)
        assert dh == pytest.approx(y[0] * u * math.cos(alpha), rel=1e-9, abs=1e-15)


def test_example1_angle_interpolates_periodically():
    # V = (multilinear in rho, v_rho, v_theta) x (a value per angle node): the
    # Q1 interpolation is exact, and the cell past the last node reaches node 0
    p = W.example1(n=(4, 3, 3, 6))
    o = oracle.Oracle(p)
    rng = np.random.default_rng(4)
    g = rng.uniform(1, 2, 6)
    c = rng.uniform(-1, 1, 4)
    i0, i1, i2, i3 = np.meshgrid(*[np.arange(k) for k in p.n], indexing="ij")
    lin = c[0] + c[1] * i0 + c[2] * i1 * i2 + c[3] * i0 * i1 * i2
    V = (lin * g[i3]).reshape(-1)
    s = np.array([1.3, 0.4, 1.7, 5.25])      # between angle node 5 and node 0
    l = c[0] + c[1] * 1.3 + c[2] * 0.4 * 1.7 + c[3] * 1.3 * 0.4 * 1.7
    assert o.interp(V, s) == pytest.approx(l * (0.75 * g[5] + 0.25 * g[0]), rel=1e-13)
    for k in (-2, 1, 3):
        assert o.interp(V, s + np.array([0, 0, 0, 6.0 * k])) == pytest.approx(o.interp(V, s), rel=1e-13)


def test_example1_thrust_off_wins_where_thrust_only_costs():
    # V constant inside the box: every control lands on the same value, so
    # the control term alpha |u| decides and the improvement switches off
    p = W.example1(n=(6, 4, 4, 6))
    o = oracle.Oracle(p)
    V = np.full(o.N, 5.0)
    Vn, codes, res, ev = o.sweep(V, mode=oracle.IMPROVE_FULL, codes=np.zeros(o.N, np.uint16))
    idx = np.array(np.unravel_index(np.arange(o.N), p.n)).T
    interior = (idx[:, 0] > 0) & (idx[:, 0] < p.n[0] - 1) & (idx[:, 1] > 0) & (idx[:, 1] < p.n[1] - 1) & \
               (idx[:, 2] > 0) & (idx[:, 2] < p.n[2] - 1)
    assert interior.any()
    assert (codes[interior] == oracle.CODE_OFF).all()
    for j in np.flatnonzero(interior)[:5]:
        x = np.array(p.lo) + idx[j] * (np.array(p.hi) - np.array(p.lo)) / (np.array(p.n) - 1)
        assert Vn[j] == pytest.approx(p.dt * o.running_cost(x, False) + p.beta * 5.0, rel=1e-14)


def test_thrust_off_wins_exact_ties_in_improvement_and_feedback():
    # with no control cost (alpha = 0) and V = 0 (every Q1 blend exactly 0,
    # whatever the weights), thrust and thrust off give exactly the same q at
    # nodes whose feet stay inside; the off control wins the tie in the
    # improvement sweep and in the feedback of Eq. (15) alike
    p = W.example1(n=(6, 4, 4, 6)).replace(cost_alpha=0.0)
    o = oracle.Oracle(p)
    V = np.zeros(o.N)
    _, codes, _, _ = o.sweep(V, mode=oracle.IMPROVE_FULL, codes=np.zeros(o.N, np.uint16))
    idx = np.array(np.unravel_index(np.arange(o.N), p.n)).T
    interior = (idx[:, 0] > 0) & (idx[:, 0] < p.n[0] - 1) & (idx[:, 1] > 0) & (idx[:, 1] < p.n[1] - 1) & \
               (idx[:, 2] > 0) & (idx[:, 2] < p.n[2] - 1)
    assert interior.sum() >= 8
    assert (codes[interior] == oracle.CODE_OFF).all()
    h = (np.array(p.hi) - np.array(p.lo)) / (np.array(p.n) - 1)
    states = np.array(p.lo) + idx[interior] * h
    fc, _ = o.feedback(V, states)
    assert (fc == oracle.CODE_OFF).all()


def test_closed_loop_coasts_where_the_feedback_switches_off():
    # V constant: the control term alone decides, the feedback switches the
    # thrust off, and the closed loop must follow the unforced RK4 steps
    p = W.example1(n=(6, 4, 4, 6))
    o = oracle.Oracle(p)
    V = np.full(o.N, 5.0)
    x0 = np.array([7000.0, 0.001, 7.546, 0.4])
    fc, _ = o.feedback(V, x0[None, :])
    assert fc[0] == oracle.CODE_OFF
    steps, h = 4, p.dt
    ta, xf = o.simulate(V, x0[None, :], t_max=steps * h)
    x = x0.copy()
    for _ in range(steps):
        x = o.rk4(x, oracle.OFF, h)
    assert ta[0] == -1.0
    assert np.array_equal(xf[0], x)


def test_policy_iteration_is_improvement_then_n_eval_evaluations():
    # the loop of modified policy iteration: a full-table improvement, n_eval
    # evaluation sweeps at the frozen policy, a walk improvement, n_eval more
    p = W.config0().replace(n=(7, 7, 7, 7))
    o = oracle.Oracle(p)
    V0 = W.random_value(p, 12)
    c0 = W.random_codes(p, 13)
    V, c, outer, evs, res = o.policy_iterate(V0=V0, codes0=c0, tol=0.0, max_outer=2, n_eval=3, walk=True)
    assert outer == 2 and evs == 6
    U, cu, _, _ = o.sweep(V0, mode=oracle.IMPROVE_FULL, codes=c0)
    for _ in range(3):
        U = o.sweep(U, mode=oracle.EVAL, codes=cu)[0]
    U, cu, _, _ = o.sweep(U, mode=oracle.IMPROVE_WALK, codes=cu)
    for _ in range(3):
        U = o.sweep(U, mode=oracle.EVAL, codes=cu)[0]
    assert np.array_equal(V, U) and np.array_equal(c, cu)


def test_value_iteration_stops_at_the_first_sweep_below_tol():
    # config 0 converges geometrically (its residual falls by about beta per
    # sweep, never to an exact zero), so the first sweep below tol is unique
    p = W.config0().replace(n=(7, 7, 7, 7))
    o = oracle.Oracle(p)
    for tol in (1e-2, 1e-3):
        V, s, res = o.value_iterate(tol=tol, max_sweeps=10000)
        U = np.zeros(o.N)
        k, r = 0, np.inf
        while r >= tol:
            U, _, r, _ = o.sweep(U, mode=oracle.VI)
            k += 1
        assert s == k and res == r and np.array_equal(V, U)


def test_example2_drag_coefficient_and_deceleration():
    # C = C_D S rho_D / (2 m) with the paper's constants, in 1/km
    C = W.example2_drag()
    assert C == pytest.approx(2.2 * 2.25 * 8.09e-14 / 700.0 * 1000.0, rel=1e-15)
    assert C == pytest.approx(5.721e-13, rel=1e-3)
    p = W.example1(n=(5, 3, 3, 4))
    o = oracle.Oracle(p)
    y = np.array([6990.0, 0.004, 7.55, 1.1])
    f0 = o.dynamics(y, oracle.OFF)
    f = o.dynamics_drag(y, oracle.OFF, C)
    # the printed components: -C v_rho^2 and -C v_theta^2; the energy then
    # falls at C (v_rho^3 + v_theta^3)
    # (no absolute tolerance: the radial term is about 1e-17 km/s^2, next to
    # f0[1] of about 3e-6, so its difference carries ~4e-5 relative rounding)
    assert f[1] - f0[1] == pytest.approx(-C * y[1] ** 2, rel=1e-3, abs=0.0)
    assert f[2] - f0[2] == pytest.approx(-C * y[2] ** 2, rel=1e-6, abs=0.0)
    dE = y[1] * (f[1] - f0[1]) + y[2] * (f[2] - f0[2])
    assert dE == pytest.approx(-C * (y[1] ** 3 + y[2] ** 3), rel=1e-6, abs=0.0)
    # an outward or inward radial speed both lose to the radial drag
    for vr in (0.006, -0.006):
        z = np.array([6990.0, vr, 7.55, 1.1])
        dz = o.dynamics_drag(z, oracle.OFF, C)[1] - o.dynamics(z, oracle.OFF)[1]
        assert dz < 0.0 and dz == pytest.approx(-C * vr * vr, rel=1e-3, abs=0.0)
    assert (o.dynamics_drag(y, 0.3, 0.0) == o.dynamics(y, 0.3)).all()


# ------------------------------------------- exact policy evaluation (Eq. 13) --

def test_policy_system_reproduces_the_evaluation_sweep():
    # the assembled rows are the evaluation sweep written as V -> b + beta W V:
    # a dropped penalty, a transposed weight or a misplaced discount breaks it
    for p, seed in [(W.config1(13).replace(n=(9, 9, 9, 9)), 1), (W.config2(13), 2), (W.example1(n=(12, 7, 7, 8)), 3)]:
        o = oracle.Oracle(p)
        codes = W.random_codes(p, seed)
        if p.off_control:
            codes[::5] = oracle.CODE_OFF
        V = W.smooth_value(p, seed + 10)
        Wm, b = o.policy_system(codes)
        got = b + o.s.beta * (Wm @ V)
        want = o.sweep(V, mode=oracle.EVAL, codes=codes)[0]
        act = o.active.astype(bool)
        assert np.abs(got - want)[act].max() <= 1e-12 * np.abs(want).max()
        # rows are convex combinations or empty
        rs = np.asarray(Wm.sum(axis=1)).ravel()
        assert np.all((np.abs(rs - 1.0) < 1e-12) | (rs == 0.0))


def test_exact_evaluation_closed_form_1d():
    # x' = 1 on a line with dt = h: every foot lands one node to the right.
    # Left of the target the value is the discounted time to go,
    # dt (1 - beta^d) / (1 - beta); right of it the trajectory leaves the box
    # after s = n - 1 - i steps and pays the penalty M one step later.
    M = 3.0
    p = W.unit_speed_1d().replace(penalty_M=M)
    o = oracle.Oracle(p)
    v = o.evaluate_exact(np.zeros(p.nodes, np.uint16)).reshape(p.n)
    n, t, dt, beta = p.n[0], 8, p.dt, p.beta
    for i in range(n):
        if i < t:
            want = dt * (1 - beta ** (t - i)) / (1 - beta)
        elif i == t:
            want = 0.0
        else:
            s = n - 1 - i
            want = dt * (1 - beta ** s) / (1 - beta) + beta ** s * (dt + beta * M)
        assert np.allclose(v[i], want, rtol=0, atol=1e-13), (i, v[i, 0, 0, 0], want)


def test_exact_evaluation_is_the_fixed_point_of_the_sweep():
    # the evaluated value is the unique fixed point of the frozen-policy sweep
    # (a beta-contraction), and Jacobi sweeps approach it at rate beta
    p = W.config1(13).replace(n=(11, 9, 9, 9))
    o = oracle.Oracle(p)
    codes = W.random_codes(p, 5)
    v = o.evaluate_exact(codes)
    v1 = o.sweep(v, mode=oracle.EVAL, codes=codes)[0]
    assert np.abs(v1 - v).max() <= 1e-12 * o.M
    V = np.zeros(p.nodes)
    e0 = np.abs(V - v).max()
    for _ in range(50):
        V = o.sweep(V, mode=oracle.EVAL, codes=codes)[0]
    assert np.abs(V - v).max() <= p.beta ** 50 * e0 * (1 + 1e-9)


def test_eval_diag_sweep_closed_form_half_step():
    # x' = 1 with dt = h / 2: every foot lies half-way to the right neighbour,
    # so a node's own weight is 1/2 and the other 1/2 sits on node j + 1:
    # V'_j = (dt + beta V_{j+1} / 2) / (1 - beta / 2)
    p = W.unit_speed_1d().replace(dt=0.5 / 16)
    o = oracle.Oracle(p)
    codes = np.zeros(p.nodes, np.uint16)
    V = W.smooth_value(p, 31)
    Vn, _ = o.eval_diag_sweep(V, codes)
    Vg, Vng = V.reshape(p.n), Vn.reshape(p.n)
    for i in range(15):
        if i == 8:
            assert Vng[i, 0, 0, 0] == 0.0
            continue
        want = (p.dt + p.beta * 0.5 * Vg[i + 1]) / (1.0 - 0.5 * p.beta)
        assert np.allclose(Vng[i], want, rtol=1e-14, atol=0)


def test_eval_diag_sweep_has_the_exact_evaluation_as_fixed_point_and_contracts():
    for p in (W.config1(13).replace(n=(11, 9, 9, 9)), W.example1(n=(12, 7, 7, 8))):
        o = oracle.Oracle(p)
        codes = W.random_codes(p, 33)
        if p.off_control:
            codes[::5] = oracle.CODE_OFF
        v = o.evaluate_exact(codes)
        v1, r = o.eval_diag_sweep(v, codes)
        assert r <= 1e-12 * np.abs(v).max()
        # a beta-contraction in the sup norm (row factor beta (1 - w) / (1 - beta w) <= beta)
        U = W.smooth_value(p, 34) * np.abs(v).max() / o.M
        X = W.smooth_value(p, 35) * np.abs(v).max() / o.M
        act = o.active.astype(bool)
        dU, _ = o.eval_diag_sweep(U, codes)
        dX, _ = o.eval_diag_sweep(X, codes)
        assert np.abs(dU - dX)[act].max() <= o.s.beta * np.abs(U - X)[act].max() * (1 + 1e-12)
        # and it converges no slower than the plain evaluation sweep
        Vp, Vd = np.zeros(p.nodes), np.zeros(p.nodes)
        for _ in range(30):
            Vp = o.sweep(Vp, mode=oracle.EVAL, codes=codes)[0]
            Vd = o.eval_diag_sweep(Vd, codes)[0]
        assert np.abs(Vd - v)[act].max() <= np.abs(Vp - v)[act].max() * (1 + 1e-12)


def test_vi_diag_sweep_closed_form_half_step():
    # x' = cos a with dt = h / 2 and the two angles 0 and pi: the foot lies
    # half-way to a neighbour, so V'_j = min over the two neighbours of
    # (dt + beta V_nb / 2) / (1 - beta / 2) (the slice i_vr = 0: an angle of
    # pi moves v_r by dt sin(pi) > 0, inside the box there)
    p = W.unit_speed_1d().replace(dt=0.5 / 16)
    o = oracle.Oracle(p)
    V = W.smooth_value(p, 36)
    V[o.target.astype(bool)] = 0.0
    Vn, _ = o.vi_diag_sweep(V)
    Vg, Vng = V.reshape(p.n), Vn.reshape(p.n)
    for i in range(17):
        if i == 8:
            continue
        cands = []
        for nb in (i - 1, i + 1):
            if 0 <= nb < 17:
                cands.append((p.dt + 0.5 * p.beta * Vg[nb, 0]) / (1 - 0.5 * p.beta))
            else:
                cands.append(np.full_like(Vg[i, 0], p.dt + p.beta * o.M))
        want = np.minimum(cands[0], cands[1])
        assert np.allclose(Vng[i, 0], want, rtol=1e-14, atol=0), i


def test_vi_diag_has_the_value_iteration_fixed_point():
    # the fixed point of Eq. (12) is also that of the diagonal-solved sweep,
    # which gets there in far fewer sweeps
    p = W.config0().replace(n=(7, 7, 7, 7), beta=0.99)
    o = oracle.Oracle(p)
    V, sweeps, res = o.value_iterate(tol=1e-11, max_sweeps=200000)
    Vd = np.zeros(p.nodes)
    n = 0
    for n in range(1, 200000):
        Vd, r = o.vi_diag_sweep(Vd)
        if r < 1e-11:
            break
    act = o.active.astype(bool)
    assert np.abs(Vd - V)[act].max() <= 1e-8 * np.abs(V).max()
    assert n < sweeps / 3
    # one sweep at the fixed point moves nothing
    V1, r1 = o.vi_diag_sweep(V)
    assert r1 <= 1e-9 * np.abs(V).max()
