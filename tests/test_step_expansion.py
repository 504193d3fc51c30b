"""The GPU evaluates the Heun step of the orbit dynamics (§3, Eq. (10)) as a
polynomial in (sin a, cos a) whose coefficients are computed once per state:

    u_r  = a0 + b0 s
    u_vr = a1 + b1 s + c (g1 + d1 c)
    u_vt = a2 + b2 s + c (g2 + e2 s)

This checks, in FP64 on the host, that the expansion is the same map as the
two-stage step (predictor, then the trapezoid average of the two drifts) for
random states and angles, including the mass coordinate's thrust scaling.
"""
import numpy as np


def _two_stage(x, a, mu, accel, mdot, dt):
    r, vr, vt, m = x
    s, c = np.sin(a), np.cos(a)

    def drift(r, vr, vt, m):
        return np.array([vr, vt * vt / r - mu / r ** 2 + accel / m * s, -vr * vt / r + accel / m * c, mdot])

    k1 = drift(r, vr, vt, m)
    k2 = drift(*(np.array(x) + dt * k1))
    return 0.5 * dt * (k1 + k2)[:3]


def _expanded(x, a, mu, accel, mdot, dt):
    r, vr, vt, m = x
    s, c = np.sin(a), np.cos(a)
    ir = 1.0 / r
    d1vr = vt * vt * ir - mu * ir * ir
    d1vt = -vr * vt * ir
    ir2 = 1.0 / (r + dt * vr)
    am, am2 = accel / m, accel / (m + dt * mdot)
    R0, P0, R1 = vr + dt * d1vr, vt + dt * d1vt, dt * am
    P1 = R1
    h = 0.5 * dt
    amm = am + am2
    a0, b0 = h * (vr + R0), h * R1
    a1 = h * (d1vr + P0 * P0 * ir2 - mu * ir2 * ir2)
    b1, g1, d1 = h * amm, h * 2 * P0 * P1 * ir2, h * P1 * P1 * ir2
    a2, b2 = h * (d1vt - R0 * P0 * ir2), -h * R1 * P0 * ir2
    g2, e2 = h * (amm - R0 * P1 * ir2), -h * R1 * P1 * ir2
    return np.array([a0 + b0 * s, a1 + b1 * s + c * (g1 + d1 * c), a2 + b2 * s + c * (g2 + e2 * s)])


def test_expanded_step_equals_two_stage_step():
    rng = np.random.default_rng(14675)
    for _ in range(200):
        x = (rng.uniform(0.95, 1.15), rng.uniform(-0.1, 0.1), rng.uniform(0.85, 1.1), rng.uniform(0.9, 1.0))
        a = rng.uniform(0, 2 * np.pi)
        accel = 10 ** rng.uniform(-4, -1)          # up to far stronger thrust than the configurations
        dt = rng.uniform(0.005, 0.1)
        want = _two_stage(x, a, 1.0, accel, -accel, dt)
        got = _expanded(x, a, 1.0, accel, -accel, dt)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_expansion_keeps_the_angle_dependence():
    # the angle-dependent part must not vanish or change sign: two angles half
    # a turn apart move the velocity components in opposite directions
    x, accel, dt = (1.0, 0.0, 1.0, 1.0), 1e-2, 0.05
    u0 = _expanded(x, 0.0, 1.0, accel, -accel, dt)
    upi = _expanded(x, np.pi, 1.0, accel, -accel, dt)
    assert (u0[2] - upi[2]) > 0.9 * dt * accel * 2 / 1.0     # cos: +accel vs -accel in v_t
    uh = _expanded(x, np.pi / 2, 1.0, accel, -accel, dt)
    u3h = _expanded(x, 3 * np.pi / 2, 1.0, accel, -accel, dt)
    assert (uh[1] - u3h[1]) > 0.9 * dt * accel * 2


def test_polar_expansion_with_the_orbital_angle():
    # the polar dynamics of the paper's Example 1: thrust acceleration fixed
    # (no mass), and the orbital angle with theta' = v_t / r
    rng = np.random.default_rng(2407)
    for _ in range(200):
        r, vr, vt = rng.uniform(0.95, 1.15), rng.uniform(-0.1, 0.1), rng.uniform(0.85, 1.1)
        a, accel, dt = rng.uniform(0, 2 * np.pi), 10 ** rng.uniform(-5, -2), rng.uniform(0.005, 0.1)
        s, c = np.sin(a), np.cos(a)

        def drift(r, vr, vt):
            return np.array([vr, vt * vt / r - 1.0 / r ** 2 + accel * s, -vr * vt / r + accel * c, vt / r])

        k1 = drift(r, vr, vt)
        k2 = drift(r + dt * k1[0], vr + dt * k1[1], vt + dt * k1[2])
        want = 0.5 * dt * (k1 + k2)
        # the expansion with a / m = a at both stages
        got3 = _expanded((r, vr, vt, 1.0), a, 1.0, accel, 0.0, dt)
        ir, ir2 = 1.0 / r, 1.0 / (r + dt * vr)
        P0, P1 = vt + dt * (-vr * vt * ir), dt * accel
        a3, g3 = 0.5 * dt * (vt * ir + P0 * ir2), 0.5 * dt * P1 * ir2
        np.testing.assert_allclose(got3, want[:3], rtol=0, atol=1e-14)
        np.testing.assert_allclose(a3 + g3 * c, want[3], rtol=0, atol=1e-14)
