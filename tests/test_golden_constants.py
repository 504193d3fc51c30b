"""The paper's printed constants (tests/golden/paper_constants.txt, each line
citing its passage) against the problem data the oracle and the GPU path both
read, plus closed-form consistency of the paper's orbits with its domain.

The paper prints no value function, policy or trajectory, so these constants
and the orbits they define are what can be pinned to the paper itself.
"""
import math
import os

import numpy as np
import pytest

from paper_2407_14675_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _constants():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, unit, passage = line.split(None, 3)
            assert passage.startswith("§"), line   # every value cites its passage
            out[name] = float(value)
    return out


C = _constants()


def test_fixture_lists_every_constant_once():
    names = [ln.split()[0] for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(names) == len(set(names)) == len(C) == 28


def test_example1_problem_uses_the_printed_constants():
    """§4 Example 1 and §2.1: the problem data of the paper's first example."""
    p = W.example1()
    assert p.mu == C["mu"]
    assert p.accel == C["thrust_accel"]
    assert (p.cost_alpha, p.cost_beta, p.cost_gamma) == (C["cost_alpha"], C["cost_beta"], C["cost_gamma"])
    assert p.dt == C["dt"]
    # the discount factor of one step of the scheme is exp(-lambda dt) (§3)
    assert p.beta == pytest.approx(math.exp(-C["discount_lambda"] * C["dt"]), rel=1e-15)
    assert p.tol == C["pi_tol"]
    assert (p.a_bar, p.e_bar, p.omega_bar) == (C["target_a"], C["target_e"], math.radians(C["target_omega_deg"]))
    # state order (rho, v_rho, v_theta, theta)
    assert p.n == (int(C["n_rho"]), int(C["n_v_rho"]), int(C["n_v_theta"]), int(C["n_theta"]))
    assert p.lo[:3] == (C["rho_lo"], C["v_rho_lo"], C["v_theta_lo"])
    assert p.hi[:3] == (C["rho_hi"], C["v_rho_hi"], C["v_theta_hi"])
    # theta covers [0, 2 pi) with n_theta nodes: the last node one step short of 2 pi
    assert p.lo[3] == 0.0
    assert p.hi[3] == pytest.approx(2.0 * math.pi * (1.0 - 1.0 / C["n_theta"]), rel=1e-15)
    # 72 angles 5 degrees apart, plus the null thrust: 73 tabulated controls
    assert p.n_angles * C["angle_step_deg"] == 360.0
    assert p.n_angles + p.off_control == int(C["tabulated_controls"])


def test_example1_grid_size_is_the_printed_order_of_magnitude():
    """§4 Example 1: 'about 3 10^6 nodes' for 110 x 30 x 30 x 30."""
    nodes = C["n_rho"] * C["n_theta"] * C["n_v_rho"] * C["n_v_theta"]
    assert nodes == 2_970_000
    assert abs(nodes - 3e6) / 3e6 < 0.02


def test_example2_drag_constant_from_the_printed_parameters():
    """§4 Example 2: C = C_D S rho_D / (2 m), here in 1/km (v in km/s, a in km/s^2)."""
    c_si = C["drag_cd"] * C["drag_area"] * C["drag_density"] / (2.0 * C["drag_mass"])   # 1/m
    assert W.example2_drag() == pytest.approx(c_si * 1000.0, rel=1e-15)
    assert W.example2_drag() == pytest.approx(5.7207857142857e-13, rel=1e-12)


def test_paper_orbits_lie_inside_the_printed_domain():
    """Closed forms: the start orbit (circular, 6978 km) and the target orbit
    (a = 7000 km, e = 0.001) lie inside the §4 domain, so the manoeuvre the
    paper flies stays on its grid."""
    mu = C["mu"]
    # circular start: rho = r0, v_rho = 0, v_theta = sqrt(mu / r0)
    x0 = W.example1_start(C["start_radius"])
    assert x0[0] == C["start_radius"] and x0[1] == 0.0
    assert x0[2] == pytest.approx(math.sqrt(mu / C["start_radius"]), rel=1e-15)
    assert C["rho_lo"] < x0[0] < C["rho_hi"]
    assert C["v_theta_lo"] < x0[2] < C["v_theta_hi"]
    # target ellipse: perigee and apogee radii, and its speeds, from the vis-viva
    # and angular-momentum relations
    a, e = C["target_a"], C["target_e"]
    rp, ra = a * (1.0 - e), a * (1.0 + e)
    p_semi = a * (1.0 - e * e)
    h = math.sqrt(mu * p_semi)
    assert C["rho_lo"] < rp < ra < C["rho_hi"]
    # v_theta = h / rho is largest at perigee, smallest at apogee
    assert C["v_theta_lo"] < h / ra < h / rp < C["v_theta_hi"]
    # the largest radial speed on the ellipse is e sqrt(mu / p)
    assert e * math.sqrt(mu / p_semi) < C["v_rho_hi"]
    # the start orbit lies below the target orbit's perigee: a raising manoeuvre
    assert x0[0] < rp
    nu = np.linspace(0.0, 2.0 * math.pi, 73)
    rho = p_semi / (1.0 + e * np.cos(nu))
    assert np.all((rho > C["rho_lo"]) & (rho < C["rho_hi"]))
