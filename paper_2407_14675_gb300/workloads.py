"""Seeded synthetic workloads for the planar low-thrust transfer problem.

This module holds problem descriptions (grid boxes, physical constants,
solver settings) and seeded random generators for inputs: initial value
fields, closed-loop initial states and batches of transfers.  It contains
none of the scheme's arithmetic (no dynamics, interpolation or Bellman
update); both the CUDA path and the CPU oracle take their inputs from here.

Problem setting: the polar form of the planar two-body dynamics of §3
("Grid and polar coordinates") with the angle coordinate dropped and the
mass added as a state, minimum-time cost (running cost 1) and a box-shaped
target around a circular orbit.  All quantities are nondimensional (mu = 1,
initial radius 1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

DYN_ORBIT = 0        # (r, v_r, v_t, m) planar orbit dynamics with mass flow
DYN_UNIT_SPEED = 1   # test dynamics x' = (cos a, sin a, 0, 0)
DYN_POLAR = 2        # (rho, v_rho, v_theta, theta), theta periodic, no mass (the paper's Example 1)

FP64 = 0
FP32 = 1


@dataclasses.dataclass
class Problem:
    """One grid + dynamics + target + control-set description."""
    n: tuple = (17, 17, 17, 17)
    lo: tuple = (0.95, -0.10, 0.85, 0.90)
    hi: tuple = (1.15, 0.10, 1.10, 1.00)
    dynamics: int = DYN_ORBIT
    mu: float = 1.0
    accel: float = 1e-3
    exhaust_c: float = 1.0
    dt: float = 0.05
    beta: float = 0.999
    penalty_M: float = 0.0          # <= 0: default dt / (1 - beta)
    target_c: tuple = (1.05, 0.0, 1.0 / math.sqrt(1.05), 0.0)
    target_w: tuple = (0.005, 0.005, 0.005, 0.0)   # open box, w <= 0: any value
    n_angles: int = 16
    refine: int = 0                 # golden-section refinement on/off
    refine_tol: float = 1e-4        # rad
    reduced: int = 0                # energy-band reduced grid
    energy_lo: float = 0.0
    energy_hi: float = 0.0
    precision: int = FP64
    # Example 1 (DYN_POLAR): thrust-off control and the running cost of Eq. (11)
    off_control: int = 0
    cost_alpha: float = 0.0
    cost_beta: float = 0.0
    cost_gamma: float = 0.0
    a_bar: float = 0.0
    e_bar: float = 0.0
    omega_bar: float = 0.0
    # solver settings (not part of the grid)
    tol: float = 1e-8
    n_eval: int = 20

    @property
    def nodes(self) -> int:
        return int(np.prod(self.n))

    def M(self) -> float:
        return self.penalty_M if self.penalty_M > 0 else self.dt / (1.0 - self.beta)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def circular_target(r_T: float, tol: float = 0.005, mu: float = 1.0):
    """Target box around the circular orbit of radius r_T (all masses)."""
    return (r_T, 0.0, math.sqrt(mu / r_T), 0.0), (tol, tol, tol, 0.0)


def energy_band(r0: float, r_T: float, margin: float = 0.02, mu: float = 1.0):
    """Specific-energy band between the initial and target circular orbits."""
    return -mu / (2.0 * r0) - margin, -mu / (2.0 * r_T) + margin


# --- the five configurations -------------------------------------------------

def config0() -> Problem:
    """17^4, FP64 value iteration, 16 angles, a = 1e-3, dt = 0.05, tol 1e-8."""
    return Problem()


def config1(n: int = 61) -> Problem:
    """61^4, FP32 modified policy iteration, 64 angles + golden, a = 2e-4."""
    return Problem(n=(n, n, n, n), accel=2e-4, dt=0.02, n_angles=64, refine=1,
                   precision=FP32, tol=1e-6, n_eval=20)


def config2(n: int = 121) -> Problem:
    """121^4 box reduced to the energy band, config-1 dynamics."""
    e_lo, e_hi = energy_band(1.0, 1.05)
    return config1(n).replace(reduced=1, energy_lo=e_lo, energy_hi=e_hi)


MU_EARTH = 398600.4   # km^3 / s^2, the Earth's gravitational parameter as the paper prints it (§2.1)


def example1(n=(110, 30, 30, 30), accel: float = 5e-7) -> Problem:
    """The paper's Example 1 (§4): target orbit a = 7000 km, e = 0.001, argument
    of perigee 0; thrust acceleration 5e-7 km/s^2; cost weights alpha = 2.04e-8,
    beta = 2.31e-2, gamma = 1.5; lambda = 1e-3 (discount exp(-lambda dt));
    dt = 10 s; rho in [6930, 7070] km, v_rho in [-0.01, 0.01] km/s, v_theta in
    [7.526, 7.566] km/s, theta in [0, 2 pi) periodic; 72 angles + thrust off.
    State order (rho, v_rho, v_theta, theta); n gives the nodes in that order
    (the paper's 110 x 30 x 30 x 30).  No target set (V > 0 everywhere)."""
    nt = n[3]
    dt, lam = 10.0, 1e-3
    beta = math.exp(-lam * dt)
    lo = (6930.0, -0.01, 7.526, 0.0)
    hi = (7070.0, 0.01, 7.566, 2.0 * math.pi * (nt - 1) / nt)
    a_bar, e_bar = 7000.0, 0.001
    # M: the discounted cost of staying forever on the worst circular orbit of
    # the box (rho at a bound, e = 0).  Larger values (the worst box corner,
    # a - a_bar ~ 180 km) spread the penalty of the velocity bounds into the
    # interior through the interpolation and stall the closed loop.
    worst = max(abs(lo[0] - a_bar), abs(hi[0] - a_bar))
    M = dt * (2.31e-2 * worst ** 2 + 1.5 * e_bar ** 2) / (1.0 - beta)
    return Problem(n=tuple(n), lo=lo, hi=hi, dynamics=DYN_POLAR, mu=MU_EARTH, accel=accel, exhaust_c=1.0,
                   dt=dt, beta=beta, penalty_M=M, target_c=(-1.0, 0.0, 0.0, 0.0), target_w=(1e-9, 0.0, 0.0, 0.0),
                   n_angles=72, refine=1, refine_tol=1e-4, precision=FP64, tol=1e-7, n_eval=20,
                   off_control=1, cost_alpha=2.04e-8, cost_beta=2.31e-2, cost_gamma=1.5,
                   a_bar=a_bar, e_bar=e_bar, omega_bar=0.0)


def example2_drag(cd: float = 2.2, area_m2: float = 2.25, mass_kg: float = 350.0,
                  density_kg_m3: float = 8.09e-14) -> float:
    """Drag coefficient C of the paper's Example 2 (§4), C = C_D S rho_D / (2 m),
    in 1/km so that -C v^2 is in km/s^2 with v in km/s."""
    c_per_m = cd * area_m2 * density_kg_m3 / (2.0 * mass_kg)
    return c_per_m * 1000.0


def example1_start(r0: float = 6978.0) -> np.ndarray:
    """Circular orbit of radius r0 km at theta = 0 (the paper's start)."""
    return np.array([r0, 0.0, math.sqrt(MU_EARTH / r0), 0.0])


def unit_speed_1d(n: int = 17, beta: float = 0.95, target_node: int = 8) -> Problem:
    """1-D minimum time with x' = cos a, a in {0, pi}, dt = h: feet land on nodes."""
    h = 1.0 / (n - 1)
    xt = 1.0 + target_node * h
    return Problem(n=(n, 2, 2, 2), lo=(1.0, 1.0, 1.0, 1.0), hi=(2.0, 2.0, 2.0, 2.0),
                   dynamics=DYN_UNIT_SPEED, dt=h, beta=beta,
                   target_c=(xt, 0.0, 0.0, 0.0), target_w=(0.25 * h, 0.0, 0.0, 0.0),
                   n_angles=2, refine=0, precision=FP64, tol=1e-12)


def unit_speed_2d(n: int = 13, beta: float = 0.97, target=(6, 4), n_angles: int = 4) -> Problem:
    """2-D minimum time with x' = (cos a, sin a), dt = h."""
    h = 1.0 / (n - 1)
    c = (1.0 + target[0] * h, 1.0 + target[1] * h, 0.0, 0.0)
    return Problem(n=(n, n, 2, 2), lo=(1.0, 1.0, 1.0, 1.0), hi=(2.0, 2.0, 2.0, 2.0),
                   dynamics=DYN_UNIT_SPEED, dt=h, beta=beta,
                   target_c=c, target_w=(0.25 * h, 0.25 * h, 0.0, 0.0),
                   n_angles=n_angles, refine=0, precision=FP64, tol=1e-12)


# --- seeded inputs -----------------------------------------------------------

def random_value(p: Problem, seed: int, lo: float = 0.0, hi: Optional[float] = None) -> np.ndarray:
    """Uniform random V over the full box (float64), in [lo, hi] (default [0, M])."""
    rng = np.random.default_rng(seed)
    hi = p.M() if hi is None else hi
    return rng.uniform(lo, hi, size=p.nodes)


def smooth_value(p: Problem, seed: int) -> np.ndarray:
    """A smooth random field over the box with values in (0, M): a sum of a few
    low-frequency cosines, used where a rough uniform field would make every
    control choice a near-tie."""
    rng = np.random.default_rng(seed)
    axes = [np.linspace(0.0, 1.0, k) for k in p.n]
    f = np.zeros(p.n)
    for _ in range(6):
        k = rng.uniform(0.5, 2.5, size=4)
        ph = rng.uniform(0, 2 * np.pi, size=4)
        a = rng.uniform(0.2, 1.0)
        term = a
        for d in range(4):
            # one axis at a time, broadcast (no full-size coordinate arrays)
            shape = [1, 1, 1, 1]
            shape[d] = p.n[d]
            term = term * np.cos(np.pi * k[d] * axes[d] + ph[d]).reshape(shape)
        f = f + term
    f = (f - f.min()) / (f.max() - f.min() + 1e-300)
    return (0.05 + 0.9 * f).reshape(-1) * p.M()


def random_codes(p: Problem, seed: int) -> np.ndarray:
    """Uniform random 16-bit angle codes per node (a frozen policy)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 65536, size=p.nodes, dtype=np.uint16)


def closed_loop_states(p: Problem, count: int, seed: int = 2407,
                       band: Optional[tuple] = None) -> np.ndarray:
    """Initial states uniform over the box minus the target, optionally kept
    only where the specific energy lies in `band` (rejection sampling).  Shape
    (count, 4), float64."""
    rng = np.random.default_rng(seed)
    lo = np.array(p.lo)
    hi = np.array(p.hi)
    c = np.array(p.target_c)
    w = np.array(p.target_w)
    out = []
    while sum(len(o) for o in out) < count:
        x = lo + (hi - lo) * rng.uniform(size=(4 * count, 4))
        in_t = np.ones(len(x), bool)
        for d in range(4):
            if w[d] > 0:
                in_t &= np.abs(x[:, d] - c[d]) < w[d]
        keep = ~in_t
        if band is not None:
            e = 0.5 * (x[:, 1] ** 2 + x[:, 2] ** 2) - p.mu / x[:, 0]
            keep &= (e >= band[0]) & (e <= band[1])
        out.append(x[keep])
    return np.concatenate(out)[:count].copy()


def transfer_start(r0: float = 1.0, m0: float = 1.0, mu: float = 1.0) -> np.ndarray:
    """State on the circular orbit of radius r0 with mass m0."""
    return np.array([r0, 0.0, math.sqrt(mu / r0), m0])


def batch_transfers(count: int = 256, seed: int = 14675, sizes=(17, 21, 25, 31, 41)) -> List[Problem]:
    """Heterogeneous batch: per-dimension sizes from `sizes`, thrust
    log-uniform in [1e-4, 2e-3], target radius U[1.02, 1.10], initial radius
    U[0.98, 1.02]; box r in [r0 - 0.05, r_T + 0.10], v_r, v_t, m as config 0;
    32 angles with golden refinement, FP32, dt 0.05, beta 0.999."""
    rng = np.random.default_rng(seed)
    sizes = np.array(sizes)
    out = []
    for _ in range(count):
        n = tuple(int(s) for s in rng.choice(sizes, size=4))
        a = float(np.exp(rng.uniform(np.log(1e-4), np.log(2e-3))))
        r_T = float(rng.uniform(1.02, 1.10))
        r0 = float(rng.uniform(0.98, 1.02))
        c, w = circular_target(r_T)
        out.append(Problem(n=n, lo=(r0 - 0.05, -0.10, 0.85, 0.90), hi=(r_T + 0.10, 0.10, 1.10, 1.00),
                           accel=a, dt=0.05, n_angles=32, refine=1, precision=FP32,
                           target_c=c, target_w=w, tol=1e-6, n_eval=20))
    return out


def mlp_init_params(seed: int = 14675, sizes=(4, 256, 256, 256, 3)):
    """Initial weights of the warm-start network: per layer [W, b] with W of
    shape (fan_out, fan_in) and every entry uniform in +-1/sqrt(fan_in)."""
    rng = np.random.default_rng(seed)
    params = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        bound = 1.0 / math.sqrt(fi)
        params.append([rng.uniform(-bound, bound, size=(fo, fi)), rng.uniform(-bound, bound, size=fo)])
    return params
