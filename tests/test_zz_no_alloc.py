"""dp_bellman_sweep_noalloc: the sweep for callers that cannot allocate device
memory (real-time code that forbids allocation after start-up, or hosts whose
device memory belongs to another allocator).  Its output must match the
allocating entry point's, dp_bellman_sweep on a grid, on two calls in a row.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2407_14675_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cases(dp):
    yield W.config0(), [dp.DP_SWEEP_VI, dp.DP_SWEEP_VI], 1e-9
    # FP64 improvement and evaluation (the grid entry point evaluates from
    # the feet its improvement stored; this call recomputes them)
    yield W.config0(), [dp.DP_SWEEP_IMPROVE_WALK, dp.DP_SWEEP_EVAL], 1e-9
    yield W.config0(), [dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_EVAL], 1e-9
    # the paper's Example 1 dynamics (periodic angle, running cost, thrust off)
    yield W.example1(n=(9, 7, 7, 8)), [dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_EVAL], 1e-9
    yield W.config1(n=17), [dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_EVAL], 1e-4
    yield W.config1(n=17), [dp.DP_SWEEP_IMPROVE_WALK, dp.DP_SWEEP_IMPROVE_WALK], 1e-4


def _compare(dp, p, modes, tol):
    """Runs `modes` on a grid and through the no-allocation call from the same
    value and policy, and compares every sweep's value, residual and codes."""
    import torch
    V0 = W.smooth_value(p, 71)
    codes0 = W.random_codes(p, 72)
    # reference: the allocating entry point on a grid
    ref = []
    with dp.Grid(p) as g:
        g.set_value(V0)
        g.set_policy(codes0)
        V_start = g.get_value()          # target nodes zeroed
        for m in modes:
            r = g.sweep(m)
            ref.append((g.get_value(), g.get_policy(), r))
    # caller-owned device buffers, no library allocation
    dt = torch.float64 if p.precision == W.FP64 else torch.float32
    a = torch.tensor(V_start, dtype=dt, device="cuda")
    b = torch.empty_like(a)
    c = torch.tensor(codes0.view(np.int16), dtype=torch.int16, device="cuda")
    desc = dp.desc_from_problem(p, stream=int(torch.cuda.current_stream().cuda_stream))
    for k, m in enumerate(modes):
        r = dp.dp_bellman_sweep_noalloc(desc, m, a.data_ptr(), b.data_ptr(), c.data_ptr())
        v_ref, c_ref, r_ref = ref[k]
        got = b.double().cpu().numpy()
        err = np.abs(got - v_ref).max()
        assert err <= tol * np.abs(v_ref).max(), (p.n, m, k, err)
        assert abs(r - r_ref) <= tol * np.abs(v_ref).max()
        if m != dp.DP_SWEEP_VI:
            assert (c.cpu().numpy().view(np.uint16) == c_ref).mean() > 0.999
        a, b = b, a


def test_noalloc_sweep_matches_grid_sweep_twice(dp):
    for p, modes, tol in _cases(dp):
        _compare(dp, p, modes, tol)


def test_noalloc_at_its_size_bound_then_a_smaller_grid(dp):
    """The largest grid the fixed scratch holds (n0 n1 = 4096, n0 n1 n2 =
    262144), then a smaller one: the tables the calls share must carry
    nothing over from the larger grid."""
    big = W.config1(n=17).replace(n=(64, 64, 64, 4), lo=(0.95, -0.10, 0.85, 0.97))
    _compare(dp, big, [dp.DP_SWEEP_IMPROVE_FULL, dp.DP_SWEEP_EVAL], 1e-4)
    _compare(dp, W.config1(n=17), [dp.DP_SWEEP_IMPROVE_WALK, dp.DP_SWEEP_EVAL], 1e-4)
    _compare(dp, W.config0(), [dp.DP_SWEEP_VI, dp.DP_SWEEP_VI], 1e-9)


def test_noalloc_rejects_what_it_cannot_hold(dp):
    import torch
    a = torch.zeros(16, device="cuda", dtype=torch.float64)
    b = torch.zeros(16, device="cuda", dtype=torch.float64)
    big = W.config1(n=121)                   # 121^3 lines > 262144
    with pytest.raises(dp.DPError) as e:
        dp.dp_bellman_sweep_noalloc(dp.desc_from_problem(big), dp.DP_SWEEP_VI, a.data_ptr(), b.data_ptr())
    assert e.value.code == dp.DP_EINVAL and "too large" in str(e.value)
    red = W.config2(n=9)
    with pytest.raises(dp.DPError) as e:
        dp.dp_bellman_sweep_noalloc(dp.desc_from_problem(red), dp.DP_SWEEP_VI, a.data_ptr(), b.data_ptr())
    assert e.value.code == dp.DP_EINVAL
    with pytest.raises(dp.DPError) as e:
        dp.dp_bellman_sweep_noalloc(dp.desc_from_problem(W.config0()), dp.DP_SWEEP_VI, a.data_ptr(), a.data_ptr())
    assert e.value.code == dp.DP_EINVAL
