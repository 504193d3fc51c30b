#!/usr/bin/env python
"""Benchmark: Bellman node-updates/s of modified policy iteration on the
121^4 energy-band reduced grid (55,976,052 stored nodes; FP32 sweeps, FP64
residual), the largest single-GPU configuration of the workload set.

One step = one outer iteration of modified policy iteration: an improvement
sweep (local walk from the previous optimum + golden-section refinement over
64 tabulated angles) followed by 20 Jacobi policy-evaluation sweeps, over the
stored nodes resident in HBM.  value = node updates / device time.  The e2e
figure runs the same step through the C ABI with host buffers: the value
(FP64) and the policy go up from pinned host memory and come back every step.
The same step on the 61^4 full box is reported as step_61x4.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
step (there is no reference implementation of this method to run).

Multi-GPU: the grid does not shard ("replicas only"): every rank
solves its own copy, value = all ranks' node updates / the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Bellman node-updates/s; time to ‖ΔV‖∞<1e-6, plain vs NN-warm-started"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the frozen-feet evaluation sweep, from one ncu capture per workload, with a
# hash of the kernel sources they were taken on: a capture of an older kernel
# is reported as stale (traffic null) instead of silently.
EVAL_TRAFFIC = {
    "61x4": {"bytes": (166.166528e6 + 18.204672e6 + 166.231552e6 + 14.960896e6) / 2, "src": "75c6a83c8a18675f"},
    "121x4_band": {"bytes": (678.591232e6 + 191.108608e6 + 677.034496e6 + 187.774976e6) / 2, "src": "75c6a83c8a18675f"},
}
KERNEL_SOURCES = ("paper_2407_14675_gb300/csrc/dp_sweep.cuh", "paper_2407_14675_gb300/csrc/dp_device.cuh")
UNIT = "node-updates/s"
L2_BYTES = 129 * 2 ** 20


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def kernel_src_hash():
    """Hash of the sources of the sweep kernels (first 16 hex digits)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(key):
    rec = EVAL_TRAFFIC.get(key) or {}
    if rec.get("bytes") is None:
        return None, "not captured for this kernel"
    if rec.get("src") != kernel_src_hash():
        return None, "stale: the kernel sources changed since the ncu capture"
    return rec["bytes"], ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel, mean of two launches "
                          "(kernel sources %s)" % rec["src"])


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    return world, rank, local


def _reduce(x, world, op):
    """All-reduce of one float over the ranks (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return float(t.item())


def _reduce_max(x, world):
    return _reduce(x, world, "max")


def _reduce_sum(x, world):
    return _reduce(x, world, "sum")


def aggregate_replicas(updates, ms, world):
    """Whole-job throughput of independent replicas: every rank's node updates
    over the slowest rank's time.  Returns (value, slowest ms)."""
    ms_max = _reduce_max(ms, world)
    return _reduce_sum(float(updates), world) / (ms_max / 1e3), ms_max


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- CPU oracle --

class OracleSample:
    """The FP64 oracle on a seeded sample of one grid's stored nodes, with a
    seeded smooth value function (built once: for the 121^4 band the box
    holds 214M nodes)."""

    def __init__(self, p, seed=2407, n_imp=2000):
        import oracle
        from paper_2407_14675_gb300 import workloads as W
        self.o = oracle.Oracle(p)
        self.p = p
        self.V = W.smooth_value(p, seed)
        self.V[self.o.target.astype(bool)] = 0
        rng = np.random.default_rng(seed)
        free = np.flatnonzero((self.o.active & ~self.o.target).astype(bool))
        self.nodes = np.sort(rng.choice(free, n_imp, replace=False))
        # previous optimum for the walk: the oracle's own full tabulation (untimed)
        _, self.start = self.o.bellman_nodes(self.V, self.nodes, mode=oracle.IMPROVE_FULL)

    def step_rate(self, seconds_target=12.0):
        """Node-updates/s for the step's mix: one walk improvement and n_eval
        evaluation sweeps at the sampled nodes, repeated to about
        seconds_target of single-thread CPU time."""
        import oracle
        o, V, nodes, start, p = self.o, self.V, self.nodes, self.start, self.p
        t0 = time.perf_counter()
        o.bellman_nodes(V, nodes, mode=oracle.IMPROVE_WALK, codes=start)
        for _e in range(p.n_eval):
            o.bellman_nodes(V, nodes, mode=oracle.EVAL, codes=start)
        once = time.perf_counter() - t0
        reps = max(1, int(seconds_target / max(once, 1e-9)))
        t0 = time.perf_counter()
        for _ in range(reps):
            o.bellman_nodes(V, nodes, mode=oracle.IMPROVE_WALK, codes=start)
            for _e in range(p.n_eval):
                o.bellman_nodes(V, nodes, mode=oracle.EVAL, codes=start)
        wall = time.perf_counter() - t0
        updates = reps * len(nodes) * (1 + p.n_eval)
        return updates / wall, {"nodes": len(nodes), "reps": reps, "seconds": wall, "updates": updates}


def _oracle_worker(task):
    """One process of the all-cores oracle baseline (spawned): the single
    thread measurement on its own seeded node sample, for a fixed time."""
    seed, seconds, n = task
    from paper_2407_14675_gb300 import workloads as W
    rate, info = OracleSample(W.config2(n=n), seed=seed).step_rate(seconds)
    return info["updates"], info["seconds"]


def oracle_parallel_rate(seconds_target=10.0, procs=None, n=121):
    """The oracle on the host cores: one spawned process per core (each holds
    the band's 214M-node box value, 1.7 GB, so at most one per 3 GB of free
    host memory), each on its own sample of the same step mix.  Aggregate
    node-updates / the slowest process's time."""
    import multiprocessing as mp
    if not procs:
        try:
            free_gb = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 2 ** 30
        except (ValueError, OSError, AttributeError):
            free_gb = 24.0
        procs = max(1, min(os.cpu_count() or 1, 64, int(free_gb // 3)))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(2407 + 97 * k, seconds_target, n) for k in range(procs)])
    updates = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return updates / wall, {"procs": procs, "seconds": wall, "updates": updates}


def run_reference(args, world, rank):
    from paper_2407_14675_gb300 import workloads as W
    if rank != 0:
        return 0
    p = W.config2()
    sample = OracleSample(p)
    steps = []
    for _ in range(args.warmup):
        sample.step_rate(seconds_target=2.0)
    for _ in range(args.steps):
        r, info = sample.step_rate(seconds_target=max(2.0, 20.0 / max(args.steps, 1)))
        steps.append((r, info))
    rate = float(np.mean([s[0] for s in steps]))
    n_upd = int(sample.o.n_active - int(sample.o.target.sum()))
    ms_step = (1 + p.n_eval) * n_upd / rate * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(p, n_upd),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: %d sampled stored nodes of the 121^4 band x (1 walk improvement + %d "
                                   "evaluations), repeated to ~%.0f s, FP64 single thread" %
                                   (steps[0][1]["nodes"], p.n_eval, steps[0][1]["seconds"])},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(p, n_upd=None):
    band = bool(p.reduced)
    d = {"workload": ("121^4 box reduced to the energy band [%.4f, %.4f] (55,976,052 stored nodes), minimum-time "
                      "orbit transfer (r, v_r, v_t, m), FP32 modified policy iteration with FP64 residual: "
                      "1 walk+golden improvement (64 angles) + 20 evaluation sweeps per step" % (p.energy_lo, p.energy_hi)
                      if band else
                      "%d^4 minimum-time orbit transfer (r, v_r, v_t, m), FP32 modified policy iteration: "
                      "1 walk+golden improvement (64 angles) + 20 evaluation sweeps per step" % p.n[0]),
         "grid": list(p.n), "box_nodes": p.nodes, "n_angles": p.n_angles, "n_eval": p.n_eval,
         "accel": p.accel, "dt": p.dt, "beta": p.beta,
         "l2": ("flushed before the timed steps (256 MiB write); every sweep streams %s > 129 MB of L2" %
                ("1.12 GB" if band else "276 MB"))}
    if n_upd is not None:
        d["node_updates_per_sweep"] = int(n_upd)
    return d


# ------------------------------------------------------------------ GPU arm --

def extra_legs(args, dp, W, torch, g1, p1):
    """FP64 value iteration on the 17^4 grid to 1e-8, and the walk against
    full tabulation in every improvement on the 61^4 cold solve (the paper
    reports about +20 % total time for exhaustive search)."""
    out = {}
    p0 = W.config0()
    st = int(torch.cuda.current_stream().cuda_stream)
    with dp.Grid(p0, stream=st) as g0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, s0 = g0.value_iterate(tol=1e-8, max_sweeps=40000)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        out["vi_fp64_17x4"] = {"seconds": secs, "converged": bool(s0.converged), "sweeps": s0.sweeps_vi,
                               "residual": s0.residual, "node_updates_per_s": s0.node_updates / secs}
        # the same with each sweep solving the node's own coefficient
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, s0 = g0.value_iterate(tol=1e-8, max_sweeps=40000, eval_solver=dp.DP_EVAL_DIAG)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        out["vi_diag_fp64_17x4"] = {"seconds": secs, "converged": bool(s0.converged), "sweeps": s0.sweeps_vi,
                                    "residual": s0.residual, "speedup": out["vi_fp64_17x4"]["seconds"] / secs}
        # FP64 policy iteration on the same grid, each policy evaluated by 20
        # Jacobi sweeps or by GMRES
        pi = {}
        for name, kw in (("jacobi20", {"n_eval": 20}),
                         ("gmres", {"eval_solver": dp.DP_EVAL_GMRES, "gmres_restart": args.gmres_restart_fp64}),
                         ("diag", {"eval_solver": dp.DP_EVAL_DIAG, "n_eval": args.diag_n_eval})):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, s0 = g0.policy_iterate(tol=1e-8, max_sweeps=args.solve_max, polish=0, **kw)
            torch.cuda.synchronize()
            pi[name] = {"seconds": time.perf_counter() - t0, "converged": bool(s0.converged),
                        "improvements": s0.sweeps_improve, "evaluation_sweeps": s0.sweeps_eval,
                        "matvecs": s0.gmres_matvecs}
        out["pi_fp64_17x4"] = pi
    res = {}
    for walk in (1, 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, s1 = g1.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=p1.n_eval, polish=1, warm=0,
                                   walk=walk)
        torch.cuda.synchronize()
        res["walk" if walk else "full_table"] = {
            "seconds": time.perf_counter() - t0, "converged": bool(s1.converged),
            "improvements": s1.sweeps_improve + s1.sweeps_improve_fp64}
    res["full_over_walk"] = res["full_table"]["seconds"] / max(res["walk"]["seconds"], 1e-9)
    out["walk_vs_full_61x4"] = res
    return out


def _kepler_a_e(x, mu):
    """Semi-major axis and eccentricity of a polar state (rho, v_rho, v_theta,
    theta), for reporting the closed loop (vis-viva; eccentricity vector)."""
    r, vr, vt = x[0], x[1], x[2]
    a = mu * r / (2.0 * mu - r * (vr * vr + vt * vt))
    er, et = r * vt * vt / mu - 1.0, -r * vr * vt / mu
    return a, math.hypot(er, et)


def example1_leg(args, dp, W, torch):
    """The paper's Example 1 (§4): 110 x 30 x 30 x 30 polar grid, running cost
    of Eq. (11), 72 angles + thrust off, FP64 policy iteration to 1e-7, with
    each policy evaluated by 20 plain evaluation sweeps, by GMRES (the paper's
    method) and by diagonal-solved Jacobi iterations; then the closed loop
    (on the last solution) from the circular orbit at
    6978 km for 1e6 s, sampled every 2,000 s: when the semi-major axis comes
    within 1 km of 7000 km, when the thrust switches off for good, and the
    final orbit; and the same on the system with drag of Example 2."""
    p = W.example1()
    out = {"grid": list(p.n), "nodes": p.nodes, "dt_s": p.dt, "tol": p.tol}
    st = int(torch.cuda.current_stream().cuda_stream)
    with dp.Grid(p, stream=st) as g:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, s = g.policy_iterate(tol=p.tol, max_sweeps=args.solve_max, n_eval=p.n_eval, polish=0)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        out["solve_jacobi"] = {"seconds": secs, "converged": bool(s.converged), "residual": s.residual,
                               "improvements": s.sweeps_improve, "evaluation_sweeps": s.sweeps_eval,
                               "node_updates_per_s": s.node_updates / secs}
        v_jacobi = g.get_value()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, s = g.policy_iterate(tol=p.tol, max_sweeps=args.solve_max, polish=0, eval_solver=dp.DP_EVAL_GMRES,
                                 gmres_restart=args.gmres_restart_fp64)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        v = g.get_value()
        out["solve"] = {"seconds": secs, "converged": bool(s.converged), "residual": s.residual,
                        "evaluation": "GMRES(%d)" % args.gmres_restart_fp64, "improvements": s.sweeps_improve,
                        "gmres_cycles": s.gmres_cycles, "matvecs": s.gmres_matvecs,
                        "max_rel_diff_to_jacobi_solution": float(np.abs(v - v_jacobi).max() / np.abs(v_jacobi).max()),
                        "speedup_over_jacobi": out["solve_jacobi"]["seconds"] / secs}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, s = g.policy_iterate(tol=p.tol, max_sweeps=args.solve_max, polish=0, eval_solver=dp.DP_EVAL_DIAG,
                                 n_eval=args.diag_n_eval)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        v = g.get_value()
        out["solve_diag"] = {"seconds": secs, "converged": bool(s.converged), "residual": s.residual,
                             "evaluation": "diagonal-solved Jacobi, %d per improvement" % args.diag_n_eval,
                             "improvements": s.sweeps_improve, "evaluation_sweeps": s.sweeps_eval,
                             "max_rel_diff_to_jacobi_solution": float(np.abs(v - v_jacobi).max() /
                                                                      np.abs(v_jacobi).max()),
                             "speedup_over_jacobi": out["solve_jacobi"]["seconds"] / secs}
        for name, drag in (("closed_loop", 0.0), ("closed_loop_with_drag", W.example2_drag())):
            # Example 2 of §4: the same feedback flown on a system with drag
            y = W.example1_start(6978.0)[None, :]
            chunk, horizon = 2000.0, 1.0e6
            t, t_near, t_last_on, worst_after = 0.0, None, None, 0.0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while t < horizon:
                alpha, _ = g.feedback(y, p.dt)
                if not np.isnan(alpha[0]):
                    t_last_on = t
                ta, y = g.simulate(y, p.dt, p.dt, chunk, drag=drag)
                t += chunk
                a, e = _kepler_a_e(y[0], p.mu)
                if t_near is None and abs(a - p.a_bar) < 1.0:
                    t_near = t
                if t_near is not None:
                    worst_after = max(worst_after, abs(a - p.a_bar))
            a, e = _kepler_a_e(y[0], p.mu)
            out[name] = {"seconds": time.perf_counter() - t0, "horizon_s": horizon, "drag_c_per_km": drag,
                         "time_a_within_1km_s": t_near, "last_thrust_on_s": t_last_on,
                         "max_a_err_after_km": worst_after, "final_a_err_km": a - p.a_bar, "final_e": e}
        out["paper"] = ("target neighbourhood after ~1e5 s, thrust off after ~5e5 s, radius error ~1e-2 km; "
                        "with drag, later adjustment manoeuvres (CPU Matlab: ~18 min for the value function)")
    return out


def batch_leg(args, dp, W, torch):
    """Batched transfers: the 256-transfer batch solved to 1e-6 in one set of
    graph-replayed persistent launches (plain and diagonal-solved
    evaluation), the evaluation sweep's HBM roofline,
    and, on a sample of the same transfers, the batched FP32 solve against
    plain FP64 policy iteration of each transfer on its own grid."""
    probs = W.batch_transfers(count=args.batch_count)
    out = {"transfers": len(probs)}
    peaks, _ = _peaks()
    with dp.Batch(probs) as b:
        info = b.info()
        out["nodes"] = info["nodes_total"]
        ie, ii = b.autotune()
        out["items"] = {"eval": ie, "improve": ii}
        b.sweep(dp.DP_SWEEP_IMPROVE_FULL)
        b.sweep(dp.DP_SWEEP_IMPROVE_WALK)
        ms_e = []
        flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
        for _ in range(6):
            flush.zero_()
            ms_e.append(b.sweep(dp.DP_SWEEP_EVAL)[1])
        r, ms_w = b.sweep(dp.DP_SWEEP_IMPROVE_WALK)
        n_upd = info["nodes_total"] - info["nodes_target"]
        ms_eval = float(np.median(ms_e[1:]))
        ach = 10.0 * n_upd / (ms_eval / 1e3) / 1e9
        out["eval_sweep"] = {"ms": ms_eval, "node_updates_per_s": n_upd / (ms_eval / 1e3),
                             "achieved_gbs": ach, "frac_of_hbm": ach / float(peaks.get("hbm_gbs", 6800.0))}
        out["walk_sweep"] = {"ms": ms_w, "node_updates_per_s": n_upd / (ms_w / 1e3)}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, tot, per = b.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=20, polish=1)
        secs = time.perf_counter() - t0
        imp = np.array([q["sweeps_improve"] + q["sweeps_improve_fp64"] for q in per])
        out["solve"] = {"seconds": secs, "converged": int(sum(q["converged"] for q in per)),
                        "node_updates": tot.node_updates, "node_updates_per_s": tot.node_updates / secs,
                        "launches": tot.launches, "max_residual": tot.residual,
                        "improvements_per_transfer": {"min": int(imp.min()), "median": float(np.median(imp)),
                                                      "max": int(imp.max())}}
        # the same solve with the diagonal-solved evaluation
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, tot, per = b.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=args.diag_n_eval, polish=1,
                                        eval_solver=dp.DP_EVAL_DIAG)
        secs = time.perf_counter() - t0
        imp = np.array([q["sweeps_improve"] + q["sweeps_improve_fp64"] for q in per])
        out["solve_diag"] = {"seconds": secs, "converged": int(sum(q["converged"] for q in per)),
                             "n_eval": args.diag_n_eval, "max_residual": tot.residual,
                             "improvements_per_transfer": {"min": int(imp.min()), "median": float(np.median(imp)),
                                                           "max": int(imp.max())},
                             "speedup_over_sweeps": out["solve"]["seconds"] / secs}
    # the same transfers, sampled: batched FP32 vs plain FP64 per grid
    pick = [int(i) for i in np.linspace(0, len(probs) - 1, args.batch_fp64_sample)]
    sample = [probs[i] for i in pick]
    with dp.Batch(sample) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, tot, per = b.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=20, polish=1)
        t_b = time.perf_counter() - t0
    t_64, conv64 = 0.0, 0
    for q in sample:
        with dp.Grid(q.replace(precision=W.FP64), stream=int(torch.cuda.current_stream().cuda_stream)) as g:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, s = g.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=20)
            torch.cuda.synchronize()
            t_64 += time.perf_counter() - t0
            conv64 += int(s.converged)
    out["vs_fp64_sample"] = {"transfers": pick, "batched_fp32_seconds": t_b,
                             "batched_fp32_converged": int(tot.converged),
                             "plain_fp64_seconds": t_64, "plain_fp64_converged": conv64,
                             "speedup": t_64 / max(t_b, 1e-9)}
    return out


def warm_start_leg(args, dp, W, torch, g1, p1, g2):
    """Learned warm start: train the network on the converged 61^4 solve
    (every stored node), then solve the 121^4 energy-band grid to 1e-6 from
    V = 0, from the network's V and policy, and from the 61^4 solution, with
    the configured evaluation sweeps and with the diagonal-solved ones;
    closed loop from 1024 seeded states on the last solution."""
    p2 = W.config2()
    out = {"grid": "121^4 box, energy band [%.4f, %.4f]" % (p2.energy_lo, p2.energy_hi)}
    with dp.Mlp(p1.lo, p1.hi, batch_capacity=262144) as net:
        dp.dp_mlp_set_params(net.h, dp.flatten_params(W.mlp_init_params()))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = dp.dp_mlp_train_grid(net.h, g1.h, epochs=args.mlp_epochs, batch=16384, lr=4e-3, lr_final=1e-3)
        torch.cuda.synchronize()
        tr = st.asdict()
        tr["wall_s"] = time.perf_counter() - t0
        tr["tflops_nominal"] = st.flops / max(st.ms, 1e-9) / 1e9
        out["train"] = tr
        out["nodes_active"] = g2.info["n_active"]
        V_cold = None
        # each start with the configured 20 evaluation sweeps per improvement,
        # then again with the diagonal-solved evaluation
        tuned = "_diag"
        runs = [(k, p2.n_eval, dp.DP_EVAL_JACOBI) for k in ("cold", "warm", "from_61x4_grid")]
        runs += [(k + tuned, args.diag_n_eval, dp.DP_EVAL_DIAG) for k in ("cold", "warm", "from_61x4_grid")]
        for start, n_eval, solver in runs:
            kind = start.split("_diag")[0]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ws_ms = 0.0
            if kind != "cold":
                if kind == "warm":
                    ws_ms = dp.dp_warm_start(net.h, g2.h)
                else:
                    # the non-learned baseline: Q1 interpolation of the 61^4 solution
                    ws_ms = dp.dp_warm_start_from_grid(g1.h, g2.h)
                if start == kind:
                    t_ws = time.perf_counter() - t0
                    err = np.abs(g2.get_value() - V_cold) / g2.info["penalty_M"]
                    out[("warm_start_error" if kind == "warm" else "from_61x4_grid_error")] = {
                        "max_over_M": float(err.max()), "rms_over_M": float(np.sqrt(np.mean(err ** 2)))}
                    t0 = time.perf_counter() - t_ws   # the host copy for the error is not timed
            rc, s2 = g2.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=n_eval, polish=1,
                                       warm=int(kind != "cold"), eval_solver=solver)
            torch.cuda.synchronize()
            if start == "cold":
                V_cold = g2.get_value()
                # the energy-band grid's evaluation sweep against the HBM roofline
                # (10 B per node-update), timed after the solve on its FP32 values
                g2.set_value(V_cold)
                rc, sk = g2.policy_iterate(tol=0.0, max_sweeps=2, n_eval=p2.n_eval, polish=0, warm=1,
                                           time_kernels=1)
                n_upd = g2.info["n_active"] - g2.info["n_target"]
                ev_ms = sk.ms_eval / max(sk.sweeps_eval, 1)
                peaks, _ = _peaks()
                out["eval_sweep_121x4_band"] = {
                    "ms": ev_ms, "node_updates_per_s": n_upd / (ev_ms / 1e3),
                    "achieved_gbs": 10.0 * n_upd / (ev_ms / 1e3) / 1e9,
                    "frac_of_hbm": 10.0 * n_upd / (ev_ms / 1e3) / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
                    "walk_ms": sk.ms_improve / max(sk.sweeps_improve, 1)}
            out[start] = {"seconds": time.perf_counter() - t0, "converged": bool(s2.converged),
                          "residual": s2.residual, "n_eval": n_eval,
                          "evaluation": "diagonal-solved Jacobi" if solver == dp.DP_EVAL_DIAG else "sweeps",
                          "warm_start_ms": ws_ms,
                          "sweeps_improve": s2.sweeps_improve, "sweeps_eval": s2.sweeps_eval,
                          "sweeps_improve_fp64": s2.sweeps_improve_fp64,
                          "sweeps_eval_fp64": s2.sweeps_eval_fp64, "node_updates": s2.node_updates}
        if args.fp64_band:
            # the plain FP64 GPU solve of the same grid (no network, no FP32
            # phase), cold, to the same tolerance: with the diagonal-solved
            # evaluation and, with --fp64-band 2, with plain sweeps too
            p64 = p2.replace(precision=W.FP64)
            kinds = [("diag", args.diag_n_eval, dp.DP_EVAL_DIAG)]
            if args.fp64_band > 1:
                kinds.append(("sweeps", p2.n_eval, dp.DP_EVAL_JACOBI))
            with dp.Grid(p64, stream=int(torch.cuda.current_stream().cuda_stream)) as g64:
                for name, n_eval, solver in kinds:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    rc, s64 = g64.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=n_eval, warm=0,
                                                 eval_solver=solver)
                    torch.cuda.synchronize()
                    out["plain_fp64_" + name] = {
                        "seconds": time.perf_counter() - t0, "converged": bool(s64.converged),
                        "residual": s64.residual, "n_eval": n_eval, "improvements": s64.sweeps_improve,
                        "evaluation_sweeps": s64.sweeps_eval}
                    if name == "diag":
                        v64 = g64.get_value()
                        err = np.abs(v64 - V_cold)
                        out["plain_fp64_diag"]["max_abs_diff_to_fp32_polish_solve"] = float(err.max())
        x0 = W.closed_loop_states(p2, 1024, band=(p2.energy_lo, p2.energy_hi))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ta, xf = g2.simulate(x0, p2.dt, p2.dt, 200.0)
        out["closed_loop"] = {"states": len(x0), "seconds": time.perf_counter() - t0,
                              "arrived": int((ta >= 0).sum()),
                              "median_time": float(np.median(ta[ta >= 0])) if (ta >= 0).any() else None}
    c, w, gr = out["cold"], out["warm"], out["from_61x4_grid"]
    out["speedup_wall"] = c["seconds"] / max(w["seconds"], 1e-9)
    out["speedup_wall_grid_start"] = c["seconds"] / max(gr["seconds"], 1e-9)
    ct, wt = out["cold" + tuned], out["warm" + tuned]
    out["speedup_wall" + tuned] = ct["seconds"] / max(wt["seconds"], 1e-9)
    if "plain_fp64_diag" in out:
        # the learned warm-started FP32 solve (network inference included,
        # training not) against the plain FP64 GPU solve of the same grid
        f64 = out["plain_fp64_diag"]
        cmp_ = {"learned_fp32_diag_seconds": wt["seconds"], "plain_fp64_diag_seconds": f64["seconds"],
                "speedup_diag": f64["seconds"] / max(wt["seconds"], 1e-9),
                "learned_fp32_sweeps_seconds": w["seconds"],
                "training_seconds": out["train"]["wall_s"]}
        if "plain_fp64_sweeps" in out:
            cmp_["plain_fp64_sweeps_seconds"] = out["plain_fp64_sweeps"]["seconds"]
            cmp_["speedup_sweeps"] = out["plain_fp64_sweeps"]["seconds"] / max(w["seconds"], 1e-9)
        out["learned_fp32_vs_plain_fp64"] = cmp_
    return out


def time_pi_step(dp, torch, g, p, steps, warmup, world, local, flush, clocks=True):
    """The benchmark step on grid g: a cold start (full tabulation) and 3 outer
    iterations, `warmup` untimed steps, then `steps` timed steps (1 walk
    improvement + n_eval evaluation sweeps each) as one policy-iteration call
    of `steps` outer iterations, between CUDA events on the grid's stream.
    L2 is flushed once before the timed region; between the steps each sweep
    streams more than L2 holds (1.12 GB on the band grid, 276 MB on 61^4)."""
    stream = torch.cuda.current_stream()
    g.policy_iterate(tol=0.0, max_sweeps=3, n_eval=p.n_eval, polish=0, warm=0)
    if warmup:
        g.policy_iterate(tol=0.0, max_sweeps=warmup, n_eval=p.n_eval, polish=0, warm=1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    _barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local) if clocks else None
    if clk:
        clk.__enter__()
    e0.record(stream)
    rc, st = g.policy_iterate(tol=0.0, max_sweeps=steps, n_eval=p.n_eval, polish=0, warm=1, time_kernels=1)
    e1.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__()
    _barrier(world)
    assert st.sweeps_improve == steps and st.sweeps_eval == steps * p.n_eval, st.asdict()
    return {"ms": e0.elapsed_time(e1), "updates": st.node_updates, "stats": [st], "steps": steps,
            "clocks": clk.summary() if clk else None}


def step_roofline(g, p, timed, key):
    """Roofline of the step's dominant kernel, the frozen-feet evaluation
    sweep: algorithmic bytes per sweep (V read 4 + policy 2 + V write 4 per
    node-update) over its CUDA-event time, against the measured HBM copy
    bandwidth."""
    stats = timed["stats"]
    n_upd = g.info["n_active"] - g.info["n_target"]
    ms_eval = sum(s.ms_eval for s in stats)
    n_eval = sum(s.sweeps_eval for s in stats)
    ms_imp = sum(s.ms_improve for s in stats)
    n_imp = sum(s.sweeps_improve for s in stats)
    launches_eval = sum(s.launches for s in stats) - n_imp
    peaks, peak_src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    eval_ms = ms_eval / max(n_eval, 1)
    eval_bytes = 10.0 * n_upd
    ach = eval_bytes / (eval_ms / 1e3) / 1e9
    traffic, tsrc = _traffic(key)
    roof = {"bound": "hbm", "kernel": "sweep_kernel<float,float,EVAL_FEET8,%s> (policy evaluation at the 8-byte frozen feet)"
                                      % ("reduced" if p.reduced else "box"),
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "peak_source": (peak_src + " (MEASURED_PEAKS.json hbm_gbs, burst copy)") if peak_src == "measured"
            else peak_src + " (6.8 TB/s)",
            "traffic": traffic, "traffic_source": tsrc,
            "algorithmic_bytes_per_sweep": eval_bytes, "avg_sweep_ms": eval_ms,
            "sweeps_per_launch": n_eval / max(launches_eval, 1),
            "share_of_step": ms_eval / max(timed["ms"], 1e-9)}
    imp_ms = ms_imp / max(n_imp, 1)
    improve = {"avg_launch_ms": imp_ms, "share_of_step": ms_imp / max(timed["ms"], 1e-9),
               "node_updates_per_s": n_upd / (imp_ms / 1e3)}
    return roof, improve, n_upd / (eval_ms / 1e3)


def e2e_pi_step(dp, torch, g, p, steps, world):
    """The same step through the C ABI with host buffers: the value and the
    policy go up from pinned host memory before each step and come back
    after it, inside the timed region.  The value travels in the grid's
    storage precision (FP32 for the FP32 grids, dp_set_value_f32 /
    dp_get_value_f32; FP64 otherwise)."""
    from paper_2407_14675_gb300 import workloads as W
    f32 = p.precision == W.FP32
    V_host = torch.empty(g.n, dtype=torch.float32 if f32 else torch.float64, pin_memory=True)
    C_host = torch.empty(g.n, dtype=torch.int16, pin_memory=True)
    C_view = C_host.numpy().view(np.uint16)
    set_v = dp.dp_set_value_f32 if f32 else dp.dp_set_value
    get_v = dp.dp_get_value_f32 if f32 else dp.dp_get_value
    get_v(g.h, g.n, out=V_host.numpy())
    C_view[:] = g.get_policy()
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    updates = 0
    for _ in range(steps):
        set_v(g.h, V_host)
        dp.dp_set_policy(g.h, C_view)
        rc, st = g.policy_iterate(tol=0.0, max_sweeps=1, n_eval=p.n_eval, polish=0, warm=1)
        get_v(g.h, g.n, out=V_host.numpy())
        dp.dp_get_policy(g.h, g.n, out=C_view)
        updates += st.node_updates
    torch.cuda.synchronize()
    secs = _reduce_max(time.perf_counter() - t0, world)
    vb = V_host.element_size()
    return {"value": _reduce_sum(float(updates), world) / secs, "unit": UNIT, "steps": steps,
            "value_transfer": "FP32" if f32 else "FP64",
            "h2d_bytes_per_step": g.n * (vb + 2), "d2h_bytes_per_step": g.n * (vb + 2)}


def run_ours(args, world, rank, local):
    import torch
    from paper_2407_14675_gb300 import build, dp
    from paper_2407_14675_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    dp.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    # --- headline: the 121^4 energy-band grid, inputs resident in HBM ---
    p2 = W.config2()
    g2 = dp.Grid(p2, stream=int(stream.cuda_stream))
    timed = time_pi_step(dp, torch, g2, p2, args.steps, args.warmup, world, local, flush)
    value, ms_max = aggregate_replicas(timed["updates"], timed["ms"], world)
    roof, improve, eval_rate = step_roofline(g2, p2, timed, "121x4_band")
    n_upd2 = g2.info["n_active"] - g2.info["n_target"]
    launches = sum(s.launches for s in timed["stats"])
    e2e = e2e_pi_step(dp, torch, g2, p2, max(1, min(args.steps, 5)), world)

    # --- the same step on the 61^4 full box ---
    p = W.config1()
    g = dp.Grid(p, stream=int(stream.cuda_stream))
    t1 = time_pi_step(dp, torch, g, p, max(1, min(args.steps, 10)), args.warmup, world, local, flush, clocks=False)
    roof1, improve1, eval_rate1 = step_roofline(g, p, t1, "61x4")
    step_61x4 = {"value": t1["updates"] / (t1["ms"] / 1e3), "unit": UNIT, "ms_per_step": t1["ms"] / t1["steps"],
                 "config": _config(p, g.info["n_active"] - g.info["n_target"]), "roofline": roof1,
                 "improve_sweep": improve1, "eval_sweep_node_updates_per_s": eval_rate1}
    # --- time to ||dV|| < 1e-6 (plain cold start, FP32 + FP64 polish) ---
    solve = None
    if args.solve:
        torch.cuda.synchronize()
        hist = np.zeros(args.solve_max)
        t0 = time.perf_counter()
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=p.n_eval, polish=1, warm=0,
                                  time_kernels=1, history=hist)
        torch.cuda.synchronize()
        h = hist[:st.history_count]
        marks = sorted(set([0, 1, 2, 5, 10, 20, 50, 100, 200, 400, 800, 1600, 3200, len(h) - 1]))
        solve = {"seconds": time.perf_counter() - t0, "converged": bool(st.converged), "residual": st.residual,
                 "sweeps_improve": st.sweeps_improve, "sweeps_eval": st.sweeps_eval,
                 "sweeps_improve_fp64": st.sweeps_improve_fp64, "sweeps_eval_fp64": st.sweeps_eval_fp64,
                 "switch_outer": st.switch_outer,
                 "gpu_ms": {"improve": st.ms_improve, "eval": st.ms_eval, "improve_fp64": st.ms_improve_fp64,
                            "eval_increments": st.ms_eval_fp64},
                 "residual_trace": {int(k): float(h[k]) for k in marks if 0 <= k < len(h)},
                 "start": "cold (V = 0, full tabulation first)"}
    solve_gmres = None
    if args.solve and rank == 0:
        # the same cold solve with each policy evaluated by GMRES on FP32 vectors
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, polish=1, warm=0, time_kernels=1,
                                  eval_solver=dp.DP_EVAL_GMRES, gmres_restart=args.gmres_restart_fp32)
        torch.cuda.synchronize()
        solve_gmres = {"seconds": time.perf_counter() - t0, "converged": bool(st.converged),
                       "residual": st.residual, "evaluation": "GMRES(%d)" % args.gmres_restart_fp32,
                       "improvements": st.sweeps_improve + st.sweeps_improve_fp64, "matvecs": st.gmres_matvecs,
                       "gpu_ms": {"improve": st.ms_improve + st.ms_improve_fp64,
                                  "gmres": st.ms_eval + st.ms_eval_fp64}}
    solve_tuned = None
    if args.solve and rank == 0:
        # the same cold solve with more evaluation sweeps per improvement: the
        # sweeps needed to propagate the value stay about the same, the
        # improvement sweeps (16 evaluation sweeps' worth each) fall
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=args.n_eval_tuned, polish=1, warm=0)
        torch.cuda.synchronize()
        solve_tuned = {"seconds": time.perf_counter() - t0, "converged": bool(st.converged), "residual": st.residual,
                       "n_eval": args.n_eval_tuned, "improvements": st.sweeps_improve + st.sweeps_improve_fp64,
                       "evaluation_sweeps": st.sweeps_eval + st.sweeps_eval_fp64}
    solve_diag = None
    if args.solve and rank == 0:
        # the same cold solve with each evaluation sweep solving the node's own
        # coefficient (the Jacobi method proper on the evaluation system)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = g.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=args.diag_n_eval, polish=1, warm=0,
                                  eval_solver=dp.DP_EVAL_DIAG, time_kernels=1)
        torch.cuda.synchronize()
        solve_diag = {"seconds": time.perf_counter() - t0, "converged": bool(st.converged), "residual": st.residual,
                      "evaluation": "diagonal-solved Jacobi", "n_eval": args.diag_n_eval,
                      "improvements": st.sweeps_improve + st.sweeps_improve_fp64,
                      "evaluation_sweeps": st.sweeps_eval + st.sweeps_eval_fp64,
                      "gpu_ms": {"improve": st.ms_improve, "eval": st.ms_eval, "improve_fp64": st.ms_improve_fp64,
                                 "eval_increments": st.ms_eval_fp64}}
    cascade = None
    if args.solve and rank == 0:
        # coarse to fine: the same problem on 16^4, then 31^4, each solved to
        # 1e-6 and interpolated onto the next grid (dp_warm_start_from_grid),
        # then solved on 61^4 to 1e-6; every level with the diagonal-solved
        # evaluation, n_eval = cascade_n_eval
        levels = [16, 31]
        grids = [dp.Grid(W.config1(n=n), stream=int(stream.cuda_stream)) for n in levels]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        per, prev = [], None
        for n, gc in zip(levels + [61], grids + [g]):
            if prev is not None:
                dp.dp_warm_start_from_grid(prev.h, gc.h)
            rc, sc = gc.policy_iterate(tol=1e-6, max_sweeps=args.solve_max, n_eval=args.cascade_n_eval, polish=1,
                                       warm=int(prev is not None), eval_solver=dp.DP_EVAL_DIAG)
            per.append({"grid": "%d^4" % n, "improvements": sc.sweeps_improve + sc.sweeps_improve_fp64,
                        "converged": bool(sc.converged), "ms": sc.ms_wall})
            prev = gc
        torch.cuda.synchronize()
        cascade = {"seconds": time.perf_counter() - t0, "converged": all(q["converged"] for q in per),
                   "evaluation": "diagonal-solved Jacobi", "n_eval": args.cascade_n_eval, "levels": per,
                   "residual": sc.residual}
        for gc in grids:
            gc.close()
    warm = warm_start_leg(args, dp, W, torch, g, p, g2) if (args.warm_start and args.solve and rank == 0) else None
    extra = extra_legs(args, dp, W, torch, g, p) if (args.extra and rank == 0) else None
    g.close()
    g2.close()
    batch = batch_leg(args, dp, W, torch) if (args.batch and rank == 0) else None
    ex1 = example1_leg(args, dp, W, torch) if (args.example1 and rank == 0) else None

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    cpu_rate, cpu_info = None, {}
    if args.cpu_seconds > 0:
        sample = OracleSample(p2)
        cpu_rate, cpu_info = sample.step_rate(seconds_target=args.cpu_seconds)
        del sample
    par_rate, par_info = (oracle_parallel_rate(args.cpu_seconds / 2) if (args.cpu_seconds > 0 and args.cpu_parallel)
                          else (None, {}))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(_config(p2, n_upd2), parallelism="replicas" if world > 1 else "single"),
        "clocks": timed["clocks"],
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roof,
        "improve_sweep": improve,
        "eval_sweep_node_updates_per_s": eval_rate,
        "cpu_baseline": None if cpu_rate is None else {
            "value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d sampled stored nodes of the 121^4 band x (1 walk improvement + %d evaluations), %d reps, "
                      "%.1f s FP64 single thread" % (cpu_info["nodes"], p2.n_eval, cpu_info["reps"],
                                                      cpu_info["seconds"])},
        "cpu_baseline_all_cores": None if par_rate is None else {
            "value": par_rate, "unit": UNIT, "cores": par_info["procs"], "kind": "oracle",
            "sample": "one spawned oracle process per core (at most one per 3 GB of free host memory), each on its "
                      "own 2,000-node sample of the "
                      "band step mix, %.1f s" % par_info["seconds"]},
        "step_61x4": step_61x4,
        "time_to_tol": solve,
        "time_to_tol_n_eval_tuned": solve_tuned,
        "time_to_tol_diag": solve_diag,
        "time_to_tol_coarse_to_fine": cascade,
        "time_to_tol_gmres": solve_gmres,
        "warm_start": warm,
        "batch": batch,
        "other_solves": extra,
        "paper_example1": ex1,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--solve", type=int, default=1, help="also time a cold solve to 1e-6")
    ap.add_argument("--solve-max", type=int, default=3000, help="improvement-sweep budget of that solve")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--warm-start", type=int, default=1, help="train the network, compare cold/warm 121^4 solves")
    ap.add_argument("--mlp-epochs", type=int, default=2)
    ap.add_argument("--fp64-band", type=int, default=1,
                    help="plain FP64 solve of the band grid: 0 none, 1 diagonal-solved evaluation, 2 also plain sweeps")
    ap.add_argument("--batch", type=int, default=1, help="time the 256-transfer batch")
    ap.add_argument("--extra", type=int, default=1, help="17^4 FP64 VI; walk vs full tabulation")
    ap.add_argument("--cpu-parallel", type=int, default=1, help="also time the oracle on every host core")
    ap.add_argument("--example1", type=int, default=1, help="the paper's Example 1 solve and closed loop")
    ap.add_argument("--n-eval-tuned", type=int, default=160, help="evaluation sweeps per improvement, tuned solve")
    ap.add_argument("--cascade-n-eval", type=int, default=20,
                    help="diagonal-solved evaluation sweeps per improvement, cascade")
    ap.add_argument("--diag-n-eval", type=int, default=40, help="diagonal-solved evaluation sweeps per improvement")
    ap.add_argument("--gmres-restart-fp64", type=int, default=60, help="GMRES restart length, FP64 grids")
    ap.add_argument("--gmres-restart-fp32", type=int, default=20, help="GMRES restart length, 61^4 FP32 grid")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-fp64-sample", type=int, default=4)
    args = ap.parse_args()
    world, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
