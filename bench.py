#!/usr/bin/env python3
"""Throughput of the active-Brownian-particle ensemble integrator on GB300.

Workload (default): the D x q parameter sweep -- 64 values of D log-spaced in [1e-3, 1]
times 32 values of q log-spaced in [0.1, 10], 1,024 trajectories per point (2,097,152
trajectories), 10^5 Euler-Maruyama steps at dt = 1e-3, FP32 state with FP64
accumulation, v0 ~ N(0, sqrt(D)), Philox seed 1.  One step of the benchmark is one pass
of the whole path: initial condition, integration with noise generation, the final
histogram of x mod L and the FP64 ensemble reduction.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s on 1 GB300 (and % FP32-pipe roofline) at oracle-matched accuracy"
UNIT = "particle-steps/s"
# Algorithmic FP32/INT32 lane operations per particle-step: drift, depot, position and
# wrap ~16, Philox4x32-10 amortised over its four steps 15, Box-Muller ~4.
N_ALG = 35
# The stochastic Heun step draws the same noise and evaluates drift, depot and position twice.
N_ALG_HEUN = 51
LANES_PER_SM = 128
# DRAM bytes (read + write) per launch of the integrator on the 2,097,152-trajectory sweep grid,
# from one ncu capture of that kernel (dram__bytes_read.sum + dram__bytes_write.sum).  Lockstep:
# the state load/store of one window, independent of its length (captured at 2,000 steps).  Work
# queue: the bench's own launch (10^5 steps in ten rounds of 10^4-step items), captured whole --
# the later rounds re-read the state from L2, the writes include its write-backs.
TRAFFIC_PER_LAUNCH = {"integrate_kernel<float,2>": (52479744 + 1671424, 2097152),
                      "persistent_kernel<float,2>": (52659712 + 19994112, 2097152)}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--ppt", type=int, default=0, help="particles per thread (0 = library default)")
    ap.add_argument("--steps-per-launch", type=int, default=0,
                    help="steps per work item (0 = autotuned)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="0 autotuned, 1 lockstep launches, 2 work queue (persistent launch)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--small", action="store_true",
                    help="the sweep grid at 2,000 steps (profiling and quick checks; not a bench line)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the pathwise-adjoint leg")
    ap.add_argument("--no-visualisation", action="store_true",
                    help="skip the per-cycle cost of reading intermediate results (iterations lost)")
    ap.add_argument("--profile-config", default="",
                    help="run only this workload of --configs (no headline, no other legs) and print its entry; "
                         "for profiling one kernel; 'uneven_slice' = the uneven batch over its first 2 x 10^4 steps, work queue")
    ap.add_argument("--adjoint-only", default="",
                    help="N_TRAJ,N_STEPS: time only the forward and backward of the differentiation workload at "
                         "this size (profiling; prints one JSON line without the bench keys)")
    ap.add_argument("--configs", default="default",
                    help="other workloads timed after the headline, comma-separated: single, single_heun, "
                         "single_xorshift, uneven, force, heun, xorshift, snapshots_slice, snapshots (the full 64M x 10^6 run, about a minute), precision, "
                         "items; 'default' = all but the full snapshots run, 'all' = every one, 'none' = skip; "
                         "reported under 'configs'")
    return ap.parse_args()


def workload(args):
    from paper_1104_2499_gb300 import workloads as W

    if args.small:  # the same grid, 2,000 steps: several waves of the integrator, a few ms per launch
        return W.sweep_grid(n_steps=2000)
    return W.sweep_grid()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "power_w_max": max(power),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle legs

def oracle_sample(w, budget_s: float, gpu_moments=None):
    """Time the FP64 oracle on whole parameter sets of the workload (all their trajectories,
    all their steps), evenly spread over the grid, until about budget_s seconds are used.
    Returns (rate, cores, sample description, parity summary)."""
    from oracle import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    base = w.traj_base()
    order = [int(round(i * (w.n_sets - 1) / 15)) for i in range(16)] if w.n_sets > 16 else list(range(w.n_sets))
    done_ps, t_used, used, z = 0, 0.0, [], []
    for i in order:
        t0 = time.perf_counter()
        r = O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, n_threads=cores)
        t_used += time.perf_counter() - t0
        done_ps += w.n_traj[i] * w.n_steps[i]
        used.append(i)
        if gpu_moments is not None:
            se = max(r["se_v"], 1e-300)
            z.append(abs(float(gpu_moments[i][0]) - r["mean_v"]) / se)
        if t_used >= budget_s:
            break
    desc = "%d whole parameter sets (%d trajectories x %d steps each, %.3g particle-steps) of the sweep" % (
        len(used), w.n_traj[used[0]], w.n_steps[used[0]], done_ps)
    parity = None
    if z:
        parity = {"sets_checked": len(z), "max_abs_dmean_over_se": max(z), "bar": 3.0, "pass": max(z) <= 3.0}
    # the same oracle on one core: 64 trajectories of the first set, all its steps
    i = order[0]
    m1 = min(64, w.n_traj[i])
    t0 = time.perf_counter()
    O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=m1, n_steps=w.n_steps[i], traj_base=base[i], v0_mode=w.v0_mode,
              n_threads=1)
    one_core = m1 * w.n_steps[i] / (time.perf_counter() - t0)
    return done_ps / t_used, cores, desc, parity, one_core


def oracle_subset_rate(w, traj_per_set: int, max_steps: int = 0):
    """The FP64 oracle's throughput on a fixed subset of workload ``w``: the first
    ``traj_per_set`` trajectories of every set, over all their steps (or the first
    ``max_steps``), on all host cores."""
    from oracle import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    base = w.traj_base()
    done, t = 0, 0.0
    for i in range(w.n_sets):
        m = min(traj_per_set, w.n_traj[i])
        n = w.n_steps[i] if max_steps <= 0 else min(max_steps, w.n_steps[i])
        if m <= 0 or n <= 0:
            continue
        t0 = time.perf_counter()
        O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=m, n_steps=n, traj_base=base[i], v0_mode=w.v0_mode,
                  n_threads=cores)
        t += time.perf_counter() - t0
        done += m * n
    desc = "first %d trajectories of each of %d sets, %s (%.3g particle-steps)" % (
        traj_per_set, w.n_sets, "all steps" if max_steps <= 0 else "%d steps" % max_steps, done)
    return {"value": done / t, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, timed on the host cores."""
    from paper_1104_2499_gb300 import workloads as W

    w = workload(args)
    if rank != 0:
        return
    from oracle import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    base = w.traj_base()
    # one step = one bounded sample of the workload: a slice of trajectories of sets spread over
    # the grid, all 10^5 steps, sized so that warm-up + timed steps take about two minutes
    total_steps = args.steps + args.warmup
    per_step_budget = max(2.0, 120.0 / max(total_steps, 1))
    t0 = time.perf_counter()
    O.run_set(w.sets[0], seed=w.seed, dt=w.dt, n_traj=16, n_steps=2000, traj_base=base[0], v0_mode=w.v0_mode,
              n_threads=cores)
    rate_probe = 16 * 2000 / max(time.perf_counter() - t0, 1e-6)
    ps_target = rate_probe * per_step_budget
    n_sets_s = 8
    m = max(1, int(ps_target / (n_sets_s * w.n_steps[0])))
    m = min(m, w.n_traj[0])
    idx = [int(round(i * (w.n_sets - 1) / (n_sets_s - 1))) for i in range(n_sets_s)]

    def step():
        for i in idx:
            O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=m, n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, n_threads=cores)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ps = n_sets_s * m * w.n_steps[0]
    value = ps / statistics.mean(times)
    sample = "%d sets spread over the %d-set sweep x %d trajectories x %d steps per step (%.3g particle-steps)" % (
        n_sets_s, w.n_sets, m, w.n_steps[0], ps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, args, {"state": "fp64 (FP64 CPU oracle, unwrapped position)",
                                            "l2": "not applicable (host cores)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(w, args, extra=None):
    d = {"workload": w.name, "parameter_sets": w.n_sets, "traj_per_set": int(w.n_traj[0]) if w.n_sets else 0,
         "total_traj": w.total_traj, "steps": int(w.n_steps[0]) if w.n_sets else 0, "dt": w.dt, "seed": w.seed,
         "particle_steps_per_step": w.particle_steps, "state": "fp32 (cell + fraction), fp64 accumulation",
         "l2": "flushed (256 MiB write) between timed steps", "hist_x_bins": w.hist_x_bins}
    if extra:
        d.update(extra)
    return d


# ----------------------------------------------------------------------------- adjoint leg

def adjoint_leg(A, stream, small=False, size=None, accuracy=True):
    """Pathwise adjoint of <v> w.r.t. (D, q, c, d, gamma0, a).

    Cost: forward (with checkpoints every 1,000 steps) and backward on the differentiation
    workload (1,048,576 trajectories x 10^5 steps, D = 0.05), timed with CUDA events.
    Accuracy: at horizons where the pathwise derivative is well conditioned (the first 4,096
    trajectories of the same set; 1,000 steps with central differences h = 1e-4 |theta|, and
    2,000 steps, where h = 1e-4 |theta| is already past the linear range of a few paths, with
    h = 1e-6 |theta|), the GPU adjoint against FP64 central differences with common random
    numbers and against the FP64 tangent-linear, both from the oracle on the same trajectories.  (Over 10^5 steps the
    frozen-noise dynamics is chaotic and the pathwise derivative grows exponentially; its
    size at the full horizon is reported as found.)"""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_1104_2499_gb300 import workloads as W

    if size is not None:
        w = W.differentiation(n_traj=size[0], n_steps=size[1])
    else:
        w = W.differentiation(n_traj=1 << 16, n_steps=20_000) if small else W.differentiation()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with A.Ensemble(w, stream=stream) as ens, torch.cuda.stream(stream):
        ens.set_params()
        ens.integrate(-1)
        ens.backward()  # warm-up (and allocation of the adjoint scratch)
        ens.reset(w.seed)
        ev[0].record(stream)
        ens.integrate(-1)
        ev[1].record(stream)
        g = ens.backward()
        ev[2].record(stream)
        stream.synchronize()
        fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        g_full = g.cpu().numpy()[0]
        # windowed adjoint (windows of 2,000 steps, t = 2): bounded where the full one is not
        win = 2000 if w.n_steps[0] >= 2000 else w.n_steps[0]
        g_win = ens.backward(window=win).cpu().numpy()[0] if win % w.checkpoint_every == 0 else None
        dv_win = ens.traj_grad()[:8192].cpu().numpy() if g_win is not None and accuracy else None
    windowed = None
    if g_win is not None and accuracy:
        # the oracle's windowed tangent on 8,192 trajectories of the same set: its mean and
        # standard error (paths decorrelate over the horizon, so this is a statistical check)
        sub = 8192
        r = O.run_set(w.sets[0], seed=w.seed, dt=w.dt, n_traj=sub, n_steps=w.n_steps[0], v0_mode=w.v0_mode,
                      want_traj_grad=True, grad_window=win)
        se = r["dvbar"].std(axis=0, ddof=1) / math.sqrt(sub)
        z = np.abs(g_win - r["grad"]) / np.maximum(se, 1e-300)
        windowed = {"window_steps": win, "grad_gpu": dict(zip(A.GRAD_PARAMS, map(float, g_win))),
                    "oracle_subset_mean": dict(zip(A.GRAD_PARAMS, map(float, r["grad"]))),
                    "oracle_subset_se": dict(zip(A.GRAD_PARAMS, map(float, se))),
                    "oracle_se_over_abs_grad": dict(zip(A.GRAD_PARAMS, map(float, se / np.maximum(np.abs(g_win),
                                                                                                  1e-300)))),
                    "max_abs_diff_over_se": float(z.max()), "oracle_subset_trajectories": sub}
        # the same trajectories on both sides: the GPU's windowed derivative of each of them against
        # the oracle's, so the noise of the estimator cancels where the FP32 and FP64 paths stay together
        d = dv_win[:sub] - r["dvbar"]
        se_d = d.std(axis=0, ddof=1) / math.sqrt(sub)
        windowed["paired"] = {"mean_diff": dict(zip(A.GRAD_PARAMS, map(float, d.mean(axis=0)))),
                              "se_of_mean_diff": dict(zip(A.GRAD_PARAMS, map(float, se_d))),
                              "se_over_abs_grad": dict(zip(A.GRAD_PARAMS, map(float, se_d / np.maximum(
                                  np.abs(g_win), 1e-300)))),
                              "max_abs_mean_diff_over_se": float(np.max(np.abs(d.mean(axis=0)) / np.maximum(se_d,
                                                                                                          1e-300))),
                              "fraction_of_trajectories_within_1e-3": float(np.mean(np.all(
                                  np.abs(d) <= 1e-3 * np.maximum(np.abs(r["dvbar"]),
                                                                 np.sqrt(np.mean(r["dvbar"] ** 2, axis=0))),
                                  axis=1)))}
    per_traj = per_trajectory_check(A, stream, w) if accuracy and size is None and not small else None

    def check(n_steps, rel_h, K):
        wa = W.differentiation(n_traj=4096, n_steps=n_steps, checkpoint_every=K)
        with A.Ensemble(wa, stream=stream) as ens, torch.cuda.stream(stream):
            ens.run()
            g_gpu = ens.backward(host=True).numpy()[0]
        base = wa.sets[0]
        kw = dict(seed=wa.seed, dt=wa.dt, n_traj=wa.n_traj[0], n_steps=wa.n_steps[0], v0_mode=wa.v0_mode)
        g_tl = O.run_set(base, want_grad=True, **kw)["grad"]
        fd = []
        for name in A.GRAD_PARAMS:
            h = rel_h * abs(base[name])
            up = O.run_set(dict(base, **{name: base[name] + h}), **kw)["mean_v"]
            dn = O.run_set(dict(base, **{name: base[name] - h}), **kw)["mean_v"]
            fd.append((up - dn) / (2 * h))
        fd = np.array(fd)
        scale = float(np.max(np.abs(fd)))
        return {"workload": wa.name, "checkpoint_every": K, "fd_h": "%g |theta|" % rel_h,
                "grad_gpu": dict(zip(A.GRAD_PARAMS, map(float, g_gpu))),
                "central_fd_fp64": dict(zip(A.GRAD_PARAMS, map(float, fd))),
                "max_err_vs_fd_over_largest": float(np.max(np.abs(g_gpu - fd)) / scale),
                "max_err_vs_tangent_linear_over_largest": float(np.max(np.abs(g_gpu - g_tl)) / scale),
                "bar": 1e-3, "fd": "oracle FP64, common random numbers"}

    acc = [check(1000, 1e-4, 200), check(2000, 1e-6, 1000)] if accuracy else None
    return {"workload": w.name, "particle_steps": w.particle_steps, "checkpoint_every": w.checkpoint_every,
            "forward_ms": fwd_ms, "backward_ms": bwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
            "max_abs_pathwise_grad_full_horizon": float(np.max(np.abs(g_full))),
            "windowed": windowed, "per_trajectory": per_traj, "accuracy": acc}


def per_trajectory_check(A, stream, w_full, n_steps=2000, n_check=4096):
    """The differentiation workload's set (all 1,048,576 trajectories, D = 0.05, seed 3) over
    its first 2,000 steps, where the frozen-noise paths of the FP32 GPU and the FP64 oracle stay
    together, so the comparison is deterministic trajectory by trajectory: the GPU's pathwise
    d vbar_i / d theta (abp_backward_traj) of the first 4,096 trajectories against the oracle's
    tangent-linear of the same trajectories.  Bar: 1e-3 max(|oracle|, rms_j), rms_j the root
    mean square of component j over the checked trajectories."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_1104_2499_gb300 import workloads as W

    w = W.differentiation(n_traj=w_full.n_traj[0], n_steps=n_steps)
    with A.Ensemble(w, stream=stream) as ens, torch.cuda.stream(stream):
        ens.run()
        g = ens.backward(host=True).numpy()[0]
        dv = ens.traj_grad()[:n_check].cpu().numpy()
    r = O.run_set(w.sets[0], seed=w.seed, dt=w.dt, n_traj=n_check, n_steps=n_steps, v0_mode=w.v0_mode,
                  want_traj_grad=True)
    ref = r["dvbar"]
    rms = np.sqrt(np.mean(ref ** 2, axis=0))
    ratio = np.abs(dv - ref) / (1e-3 * np.maximum(np.abs(ref), rms))
    return {"workload": w.name, "trajectories_checked": n_check, "bar": "1e-3 max(|oracle|, rms over trajectories)",
            "max_ratio": dict(zip(A.GRAD_PARAMS, map(float, ratio.max(axis=0)))),
            "fraction_within_bar": float(np.mean(np.all(ratio <= 1.0, axis=1))),
            "gpu_set_gradient_all_trajectories": dict(zip(A.GRAD_PARAMS, map(float, g))),
            "oracle_mean_checked_trajectories": dict(zip(A.GRAD_PARAMS, map(float, r["grad"])))}


# ----------------------------------------------------------------------------- visualisation leg

def visualisation_leg(A, stream):
    """The cost of looking at intermediate results, in the form of the paper's Table 1
    (Sec. 3.2): the number of iterations that could have run in the time a display cycle
    spends outside the integration.  Work items = parameter sets of the load sweep (one
    trajectory each, as the paper's work items); a cycle integrates T steps, reduces the
    ensemble (the mean-velocity-versus-load curve, Fig. 2) and waits for it.  'device': the
    result stays in device memory (the analogue of shared CL/GL buffers); 'host': it is copied
    into pinned host memory every cycle (the analogue of the non-shared method).  Cycle time
    is fitted linearly in T; offset / slope = iterations lost.  'live_T*': the library streams a
    snapshot (moments of every set) every T steps to pinned host memory on its own stream while
    the integration goes on (abp_live); iterations lost = the extra time per snapshot over the
    same run without live results, in iterations."""
    import numpy as np
    import torch
    from paper_1104_2499_gb300 import workloads as W

    out = {}
    Ts = [250, 500, 1000, 2000, 4000]
    reps = 20
    for n_items in (64, 8192):
        w = W.force_sweep(n_F=n_items, traj_per_set=1, n_steps=(sum(Ts) * reps) + 1000)
        res = {}
        with A.Ensemble(w, stream=stream) as ens, torch.cuda.stream(stream):
            ens.set_params()
            ens.integrate(1000)  # warm-up
            mom_d = torch.empty((n_items, 8), dtype=torch.float64, device="cuda")
            mom_h = torch.empty((n_items, 8), dtype=torch.float64, pin_memory=True)
            for method, dst in (("device", mom_d), ("host", mom_h)):
                xs, ys = [], []
                for T in Ts:
                    stream.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(reps // 2):
                        A.abp_integrate(ens.ctx, T)
                        A.abp_reduce(ens.ctx, dst, None, None)
                        stream.synchronize()
                    xs.append(T)
                    ys.append((time.perf_counter() - t0) / (reps // 2))
                slope, offset = np.polyfit(np.array(xs, float), np.array(ys), 1)
                res[method] = {"us_per_iteration": slope * 1e6, "offset_us": offset * 1e6,
                               "iterations_lost": offset / slope}
        # live results: snapshots every T steps streamed to pinned host memory by the library
        # while the integration continues; cost = extra time per snapshot over the same steps
        # integrated without live results
        for T in (250, 1000):
            n_cycles = 40
            wl = W.force_sweep(n_F=n_items, traj_per_set=1, n_steps=n_cycles * T)
            wl.snapshot_every = T
            with A.Ensemble(wl, stream=stream) as ens, torch.cuda.stream(stream):
                ens.set_params()
                mom_l = torch.empty((ens.n_snapshots(), n_items, 8), dtype=torch.float64, pin_memory=True)
                times = {}
                for mode in ("plain", "live", "plain", "live"):
                    A.abp_live(ens.ctx, mom_l if mode == "live" else None, None, None)
                    ens.reset()
                    ens.synchronize()
                    t0 = time.perf_counter()
                    ens.integrate(-1)
                    ens.synchronize()
                    times[mode] = time.perf_counter() - t0
                assert A.abp_live_ready(ens.ctx) == n_cycles
                A.abp_live(ens.ctx, None, None, None)
            per_it = times["plain"] / (n_cycles * T)
            extra = (times["live"] - times["plain"]) / n_cycles
            res["live_T%d" % T] = {"us_per_iteration": per_it * 1e6, "extra_us_per_snapshot": extra * 1e6,
                                   "iterations_lost": extra / per_it}
        out["%d_work_items" % n_items] = res
    return out


# ----------------------------------------------------------------------------- other workloads

def time_workload(A, stream, w, reps=1, lane_peak=None, **kw):
    """Integrate and reduce workload ``w`` ``reps`` times from a fresh initial condition (inputs
    resident on the device), timed with CUDA events on the library's stream."""
    import torch

    with A.Ensemble(w, stream=stream, **kw) as ens, torch.cuda.stream(stream):
        ens.set_params()
        ens.integrate(min(512, max(w.n_steps)))  # warm-up (first launches, autotuned choice)
        ens.results()
        times, res = [], None
        for _ in range(reps):
            ens.reset(w.seed)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ens.integrate(-1)
            res = ens.results()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b) * 1e-3)
        t = statistics.median(times)
        out = {"workload": w.name, "sets": w.n_sets, "trajectories": w.total_traj,
               "particle_steps": w.particle_steps, "seconds": t, "value": w.particle_steps / t, "unit": UNIT,
               "reps": reps, "tuning": ens.tuning(), "tiles": ens.tiles(), "timing": "CUDA events, integrate + reduce"}
        if lane_peak:
            # the same algorithmic count as the headline (the Heun step evaluates the drift twice)
            n_alg = N_ALG_HEUN if w.scheme == 1 else N_ALG
            out["roofline_frac"] = n_alg * out["value"] / (lane_peak * 1e12)
            out["roofline_basis"] = "%d lane-ops per particle-step over the whole workload time" % n_alg
        return out, res


def precision_leg(A, stream):
    """FP32 state against FP64 state on the same noise: 1,048,576 trajectories x 10^5 steps of the
    large-ensemble workload's parameters (D = 0.2, x0 uniform, v0 = e0 = 0, seed 4), final
    1,024-bin histograms of x mod L and v.  Reports the difference of the ensemble means in
    standard errors and the two-sample chi^2 of the histograms."""
    import numpy as np
    from paper_1104_2499_gb300 import workloads as W

    w = W.shrink(W.large_snapshots(), max_traj=1 << 20, max_steps=100_000, name="precision_1Mx1e5")
    w.snapshot_every = 0
    r32, m32 = time_workload(A, stream, w, 1)
    r64, m64 = time_workload(A, stream, w, 1, state_fp64=True)
    a, b = m32["moments"].cpu().numpy()[0], m64["moments"].cpu().numpy()[0]
    out = {"fp32": {"value": r32["value"], "mean_v": a[0], "se": a[1], "d_eff": a[3]},
           "fp64": {"value": r64["value"], "mean_v": b[0], "se": b[1], "d_eff": b[3]},
           "delta_mean_v_in_se": abs(a[0] - b[0]) / b[1], "d_eff_rel_diff": abs(a[3] - b[3]) / abs(b[3])}
    for key in ("hist_x", "hist_v"):
        h32 = m32[key].cpu().numpy()[-1, 0].astype(float)
        h64 = m64[key].cpu().numpy()[-1, 0].astype(float)
        k = (h32 + h64) > 0
        chi2 = float((((h32 - h64) ** 2)[k] / (h32 + h64)[k]).sum())
        out[key + "_chi2"] = {"chi2": chi2, "dof": int(k.sum()) - 1}
        try:
            from scipy import stats

            out[key + "_chi2"]["p"] = float(stats.chi2.sf(chi2, int(k.sum()) - 1))
        except Exception:
            pass
    return out


def items_leg(A, stream):
    """Time against the number of work items with the paper's protocol (Sec. 3.1): for every
    power of two from 2^0 to 2^16 parameter sets of the load sweep (one trajectory each, the
    paper's work items), 20 cycles of T steps each followed by the device reduction; the mean of
    the last 15 cycles is reported, for T = 10^3 and T = 10^4."""
    import torch
    from paper_1104_2499_gb300 import workloads as W

    out = []
    for T in (1000, 10_000):
        for k in range(0, 17):
            n = 1 << k
            w = W.force_sweep(n_F=n, traj_per_set=1, n_steps=20 * T)
            with A.Ensemble(w, stream=stream) as ens, torch.cuda.stream(stream):
                ens.set_params()
                mom = torch.empty((n, 8), dtype=torch.float64, device="cuda")
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
                for a, b in ev:
                    a.record(stream)
                    A.abp_integrate(ens.ctx, T)
                    A.abp_reduce(ens.ctx, mom, None, None)
                    b.record(stream)
                stream.synchronize()
                ms = statistics.mean(a.elapsed_time(b) for a, b in ev[5:])
                tl = ens.tiles()
            out.append({"steps": T, "work_items": n, "ms_per_cycle": ms, "value": n * T / (ms * 1e-3),
                        "tiles": tl["tiles"], "packed_tiles": tl["packed"], "narrow": tl["narrow"]})
    return out


def force_leg(A, stream, lane_peak=None):
    """The paper's benchmark observable (Fig. 2): mean velocity against the load F0, 64 values in
    [-1, 1], 4,096 trajectories x 10^5 steps each.  Reports the curve, the stall force (where
    <v> crosses zero, linear interpolation) and the efficiency -F0 <v> / q (power delivered
    against the load per unit energy influx into the depot)."""
    import numpy as np
    from paper_1104_2499_gb300 import workloads as W

    w = W.force_sweep()
    r, res = time_workload(A, stream, w, 1, lane_peak)
    mom = res["moments"].cpu().numpy()
    F = np.array([p["F0"] for p in w.sets])
    v, se = mom[:, 0], mom[:, 1]
    stall = []
    for i in range(len(F) - 1):
        if v[i] == 0.0 or (v[i] < 0.0) != (v[i + 1] < 0.0):
            stall.append(float(F[i] - v[i] * (F[i + 1] - F[i]) / (v[i + 1] - v[i])) if v[i + 1] != v[i] else float(F[i]))
    eff = -F * v / np.array([p["q"] for p in w.sets])
    r.update({"F0": F.tolist(), "mean_v": v.tolist(), "se": se.tolist(), "stall_force": stall,
              "max_efficiency": float(eff.max()), "F0_at_max_efficiency": float(F[int(eff.argmax())])})
    return r


def configs_leg(A, stream, names, lane_peak):
    """Every other workload of the benchmark suite, each timed with CUDA events on the library's
    stream (inputs resident, integrate + reduce), with its throughput and its fraction of the
    FP32-lane roofline."""
    from paper_1104_2499_gb300 import workloads as W

    if names == ["default"]:
        names = ["single", "single_heun", "single_xorshift", "uneven", "force", "heun", "xorshift",
                 "snapshots_slice", "precision", "items"]
    elif names == ["all"]:
        names = ["single", "single_heun", "single_xorshift", "uneven", "force", "heun", "xorshift",
                 "snapshots_slice", "snapshots", "precision", "items"]
    out = {}
    for name in names:
        t0 = time.perf_counter()
        if name == "single":
            out[name] = time_workload(A, stream, W.single_set(), 5, lane_peak)[0]
        elif name in ("single_heun", "single_xorshift"):
            # the same set with the stochastic Heun step, or with xorshift noise
            w = W.single_set()
            if name == "single_heun":
                w.scheme = 1
            else:
                w.noise = 1
            w.name += name[len("single"):]
            out[name] = time_workload(A, stream, w, 5, lane_peak)[0]
        elif name == "uneven":
            w = W.uneven_batch()
            r = time_workload(A, stream, w, 1, lane_peak)[0]
            # the schedule the autotuner did not choose, at its best trajectories per thread
            other = 2 if r["tuning"]["schedule"] == 1 else 1
            alt = time_workload(A, stream, w, 1, lane_peak, schedule=other)[0]
            r["other_schedule"] = {k: alt[k] for k in ("value", "seconds", "tuning", "roofline_frac")}
            r["cpu_oracle"] = oracle_subset_rate(w, 16)
            out[name] = r
        elif name == "force":
            out[name] = force_leg(A, stream, lane_peak)
        elif name == "snapshots":
            w = W.large_snapshots()
            out[name] = time_workload(A, stream, w, 1, lane_peak)[0]
            out[name]["cpu_oracle"] = oracle_subset_rate(w, 65536, 10_000)
        elif name == "snapshots_slice":
            # every trajectory of the large ensemble (67,108,864) over its first 2 x 10^4 steps, with
            # its 1,024-bin histograms of x mod L and of v every 10^4 steps
            w = W.large_snapshots(n_steps=20_000)
            w.name = "snapshots_67108864x20000_slice"
            out[name] = time_workload(A, stream, w, 1, lane_peak)[0]
            out[name]["cpu_oracle"] = oracle_subset_rate(w, 65536, 10_000)
        elif name == "uneven_slice":
            # all 512 sets of the uneven batch over their first 2 x 10^4 steps (1.3e11 particle-steps)
            # in the configuration chosen for the whole batch (work queue, 2 trajectories per thread,
            # items of 10^4 steps): its kernel in a launch short enough to profile
            w = W.shrink(W.uneven_batch(), max_steps=20_000, name="uneven_512sets_2e4steps")
            out[name] = time_workload(A, stream, w, 1, lane_peak, schedule=2, particles_per_thread=2,
                                      steps_per_launch=10_000)[0]
        elif name == "heun":
            w = W.sweep_grid()
            w.scheme, w.name = 1, w.name + "_heun"
            out[name] = time_workload(A, stream, w, 1, lane_peak)[0]
        elif name == "xorshift":
            w = W.sweep_grid()
            w.noise, w.name = 1, w.name + "_xorshift"
            out[name] = time_workload(A, stream, w, 1, lane_peak)[0]
        elif name == "precision":
            out[name] = precision_leg(A, stream)
        elif name == "items":
            out[name] = items_leg(A, stream)
        else:
            raise SystemExit("unknown workload in --configs: " + name)
        if isinstance(out[name], dict):
            out[name]["leg_wall_s"] = time.perf_counter() - t0
    return out


# ----------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1104_2499_gb300 import abp as A
    from paper_1104_2499_gb300 import build as B
    from paper_1104_2499_gb300 import shard

    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
        B.build()
    A.lib()

    stream = torch.cuda.Stream()
    if args.adjoint_only:
        n_traj, n_steps = (int(v) for v in args.adjoint_only.split(","))
        print(json.dumps({"adjoint": adjoint_leg(A, stream, size=(n_traj, n_steps), accuracy=False)}), flush=True)
        return
    w = workload(args)
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    if args.profile_config:
        pk, _ = peaks()
        lane_peak = n_sm * LANES_PER_SM * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        print(json.dumps({"configs": configs_leg(A, stream, [args.profile_config], lane_peak)}), flush=True)
        return
    # weak scaling: every rank integrates its own copy of the sweep with distinct trajectory ids
    ens = A.Ensemble(w, stream=stream, particles_per_thread=args.ppt, steps_per_launch=args.steps_per_launch,
                     traj_base=shard.replica_traj_base(rank, w.total_traj), schedule=args.schedule)
    S = w.n_sets
    mom = torch.empty((S, 8), dtype=torch.float64, device="cuda")
    ns = 1
    hx = torch.empty((ns, S, w.hist_x_bins), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    with torch.cuda.stream(stream):
        ens.set_params()
    tuning = ens.tuning()
    spl = tuning["steps_per_item"]
    queue = tuning["schedule"] == 2
    # work queue: one persistent launch per step; lockstep: one launch per steps_per_launch
    n_launch = 1 if queue else math.ceil(w.n_steps[0] / spl)
    chunk = -1 if queue else spl

    def gpu_step(ev_k=None):
        ens.reset(w.seed)
        for j in range(n_launch):
            if ev_k is not None:
                ev_k[j][0].record(stream)
            ens.integrate(chunk)
            if ev_k is not None:
                ev_k[j][1].record(stream)
        A.abp_reduce(ens.ctx, mom, hx, None)
        if dist is not None:
            with torch.cuda.stream(stream):
                shard.all_reduce_sums_(mom, dist.all_reduce, [m * world for m in w.n_traj], w.n_steps, w.dt, stream)

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            gpu_step()
    stream.synchronize()

    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev_kern = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_launch)]
               for _ in range(args.steps)]
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else None
    except Exception:
        gpu_id = None
    launches0 = ens.launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev_step[k][0].record(stream)
                gpu_step(ev_kern[k])
                ev_step[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    launches = ens.launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    total_ms = sum(step_ms)
    kern_ms = [a.elapsed_time(b) for row in ev_kern for a, b in row]
    t_max = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_ms = float(t_max.item())
    ps_step = w.particle_steps
    value = world * ps_step * args.steps / (total_ms * 1e-3)
    moments = mom.cpu().numpy()
    clocks = clk.summary()

    # e2e: the same step through the C ABI with host buffers (params uploaded from host
    # memory, moments and histograms read back into pinned host memory)
    e2e = None
    if not args.no_e2e:
        mom_h = torch.empty((S, 8), dtype=torch.float64, pin_memory=True)
        hx_h = torch.empty((ns, S, w.hist_x_bins), dtype=torch.int32, pin_memory=True)
        n_tiles = sum(math.ceil(m / (256 * tuning["particles_per_thread"])) for m in w.n_traj)
        n_rounds = math.ceil(w.n_steps[0] / spl) if queue else 0
        # what abp_set_params uploads -- parameters and step counts, set tile ranges, set
        # offsets and order, the tile table (first trajectory, count, set) and the work-queue
        # order -- plus the work queue's round starts
        h2d = S * (72 + 8) + 4 * (S + 1) + 8 * (S + 1) + 4 * S + (8 + 4 + 4 + 4) * n_tiles + (
            4 * (n_rounds + 1) if queue else 0)
        d2h = mom_h.numel() * 8 + hx_h.numel() * 4
        times = []
        # the inputs as a user holds them on the host: the parameter grid [sets, 9] float64,
        # ensemble sizes and step counts (marshalled without copies, uploaded by the call)
        p_h, m_h, n_h = w.param_matrix(), np.asarray(w.n_traj, np.int64), np.asarray(w.n_steps, np.int64)
        with torch.cuda.stream(stream):
            for k in range(max(1, args.steps)):
                flush.zero_()
                stream.synchronize()
                t0 = time.perf_counter()
                A.abp_set_params(ens.ctx, p_h, m_h, n_h)
                A.abp_integrate(ens.ctx, -1)
                A.abp_reduce(ens.ctx, mom_h, hx_h, None)
                times.append(time.perf_counter() - t0)
        e2e = {"value": world * ps_step / statistics.mean(times), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    pk, pk_kind = peaks()
    f_max = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    peak = n_sm * LANES_PER_SM * f_max / 1e12  # T lane-ops/s
    ps_launch = ps_step // n_launch
    kern_avg = statistics.mean(kern_ms) * 1e-3
    achieved = N_ALG * ps_launch / kern_avg / 1e12
    kname = ("persistent_kernel<float,%d>" if queue else "integrate_kernel<float,%d>") % tuning["particles_per_thread"]
    traffic = None
    # the work-queue figure holds for the launch it was taken from (items of 10^4 steps)
    if kname in TRAFFIC_PER_LAUNCH and not args.small and (not queue or spl == 10_000):
        b_cap, t_cap = TRAFFIC_PER_LAUNCH[kname]
        traffic = b_cap * w.total_traj / t_cap
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-op/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch", "kernel": kname, "n_alg_per_particle_step": N_ALG,
            "peak_basis": "%d SMs x %d FP32 lanes x %.0f MHz (%s sm_max_mhz)" % (n_sm, LANES_PER_SM, f_max / 1e6,
                                                                                pk_kind),
            "launch_ms_avg": kern_avg * 1e3, "particle_steps_per_launch": ps_launch,
            "particle_steps_per_s_in_kernel": ps_launch / kern_avg}
    if clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (n_sm * LANES_PER_SM * clocks["sm_mhz"] * 1e6 / 1e12)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, desc, parity, one_core = oracle_sample(w, args.cpu_seconds, gpu_moments=moments)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "value_1_core": one_core}
        if parity:
            cpu["parity_mean_v"] = parity

    adj = None
    if rank == 0 and world == 1 and not args.no_adjoint:
        adj = adjoint_leg(A, stream, small=args.small)
    vis = visualisation_leg(A, stream) if (rank == 0 and world == 1 and not args.no_visualisation) else None
    cfg_names = [c for c in args.configs.split(",") if c and c != "none"]
    cfgs = configs_leg(A, stream, cfg_names, peak) if (rank == 0 and world == 1 and cfg_names) else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(w, args, {"schedule": "work queue" if queue else "lockstep",
                                                "steps_per_item": spl,
                                                "particles_per_thread": tuning["particles_per_thread"],
                                                "resident_blocks": tuning["blocks"],
                                                "integrator_launches_per_step": n_launch,
                                                "parallelism": "dp%d (independent replicas)" % world}),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "adjoint": adj, "visualisation": vis, "configs": cfgs,
                "wall_s_timed": wall, "sm_count": n_sm, "device": props.name}
        print(json.dumps(line), flush=True)
    ens.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
