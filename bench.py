"""Benchmark of the LLG + cavity hot path on GB300.

Default workload: the largest grid -- a CPW-like Permalloy film of 1024 x 1024
x 8 cells of 4 nm (8.4 M cells; Ms 8e5 A/m, A 1.3e-11 J/m, alpha 0.01, bias
30 mT along x), coupled to the cavity through a Lorentzian profile
g(x) = g0 / (1 + (x / 500 nm)^2), g0/2pi = 20 MHz, omega_c at the uniform
mode, kappa/2pi = 10 MHz, integrated by Dormand-Prince (tol 1e-6).  One step =
one Dormand-Prince attempt.  Other workloads: --workload yig_wire (the 21-value
omega_c sweep of a 256x64x16 YIG wire, one batch), batched (64 mixed-grid
instances, CUDA graphs), adjoint (forward + discrete adjoint), film.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

Prints one JSON line.  `value` counts accepted cell-steps (cells x accepted
steps, summed over instances and ranks) per second of device time; the
roofline object reports the dominant kernel's algorithmic bytes per launch over
its event-timed duration, against the measured HBM copy bandwidth.  `parity`
gives the error against the FP64 oracle, which replays the accepted steps of
the first two (warm-up) attempts of instance 0 from the same initial state;
the time of that replay is the CPU baseline.
Multi-GPU (torchrun): every rank integrates its own instances (independent,
no data exchange; weak scaling).  The reference arm times the FP64 CPU oracle
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LLG cell-steps/s on 1 GB300 (plain vs batched) at max|Δm|≤1e-5; % HBM roofline"
FALLBACK_HBM_GBS = 6800.0
SRC_DIR = os.path.join(ROOT, "paper_2410_00966_gb300", "csrc")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def source_hash() -> str:
    h = hashlib.sha256()
    for fn in sorted(os.listdir(SRC_DIR)):
        with open(os.path.join(SRC_DIR, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None
    when there is none or the kernel sources changed since it was taken."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    cur = source_hash()
    with open(TRAFFIC_FILE) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kv = dict(zip(*[iter(line.split())] * 2))
            if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("source") == cur:
                return float(kv["bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def workload_instances(name: str, rank: int):
    import synthetic
    if name == "yig_wire":
        w = synthetic.yig_wire_sweep()
    elif name == "film":
        w = synthetic.film_32()
    elif name == "large":
        w = synthetic.large_cpw()
    elif name == "batched":
        w = synthetic.batched_map()
    else:
        raise SystemExit(f"unknown workload {name}")
    if rank:
        # weak scaling: each rank integrates its own sweep (different seeds)
        w.instances = [synthetic.replace(I, seed=synthetic.derive_seed(100 + rank, k)) for k, I in
                       enumerate(w.instances)]
    return w


def reduce_over_ranks(dist, device, ms: float, cell_steps: float):
    """Whole-job timing: the slowest rank's time and the sum of every rank's work."""
    if dist is None:
        return ms, float(cell_steps)
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(cell_steps)], device=device, dtype=torch.float64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def oracle_for(I, w):
    """The FP64 oracle set up like instance I of workload w (E-mode cavity)."""
    import numpy as np
    import oracle
    o = oracle.Oracle(I.nx, I.ny, I.nz, I.d, I.d, I.d, I.Ms, I.Aex, I.alpha, Ku=I.Ku, axis=I.axis)
    o.set_m(I.m0().astype(np.float64))
    o.set_bias(I.bias)
    prof = I.coupling_profile()
    o.set_cavity(I.omega_c, I.kappa, I.g, profile=None if prof is None else prof.astype(np.float64))
    o.set_integrator(oracle.DP45 if w.integrator == "dp45" else oracle.RK4, w.tol, oracle.CAV_E)
    return o


def cpu_oracle_sample(w, attempts: int):
    """Time the FP64 oracle on instance 0 of the workload for `attempts` steps
    (then on until about 10 s of CPU work)."""
    o = oracle_for(w.instances[0], w)
    o.step(1, w.dt)   # first attempt outside the timing (sets the trial step)
    t0 = time.perf_counter()
    acc = 0
    done = 0
    while done < attempts or (time.perf_counter() - t0 < 10.0 and done < 50 * attempts):
        acc += o.step(1, 0.0 if w.integrator == "dp45" else w.dt)
        done += 1
    dt = time.perf_counter() - t0
    return acc * w.instances[0].n / dt, dt, acc


def oracle_replay_parity(w, prefix):
    """Replay the GPU's accepted steps of the prefix (instance 0) in the oracle
    from the same initial state; returns the error figures and the replay's
    CPU throughput (the CPU baseline of the large workload)."""
    import numpy as np
    import oracle
    I = w.instances[0]
    t_setup = time.perf_counter()
    o = oracle_for(I, w)
    t_setup = time.perf_counter() - t_setup
    hist = prefix["dt_history"]
    t0 = time.perf_counter()
    if w.integrator == "dp45":
        o.replay(hist)
    else:
        o.step(len(hist), w.dt)
    el = time.perf_counter() - t0
    m_o = o.get_m()
    dm = float(np.abs(prefix["m"].astype(np.float64) - m_o).max())
    oc = o.cavity()
    c = prefix["cavity"]
    a_o = complex(oc["re_alpha"], oc["im_alpha"])
    a_g = complex(c["re_alpha"], c["im_alpha"])
    return {"max_dm": dm, "alpha_rel_err": abs(a_g - a_o) / abs(a_o) if a_o != 0 else None,
            "alpha_gpu": [a_g.real, a_g.imag], "alpha_oracle": [a_o.real, a_o.imag],
            "steps_replayed": len(hist), "t_replayed": float(np.sum(hist)), "instance": 0,
            "oracle_setup_s": t_setup, "oracle_replay_s": el,
            "bar": "max|dm| <= 1e-5 per component"}, len(hist) * I.n / el, el


def run_reference(args):
    """The FP64 oracle on instance 0 of the workload, one attempt (step) at a
    time on the host cores; the number of timed steps is capped so that the
    run ends within a few minutes (one attempt of the largest grid takes tens
    of seconds)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = workload_instances(args.workload, 0)
    I = w.instances[0]
    dp = w.integrator == "dp45"
    o = oracle_for(I, w)
    budget_s = 60.0 if args.workload == "large" else 240.0
    warm = 1 if args.workload == "large" else args.warmup
    o.step(1, w.dt)
    for _ in range(warm - 1):
        o.step(1, 0.0 if dp else w.dt)
    t0 = time.perf_counter()
    acc = 0
    steps = 0
    while steps < args.steps and (steps == 0 or time.perf_counter() - t0 < budget_s):
        acc += o.step(1, 0.0 if dp else w.dt)
        steps += 1
    el = time.perf_counter() - t0
    value = acc * I.n / el
    cores = oracle.set_threads(0)
    sample = (f"instance 0 of the workload ({I.nx}x{I.ny}x{I.nz} cells), {steps} {w.integrator} attempts "
              f"({acc} accepted) after {warm} untimed, {el:.1f} s; steps capped by a {budget_s:.0f} s budget")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": args.gpus,
        "steps": steps, "steps_requested": args.steps, "warmup": warm, "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "instances_timed": 1, "cells_per_instance": I.n, "integrator": w.integrator},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2410_00966_gb300 as pkg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = workload_instances(args.workload, rank)
    if args.instances:
        w.instances = w.instances[:args.instances]
    if args.grid:
        # the same workload on another grid (profiling a smaller case of the same kernels)
        import synthetic
        nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
        w.instances = [synthetic.scaled(I, nx, ny, nz) for I in w.instances]
    I0 = w.instances[0]
    B = len(w.instances)
    dp = w.integrator == "dp45"
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        sim = pkg.Sim(I0.nx, I0.ny, I0.nz, I0.d, I0.d, I0.d, I0.Ms, I0.Aex, I0.alpha, Ku=I0.Ku, axis=I0.axis,
                      batch=B, device=local)
        prof = I0.coupling_profile()
        m0 = [I.m0() for I in w.instances]
        for b, I in enumerate(w.instances):
            sim.set_m(m0[b], inst=b)
            sim.set_bias(I.bias, inst=b)
            sim.set_cavity(I.omega_c, I.kappa, I.g, profile=prof if b == 0 else None, inst=b)
        sim.set_integrator(pkg.MMCQ_DP45 if dp else pkg.MMCQ_RK4, w.tol, pkg.MMCQ_CAVITY_E)
        if dp:
            sim.set_horizon(w.horizon)
        info = sim.info()
        if args.plan:
            # a given launch plan (e.g. the one a plain run chose, to profile
            # the same kernels under ncu, whose timings would mislead the tuner)
            sim.set_tuning(json.loads(args.plan))
            tuning = sim.tuning()
        else:
            tuning = sim.autotune(reps=7)   # launch parameters of this grid, chosen by timing
        # warm-up; the state of instance 0 after the first two attempts is
        # kept for the parity check against the oracle (after the timing)
        sim.step(1, w.dt)
        sim.step(1, 0.0 if dp else w.dt)
        prefix = None
        if rank == 0 and not args.no_cpu_baseline:
            prefix = {"m": sim.get_m(0), "cavity": sim.cavity(0), "dt_history": sim.dt_history(0)}
        sim.step(max(args.warmup - 2, 0), 0.0 if dp else w.dt)
        sim.sync()
        acc0 = sum(c["accepted"] for c in sim.cavity(-1))
        launches0 = sim.launch_count()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sim.profile(True)
        e0.record(stream)
        sim.step(args.steps, 0.0 if dp else w.dt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sim.profile(False)
        if dist:
            dist.barrier()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        cav = sim.cavity(-1)
        sim.sync()
        acc1 = sum(c["accepted"] for c in cav)
        rej = sum(c["rejected"] for c in cav)
        launches = sim.launch_count() - launches0
        kstats = sim.profile_read()
        cell_steps = (acc1 - acc0) * I0.n
        ms_max, total_cell_steps = reduce_over_ranks(dist, dev, ms, cell_steps)
        value = total_cell_steps / (ms_max / 1e3)

        # dominant kernel and its roofline
        top = max(kstats, key=lambda k: k["total_ms"]) if kstats else None
        peak, peak_kind = measured_peak()
        roof = None
        if top:
            per_launch_bytes = top["bytes"] / top["launches"]
            avg_s = top["total_ms"] / top["launches"] / 1e3
            achieved = per_launch_bytes / avg_s / 1e9
            traffic = ncu_traffic(top["name"], args.workload)
            roof = {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_s * 1e3,
                    "share_of_step": top["total_ms"] / sum(k["total_ms"] for k in kstats)}
        kernels = [{"name": k["name"], "launches": k["launches"], "ms": round(k["total_ms"], 3),
                    "GB/s": round(k["bytes"] / (k["total_ms"] / 1e3) / 1e9, 1) if k["total_ms"] > 0 else None}
                   for k in kstats]
        step_bytes = sum(k["bytes"] for k in kstats)

        # end to end through the C ABI with host buffers: pinned m of every
        # instance in, one step, the cavity read-out of every instance back
        # each step, the final m of every instance back.
        e2e = None
        if not args.no_e2e:
            host_m = torch.empty((B, I0.n, 3), dtype=torch.float32, pin_memory=True)
            for b in range(B):
                host_m[b].copy_(torch.from_numpy(sim.get_m(b)))
            out_m = torch.empty((B, I0.n, 3), dtype=torch.float32, pin_memory=True)
            acc_a = sum(c["accepted"] for c in sim.cavity(-1))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for b in range(B):
                sim.set_m(host_m[b], inst=b)
            # every step's read-out comes back; step k + 1 is enqueued before
            # the host waits for the read-out of step k
            sim.step(1, 0.0 if dp else w.dt)
            sim.post_cavity()
            for _ in range(args.steps - 1):
                sim.step(1, 0.0 if dp else w.dt)
                sim.post_cavity()
                cv = sim.take_cavity()
            cv = sim.take_cavity()
            for b in range(B):
                sim.get_m(b, out=out_m[b])
            el = time.perf_counter() - t0
            acc_b = sum(c["accepted"] for c in cv)
            e2e_val = (acc_b - acc_a) * I0.n / el
            if dist:
                t = torch.tensor([e2e_val], device=dev, dtype=torch.float64)
                dist.all_reduce(t, op=dist.ReduceOp.SUM)
                e2e_val = float(t.item())
            h2d = B * I0.n * 3 * 4 / args.steps
            d2h = (B * I0.n * 3 * 4) / args.steps + B * ctypes_sizeof_cavity(pkg)
            e2e = {"value": e2e_val, "unit": "cell-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "note": "C-ABI calls with pinned host buffers; per step one attempt + read-out of all instances "
                           "(pipelined: mmcq_post_cavity / mmcq_take_cavity one step behind)"}
        sim.close()

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = oracle.set_threads(0)
        if args.workload == "large":
            # the replay of the warm-up prefix is both the parity check and the
            # CPU baseline (one attempt of this grid is tens of seconds of CPU)
            parity, v, el = oracle_replay_parity(w, prefix)
            cpu = {"value": v, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                   "sample": f"FP64 replay of the {parity['steps_replayed']} accepted {w.integrator} steps of the "
                             f"first two attempts of instance 0 ({I0.nx}x{I0.ny}x{I0.nz} cells), {el:.1f} s"}
        else:
            attempts = 3 if args.workload == "yig_wire" else 20
            v, el, acc = cpu_oracle_sample(w, attempts)
            oracle.set_threads(1)
            v1, el1, acc_1 = cpu_oracle_sample(w, 1)
            oracle.set_threads(0)
            cpu = {"value": v, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                   "sample": f"{acc} accepted {w.integrator} steps of instance 0 ({I0.nx}x{I0.ny}x{I0.nz} cells), "
                             f"{el:.1f} s",
                   "single_thread": {"value": v1, "sample": f"{acc_1} accepted steps, {el1:.1f} s"}}
            if prefix is not None:
                parity, _, _ = oracle_replay_parity(w, prefix)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "instances_per_gpu": B, "grid": [I0.nx, I0.ny, I0.nz],
                       "cells_per_instance": I0.n, "integrator": w.integrator, "tol": w.tol,
                       "cavity_mode": "E", "parallelism": "independent instances per rank",
                       "accepted_steps": acc1 - acc0, "rejected_steps": rej,
                       "l2": f"inputs larger than L2 ({info['device_bytes'] / 1e9:.2f} GB resident)",
                       "padded": [info["px"], info["py"], info["pz"]], "tile": info["tile"], "tuning": tuning,
                       "algorithmic_bytes_per_step": step_bytes / args.steps,
                       "field_evals_per_s": B * (6 if dp else 4) * args.steps / (ms_max / 1e3),
                       "step_model_efficiency": (step_bytes / args.steps) / (ms_max / args.steps / 1e3) / 1e9 / peak},
            "roofline": roof,
            "cpu_baseline": cpu,
            "parity": parity,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches,
            "kernels": kernels,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """The batched anticrossing map: 64 Permalloy instances on four grid sizes
    (32x32x1, 64x64x2, 128x128x2, 256x256x4), one batched handle per grid
    size, each with launch parameters chosen by mmcq_autotune, all stepped
    together as one CUDA graph per chunk of RK4 steps (mmcq_group_*).  A step
    advances every instance by one RK4 step.  The line also gives the same
    graphs under the fixed launch rules."""
    import torch

    import paper_2410_00966_gb300 as pkg
    import synthetic

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synthetic.batched_map()
    shapes = {}
    for I in w.instances:
        shapes.setdefault((I.nx, I.ny, I.nz), []).append(I)
    chunk = 25
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        sims = []
        for (nx, ny, nz), insts in sorted(shapes.items()):
            I0 = insts[0]
            sim = pkg.Sim(nx, ny, nz, I0.d, I0.d, I0.d, I0.Ms, I0.Aex, I0.alpha, batch=len(insts), device=local)
            for b, I in enumerate(insts):
                sim.set_m(I.m0(), inst=b)
                sim.set_bias(I.bias, inst=b)
                sim.set_cavity(I.omega_c, I.kappa, I.g, inst=b)
            sim.set_integrator(pkg.MMCQ_RK4, w.tol, pkg.MMCQ_CAVITY_E)
            sims.append(sim)
        cells = sum(s.n * s.batch for s in sims)
        # launch parameters per grid shape, chosen by timing (mmcq_autotune)
        tuning = {"x".join(map(str, s.shape[::-1])): s.autotune(reps=7) for s in sims}
        g = pkg.Group(sims, chunk=chunk)
        steps = max(chunk, (args.steps // chunk) * chunk)

        def timed(fn):
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            # the group's last work is ordered before each handle's stream
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1)

        g.step(max(args.warmup, 1) * chunk, w.dt)
        for s in sims:
            s.step(args.warmup, w.dt)
        launches0 = sum(s.launch_count() for s in sims)
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        ms_graph = timed(lambda: g.step(steps, w.dt))
        clk = clocks.stop()
        launches = sum(s.launch_count() for s in sims) - launches0

        def eager():
            for s in sims:
                s.step(steps, w.dt)
        ms_eager = timed(eager)
        # the same graphs with the fixed launch rules instead of the tuned plans
        g.close()
        for s in sims:
            s.set_tuning(None)
        g = pkg.Group(sims, chunk=chunk)
        g.step(chunk, w.dt)
        ms_rules = timed(lambda: g.step(steps, w.dt))
        for s, (_, t) in zip(sims, tuning.items()):
            s.set_tuning(t)
        for s in sims:
            s.profile(True)
        ms_prof = timed(lambda: [s.step(chunk, w.dt) for s in sims])
        stats = {}
        for s in sims:
            for k in s.profile_read():
                d = stats.setdefault(k["name"], {"launches": 0, "total_ms": 0.0, "bytes": 0.0})
                d["launches"] += k["launches"]; d["total_ms"] += k["total_ms"]; d["bytes"] += k["bytes"]
            s.profile(False)
        g.close()
        for s in sims:
            s.close()
    value = cells * steps / (ms_graph / 1e3)
    peak, peak_kind = measured_peak()
    top_name = max(stats, key=lambda k: stats[k]["total_ms"])
    top = stats[top_name]
    achieved = top["bytes"] / (top["total_ms"] / 1e3) / 1e9
    # every handle's algorithmic bytes of one step (the profiled pass ran
    # `chunk` steps), over the graph's time per step: the whole map's share
    # of the peak while its handles run side by side
    step_bytes = sum(d["bytes"] for d in stats.values()) / chunk
    step_eff = step_bytes / (ms_graph / steps / 1e3) / 1e9 / peak
    line = {
        "metric": "LLG cell-steps/s, batched anticrossing map (mixed grids, CUDA graph)", "value": value,
        "unit": "cell-steps/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms_graph / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "instances": len(w.instances),
                   "grids": {f"{a}x{b}x{c}": len(v) for (a, b, c), v in sorted(shapes.items())},
                   "cells_per_step": cells, "integrator": "rk4", "dt": w.dt, "graph_chunk": chunk,
                   "eager_value": cells * steps / (ms_eager / 1e3),
                   "fixed_rules_value": cells * steps / (ms_rules / 1e3),
                   "tuning": tuning,
                   "algorithmic_bytes_per_step": step_bytes, "step_model_efficiency": step_eff,
                   "l2": "working set below L2 (small grids; latency and launch bound)"},
        "roofline": {"bound": "hbm", "kernel": top_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                     "note": "from an eager profiled pass (per-launch events, handles one after another); "
                             "config.step_model_efficiency is the graph run with the handles side by side"},
        "clocks": clk, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args):
    """Gradient workload: the vortex disk (128x128x4 cells of 2 nm, Ms map,
    65 536 cells), `steps` RK4 steps forward and the discrete adjoint back
    (checkpoints every 64 steps), objective = photon number averaged over the
    last fifth of the run.  value = cells x steps / (forward + adjoint time)."""
    import torch

    import paper_2410_00966_gb300 as pkg
    import synthetic

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    I, ms, m0 = synthetic.disk_vortex()
    dt = 5e-14
    steps = max(args.steps, 8)
    sim = pkg.Sim(I.nx, I.ny, I.nz, I.d, I.d, I.d, I.Ms, I.Aex, I.alpha, device=local)
    sim.set_ms_map(ms)
    sim.set_m(m0)
    sim.set_cavity(I.omega_c, I.kappa, I.g)

    def run(n):
        sim.set_m(m0)
        sim.reset_cavity()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = sim.adjoint_rk4(n, dt, wavg=1.0, window=max(1, n // 5), ckpt_every=64, ms_grad=True)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, out

    for _ in range(max(args.warmup, 1)):
        run(8)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    el, (J, g, gms) = run(steps)
    clk = clocks.stop()
    sim.set_m(m0)
    sim.reset_cavity()
    sim.set_integrator(pkg.MMCQ_RK4, 0.0, pkg.MMCQ_CAVITY_E)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sim.step(steps, dt)
    sim.sync()
    el_f = time.perf_counter() - t0
    cells = I.n
    line = {
        "metric": "LLG cell-steps/s, forward + discrete adjoint (gradients w.r.t. bias, g, omega_c, kappa, Ms map)",
        "value": cells * steps / el, "unit": "cell-steps/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "vortex disk 128x128x4 @2nm, Ms map, photon-number objective", "cells": cells,
                   "dt": dt, "checkpoint_every": 64, "forward_only_value": cells * steps / el_f,
                   "J": float(J[0]), "grad": [float(v) for v in g[0]],
                   "timing": "host clock around the synchronous adjoint call"},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    sim.close()
    return 0


def ctypes_sizeof_cavity(pkg):
    import ctypes
    return ctypes.sizeof(pkg.mmcq_cavity)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "yig_wire", "film", "batched", "adjoint"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--instances", type=int, default=0, help="use only the first N instances (profiling)")
    ap.add_argument("--grid", default="", help="NXxNYxNZ: run the workload on this grid instead (profiling)")
    ap.add_argument("--plan", default="", help="launch plan as JSON (x_rows, col_groups, z_split, x_pipe) "
                                               "instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    from paper_2410_00966_gb300 import build
    build.build()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
