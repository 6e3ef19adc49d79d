#!/usr/bin/env python
"""Projection-step throughput of the GB300 pressure-Poisson path.

One step = one pass of the whole hot path on a 256^3 grid: geometry setup
from phi (curvature, ghost-fluid faces, jump source, coarse hierarchy,
coarsest inverse), rhs = div u* with the jump, the pressure solve to relative
residual 1e-10 (MG-preconditioned CG; FP64, or mixed FP32/FP64 refinement),
the gauge and the face-velocity correction.  Every step gets a fresh seeded
16-mode u*.  The headline value is the mixed-precision form; the plain FP64
form is measured on the same inputs and reported under "modes".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs independent replicas (the solve does
not shard: one grid per GPU); value = steps of all ranks / max time.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pressure solves/s at 256³ to res 1e-10: FP64 MG vs mixed+learned; HBM % peak"
UNIT = "solves/s"
WORKLOAD = "bubble256"
TOL = 1e-10


def workload_desc(n):
    return ("bubble256: %d^3 cells on the unit cube, periodic x,y / wall z, one gas bubble "
            "R=0.15 at (0.5,0.5,0.4), rho_l=1, rho_g=1e-3, sigma=0.07, fresh seeded 16-mode u* "
            "per step, solve to relative residual 1e-10" % n)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(index)], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = self.t1 = None
        time.sleep(0.5)  # let the sampler start before the timed region

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                rows.append(dict(ts=ts, sm=float(parts[2]), max=float(parts[3]),
                                 power=float(parts[4]), hw=parts[6], hwt=parts[7], swt=parts[8],
                                 pcap=parts[9]))
            except ValueError:
                continue
        os.unlink(self.path)
        # samples taken inside the timed region (all of them if none fell inside)
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if self.t0 <= r["ts"] <= self.t1]
            if inside:
                rows = inside
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["max"] for r in rows),
                "power_w_max": max(r["power"] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# --------------------------------------------------------------- CPU oracle
def cpu_baseline(n, cg_iters=100):
    """The FP64 CPU oracle as it stands, on this host's cores: assembly and
    projection plus `cg_iters` Jacobi-PCG iterations at n^3 are timed; the
    iterations a solve to 1e-10 needs come from a full oracle solve of the
    same workload at (n/2)^3, doubled (CG iterations grow linearly in n)."""
    import oracle
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    bc = (synth.PERIODIC, synth.PERIODIC, synth.NEUMANN)
    cores = os.cpu_count() or 1
    # iteration count from the half-size solve (untimed)
    m = n // 2
    hm = 1.0 / m
    phi_m = synth.level_set((m, m, m), hm, w["bubbles"])
    u_m = synth.velocity(w["useed"], (m, m, m), hm)
    res_m = oracle.solve(phi_m, oracle.divergence(*u_m, hm), hm, w["rho_l"], w["rho_g"],
                         w["sigma"], bc, tol=TOL)
    iters_est = 2 * max(res_m["iters"], 1)
    h = 1.0 / n
    phi = synth.level_set((n, n, n), h, w["bubbles"])
    u = synth.velocity(w["useed"], (n, n, n), h)
    t0 = time.perf_counter()
    rhs = oracle.divergence(*u, h)
    kap, f, J, b = oracle.assemble(phi, rhs, h, w["rho_l"], w["rho_g"], w["sigma"], bc)
    t1 = time.perf_counter()
    x, _, _ = oracle.cg(f, b, h, bc, tol=1e-30, maxit=cg_iters)
    t2 = time.perf_counter()
    oracle.project(phi, kap, f, x, *u, h, w["sigma"], bc)
    t3 = time.perf_counter()
    t_solve = (t1 - t0) + (t3 - t2) + (t2 - t1) / cg_iters * iters_est
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": ("C oracle (OpenMP, %d threads): assembly + projection + %d Jacobi-PCG "
                       "iterations timed at %d^3 (%.2f s); %d iterations to 1e-10 estimated as 2x "
                       "a full oracle solve of the same workload at %d^3 (%d iterations)"
                       % (cores, cg_iters, n, t3 - t0, iters_est, m, res_m["iters"])),
            "seconds_per_solve_est": t_solve}


def run_reference(args, rank):
    """Reference arm: the CPU oracle itself on this host's cores."""
    if rank != 0:
        return
    n = args.n
    cg_iters = 40
    import oracle
    import synth
    oracle.build()
    w = synth.WORKLOADS[WORKLOAD]
    bc = (synth.PERIODIC, synth.PERIODIC, synth.NEUMANN)
    m = n // 2
    hm = 1.0 / m
    phi_m = synth.level_set((m, m, m), hm, w["bubbles"])
    u_m = synth.velocity(w["useed"], (m, m, m), hm)
    res_m = oracle.solve(phi_m, oracle.divergence(*u_m, hm), hm, w["rho_l"], w["rho_g"],
                         w["sigma"], bc, tol=TOL)
    iters_est = 2 * max(res_m["iters"], 1)
    h = 1.0 / n
    phi = synth.level_set((n, n, n), h, w["bubbles"])
    times = []
    for step in range(args.warmup + args.steps):
        u = synth.velocity(1000 + step, (n, n, n), h)
        t0 = time.perf_counter()
        rhs = oracle.divergence(*u, h)
        kap, f, J, b = oracle.assemble(phi, rhs, h, w["rho_l"], w["rho_g"], w["sigma"], bc)
        t1 = time.perf_counter()
        x, _, _ = oracle.cg(f, b, h, bc, tol=1e-30, maxit=cg_iters)
        t2 = time.perf_counter()
        oracle.project(phi, kap, f, x, *u, h, w["sigma"], bc)
        t3 = time.perf_counter()
        if step >= args.warmup:
            times.append((t1 - t0) + (t3 - t2) + (t2 - t1) / cg_iters * iters_est)
    t = sum(times)
    value = len(times) / t
    cores = os.cpu_count() or 1
    sample = ("each step: C oracle (OpenMP, %d threads) assembly + projection + %d Jacobi-PCG "
              "iterations at %d^3, CG time scaled to %d iterations (2x a full oracle solve at "
              "%d^3: %d iterations)" % (cores, cg_iters, n, iters_est, m, res_m["iters"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(n), "grid": [n, n, n]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- multi-rank
def max_over_ranks(ms, world, device=None):
    """The slowest rank's timed-region length (ms): replicas run the same
    number of steps, so whole-job throughput is world * K / max(ms)."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, ms_max):
    """Whole-job solves per second: every rank solves `steps` problems."""
    return world * steps / (ms_max * 1e-3)


# ------------------------------------------------------------------- GPU arm
def run_mine(args, rank, world, local_rank):
    import torch
    import synth
    from paper_2312_11740_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2312_11740_gb300 import Net, Poisson, mp_poisson_project_step_host
    from paper_2312_11740_gb300 import mp_poisson_set_net

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = args.n
    h = 1.0 / n
    shape = (n, n, n)
    w = synth.WORKLOADS[WORKLOAD]
    bc = (synth.PERIODIC, synth.PERIODIC, synth.NEUMANN)
    phi = torch.from_numpy(synth.level_set(shape, h, w["bubbles"])).to(dev)
    nprof = min(args.steps, 3)
    nsteps = args.warmup + args.steps + nprof
    seeds = [100000 * (rank + 1) + s for s in range(nsteps)]

    def fresh_u(count=nsteps):
        return [synth.velocity(sd, shape, h, device=dev) for sd in seeds[:count]]

    stream = torch.cuda.Stream(device=dev)
    results = {}
    # (precision, initial guess): fp64 and mixed from zero; learned = mixed with the
    # packaged network (trained at 128^3) run on the half-resolution grid
    mode_cfg = {"fp64": (0, 0), "mixed": (1, 0), "learned": (1, 2)}
    names = args.modes.split(",")
    headline = names[-1]
    for name in names:
        precision, guess = mode_cfg[name]
        us = fresh_u()
        ps = [torch.zeros(shape, dtype=torch.float64, device=dev) for _ in range(nsteps)]
        torch.cuda.synchronize()
        s = Poisson(phi, h, bc, w["rho_l"], w["rho_g"], w["sigma"], precision=precision,
                    stream=stream)
        net = None
        if guess == 2:
            net = Net(n // 2, n // 2, n // 2, stream=stream)
            net.load()
            mp_poisson_set_net(s.handle, net)
            s.set_opts(initial_guess=2, net_check=args.net_check)
        used = []

        def step(k):
            s.set_geometry(phi, w["rho_l"], w["rho_g"], w["sigma"])
            it = s.project_step(*us[k], ps[k], tol=TOL)
            st = s.stats()
            used.append(st["used_net"])
            return it, st["relres"]

        for k in range(args.warmup):
            step(k)
        # timed region: launch counting only (no per-launch events)
        s.set_profiling(False)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(local_rank) if name == headline else None
        n0 = net.launches() if net else 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.mark_start()
        e0.record(stream)
        its, relres = [], []
        for k in range(args.warmup, args.warmup + args.steps):
            it, rr = step(k)
            its.append(it)
            relres.append(rr)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        if sampler:
            sampler.mark_end()
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        launches = sum(e["launches"] for e in s.profile()) + (net.launches() - n0 if net else 0)
        used_timed = used[args.warmup:]
        # profiled pass on further inputs: every launch bracketed by CUDA events on
        # the library's stream (per-kernel durations for the roofline)
        s.set_profiling(True)
        for k in range(args.warmup + args.steps, nsteps):
            step(k)
        prof = s.profile()
        s.set_profiling(False)
        st = s.stats()
        results[name] = dict(ms=ms, iters=its, relres=max(relres), prof=prof, clocks=clocks,
                             levels=st["levels"], outer=st["outer_steps"], launches=launches,
                             prof_steps=nprof, guess_used=used_timed)
        # end to end through the host-buffer entry point (pinned host memory)
        if name == headline:
            hx = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(3)]
            hp = torch.empty(shape, dtype=torch.float64).pin_memory()
            e2e_steps = max(2, min(args.steps, 5))
            src = fresh_u(e2e_steps)
            host_u = [[c.cpu().pin_memory() for c in u3] for u3 in src]
            torch.cuda.synchronize()
            t_e2e = 0.0
            for k in range(e2e_steps):
                for dst, srcc in zip(hx, host_u[k]):
                    dst.copy_(srcc)
                t0 = time.perf_counter()
                s.set_geometry(phi, w["rho_l"], w["rho_g"], w["sigma"])
                mp_poisson_project_step_host(s.handle, hx[0], hx[1], hx[2], hp, TOL)
                t_e2e += time.perf_counter() - t0
            results[name]["e2e"] = dict(steps=e2e_steps, seconds=t_e2e)
        if net:
            mp_poisson_set_net(s.handle, None)
            net.close()
        s.close()
        del us, ps
        torch.cuda.empty_cache()

    if rank != 0:
        return
    K = args.steps
    mixed = results[headline]
    fp64 = results.get("fp64", mixed)
    value = job_value(world, K, mixed["ms"])
    # dominant (kernel, level) by time in the headline mode's profiled steps
    prof = mixed["prof"]
    top = max(prof, key=lambda e: e["total_ms"])
    hbm, peak_kind = peaks()
    achieved = top["alg_bytes"] / (top["total_ms"] * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            tr = json.load(open(tpath))
            key = "%s@L%d" % (top["name"], top["level"])
            if key in tr and tr[key].get("cells") == top["cells"]:
                traffic = tr[key]["dram_bytes_per_launch"]
        except Exception:
            traffic = None
    launches = mixed["launches"]
    total_prof_ms = sum(e["total_ms"] for e in prof)

    def mode_line(r):
        d = {"solves_per_s": job_value(world, K, r["ms"]), "ms_per_step": r["ms"] / K,
             "iterations": r["iters"], "outer_steps_last": r["outer"],
             "max_relres": r["relres"], "levels": r["levels"]}
        if any(r["guess_used"]):
            d["learned_guess_kept"] = sum(r["guess_used"])
        return d

    modes_out = {k: mode_line(v) for k, v in results.items()}
    if "fp64" in results:
        for k in results:
            if k != "fp64":
                modes_out["%s_over_fp64" % k] = results["fp64"]["ms"] / results[k]["ms"]
    forms = {"fp64": "FP64 MG-preconditioned CG",
             "mixed": "mixed FP32/FP64 (FP32 MG-preconditioned CG with FP64 reliable updates)",
             "learned": "mixed FP32/FP64 + learned initial guess (U-Net trained at 128^3, run "
                        "on the half-resolution grid, energy-optimal scale, residual check)"}

    e2e = mixed["e2e"]
    nbytes = n * n * n * 8
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": mixed["ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64", "learned": "f32+f64+bf16"}[headline],
        "data": "synthetic",
        "config": {"workload": workload_desc(n), "grid": [n, n, n], "tol": TOL,
                   "form": forms[headline],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: each step touches ~2 GB of fields"},
        "modes": modes_out,
        "roofline": {"kernel": "%s@L%d" % (top["name"], top["level"]), "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_source": peak_kind, "traffic": traffic,
                     "share_of_profiled_time": top["total_ms"] / total_prof_ms,
                     "timing": "CUDA events around every launch on the library stream, "
                               "%d further steps after the timed region" % mixed["prof_steps"],
                     "launches": top["launches"],
                     "alg_bytes_per_launch": top["alg_bytes"] / top["launches"],
                     "avg_launch_us": 1e3 * top["total_ms"] / top["launches"]},
        "e2e": {"value": e2e["steps"] / e2e["seconds"], "unit": UNIT,
                "h2d_bytes_per_step": 3 * nbytes, "d2h_bytes_per_step": 4 * nbytes},
        "gpu_launches": launches,
        "clocks": mixed["clocks"],
    }
    if world == 1 and not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            line["cpu_baseline"] = cpu_baseline(n)
        except Exception as ex:  # reported, never silently replaced
            line["cpu_baseline"] = {"value": None, "error": repr(ex)}
    if args.profile_out:
        with open(args.profile_out, "w") as f:
            json.dump({k: v["prof"] for k, v in results.items()}, f, indent=1)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--n", type=int, default=256, help="grid cells per axis (default 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--modes", default="fp64,mixed,learned",
                    help="comma list of fp64, mixed, learned; the last one is the headline value")
    ap.add_argument("--profile-out", default=None, help="write per-kernel profile JSON here")
    ap.add_argument("--net-check", type=int, default=0, choices=(0, 1),
                    help="learned guess kept if its residual is below ||b|| (0, default) or "
                         "whenever its energy-optimal scale is nonzero (1)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_mine(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
