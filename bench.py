#!/usr/bin/env python
"""Projection-step throughput of the GB300 pressure-Poisson path.

One step = one pass of the whole hot path on a 256^3 grid: geometry data
from phi (curvature, ghost-fluid faces, jump source, coarse hierarchy,
coarsest inverse, gas components), rhs = div u* with the jump, the pressure
solve to relative residual 1e-10 (MG-preconditioned CG, deflated by the gas
components; FP64, or mixed FP32/FP64 with FP64 reliable updates, optionally
from the learned guess), the gauge and the face-velocity correction.

The timed workload is the metric's configuration: a liquid pool with 32
bubbles, a sequence of steps whose u* differ by 5% seeded noise.  The
headline value is the mixed + learned form; FP64, mixed, and mixed from the
previous step's pressure are measured on the same inputs under "modes", and
the one-bubble 256^3 workload as a second block there.

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
WORKLOAD = "pool256"      # the metric's configuration: pool + 32 bubbles, 50-step sequence
SECONDARY = "bubble256"   # one bubble, fresh u* per step (reported under "modes")
TOL = 1e-10
SEQ_LEN, SEQ_AMP, SEQ_SEED0 = 50, 0.05, 5001

# (precision, initial guess): 0/1 = FP64/mixed; guess 0 zero, 1 previous pressure, 2 network
MODE_CFG = {"fp64": (0, 0), "mixed": (1, 0), "previous": (1, 1), "learned": (1, 2)}
FORMS = {"fp64": "FP64 MG-preconditioned CG from the zero guess",
         "mixed": "mixed FP32/FP64 (FP32 MG-preconditioned CG with FP64 reliable updates) "
                  "from the zero guess",
         "previous": "mixed FP32/FP64 from the previous step's pressure",
         "learned": "mixed FP32/FP64 + learned initial guess (U-Net trained at 128^3, run on the "
                    "half-resolution grid, energy-optimal scale, residual check)"}


def workload_desc(name, n):
    if name == "pool256":
        return ("pool256: %d^3 cells on the unit cube, periodic x,y / wall z, liquid pool below "
                "z=0.3 (gas above) with 32 seeded gas bubbles R~U[0.02,0.06] in it (geometry "
                "seed 5), rho_l=1, rho_g=1e-3, sigma=0.07; a sequence of projection steps with "
                "u*_n = u*_0 + 0.05 xi_n (u*_0 seed 5, xi_n fresh max-normalised 16-mode fields "
                "of seeds 5001..5050; step k takes n = k mod 50), each solved to relative "
                "residual 1e-10; every step recomputes the geometry data" % n)
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
def _oracle_problem(name, n):
    """phi, u*_0 and parameters of a workload at n^3, from the generators."""
    import synth
    w = dict(synth.WORKLOADS[name])
    h = 1.0 / n
    bubbles = w.get("bubbles") or synth.random_bubbles(w["gseed"], w["nbubbles"], w["rmin"],
                                                        w["rmax"], n, pool_z0=w["pool_z0"])
    phi = synth.level_set((n, n, n), h, bubbles, w["pool_z0"])
    return phi, w, h


def _solve_count(name, n):
    """Iterations of a full oracle solve of the workload to 1e-10 at n^3,
    measured by oracle/calibrate.py (a committed file written by that script)."""
    from oracle import calibrate
    cal = calibrate.load().get(name)
    if cal is None or cal.get("n") != n:
        raise RuntimeError("no measured oracle iteration count for %s at %d^3: run python -m "
                           "oracle.calibrate %s" % (name, n, name))
    return cal


def _oracle_sample(phi, u, h, w, cg_iters):
    """One bounded oracle step: divergence, assembly, `cg_iters` Jacobi-PCG
    iterations, projection.  Returns (t_assembly, t_cg, t_projection)."""
    import oracle
    bc = (0, 0, 1)
    t0 = time.perf_counter()
    rhs = oracle.divergence(*u, h)
    kap, f, J, b = oracle.assemble(phi, rhs, h, w["rho_l"], w["rho_g"], w["sigma"], bc)
    t1 = time.perf_counter()
    x, _, _ = oracle.cg(f, b, h, bc, tol=1e-30, maxit=cg_iters)
    t2 = time.perf_counter()
    oracle.project(phi, kap, f, x, *u, h, w["sigma"], bc)
    t3 = time.perf_counter()
    return t1 - t0, t2 - t1, t3 - t2


def cpu_baseline(n, cg_iters=300):
    """The FP64 CPU oracle as it stands, on this host's cores, on the bench
    workload's first right-hand side: the assembly, the projection and
    `cg_iters` Jacobi-PCG iterations are timed, and the solve time is the
    assembly + projection + the measured time per iteration times the
    iterations a full oracle solve of this problem took (measured, stored by
    oracle/calibrate.py)."""
    import synth
    cores = os.cpu_count() or 1
    cal = _solve_count(WORKLOAD, n)
    phi, w, h = _oracle_problem(WORKLOAD, n)
    u = synth.velocity(w["useed"], (n, n, n), h)
    ta, tc, tp = _oracle_sample(phi, u, h, w, cg_iters)
    t_solve = ta + tp + tc / cg_iters * cal["iterations"]
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": ("C oracle (OpenMP, %d threads) on %s: divergence + assembly (%.2f s), "
                       "%d Jacobi-PCG iterations (%.2f s, %.1f ms each) and the projection "
                       "(%.2f s) timed at %d^3; per solve: assembly + projection + %d iterations, "
                       "the count of a full oracle solve of this problem to 1e-10 (measured: "
                       "%.0f s with %d threads on %s)"
                       % (cores, WORKLOAD, ta, cg_iters, tc, 1e3 * tc / cg_iters, tp, n,
                          cal["iterations"], cal["seconds"], cal["threads"], cal["host"].strip())),
            "seconds_per_solve": t_solve, "oracle_iterations": cal["iterations"]}


def run_reference(args, rank):
    """Reference arm: the CPU oracle itself on this host's cores, on the same
    workload and sequence; every step is a bounded sample (assembly, 40
    Jacobi-PCG iterations, projection) and counts as the fraction of a full
    solve that its iterations are of the measured full-solve count."""
    if rank != 0:
        return
    n = args.n
    cg_iters = 40
    import oracle
    import synth
    oracle.build()
    cal = _solve_count(WORKLOAD, n)
    phi, w, h = _oracle_problem(WORKLOAD, n)
    u0 = synth.velocity(w["useed"], (n, n, n), h)
    step_s, solve_s = [], []
    for step in range(args.warmup + args.steps):
        xi = synth.velocity(SEQ_SEED0 + step % SEQ_LEN, (n, n, n), h)
        u = tuple(np.ascontiguousarray(a + SEQ_AMP * b) for a, b in zip(u0, xi))
        ta, tc, tp = _oracle_sample(phi, u, h, w, cg_iters)
        if step >= args.warmup:
            step_s.append(ta + tc + tp)
            solve_s.append(ta + tp + tc / cg_iters * cal["iterations"])
    value = len(solve_s) / sum(solve_s)
    cores = os.cpu_count() or 1
    sample = ("each step: C oracle (OpenMP, %d threads) divergence + assembly + %d Jacobi-PCG "
              "iterations + projection of u*_n at %d^3 (the step's measured time is "
              "ms_per_step); a solve = assembly + projection + %d iterations, the count of a "
              "full oracle solve of this problem to 1e-10 (measured by oracle/calibrate.py), so "
              "value = steps / sum of the per-step solve times" % (cores, cg_iters, n,
                                                                   cal["iterations"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(step_s) / len(step_s),
            "ms_per_solve": 1e3 * sum(solve_s) / len(solve_s),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(WORKLOAD, n), "grid": [n, n, n], "tol": TOL,
                       "form": "FP64 Jacobi-preconditioned CG (CPU oracle)"},
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
def _gpu_inputs(name, n, rank, dev):
    """phi on the device and a maker of the step-k velocity u*_k (device)."""
    import synth
    w = synth.WORKLOADS[name]
    h = 1.0 / n
    shape = (n, n, n)
    bubbles = w.get("bubbles") or synth.random_bubbles(w["gseed"], w["nbubbles"], w["rmin"],
                                                        w["rmax"], n, pool_z0=w["pool_z0"])
    phi = synth.level_set(shape, h, bubbles, w["pool_z0"], device=dev)
    if name == WORKLOAD:
        u0 = synth.velocity(w["useed"], shape, h, device=dev)

        def make(k):
            xi = synth.velocity(SEQ_SEED0 + k % SEQ_LEN, shape, h, device=dev)
            return tuple((a + SEQ_AMP * b).contiguous() for a, b in zip(u0, xi))
    else:
        def make(k):
            return synth.velocity(100000 * (rank + 1) + k, shape, h, device=dev)
    return phi, w, h, make


def run_mode(name, mode, args, n, dev, stream, world, local_rank, rank, steps, warmup, nprof,
             headline):
    """W untimed steps, K timed steps (CUDA events on the library stream,
    barrier + synchronize on both sides), then `nprof` steps with every
    launch bracketed by CUDA events (per-kernel durations for the roofline)
    and, for the headline mode, the same K steps end to end through the
    host-buffer entry point."""
    import torch
    from paper_2312_11740_gb300 import Net, Poisson, mp_poisson_project_step_host
    from paper_2312_11740_gb300 import mp_poisson_set_net
    phi, w, h, make = _gpu_inputs(name, n, rank, dev)
    shape = (n, n, n)
    bc = (0, 0, 1)
    precision, guess = MODE_CFG[mode]
    count = warmup + steps + nprof
    us = [make(k) for k in range(count)]
    p = torch.zeros(shape, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    s = Poisson(phi, h, bc, w["rho_l"], w["rho_g"], w["sigma"], precision=precision,
                stream=stream)
    net = None
    if guess == 2:
        net = Net(n // 2, n // 2, n // 2, stream=stream)
        net.load()
        mp_poisson_set_net(s.handle, net)
    s.set_opts(initial_guess=guess, net_check=args.net_check)
    used = []

    def step(u3):
        s.set_geometry(phi, w["rho_l"], w["rho_g"], w["sigma"])
        it = s.project_step(*u3, p, tol=TOL)
        st = s.stats()
        used.append(st["used_net"])
        return it, st["relres"]

    for k in range(warmup):
        step(us[k])
    s.set_profiling(False)  # timed region: launch counting only (no per-launch events)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local_rank) if headline else None
    n0 = net.launches() if net else 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.mark_start()
    e0.record(stream)
    its, relres = [], []
    for k in range(warmup, warmup + steps):
        it, rr = step(us[k])
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
    used_timed = used[warmup:]
    prof = None
    if nprof:
        s.set_profiling(True)
        for k in range(warmup + steps, count):
            step(us[k])
        prof = s.profile()
        s.set_profiling(False)
    st = s.stats()
    del us
    out = dict(ms=ms, iters=its, relres=max(relres), prof=prof, clocks=clocks,
               levels=st["levels"], outer=st["outer_steps"], launches=launches,
               prof_steps=nprof, guess_used=used_timed, components=st["components"])
    if headline:
        # end to end: every timed step again through mp_poisson_project_step_host,
        # u*_k staged in pinned host buffers before its call (outside the timing)
        hx = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(3)]
        hp = torch.zeros(shape, dtype=torch.float64).pin_memory()
        t_e2e = 0.0
        for k in range(warmup, warmup + steps):
            for dst, src in zip(hx, make(k)):
                dst.copy_(src)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.set_geometry(phi, w["rho_l"], w["rho_g"], w["sigma"])
            mp_poisson_project_step_host(s.handle, hx[0], hx[1], hx[2], hp, TOL)
            t_e2e += time.perf_counter() - t0
        out["e2e"] = dict(steps=steps, seconds=t_e2e)
    if net:
        mp_poisson_set_net(s.handle, None)
        net.close()
    s.close()
    torch.cuda.empty_cache()
    return out


def run_mine(args, rank, world, local_rank):
    import torch
    from paper_2312_11740_gb300 import build as pkg_build
    pkg_build.build()

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = args.n
    stream = torch.cuda.Stream(device=dev)
    names = args.modes.split(",")
    headline = args.headline if args.headline in names else names[-1]
    K, W = args.steps, args.warmup
    nprof = min(K, 3)
    results = {}
    for name in names:
        results[name] = run_mode(WORKLOAD, name, args, n, dev, stream, world, local_rank, rank,
                                 K, W, nprof, name == headline)
    secondary = {}
    if not args.no_secondary:
        k2, w2 = min(K, 10), min(W, 3)
        for name in ("fp64", "mixed", "learned"):
            secondary[name] = run_mode(SECONDARY, name, args, n, dev, stream, world, local_rank,
                                       rank, k2, w2, 0, False)
    if rank != 0:
        return
    top_mode = results[headline]
    value = job_value(world, K, top_mode["ms"])
    # dominant (kernel, level) by time in the headline mode's profiled steps
    prof = top_mode["prof"]
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
    total_prof_ms = sum(e["total_ms"] for e in prof)

    def mode_line(r, k, name):
        d = {"solves_per_s": job_value(world, k, r["ms"]), "ms_per_step": r["ms"] / k,
             "iterations": r["iters"], "outer_steps_last": r["outer"],
             "max_relres": r["relres"], "levels": r["levels"], "components": r["components"]}
        if name == "learned":  # timed steps whose learned guess passed the residual check
            d["learned_guess_kept"] = int(sum(r["guess_used"] or []))
            d["learned_guess_offered"] = len(r["guess_used"] or [])
        return d

    modes_out = {k: mode_line(v, K, k) for k, v in results.items()}
    if "fp64" in results:
        for k in results:
            if k != "fp64":
                modes_out["%s_over_fp64" % k] = results["fp64"]["ms"] / results[k]["ms"]
    if secondary:
        k2 = min(K, 10)
        sec = {k: mode_line(v, k2, k) for k, v in secondary.items()}
        for k in ("mixed", "learned"):
            sec["%s_over_fp64" % k] = secondary["fp64"]["ms"] / secondary[k]["ms"]
        sec["workload"] = workload_desc(SECONDARY, n)
        sec["steps"] = k2
        modes_out[SECONDARY] = sec
    e2e = top_mode["e2e"]
    nbytes = n * n * n * 8
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": top_mode["ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64", "previous": "f32+f64",
                  "learned": "f32+f64+bf16"}[headline],
        "data": "synthetic",
        "config": {"workload": workload_desc(WORKLOAD, n), "grid": [n, n, n], "tol": TOL,
                   "form": FORMS[headline],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: each step touches ~2 GB of fields"},
        "modes": modes_out,
        "roofline": {"kernel": "%s@L%d" % (top["name"], top["level"]), "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_source": peak_kind, "traffic": traffic,
                     "share_of_profiled_time": top["total_ms"] / total_prof_ms,
                     "timing": "CUDA events around every launch on the library stream, "
                               "%d further steps after the timed region" % top_mode["prof_steps"],
                     "launches": top["launches"],
                     "alg_bytes_per_launch": top["alg_bytes"] / top["launches"],
                     "avg_launch_us": 1e3 * top["total_ms"] / top["launches"]},
        "e2e": {"value": job_value(world, e2e["steps"], 1e3 * e2e["seconds"]), "unit": UNIT,
                "h2d_bytes_per_step": 3 * nbytes, "d2h_bytes_per_step": 4 * nbytes,
                "steps": e2e["steps"]},
        "gpu_launches": top_mode["launches"],
        "clocks": top_mode["clocks"],
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
    ap.add_argument("--modes", default="fp64,mixed,previous,learned",
                    help="comma list of fp64, mixed, previous, learned (pool256 sequence)")
    ap.add_argument("--headline", default="learned",
                    help="mode reported as the value (default: learned, the metric's form)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the one-bubble 256^3 block under modes")
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
