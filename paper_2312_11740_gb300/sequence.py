"""A sequence of projection steps on one geometry: the time-stepping use of
the solve.  Step n projects u*_n = u*_0 + amp * xi_n (xi_n a fresh seeded
16-mode field, max-normalised) to tolerance tol, as in a simulation whose
velocity changes a little between steps.

Modes:
  fp64      FP64 MG-preconditioned CG from the zero guess
  mixed     mixed FP32/FP64 from the zero guess
  learned   mixed + the packaged network's guess (half-resolution grid,
            energy-optimal scale, residual check)
  previous  mixed from the previous step's pressure (initial_guess = 1)

    python -m paper_2312_11740_gb300.sequence --workload pool256 --count 50 --mode learned
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import torch

from . import Net, Poisson, mp_poisson_set_net

MODES = {"fp64": (0, 0), "mixed": (1, 0), "learned": (1, 2), "previous": (1, 1)}


def _synth():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth
    return synth


def inputs(workload, count, amp=0.05, seed0=5001, device="cuda"):
    """(phi, params, [u*_n]) of a named workload, generated on the device:
    u*_n = u*_0 + amp * xi_n with xi_n the 16-mode field of seed seed0 + n."""
    synth = _synth()
    w = synth.WORKLOADS[workload]
    n = w["n"]
    h = 1.0 / n
    shape = (n, n, n)
    bc = (synth.PERIODIC, synth.PERIODIC, synth.NEUMANN)
    bubbles = w.get("bubbles") or synth.random_bubbles(w["gseed"], w["nbubbles"], w["rmin"],
                                                        w["rmax"], n, pool_z0=w["pool_z0"])
    phi = synth.level_set(shape, h, bubbles, w["pool_z0"], device=device)
    u0 = synth.velocity(w["useed"], shape, h, device=device)
    us = []
    for k in range(count):
        xi = synth.velocity(seed0 + k, shape, h, device=device)
        us.append(tuple(a + amp * b for a, b in zip(u0, xi)))
    prm = dict(h=h, rho_l=w["rho_l"], rho_g=w["rho_g"], sigma=w["sigma"], bc=bc,
               bubbles=bubbles, pool_z0=w["pool_z0"])
    return phi, prm, us


def run(phi, prm, us, mode="learned", tol=1e-10, warmup=2, keep=False, stream=None):
    """Project every u* of the sequence in order; returns timing, iterations,
    guess use and residuals (and the pressures when keep=True).  The first
    `warmup` steps (graph capture, first-touch) are excluded from the timing
    and repeated afterwards so that every step is timed once."""
    precision, guess = MODES[mode]
    n = phi.shape[2]
    s = Poisson(phi, prm["h"], prm["bc"], prm["rho_l"], prm["rho_g"], prm["sigma"],
                precision=precision, stream=stream)
    net = None
    if guess == 2:
        net = Net(n // 2, n // 2, n // 2, stream=stream)
        net.load()
        mp_poisson_set_net(s.handle, net)
    s.set_opts(initial_guess=guess)
    p = torch.zeros(phi.shape, dtype=torch.float64, device=phi.device)
    for k in range(min(warmup, len(us))):
        s.project_step(*[c.clone() for c in us[k]], p.zero_(), tol=tol)
    p.zero_()
    its, used, rel, ps = [], [], [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for u in us:
        uc = [c.clone() for c in u]
        if guess != 1:
            p.zero_()
        its.append(s.project_step(*uc, p, tol=tol))
        st = s.stats()
        used.append(st["used_net"])
        rel.append(st["relres"])
        if keep:
            ps.append(p.clone())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if net:
        mp_poisson_set_net(s.handle, None)
        net.close()
    s.close()
    out = dict(mode=mode, solves=len(us), seconds=dt, solves_per_s=len(us) / dt,
               iterations=its, mean_iterations=sum(its) / len(its), guess_kept=sum(used),
               max_relres=max(rel))
    if keep:
        out["pressures"] = ps
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="pool256")
    ap.add_argument("--count", type=int, default=50)
    ap.add_argument("--mode", default="learned", choices=sorted(MODES))
    ap.add_argument("--tol", type=float, default=1e-10)
    a = ap.parse_args(argv)
    phi, prm, us = inputs(a.workload, a.count)
    r = run(phi, prm, us, a.mode, a.tol)
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
