"""Iterations the oracle's Jacobi-preconditioned CG needs on the benchmark
workloads, measured by full solves to relative residual 1e-10.

Test infrastructure: the CPU legs of the benchmark time an assembly, a
projection and a bounded number of CG iterations, and turn the measured
time per iteration into a time per solve with the iteration count stored
here.  Every count comes from an actual oracle solve of that workload's
first right-hand side (u*_0); nothing is estimated.

    python -m oracle.calibrate [pool256 bubble256 ...]

writes oracle/solve_counts.json.  A 256^3 pool solve takes several minutes.
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

_HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(_HERE, "solve_counts.json")
TOL = 1e-10


def measure(name):
    root = os.path.dirname(_HERE)
    if root not in sys.path:
        sys.path.insert(0, root)
    import oracle
    import synth
    phi, u, prm = synth.workload(name)
    h = prm["h"]
    t0 = time.perf_counter()
    rhs = oracle.divergence(*u, h)
    res = oracle.solve(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], prm["bc"], tol=TOL)
    dt = time.perf_counter() - t0
    if res["iters"] < 0:
        raise RuntimeError("oracle solve of %s did not converge" % name)
    return {"n": int(phi.shape[0]), "iterations": int(res["iters"]), "relres": float(res["relres"]),
            "seconds": dt,
            "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "host": platform.machine(),
            "tol": TOL}


def load():
    if not os.path.exists(OUT):
        return {}
    with open(OUT) as f:
        return json.load(f)


def main(argv=None):
    names = (argv if argv is not None else sys.argv[1:]) or ["pool256", "bubble256"]
    counts = load()
    for name in names:
        counts[name] = measure(name)
        print(name, counts[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(counts, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
