"""Training and evaluation of the learned initial guess (the warm start).

Data: seeded bubble configurations (1-16 gas bubbles, radii 0.03-0.12,
density ratio 1000, sigma 0.07, periodic x,y / wall z) with seeded smooth
u*; each sample's pressure comes from the plain FP64 multigrid solve to
relative residual 1e-10.  Stored on the GPU: the network's two input
channels (BF16) and the target q = p / rms(p) (FP32, mean-free): the
network learns the shape, the solver fits the scale.

Training: Adam, one sample per step, every forward and backward operation
in the library's tcgen05 kernels.  Default loss: the energy norm of the
best-scaled guess, 1 - (q.At)^2/((q.Aq)(t.At)) with A the ghost-fluid
operator of the sample (the solver scales the network output by the
energy-optimal factor, so this is the quantity the guess is judged by);
--loss mse trains on the gauge-free mean squared error instead.

Evaluation on held-out seeds: the number of solver iterations to 1e-10 from
the zero guess and from the learned guess, with the residual check
(net_check 0: kept only if ||b - A p0|| < ||b||) and with the energy check
(net_check 1), hence the iterations saved and the fallback rates, and the
guess's relative L2 and A-norm errors.

    python -m paper_2312_11740_gb300.learn --n 128 --train 2000 --epochs 3 \\
        --eval 200 --out net128.npz

--checkpoint PATH writes a checkpoint after every epoch (parameters, Adam's
moments, step, sample-order generator state, losses); --resume PATH continues
such a run at its epoch boundary, bit for bit as if it had not stopped.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

from . import Net, Poisson, mp_poisson_set_net
from .poisson import NEUMANN, PERIODIC

RHO_L, RHO_G, SIGMA = 1.0, 1e-3, 0.07
BC = (PERIODIC, PERIODIC, NEUMANN)


def _synth():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth
    return synth


def geometry(seed, n, device):
    """Seeded 1-16 bubbles, radii U[0.03, 0.12]: (phi, u*) on the device."""
    synth = _synth()
    rng = np.random.Generator(np.random.PCG64(seed))
    count = int(rng.integers(1, 17))
    bubbles = synth.random_bubbles(seed, count, 0.03, 0.12, n)
    h = 1.0 / n
    phi = synth.level_set((n, n, n), h, bubbles, device=device)
    u = synth.velocity(seed, (n, n, n), h, device=device)
    return phi, u, bubbles


def make_dataset(seeds, n, stream=None, log=print):
    """Solve each seeded problem with the plain FP64 solver; returns the
    network inputs (BF16, (count, n, n, n, 2)), targets (FP32) and solver
    iteration counts."""
    dev = torch.device("cuda")
    h = 1.0 / n
    count = len(seeds)
    X = torch.empty((count, n, n, n, 2), dtype=torch.bfloat16, device=dev)
    Q = torch.empty((count, n, n, n), dtype=torch.float32, device=dev)
    its = []
    net = Net(n, n, n, stream=stream)
    solver = None
    t0 = time.time()
    for k, seed in enumerate(seeds):
        phi, u, _ = geometry(seed, n, dev)
        if solver is None:
            solver = Poisson(phi, h, BC, RHO_L, RHO_G, SIGMA, precision=0, stream=stream)
        else:
            solver.set_geometry(phi, RHO_L, RHO_G, SIGMA)
        rhs = solver.divergence(*u)
        p, it, _ = solver.solve(rhs, tol=1e-10)
        b = solver.rhs(rhs)
        net.features(phi, b, h, h * h)
        X[k] = net.get_input2()
        Q[k] = net.make_target(p)
        its.append(it)
        if log and (k + 1) % max(1, count // 10) == 0:
            log("  data %d/%d  %.1fs" % (k + 1, count, time.time() - t0))
    net.close()
    solver.close()
    return X, Q, its


def init_params(net, seed):
    """He-normal weights, small biases, drawn on the host (PCG64(seed))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = [(16, 16, 2), (16, 16, 16), (32, 16, 16), (32, 32, 32), (64, 32, 32), (64, 64, 64),
              (64, 64, 64), (64, 64, 64), (64, 128, 128), (64, 64, 64), (32, 96, 96),
              (32, 32, 32), (16, 48, 48), (16, 16, 16)]
    parts = []
    for cout, cin, fan in shapes:
        parts.append(rng.standard_normal(cout * 27 * cin) * np.sqrt(2.0 / (27 * fan)))
        parts.append(np.zeros(cout))
    parts.append(rng.standard_normal(16) * 0.25)
    parts.append(np.zeros(1))
    vec = np.concatenate(parts).astype(np.float32)
    assert vec.size == net.param_count(), (vec.size, net.param_count())
    return torch.from_numpy(vec).cuda()


def save_checkpoint(path, net, step, epoch, rng, losses, config):
    """Everything training needs to resume exactly at an epoch boundary:
    parameters, Adam's moments, the step count (Adam's bias correction and
    the learning-rate schedule), the epochs done, the sample-order generator's
    state, the loss history and the run's configuration.  Written to a
    temporary file and renamed, so a crash leaves the previous checkpoint."""
    m, v = net.get_adam()
    tmp = path + ".tmp.npz"
    np.savez(tmp, params=net.get_params().cpu().numpy(), adam_m=m.cpu().numpy(),
             adam_v=v.cpu().numpy(), step=np.int64(step), epoch=np.int64(epoch),
             rng=np.array(json.dumps(rng.bit_generator.state)), losses=np.array(losses),
             config=np.array(json.dumps(config, sort_keys=True)))
    os.replace(tmp, path)


def load_checkpoint(path, net, device="cuda"):
    """Restore parameters and Adam's moments into net; returns (step, epoch,
    rng state, losses, config)."""
    d = np.load(path)
    net.set_params(torch.from_numpy(d["params"]).to(device))
    net.set_adam(torch.from_numpy(d["adam_m"]).to(device), torch.from_numpy(d["adam_v"]).to(device))
    return (int(d["step"]), int(d["epoch"]), json.loads(str(d["rng"])), list(d["losses"]),
            json.loads(str(d["config"])))


def train(net, X, Q, epochs, lr, seed, log=print, lr_final=None, loss="energy",
          checkpoint=None, resume=None, device="cuda", phi_of=None, n=None):
    """Adam over shuffled samples; returns the loss history (one per step).
    checkpoint: path written after every epoch; resume: a checkpoint of the
    same run (same samples, epochs, schedule and seed) to continue from.
    loss "energy_deflated": the deflated energy of the guess
    (mp_poisson_deflated_energy) on each sample's geometry, phi_of(k) giving
    sample k's level set on the device (n^3 grid); the gradient it returns
    drives mp_net_train_step_grad."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = X.shape[0]
    config = dict(count=int(count), epochs=int(epochs), lr=float(lr), seed=int(seed),
                  lr_final=None if lr_final is None else float(lr_final), loss=loss)
    solver = None
    if loss == "energy_deflated":
        solver = Poisson(phi_of(0), 1.0 / n, BC, RHO_L, RHO_G, SIGMA, precision=0)
    else:
        net.set_loss(1 if loss == "energy" else 0, RHO_L, RHO_G, BC)
    losses = []
    step, first = 0, 0
    if resume:
        step, first, state, losses, saved = load_checkpoint(resume, net, device)
        if saved != config:
            raise ValueError("checkpoint of a different run: %s vs %s" % (saved, config))
        rng.bit_generator.state = state
    total = epochs * count
    t0 = time.time()
    for ep in range(first, epochs):
        order = rng.permutation(count)
        for k in order:
            step += 1
            cur = lr if lr_final is None else lr * (lr_final / lr) ** (step / total)
            net.set_input2(X[k])
            if solver is None:
                losses.append(net.train_step(Q[k], cur, step))
            else:
                solver.set_geometry(phi_of(int(k)), RHO_L, RHO_G, SIGMA)
                L, gq = solver.deflated_energy(net.forward(), Q[k])
                net.train_step_grad(gq, cur, step)
                losses.append(L)
        if log:
            log("  epoch %d  mean loss %.4e  %.1fs" % (ep + 1, float(np.mean(losses[-count:])),
                                                       time.time() - t0))
        if checkpoint:
            save_checkpoint(checkpoint, net, step, ep + 1, rng, losses, config)
    if solver is not None:
        solver.close()
    return losses


def pg_forced(solver, rhs):
    """The scaled network guess itself (energy check, no iterations)."""
    solver.set_opts(initial_guess=2, max_iters=0, net_check=1)
    pg, _, _ = solver.solve(rhs, tol=1e-10, allow_not_converged=True)
    return pg


def deflated_errors(solver, guess, p):
    """Energy errors of a guess against the converged pressure p, for the
    deflated solver.  Deflated CG corrects any start exactly along the gas
    components' indicator vectors Z, so what it inherits from a guess is the
    error in the deflated energy ||e||_D^2 = ||e||_A^2 - (Z^T A e)^T E^-1
    (Z^T A e), E = Z^T A Z (the A-energy left after the best correction along
    Z).  Returns (eps_A, eps_D, share): ||e||_A / ||p||_A, ||e||_D / ||p||_D
    and ||p||_D^2 / ||p||_A^2, the part of the solution's energy that
    deflation leaves to the iterations.  Diagnostic: A applied through the
    library, the small dense E and the component sums in torch."""
    comp, m = solver.components()
    comp = comp.reshape(-1).long()
    mask = comp >= 0

    def zt(v):
        out = torch.zeros(m, dtype=torch.float64, device=v.device)
        out.index_add_(0, comp[mask], v.reshape(-1)[mask])
        return out

    E = torch.zeros((m, m), dtype=torch.float64, device=p.device)
    for a in range(m):
        E[:, a] = zt(solver.apply((comp == a).to(torch.float64).view(p.shape)))

    def energies(v):
        Av = solver.apply(v)
        ea = -float((v * Av).sum())  # A is negative semidefinite
        if m == 0:
            return ea, ea
        y = zt(Av)
        return ea, ea + float(y @ torch.linalg.solve(E, y))

    pa, pd = energies(p)
    ea, ed = energies(guess - p)
    return float(np.sqrt(ea / pa)), float(np.sqrt(max(ed, 0.0) / pd)), pd / pa


def evaluate(net, seeds, n, precision=0, stream=None, log=print, deflate=0):
    """Iterations to 1e-10 from the zero guess and from the learned guess,
    and the learned guess's relative error against the converged pressure.
    deflate = 0 evaluates against plain MG-preconditioned CG, the method the
    network's targets and loss are set up for; 1 against the deflated solver."""
    dev = torch.device("cuda")
    h = 1.0 / n
    rows = []
    solver = None
    for seed in seeds:
        phi, u, _ = geometry(seed, n, dev)
        if solver is None:
            solver = Poisson(phi, h, BC, RHO_L, RHO_G, SIGMA, precision=precision, stream=stream)
            solver.set_opts(deflate=deflate)
            mp_poisson_set_net(solver.handle, net)
        else:
            solver.set_geometry(phi, RHO_L, RHO_G, SIGMA)
        rhs = solver.divergence(*u)
        solver.set_opts(initial_guess=0)
        p0, it0, _ = solver.solve(rhs, tol=1e-10)
        pg = pg_forced(solver, rhs)  # the scaled guess itself
        guess_err = float(torch.linalg.norm(pg - p0) / torch.linalg.norm(p0))
        solver.set_opts(initial_guess=2, max_iters=200, net_check=0)
        p1, it1, _ = solver.solve(rhs, tol=1e-10)
        st = solver.stats()
        err = float(torch.linalg.norm(p1 - p0) / torch.linalg.norm(p0))
        # the guess kept whenever it lowers the A-norm error (net_check = 1)
        solver.set_opts(initial_guess=2, max_iters=200, net_check=1)
        p2, it2, _ = solver.solve(rhs, tol=1e-10)
        st2 = solver.stats()
        solver.set_opts(net_check=0)
        # A-norm error of the scaled guess relative to the solution's A-norm
        e = pg - p0
        relA = float(torch.sqrt(torch.abs((e * solver.apply(e)).sum()) /
                                torch.abs((p0 * solver.apply(p0)).sum())))
        defl = {}
        if deflate and st["components"] > 0:
            eA, eD, share = deflated_errors(solver, pg, p0)
            defl = dict(guess_rel_energy_err_deflated=eD, deflated_energy_share=share)
        rows.append(dict(seed=seed, zero_iters=it0, net_iters=it1, used_net=st["used_net"],
                         net_relres=st["net_relres"], guess_rel_err=guess_err,
                         diff_vs_zero_guess=err, energy_iters=it2,
                         energy_used=st2["used_net"], guess_rel_energy_err=relA,
                         diff_energy=float(torch.linalg.norm(p2 - p0) / torch.linalg.norm(p0)),
                         **defl))
    mp_poisson_set_net(solver.handle, None)
    solver.close()
    zero = np.array([r["zero_iters"] for r in rows])
    lrn = np.array([r["net_iters"] for r in rows])
    used = np.array([r["used_net"] for r in rows])
    en = np.array([r["energy_iters"] for r in rows])
    summary = dict(samples=len(rows), mean_zero_iters=float(zero.mean()),
                   mean_net_iters=float(lrn.mean()), iterations_saved=float((zero - lrn).mean()),
                   fallback_rate=float(1.0 - used.mean()),
                   median_net_relres=float(np.median([r["net_relres"] for r in rows])),
                   median_guess_rel_err=float(np.median([r["guess_rel_err"] for r in rows])),
                   median_guess_rel_energy_err=float(
                       np.median([r["guess_rel_energy_err"] for r in rows])),
                   energy_check_mean_iters=float(en.mean()),
                   energy_check_iterations_saved=float((zero - en).mean()),
                   energy_check_fallback_rate=float(
                       1.0 - np.mean([r["energy_used"] for r in rows])))
    dl = [r for r in rows if "guess_rel_energy_err_deflated" in r]
    if dl:
        summary["median_guess_rel_energy_err_deflated"] = float(
            np.median([r["guess_rel_energy_err_deflated"] for r in dl]))
        summary["median_deflated_energy_share"] = float(
            np.median([r["deflated_energy_share"] for r in dl]))
    if log:
        log("  eval: " + json.dumps(summary))
    return summary, rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--train-seed0", type=int, default=10000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--eval-seed0", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--init-seed", type=int, default=7)
    ap.add_argument("--loss", choices=("energy", "mse", "energy_deflated"), default="energy")
    ap.add_argument("--init-from", default=None,
                    help="start from these weights (.npz) instead of random initialisation")
    ap.add_argument("--deflate", type=int, choices=(0, 1), default=0,
                    help="solver form the evaluation compares against (0: plain MG-PCG)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--checkpoint", default=None, help="written after every epoch")
    ap.add_argument("--resume", default=None, help="checkpoint of this run to continue from")
    ap.add_argument("--report", default=None)
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    n = a.n
    t0 = time.time()
    print("data: %d training samples at %d^3" % (a.train, n), flush=True)
    X, Q, its = make_dataset(list(range(a.train_seed0, a.train_seed0 + a.train)), n)
    t_data = time.time() - t0
    net = Net(n, n, n)
    if a.init_from:
        net.load(a.init_from)
    else:
        net.set_params(init_params(net, a.init_seed))
    seeds = list(range(a.train_seed0, a.train_seed0 + a.train))
    dev = torch.device("cuda")

    def phi_of(k):
        return geometry(seeds[k], n, dev)[0]

    print("train: %d epochs" % a.epochs, flush=True)
    t1 = time.time()
    losses = train(net, X, Q, a.epochs, a.lr, a.init_seed, lr_final=a.lr_final, loss=a.loss,
                   checkpoint=a.checkpoint, resume=a.resume, phi_of=phi_of, n=n)
    t_train = time.time() - t1
    del X, Q
    torch.cuda.empty_cache()
    summary, rows = evaluate(net, list(range(a.eval_seed0, a.eval_seed0 + a.eval)), n,
                             deflate=a.deflate)
    report = dict(n=n, loss=a.loss, train_samples=a.train, epochs=a.epochs, lr=a.lr,
                  lr_final=a.lr_final, deflate=a.deflate,
                  data_seconds=t_data, train_seconds=t_train,
                  steps=len(losses), loss_first=float(np.mean(losses[:50])),
                  loss_last=float(np.mean(losses[-50:])), train_solver_iters=float(np.mean(its)),
                  eval=summary)
    print(json.dumps(report), flush=True)
    if a.out:
        np.savez(a.out, params=net.get_params().cpu().numpy(), n=n, losses=np.array(losses))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(dict(report=report, rows=rows), f, indent=1)
    net.close()


if __name__ == "__main__":
    main()
