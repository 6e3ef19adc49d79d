"""The larger workloads: 50-step pool sequences (256^3, 32 bubbles under a
liquid pool, u* perturbed by 5% per step) in every mode, and the 512^3
64-bubble mixed solve.  At these sizes the oracle checks each GPU pressure
through its own assembly and operator (its residual of the GPU solution);
the modes must also agree with one another to the parity bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_11740_gb300 import Poisson, sequence

pytestmark = pytest.mark.gpu

TOL = 1e-10
SEQ_AGREE = 5e-8   # two GPU forms that each stop at relres <= 1e-10 (see below)


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def oracle_relres(phi, u, prm, p):
    """||b - A p|| / ||b|| with b, A from the oracle (FP64 CPU)."""
    h, bc = prm["h"], prm["bc"]
    rhs = oracle.divergence(*[c.cpu().numpy() for c in u], h)
    _, f, _, b = oracle.assemble(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc)
    _, rn = oracle.residual(f, b, p.cpu().numpy(), h, bc)
    return rn / np.linalg.norm(b)


def test_pool256_sequence_all_modes():
    phi, prm, us = sequence.inputs("pool256", 4)
    ref = sequence.run(phi, prm, us, "fp64", warmup=0, keep=True)
    assert ref["max_relres"] <= TOL
    phi_h = phi.cpu().numpy()
    # the first FP64 pressure through the oracle's own operator
    assert oracle_relres(phi_h, us[0], prm, ref["pressures"][0]) <= 1.5 * TOL
    for mode in ("mixed", "learned", "previous"):
        r = sequence.run(phi, prm, us, mode, warmup=0, keep=True)
        assert r["max_relres"] <= TOL, mode
        for k, (a, b) in enumerate(zip(r["pressures"], ref["pressures"])):
            # every pressure meets the target through the oracle's operator
            assert oracle_relres(phi_h, us[k], prm, a) <= 1.5 * TOL, (mode, k)
            # two solutions that each meet ||b - Ap|| <= 1e-10 ||b|| differ by up to
            # cond x 1e-10 (the oracle parity bar, 1e-8 against a reference solved
            # 10x tighter, is checked element-wise at the sizes the oracle solves).
            # Measured on this machine geometry (density ratio 1000): zero-guess forms
            # stopping at relres ~9.9e-11 on different Krylov paths differ by 1.5e-8,
            # warm starts, which stop at a different point of the iteration, by 5e-8
            assert rel(a, b) <= (1e-6 if mode == "previous" else SEQ_AGREE), (mode, k)


def test_bubbles512_mixed_full_size():
    phi, prm, us = sequence.inputs("bubbles512", 1, amp=0.0)
    s = Poisson(phi, prm["h"], prm["bc"], prm["rho_l"], prm["rho_g"], prm["sigma"], precision=1)
    rhs = s.divergence(*us[0])
    p, it, hist = s.solve(rhs, tol=TOL)
    assert s.stats()["relres"] <= TOL
    del rhs
    phi_h = phi.cpu().numpy()
    assert oracle_relres(phi_h, us[0], prm, p) <= 1.5 * TOL
    s.close()
