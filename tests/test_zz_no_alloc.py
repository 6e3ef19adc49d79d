"""The allocation-free right-hand-side entry point, for callers that cannot
allocate device memory (their application owns every allocation, or their
path must not call cudaMalloc).  Its output must match the handle-based
mp_poisson_rhs, on two calls in a row (the shared scratch keeps the first
call's contents).  Collected last so a run that stops at the first failure
has run every other test first."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2312_11740_gb300 import Poisson, _lib, mp_poisson_rhs_noalloc

pytestmark = pytest.mark.gpu


def test_rhs_noalloc_matches_handle_entry_point():
    phi, u, prm = synth.workload("bubble32")
    h = prm["h"]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    s = Poisson(d(phi), h, prm["bc"], prm["rho_l"], prm["rho_g"], prm["sigma"])
    J = s.fields()["J"]
    rhs1 = d(oracle.divergence(*u, h))
    rhs2 = d(np.random.Generator(np.random.PCG64(3)).standard_normal(phi.shape))
    for rhs in (rhs1, rhs2):  # two calls in a row through the shared scratch
        ref = s.rhs(rhs)
        b = torch.full_like(rhs, np.nan)
        mp_poisson_rhs_noalloc(rhs, J, b)
        torch.cuda.synchronize()
        err = (b - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-11, err
        assert abs(b.sum().item()) < 1e-9 * b.abs().sum().item()
    s.close()


def test_rhs_noalloc_rejects_bad_sizes():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    lib = _lib.load()
    too_big = _lib.MP_NOALLOC_MAX_CELLS + 1
    assert lib.mp_poisson_rhs_noalloc(too_big, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                      None) == _lib.MP_ERR_INVALID_ARG
    assert lib.mp_poisson_rhs_noalloc(0, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                      None) == _lib.MP_ERR_INVALID_ARG
    with pytest.raises(ValueError):  # binding checks sizes before calling the library
        mp_poisson_rhs_noalloc(x, x, torch.zeros(7, dtype=torch.float64, device="cuda"))
