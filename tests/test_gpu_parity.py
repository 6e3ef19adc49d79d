"""CUDA path vs the FP64 CPU oracle, element by element, through the C-ABI.

Small grids (several launch tiles plus ragged tails) are compared in full;
the 256^3 one-bubble workload (the benchmark's launch configuration) is
checked through properties the oracle evaluates at any size: its own
residual of the GPU pressure, and sampled setup fields.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2312_11740_gb300 import Poisson, MPError
from paper_2312_11740_gb300 import _lib

pytestmark = pytest.mark.gpu

P, N = synth.PERIODIC, synth.NEUMANN
TOL = 1e-10          # solver target (relative residual)
PARITY = 1e-8        # relative L2 of the gauge-fixed pressure vs the oracle
REF_TOL = 1e-11      # oracle reference tolerance (10x tighter than the GPU target;
                     # 1e-12 sits at the FP64 floor of the all-wall grids)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def owned(f):
    """oracle faces (n+1 per axis) -> low-face-owned layout (n per axis)"""
    return f.fx[:, :, :-1], f.fy[:, :-1, :], f.fz[:-1, :, :]


def band(phi, bc):
    """Cells with a face neighbour of the other fluid (periodic axes wrap;
    across a wall there is no neighbour)."""
    gas = phi > 0
    out = np.zeros_like(gas)
    for axis, kind in enumerate(bc):
        ax = 2 - axis
        for shift in (1, -1):
            nb = np.roll(gas, shift, axis=ax)
            diff = nb != gas
            if kind == N:
                edge = [slice(None)] * 3
                edge[ax] = 0 if shift == 1 else -1
                diff[tuple(edge)] = False
            out |= diff
    return out


def rel_max(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def case(name):
    if name == "bubble32":
        phi, u, prm = synth.workload("bubble32")
        return phi, u, prm
    if name == "ragged":  # 40 x 24 x 56 cells, two bubbles, tails past 32/8 tiles
        shape, h = (56, 24, 40), 1.0 / 40
        bub = [((0.3, 0.25, 0.5), 0.13), ((0.7, 0.3, 0.9), 0.1)]
        bc = (P, P, N)
        phi = synth.level_set(shape, h, bub, bc=bc)
        u = synth.velocity(7, shape, h, bc=bc)
        return phi, u, dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.07, bc=bc)
    if name == "walls":  # walls on every axis, pool + bubble
        shape, h = (32, 16, 48), 1.0 / 48
        bc = (N, N, N)
        phi = synth.level_set(shape, h, [((0.5, 0.15, 0.25), 0.1)], pool_z0=0.45, bc=bc)
        u = synth.velocity(9, shape, h, bc=bc)
        return phi, u, dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.05, bc=bc)
    if name == "periodic":  # periodic on every axis
        shape, h = (16, 32, 32), 1.0 / 32
        bc = (P, P, P)
        phi = synth.level_set(shape, h, [((0.5, 0.5, 0.25), 0.2)], bc=bc)
        u = synth.velocity(11, shape, h, bc=bc)
        return phi, u, dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.03, bc=bc)
    if name == "wide":  # 128 x 24 x 40: whole 64-cell x tiles; level 1 (ny = 12) overhangs a wall
        shape, h = (40, 24, 128), 1.0 / 128
        bc = (P, N, N)
        bub = [((0.3, 0.09, 0.1), 0.06), ((0.8, 0.1, 0.12), 0.05)]
        phi = synth.level_set(shape, h, bub, pool_z0=0.25, bc=bc)
        u = synth.velocity(13, shape, h, bc=bc)
        return phi, u, dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.07, bc=bc)
    if name == "slab":  # 128 x 12 x 16: the finest level's second tile row wraps (periodic y)
        shape, h = (16, 12, 128), 1.0 / 128
        bc = (P, P, N)
        phi = synth.level_set(shape, h, [((0.5, 0.05, 0.06), 0.035)], pool_z0=0.1, bc=bc)
        u = synth.velocity(15, shape, h, bc=bc)
        return phi, u, dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.07, bc=bc)
    raise KeyError(name)


CASES = ["bubble32", "ragged", "walls", "periodic"]


def make(phi, prm, **opts):
    return Poisson(dev(phi), prm["h"], prm["bc"], prm["rho_l"], prm["rho_g"], prm["sigma"],
                   **opts)


@pytest.mark.parametrize("name", CASES)
def test_setup_fields_match_oracle(name):
    phi, u, prm = case(name)
    h, bc = prm["h"], prm["bc"]
    s = make(phi, prm)
    got = {k: host(v) for k, v in s.fields().items()}
    kap = oracle.curvature(phi, h, bc)
    f = oracle.faces(phi, prm["rho_l"], prm["rho_g"], bc)
    J = oracle.jump(phi, kap, f, h, prm["sigma"], bc)
    # curvature is evaluated in the interface band (the only cells the jump
    # reads) and is zero elsewhere
    bnd = band(phi, bc)
    assert bnd.any()
    assert rel_max(got["kappa"][bnd], kap[bnd]) < 1e-12
    assert np.all(got["kappa"][~bnd] == 0.0)
    for g, o in zip((got["bx"], got["by"], got["bz"]), owned(f)):
        assert rel_max(g, o) < 1e-13
    assert rel_max(got["J"], J) < 1e-11
    assert abs(got["J"].sum()) < 1e-9 * np.abs(got["J"]).sum()
    s.close()


@pytest.mark.parametrize("name", CASES)
def test_divergence_rhs_apply_match_oracle(name):
    phi, u, prm = case(name)
    h, bc = prm["h"], prm["bc"]
    s = make(phi, prm)
    div = host(s.divergence(*[dev(c) for c in u]))
    div_o = oracle.divergence(*u, h)
    assert rel_max(div, div_o) < 1e-12
    kap, f, J, b_o = oracle.assemble(phi, div_o, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc)
    b = host(s.rhs(dev(div_o)))
    assert rel_max(b, b_o) < 1e-11
    x = np.random.Generator(np.random.PCG64(5)).standard_normal(phi.shape)
    y = host(s.apply(dev(x)))
    assert rel_max(y, oracle.apply(f, x, h, bc)) < 1e-12
    s.close()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,method", [(0, 0), (1, 0), (0, 1)])
def test_solve_matches_oracle(name, precision, method):
    phi, u, prm = case(name)
    h, bc = prm["h"], prm["bc"]
    rhs = oracle.divergence(*u, h)
    ref = oracle.solve(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc, tol=REF_TOL)
    assert ref["iters"] >= 0
    s = make(phi, prm, precision=precision, method=method, max_iters=400)
    # The stationary V-cycle leaves its error in smooth modes, which the
    # residual underweights: on the all-wall grid it needs 2e-11 to stay
    # within the 1e-8 parity bar (at 1e-10 it measured 1.3e-8).
    tol = TOL if method == 0 else 2e-11
    p, it, hist = s.solve(dev(rhs), tol=tol)
    st = s.stats()
    pg = host(p)
    assert abs(pg.mean()) < 1e-12 * np.abs(pg).max()
    assert st["relres"] <= tol
    assert hist[0] == pytest.approx(st["r0"])
    assert hist[-1] <= tol
    # residual of the GPU pressure evaluated by the oracle's own operator
    _, rn = oracle.residual(ref["faces"], ref["b"], pg, h, bc)
    assert rn / np.linalg.norm(ref["b"]) <= 1.5 * TOL
    assert rel_l2(pg, ref["p"]) <= PARITY
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_project_step_matches_oracle(precision):
    phi, u, prm = case("bubble32")
    h, bc, sig = prm["h"], prm["bc"], prm["sigma"]
    rhs = oracle.divergence(*u, h)
    ref = oracle.solve(phi, rhs, h, prm["rho_l"], prm["rho_g"], sig, bc, tol=REF_TOL)
    fx, fy, fz = oracle.project(phi, ref["kappa"], ref["faces"], ref["p"], *u, h, sig, bc)
    s = make(phi, prm, precision=precision)
    ux, uy, uz = [dev(c) for c in u]
    p = torch.zeros_like(ux)
    s.project_step(ux, uy, uz, p, tol=TOL)
    # the velocity error is the pressure's A-norm error (||u - u_ref||_beta =
    # ||p - p_ref||_A), which a solve stopped below relative residual 1e-10
    # bounds only to ~1e-9: the same parity bar as the pressure
    for g, o in zip((ux, uy, uz), (fx[:, :, :-1], fy[:, :-1, :], fz[:-1, :, :])):
        assert rel_l2(host(g), o) < PARITY
    # div u = b - A p on every cell: bounded by the solve's relative residual times ||b||
    div = oracle.divergence(host(ux), host(uy), host(uz), h)
    assert np.linalg.norm(div) <= 2 * TOL * np.linalg.norm(ref["b"])
    assert np.all(host(uz)[0] == 0.0)
    # host-buffer entry point gives the same bits as the device one
    hx, hy, hz = [torch.from_numpy(np.ascontiguousarray(c)).pin_memory() for c in u]
    hp = torch.zeros(phi.shape, dtype=torch.float64).pin_memory()
    from paper_2312_11740_gb300 import mp_poisson_project_step_host
    # (z-slab copy pipeline on a second stream: slabs of whole z-blocks, the
    # assembly of a slab after it and the next have arrived)
    mp_poisson_project_step_host(s.handle, hx, hy, hz, hp, TOL)
    assert np.array_equal(hp.numpy(), host(p))
    for hc, dc in zip((hx, hy, hz), (ux, uy, uz)):
        assert np.array_equal(hc.numpy(), host(dc))
    # pageable host buffers: the same bits
    gx, gy, gz = [torch.from_numpy(np.ascontiguousarray(c)) for c in u]
    gp = torch.zeros(phi.shape, dtype=torch.float64)
    mp_poisson_project_step_host(s.handle, gx, gy, gz, gp, TOL)
    assert np.array_equal(gp.numpy(), host(p))
    for hc, dc in zip((gx, gy, gz), (ux, uy, uz)):
        assert np.array_equal(hc.numpy(), host(dc))
    s.close()


def test_deterministic_and_resume():
    phi, u, prm = case("bubble32")
    rhs = dev(oracle.divergence(*u, prm["h"]))
    s = make(phi, prm)
    p1, it1, h1 = s.solve(rhs)
    p2, it2, h2 = s.solve(rhs)
    assert it1 == it2 and h1 == h2
    assert torch.equal(p1, p2)
    # stationary iteration: stop after k cycles, resume from p_k
    s.set_opts(method=1, max_iters=4)
    pk, itk, hk = s.solve(rhs, allow_not_converged=True)
    assert itk == 4
    s.set_opts(method=1, max_iters=400, initial_guess=1)
    pr, itr, hr = s.solve(rhs, p=pk.clone())
    s.set_opts(method=1, max_iters=400, initial_guess=0)
    pf, itf, hf = s.solve(rhs)
    assert abs(itf - (itk + itr)) <= 1
    assert rel_l2(host(pr), host(pf)) < 1e-8
    s.close()


def test_edge_cases():
    h = 1.0 / 8
    # single-level grid: the coarsest direct solve is the whole solve
    phi = synth.level_set((4, 4, 4), 0.25, [((0.5, 0.5, 0.5), 0.3)])
    prm = dict(h=0.25, rho_l=1.0, rho_g=1e-3, sigma=0.02, bc=(P, P, N))
    rhs = np.random.Generator(np.random.PCG64(1)).standard_normal((4, 4, 4))
    ref = oracle.solve(phi, rhs, 0.25, 1.0, 1e-3, 0.02, (P, P, N), tol=1e-13)
    s = make(phi, prm)
    p, it, _ = s.solve(dev(rhs))
    assert it <= 2 and rel_l2(host(p), ref["p"]) < 1e-9
    st = s.stats()
    assert st["levels"] == 1 and st["coarse_n"] == 64
    # zero right-hand side without interface: p = 0 exactly
    s.set_geometry(dev(-np.ones((4, 4, 4))), 1.0, 1e-3, 0.02)
    p, it, hist = s.solve(dev(np.zeros((4, 4, 4))))
    assert torch.count_nonzero(p) == 0 and it == 0
    s.close()
    # odd wall-bounded axis: no coarsening possible, direct solve of 448 cells
    phi = synth.level_set((7, 8, 8), h, [((0.5, 0.5, 0.4), 0.25)])
    prm = dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.01, bc=(P, P, N))
    rhs = np.random.Generator(np.random.PCG64(2)).standard_normal((7, 8, 8))
    ref = oracle.solve(phi, rhs, h, 1.0, 1e-3, 0.01, (P, P, N), tol=1e-13)
    s = make(phi, prm)
    p, it, _ = s.solve(dev(rhs))
    assert rel_l2(host(p), ref["p"]) < 1e-9
    s.close()
    # equal densities, no surface tension: constant-coefficient Poisson
    phi, u, prm = case("bubble32")
    prm = dict(prm, rho_g=1.0, sigma=0.0)
    rhs = oracle.divergence(*u, prm["h"])
    ref = oracle.solve(phi, rhs, prm["h"], 1.0, 1.0, 0.0, prm["bc"], tol=REF_TOL)
    s = make(phi, prm)
    p, it, _ = s.solve(dev(rhs))
    assert rel_l2(host(p), ref["p"]) < PARITY and it <= 12
    s.close()


def test_errors_are_reported():
    phi, u, prm = case("bubble32")
    rhs = oracle.divergence(*u, prm["h"])
    # odd periodic axis
    with pytest.raises(MPError) as e:
        Poisson(dev(np.zeros((8, 8, 9))), 1.0 / 9, (P, P, N))
    assert e.value.status == _lib.MP_ERR_INVALID_ARG
    # coarsest level too large (18 -> 9: 729 cells)
    with pytest.raises(MPError) as e:
        Poisson(dev(np.zeros((18, 18, 18))), 1.0 / 18, (N, N, N))
    assert e.value.status == _lib.MP_ERR_INVALID_ARG
    with pytest.raises(MPError):
        Poisson(dev(phi), prm["h"], prm["bc"], rho_l=-1.0)
    s = make(phi, prm, max_iters=2)
    with pytest.raises(MPError) as e:
        s.solve(dev(rhs))
    assert e.value.status == _lib.MP_ERR_NOT_CONVERGED
    p, it, hist = s.solve(dev(rhs), allow_not_converged=True)
    assert it == 2 and len(hist) == 3
    s.set_opts(max_iters=50)
    bad = rhs.copy()
    bad[3, 4, 5] = np.nan
    with pytest.raises(MPError) as e:
        s.solve(dev(bad))
    assert e.value.status == _lib.MP_ERR_DIVERGED
    s.set_opts(initial_guess=2)
    with pytest.raises(MPError) as e:
        s.solve(dev(rhs))
    assert e.value.status == _lib.MP_ERR_NO_NET
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_256_properties(precision):
    """256^3 one-bubble workload: the oracle's own assembly and operator
    confirm the GPU pressure solves its system to the target; setup fields
    agree at sampled cells."""
    phi, u, prm = synth.workload("bubble256")
    h, bc = prm["h"], prm["bc"]
    rhs = oracle.divergence(*u, h)
    kap, f, J, b = oracle.assemble(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc)
    s = make(phi, prm, precision=precision)
    p, it, hist = s.solve(dev(rhs), tol=TOL)
    pg = host(p)
    _, rn = oracle.residual(f, b, pg, h, bc)
    assert rn / np.linalg.norm(b) <= 1.5 * TOL
    g = s.fields()
    idx = np.random.Generator(np.random.PCG64(3)).integers(0, phi.size, 4096)
    bidx = np.flatnonzero(band(phi, bc).ravel())
    bidx = bidx[np.random.Generator(np.random.PCG64(4)).integers(0, bidx.size, 4096)]
    for key, ref, ix in (("kappa", kap, bidx), ("bx", owned(f)[0], idx), ("bz", owned(f)[2], idx),
                         ("J", J, idx), ("J", J, bidx)):
        got = host(g[key]).ravel()[ix]
        assert np.max(np.abs(got - ref.ravel()[ix])) <= 1e-11 * max(np.abs(ref).max(), 1e-300)
    s.close()



def _components_reference(phi, bc):
    """Gas components (face neighbours, periodic axes wrapped) by scipy, with
    ids in the order of each component's lowest cell index."""
    from scipy import ndimage
    gas = phi > 0
    lab, nl = ndimage.label(gas)
    parent = list(range(nl + 1))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    for axis, kind in enumerate(bc):
        if kind != P:
            continue
        ax = 2 - axis
        a, b = np.take(lab, 0, axis=ax), np.take(lab, -1, axis=ax)
        m = (a > 0) & (b > 0)
        for x, y in set(zip(a[m].tolist(), b[m].tolist())):
            rx, ry = find(x), find(y)
            if rx != ry:
                parent[max(rx, ry)] = min(rx, ry)
    flat = lab.ravel()
    roots = np.array([find(v) if v > 0 else 0 for v in range(nl + 1)])[flat]
    comp = np.full(flat.shape, -1)
    first = {}
    for idx in np.flatnonzero(roots):
        first.setdefault(roots[idx], idx)
    order = {r: k for k, r in enumerate(sorted(first, key=first.get))}
    for idx in np.flatnonzero(roots):
        comp[idx] = order[roots[idx]]
    return comp.reshape(phi.shape), len(order)


@pytest.mark.parametrize("bc", [(P, P, N), (N, N, N), (P, P, P)])
def test_gas_components_match_scipy_labelling(bc):
    """Union-find labelling of the gas cells on the GPU (deflation vectors):
    the partition and the id order equal scipy's labelling with periodic
    merging, including bubbles cut by periodic boundaries."""
    shape = (40, 32, 48)
    h = 1.0 / 48
    bubbles = [((0.02, 0.5, 0.5), 0.12), ((0.5, 0.03, 0.3), 0.1), ((0.6, 0.6, 0.7), 0.08),
               ((0.3, 0.3, 0.25), 0.05), ((0.8, 0.2, 0.15), 0.06)]
    phi = synth.level_set(shape, h, bubbles, bc=bc)
    prm = dict(h=h, bc=bc, rho_l=1.0, rho_g=1e-3, sigma=0.07)
    s = make(phi, prm)
    comp, m = s.components()
    ref, mref = _components_reference(phi, bc)
    assert m == mref
    assert np.array_equal(comp.cpu().numpy(), ref)
    s.close()


def test_gas_components_pool_layer_spans_every_tile():
    """A gas layer above a liquid pool is one component crossing every
    labelling tile (32 x 8 x 8 cells) and both periodic wraps; the bubbles
    below it, some cut by the periodic boundaries, are separate components.
    80 cells per axis: three tiles in x (the last one partial), ten in y."""
    n = 80
    h = 1.0 / n
    bc = (P, P, N)
    bub = [((0.02, 0.5, 0.3), 0.1), ((0.5, 0.97, 0.25), 0.08), ((0.6, 0.6, 0.2), 0.06)]
    phi = synth.level_set((n, n, n), h, bub, pool_z0=0.55, bc=bc)
    s = make(phi, dict(h=h, bc=bc, rho_l=1.0, rho_g=1e-3, sigma=0.07))
    comp, m = s.components()
    ref, mref = _components_reference(phi, bc)
    assert m == mref == 4
    assert np.array_equal(comp.cpu().numpy(), ref)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_deflation_same_answer_fewer_iterations(precision):
    """Deflating CG by the bubbles' indicator vectors changes the iteration,
    not the answer: both solves meet the target, agree with each other, and
    the deflated one takes fewer V-cycles on a multi-bubble problem."""
    n = 64
    h = 1.0 / n
    shape = (n, n, n)
    bubbles = synth.random_bubbles(10, 12, 0.04, 0.1, n)
    phi = synth.level_set(shape, h, bubbles)
    u = synth.velocity(11, shape, h)
    prm = dict(h=h, bc=(P, P, N), rho_l=1.0, rho_g=1e-3, sigma=0.07)
    s = make(phi, prm, precision=precision)
    rhs = s.divergence(*[dev(c) for c in u])
    p1, it1, _ = s.solve(rhs, tol=TOL)
    st = s.stats()
    assert st["components"] == 12 and st["relres"] <= TOL
    s.set_opts(deflate=0)
    p0, it0, _ = s.solve(rhs, tol=TOL)
    assert s.stats()["components"] == 0 and s.stats()["relres"] <= TOL
    assert it1 < it0, (it1, it0)
    assert float(torch.linalg.norm(p1 - p0) / torch.linalg.norm(p0)) < 1e-7
    s.close()


def test_fresh_handles_on_nonblocking_streams():
    """A handle created and used at once on a non-blocking caller stream gives
    bitwise the answer of one on the legacy default stream: the zero fills of
    the new buffers are complete before the first geometry setup (they once
    were not, and an early solve could read half-cleared work arrays)."""
    n = 128
    h = 1.0 / n
    shape = (n, n, n)
    bubbles = synth.random_bubbles(21, 16, 0.03, 0.08, n)
    phi = dev(synth.level_set(shape, h, bubbles))
    u = [dev(c) for c in synth.velocity(22, shape, h)]
    prm = dict(h=h, bc=(P, P, N), rho_l=1.0, rho_g=1e-3, sigma=0.07)
    ref = Poisson(phi, h, prm["bc"], prm["rho_l"], prm["rho_g"], prm["sigma"], precision=0)
    rhs = ref.divergence(*u)
    p_ref, it_ref, _ = ref.solve(rhs, tol=TOL)
    ref.close()
    for precision in (0, 1, 0):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = Poisson(phi, h, prm["bc"], prm["rho_l"], prm["rho_g"], prm["sigma"],
                        precision=precision, stream=st)
            p, it, _ = s.solve(rhs, tol=TOL)
            stats = s.stats()
        st.synchronize()
        assert stats["relres"] <= TOL and stats["components"] == 16
        if precision == 0:
            assert it == it_ref and torch.equal(p, p_ref)
        else:
            assert float(torch.linalg.norm(p - p_ref) / torch.linalg.norm(p_ref)) < 1e-7
        s.close()


def test_precision_switch_after_geometry():
    """The per-precision arrays (FP64 1/diag; FP32 and FP16 faces) are formed
    for the precision the geometry was set in, and added at the first solve in
    the other precision: switching after set_geometry gives bitwise the answer
    of a handle created in that precision."""
    phi, u, prm = case("ragged")
    rhs = dev(oracle.divergence(*u, prm["h"]))
    results = {}
    for first, second in ((0, 1), (1, 0)):
        s = make(phi, prm, precision=first)
        s.set_geometry(dev(phi), prm["rho_l"], prm["rho_g"], prm["sigma"])
        s.solve(rhs)
        s.set_opts(precision=second)
        p, it, _ = s.solve(rhs)
        results[second] = (p, it)
        s.close()
    for prec in (0, 1):
        s = make(phi, prm, precision=prec)
        p, it, _ = s.solve(rhs)
        assert it == results[prec][1] and torch.equal(p, results[prec][0]), prec
        s.close()


@pytest.mark.parametrize("rho_g", [1e-5, 10.0])
def test_mixed_extreme_density_ratios(rho_g):
    """The FP16 face copies of the FP32 V-cycle are scaled by a power of two
    set from 1/min(rho): at density ratio 1e5 (faces up to 1e5) and with the
    gas heavier than the liquid (faces down to 0.1) the mixed solve still
    reaches 1e-10 and agrees with the FP64 one."""
    phi, u, prm = case("bubble32")
    prm = dict(prm, rho_g=rho_g)
    rhs = dev(oracle.divergence(*u, prm["h"]))
    out = {}
    for prec in (0, 1):
        s = make(phi, prm, precision=prec, max_iters=400)
        p, it, _ = s.solve(rhs, tol=TOL)
        assert s.stats()["relres"] <= TOL
        out[prec] = host(p)
        s.close()
    assert rel_l2(out[1], out[0]) < 1e-7


def _pool_case(n, seed=5):
    """Pool + 16 bubbles on an n^3 grid (several fused-sweep z-chunks)."""
    h = 1.0 / n
    bub = synth.random_bubbles(seed, 16, 0.03, 0.08, n, pool_z0=0.6)
    phi = synth.level_set((n, n, n), h, bub, pool_z0=0.6)
    u = synth.velocity(seed, (n, n, n), h)
    return phi, u, dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.07, bc=(P, P, N))


@pytest.mark.parametrize("name,opts", [("ragged", {}), ("walls", {}), ("periodic", {}),
                                       ("bubble32", {"nu1": 3, "nu2": 3}), ("wide", {}),
                                       ("slab", {}),
                                       ("pool128", {}),
                                       ("pool128", {"deflate": 0, "method": 1, "max_iters": 20})])
def test_fused_sweep_bitwise_equals_per_colour_launches(name, opts):
    """The fused red-black pass (both colours in one z-marching launch) and
    the two in-place launches per sweep update every cell with the same
    operands in the same order, so whole mixed-precision solves agree bit for
    bit: pressure, iteration count and residual history.  The cases cover
    tiles that overhang the grid (nx = 40 < 64, ny = 24 = 3 tiles), wall and
    periodic axes in x, y and z, an odd number of sweeps (the last one per
    colour), a 128^3 pool with many z-chunks per tile, and the stationary
    V-cycle iteration; both staging modes: tensor copies of the main rows
    (nx a multiple of 64: pool128; wide, whose level 1 overhangs a wall in
    y; slab, whose finest level wraps a periodic y) and 16-byte copies (the
    other grids and the coarser levels).  The small grids run without the cluster tail, which
    would otherwise take every level the fused sweep runs on."""
    if name == "pool128":
        phi, u, prm = _pool_case(128)
    else:
        phi, u, prm = case(name)
        opts = dict(opts, coarse_cluster=0)
    rhs = dev(oracle.divergence(*u, prm["h"]))
    out = []
    for smoother in (1, 0):
        s = make(phi, prm, precision=1, smoother=smoother, **opts)
        # (the stationary V-cycle is cut off after max_iters: same bits either way)
        p, it, hist = s.solve(rhs, tol=TOL, allow_not_converged="max_iters" in opts)
        out.append((host(p), it, list(hist), s.stats()["relres"]))
        if smoother == 1:
            prof = {(e["name"], e["level"]) for e in s.profile()}
            assert any(k[0] == "rbgs_f32_fused" for k in prof), prof
        s.close()
    (p1, it1, h1, r1), (p0, it0, h0, r0) = out
    assert it1 == it0 and h1 == h0 and r1 == r0
    assert np.array_equal(p1.view(np.uint64), p0.view(np.uint64))


def test_fused_sweep_bitwise_full_size_pool():
    """The benchmark's 256^3 pool workload (7 z-chunks of 36-37 planes at the
    finest level): fused and per-colour smoothing give the same bits."""
    phi, u, prm = synth.workload("pool256")
    d = [dev(c) for c in u]
    out = []
    for smoother in (1, 0):
        s = Poisson(dev(phi), prm["h"], prm["bc"], prm["rho_l"], prm["rho_g"], prm["sigma"],
                    precision=1, smoother=smoother)
        rhs = s.divergence(*d)
        p, it, hist = s.solve(rhs, tol=TOL)
        out.append((p, it, list(hist)))
        s.close()
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert torch.equal(out[0][0], out[1][0])


def test_labelling_bound_turns_deflation_off_and_the_solve_still_converges():
    """When a find walk or union retry of the gas-component labelling reaches
    mp_opts.label_limit (here 1, so any walk longer than a step does), the
    geometry is solved without deflation: no components, the same converged
    pressure, and deflation returns with the default bound."""
    phi, u, prm = _pool_case(64, seed=9)
    rhs = dev(oracle.divergence(*u, prm["h"]))
    s = make(phi, prm, precision=1)
    p_ref, _, _ = s.solve(rhs, tol=TOL)
    assert s.stats()["components"] > 1
    s.set_opts(label_limit=1)
    s.set_geometry(dev(phi), prm["rho_l"], prm["rho_g"], prm["sigma"])
    assert s.components()[1] == 0
    p, it, _ = s.solve(rhs, tol=TOL)
    st = s.stats()
    assert st["components"] == 0 and st["relres"] <= TOL
    assert rel_l2(host(p), host(p_ref)) < PARITY
    s.set_opts(label_limit=8192)
    s.set_geometry(dev(phi), prm["rho_l"], prm["rho_g"], prm["sigma"])
    s.solve(rhs, tol=TOL)
    assert s.stats()["components"] > 1
    s.close()


# ---------------------------------------------------- outflow (p = 0) sides
D, ND, DN = oracle.DIRICHLET, oracle.NEUMANN_DIRICHLET, oracle.DIRICHLET_NEUMANN


def _outflow_case(name):
    g = rng_np(17)
    if name == "pool_outflow_top":   # liquid pool + bubble, wall bottom, outflow top
        shape, h, bc = (32, 32, 32), 1.0 / 32, (P, P, ND)
        phi = synth.level_set(shape, h, [((0.5, 0.5, 0.3), 0.15)], pool_z0=0.6, bc=bc)
    elif name == "channel":          # outflow at both x ends, walls in y, periodic z
        shape, h, bc = (16, 24, 40), 1.0 / 40, (D, N, P)
        phi = synth.level_set(shape, h, [((0.3, 0.3, 0.5), 0.12), ((0.75, 0.6, 0.4), 0.1)], bc=bc)
    elif name == "inflow_outflow":   # the paper's TOML pattern: inflow low x, outflow high x
        shape, h, bc = (24, 16, 48), 1.0 / 48, (ND, DN, N)
        phi = synth.level_set(shape, h, [((0.5, 0.4, 0.3), 0.2)], bc=bc)
    else:                            # outflow on every side
        shape, h, bc = (16, 16, 24), 1.0 / 24, (D, D, D)
        phi = synth.level_set(shape, h, [((0.5, 0.5, 0.5), 0.25)], bc=bc)
    rhs = g.standard_normal(shape)
    return phi, rhs, dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.05, bc=bc)


def rng_np(seed):
    return np.random.Generator(np.random.PCG64(seed))


OUT_CASES = ["pool_outflow_top", "channel", "inflow_outflow", "all_outflow"]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", OUT_CASES)
def test_outflow_solve_matches_oracle(name, precision):
    """p = 0 on outflow faces (antisymmetric ghost): the operator is
    nonsingular, b keeps its mean, no gauge.  GPU pressure against the
    oracle's, element by element (relative L2 <= 1e-8), FP64 and mixed;
    deflation and the fused sweep switch themselves off."""
    phi, rhs, prm = _outflow_case(name)
    ref = oracle.solve(phi, rhs, prm["h"], prm["rho_l"], prm["rho_g"], prm["sigma"], prm["bc"],
                       tol=REF_TOL)
    assert ref["iters"] >= 0
    s = make(phi, prm, precision=precision)
    p, it, _ = s.solve(dev(rhs), tol=TOL)
    st = s.stats()
    assert st["relres"] <= TOL and st["components"] == 0
    assert rel_l2(host(p), ref["p"]) < PARITY
    assert abs(host(p).mean()) > 1e-6 * np.abs(host(p)).max()  # not gauged to mean zero
    s.close()


@pytest.mark.parametrize("name", OUT_CASES)
def test_outflow_apply_and_rhs_match_oracle(name):
    phi, rhs, prm = _outflow_case(name)
    h, bc = prm["h"], prm["bc"]
    s = make(phi, prm)
    x = rng_np(23).standard_normal(phi.shape)
    f = oracle.faces(phi, prm["rho_l"], prm["rho_g"], bc)
    assert rel_max(host(s.apply(dev(x))), oracle.apply(f, x, h, bc)) < 1e-12
    _, _, _, b = oracle.assemble(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc)
    assert rel_max(host(s.rhs(dev(rhs))), b) < 1e-11
    s.close()


def test_outflow_rejects_face_velocity_calls_and_learned_guess():
    """The low-face-owned velocity layout has one boundary slot per
    non-periodic axis: the fused divergence/correction calls refuse outflow
    handles."""
    phi, rhs, prm = _outflow_case("pool_outflow_top")
    s = make(phi, prm)
    u = [dev(np.zeros(phi.shape)) for _ in range(3)]
    for call in (lambda: s.divergence(*u), lambda: s.project_step(*u, dev(np.zeros(phi.shape))),
                 lambda: s.project(dev(np.zeros(phi.shape)), *u)):
        with pytest.raises(MPError) as e:
            call()
        assert e.value.status == _lib.MP_ERR_INVALID_ARG
    s.close()


# ------------------------------------------- phase change: the flux jump
def _mdot(phi, h, scale=0.05):
    nz, ny, nx = phi.shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h,
                          (np.arange(nx) + 0.5) * h, indexing="ij")
    return np.ascontiguousarray(scale * (1.0 + x + 0.5 * y * z))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["bubble32", "ragged", "pool_outflow_top", "channel"])
def test_mass_flux_source_and_solve_match_oracle(name, precision):
    """Evaporation (mp_poisson_set_mass_flux): the jump source with the
    flux-jump shares, the right-hand side and the pressure against the
    oracle's, element by element; with no outflow side the net source goes
    with the mean of b.  Clearing the mass flux restores the plain source."""
    if name in ("bubble32", "ragged"):
        phi, u, prm = case(name)
        rhs = oracle.divergence(*u, prm["h"])
    else:
        phi, rhs, prm = _outflow_case(name)
    h, bc = prm["h"], prm["bc"]
    md = _mdot(phi, h)
    s = make(phi, prm, precision=precision)
    s.set_mass_flux(dev(md))
    kap, f, J, b = oracle.assemble(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc,
                                   mdot=md)
    Jflux = oracle.flux_jump(phi, md, f, h, prm["rho_l"], prm["rho_g"], bc)
    assert np.abs(Jflux).max() > 0.1 * np.abs(J - Jflux).max()  # the source matters
    assert rel_max(host(s.fields()["J"]), J) < 1e-11
    assert rel_max(host(s.rhs(dev(rhs))), b) < 1e-11
    ref = oracle.solve(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc, tol=REF_TOL,
                       mdot=md)
    p, _, _ = s.solve(dev(rhs), tol=TOL)
    assert s.stats()["relres"] <= TOL
    assert rel_l2(host(p), ref["p"]) < PARITY
    s.set_mass_flux(None)
    assert rel_max(host(s.fields()["J"]), J - Jflux) < 1e-11
    s.close()


@pytest.mark.parametrize("name", ["bubble32", "walls"])
def test_mass_flux_projection_matches_oracle(name):
    """The projection step with a mass flux: the corrected face velocities
    (liquid side on interface faces) against the oracle's; every liquid cell
    is divergence-free to the solve's tolerance.  The flux stays set across
    set_geometry."""
    phi, u, prm = case(name)
    h, bc = prm["h"], prm["bc"]
    md = _mdot(phi, h, 0.02)
    rhs = oracle.divergence(*u, h)
    ref = oracle.solve(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc, tol=REF_TOL,
                       mdot=md)
    fx, fy, fz = oracle.project(phi, ref["kappa"], ref["faces"], ref["p"], *u, h, prm["sigma"],
                                bc, mdot=md, rho_l=prm["rho_l"], rho_g=prm["rho_g"])
    s = make(phi, prm)
    s.set_mass_flux(dev(md))
    s.set_geometry(dev(phi), prm["rho_l"], prm["rho_g"], prm["sigma"])
    ux, uy, uz = [dev(c) for c in u]
    p = torch.zeros_like(ux)
    s.project_step(ux, uy, uz, p, tol=TOL)
    for g, o in zip((ux, uy, uz), (fx[:, :, :-1], fy[:, :-1, :], fz[:-1, :, :])):
        assert rel_l2(host(g), o) < PARITY
    div = oracle.divergence(host(ux), host(uy), host(uz), h)
    liquid = phi <= 0
    # singular problem: the mean of b (the created volume) is spread over every cell
    assert np.abs(div[liquid] - div[liquid].mean()).max() <= 1e-8 * np.linalg.norm(ref["b"])
    s.close()


# ------------------------------------------------ cluster coarse tail
@pytest.mark.parametrize("name", ["bubble32", "periodic", "pool128"])
def test_cluster_tail_matches_per_level_launches(name):
    """The FP32 coarse tail on an 8-CTA thread-block cluster (coarse_cluster
    = 1) runs the same V-cycle as the per-level launches down to the one-CTA
    tail, except that its top level smooths on FP32 instead of FP16 faces:
    one stationary V-cycle from zero agrees to 1e-2, the kernel does run, and
    both forms solve to the target with the oracle's pressure and iteration
    counts within two."""
    if name == "pool128":
        phi, u, prm = _pool_case(128)
    else:
        phi, u, prm = case(name)
    h, bc = prm["h"], prm["bc"]
    rhs = dev(oracle.divergence(*u, h))
    out = {}
    for cl in (1, 0):
        s = make(phi, prm, precision=1, coarse_cluster=cl, method=1, max_iters=1)
        p1, _, _ = s.solve(rhs, tol=TOL, allow_not_converged=True)
        ran = sum(e["launches"] for e in s.profile() if e["name"] == "coarse_cluster_f32")
        s.set_opts(precision=1, coarse_cluster=cl, method=0, max_iters=200)
        p, it, _ = s.solve(rhs, tol=TOL)
        assert s.stats()["relres"] <= TOL
        out[cl] = (host(p1), host(p), it, ran)
        s.close()
    assert out[1][3] > 0 and out[0][3] == 0
    assert rel_l2(out[1][0], out[0][0]) < 1e-2
    assert abs(out[1][2] - out[0][2]) <= 2
    if name != "pool128":
        ref = oracle.solve(phi, oracle.divergence(*u, h), h, prm["rho_l"], prm["rho_g"],
                           prm["sigma"], bc, tol=REF_TOL)
        for cl in (1, 0):
            assert rel_l2(out[cl][1], ref["p"]) < PARITY


def test_all_gas_and_all_liquid_domains():
    """A domain that is one gas component (its indicator is the operator's
    null space, so its E entry is zero and the component is left out of the
    deflation) and an all-liquid domain (no components): both solve to the
    oracle's pressure, FP64 and mixed, with and without deflation."""
    shape, h = (24, 16, 32), 1.0 / 32
    bc = (P, P, N)
    g = np.random.Generator(np.random.PCG64(8))
    rhs = g.standard_normal(shape)
    for sign in (1.0, -1.0):
        phi = sign * (0.5 + g.random(shape))  # gas everywhere / liquid everywhere
        prm = dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.05, bc=bc)
        ref = oracle.solve(phi, rhs, h, 1.0, 1e-3, 0.05, bc, tol=REF_TOL)
        for precision in (0, 1):
            for deflate in (1, 0):
                s = make(phi, prm, precision=precision, deflate=deflate)
                p, _, _ = s.solve(dev(rhs), tol=TOL)
                assert s.stats()["relres"] <= TOL
                assert rel_l2(host(p), ref["p"]) < PARITY, (sign, precision, deflate)
                s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_outflow_mass_flux_properties(precision):
    """256^3 pool + 32 bubbles under an outflow top with an evaporating mass
    flux (the bench geometry with the paper's outflow and phase-change
    options): the oracle's own assembly (flux-jump source included) and
    operator confirm the GPU pressure solves its system to the target; the
    jump source agrees at sampled cells."""
    phi, u, prm = synth.workload("pool256")
    h = prm["h"]
    bc = (P, P, oracle.NEUMANN_DIRICHLET)
    nz, ny, nx = phi.shape
    z = (np.arange(nz) + 0.5)[:, None, None] * h
    md = np.ascontiguousarray(np.broadcast_to(0.02 * (1.0 + z), phi.shape))
    rhs = oracle.divergence(*u, h)
    prm = dict(prm, bc=bc)
    kap, f, J, b = oracle.assemble(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc,
                                   mdot=md)
    s = make(phi, prm, precision=precision)
    s.set_mass_flux(dev(md))
    p, it, _ = s.solve(dev(rhs), tol=TOL)
    _, rn = oracle.residual(f, b, host(p), h, bc)
    assert rn / np.linalg.norm(b) <= 1.5 * TOL
    idx = np.flatnonzero(band(phi, bc).ravel())
    idx = idx[np.random.Generator(np.random.PCG64(5)).integers(0, idx.size, 4096)]
    got = host(s.fields()["J"]).ravel()[idx]
    assert np.max(np.abs(got - J.ravel()[idx])) <= 1e-11 * np.abs(J).max()
    s.close()


@pytest.mark.parametrize("shape", [(64, 32, 16), (32, 64, 64)])
def test_cluster_tail_on_anisotropic_grids(shape):
    """Grids whose axes coarsen to different sizes (the cluster tail's slabs
    then hold planes of unequal sides, and its coarsest level is not cubic):
    mixed solves with the cluster tail reach the oracle's pressure."""
    nz, ny, nx = shape
    h = 1.0 / nx
    bc = (P, P, N)
    phi = synth.level_set(shape, h, [((0.5, 0.5 * ny / nx, 0.3 * nz / nx), 0.2 * min(ny, nz) / nx)],
                          bc=bc)
    u = synth.velocity(12, shape, h, bc=bc)
    prm = dict(h=h, rho_l=1.0, rho_g=1e-3, sigma=0.05, bc=bc)
    rhs = oracle.divergence(*u, h)
    ref = oracle.solve(phi, rhs, h, 1.0, 1e-3, 0.05, bc, tol=REF_TOL)
    s = make(phi, prm, precision=1)
    p, _, _ = s.solve(dev(rhs), tol=TOL)
    assert s.stats()["relres"] <= TOL
    assert rel_l2(host(p), ref["p"]) < PARITY
    print(shape, [(e["name"], e["level"]) for e in s.profile() if e["name"] == "coarse_cluster_f32"])
    s.close()
