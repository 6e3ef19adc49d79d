"""Pins of the FP64 CPU oracle against facts fixed outside the oracle.

Each test checks the oracle against a closed form, an invariant, a special
case with a textbook solution, an exact continuum solution, a dense direct
solve, or a convergence rate -- never against a retyped copy of its own
formulas.  A dropped term, a wrong sign, a swapped theta or a transposed
index in the oracle fails at least one of them.
"""
import os
import tomllib

import numpy as np
import pytest

import oracle
import synth
from numpy.polynomial import Polynomial as Poly

P, N = synth.PERIODIC, synth.NEUMANN
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_params():
    with open(os.path.join(GOLDEN, "paper_runtime_params.toml"), "rb") as f:
        t = tomllib.load(f)
    return t["Multiphase"]["mph_rhoGas"], t["Multiphase"]["mph_invWeber"]


def centres(shape, h):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(synth.cell_centres(nz, h), synth.cell_centres(ny, h),
                          synth.cell_centres(nx, h), indexing="ij")
    return x, y, z


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


BCS = [(P, P, N), (N, N, N), (P, P, P), (N, P, N)]


@pytest.mark.parametrize("bc", BCS)
def test_operator_symmetric_nullspace_negative(bc):
    """A is symmetric, annihilates constants and is negative semidefinite."""
    shape, h = (10, 12, 14), 1.0 / 14
    bub = [((0.4, 0.5, 0.35), 0.22), ((0.1, 0.15, 0.6), 0.12)]
    phi = synth.level_set(shape, h, bub, bc=bc)
    phi += 0.01 * rng(1).standard_normal(shape)  # break symmetries of the geometry
    f = oracle.faces(phi, 1.0, 1e-3, bc)
    g = rng(2)
    for _ in range(5):
        x, y = g.standard_normal(shape), g.standard_normal(shape)
        yAx = (y * oracle.apply(f, x, h, bc)).sum()
        xAy = (x * oracle.apply(f, y, h, bc)).sum()
        scale = np.linalg.norm(y) * np.linalg.norm(oracle.apply(f, x, h, bc))
        assert abs(yAx - xAy) <= 1e-13 * scale
        assert (x * oracle.apply(f, x, h, bc)).sum() <= 0.0
    assert np.all(oracle.apply(f, np.full(shape, 3.25), h, bc) == 0.0)


def _eig_axis(n, kind):
    """Eigen-decomposition of the 1-D cell-centred second difference (h=1)."""
    i = np.arange(n)
    if kind == P:  # periodic: Fourier modes
        m = np.arange(n)
        lam = 2.0 * np.cos(2.0 * np.pi * m / n) - 2.0
        V = np.exp(2j * np.pi * np.outer(i, m) / n) / np.sqrt(n)
    else:  # zero-flux walls: DCT-II modes cos(pi m (i + 1/2) / n)
        m = np.arange(n)
        lam = 2.0 * np.cos(np.pi * m / n) - 2.0
        V = np.cos(np.pi * np.outer(i + 0.5, m) / n)
        V /= np.linalg.norm(V, axis=0)
    return lam, V


def spectral_solve(b, h, beta, bc):
    """Exact discrete solution of beta * L p = b, mean(p) = 0 (L = 7-point
    Laplacian with the given boundaries) by diagonalisation."""
    nz, ny, nx = b.shape
    lx, Vx = _eig_axis(nx, bc[0])
    ly, Vy = _eig_axis(ny, bc[1])
    lz, Vz = _eig_axis(nz, bc[2])
    bh = np.einsum("kji,ia,jb,kc->cba", b.astype(complex), Vx.conj(), Vy.conj(), Vz.conj())
    lam = (lz[:, None, None] + ly[None, :, None] + lx[None, None, :]) * beta / (h * h)
    ph = np.zeros_like(bh)
    nz_mask = np.abs(lam) > 1e-9 * np.abs(lam).max()
    ph[nz_mask] = bh[nz_mask] / lam[nz_mask]
    p = np.einsum("cba,ia,jb,kc->kji", ph, Vx, Vy, Vz).real
    return p - p.mean()


@pytest.mark.parametrize("bc", [(P, P, N), (N, N, N), (P, P, P)])
def test_constant_coefficient_matches_spectral(bc):
    """rho_l = rho_g, sigma = 0: the system is beta times the 7-point
    Laplacian, solved exactly by Fourier (periodic) / DCT-II (walls)."""
    shape, h = (8, 12, 16), 1.0 / 16
    phi = synth.level_set(shape, h, [((0.5, 0.4, 0.3), 0.2)], bc=bc)
    rhs = rng(3).standard_normal(shape)
    res = oracle.solve(phi, rhs, h, 0.5, 0.5, 0.0, bc, tol=1e-13)
    assert res["iters"] >= 0
    assert np.all(res["J"] == 0.0)
    exact = spectral_solve(rhs - rhs.mean(), h, 2.0, bc)
    err = np.linalg.norm(res["p"] - exact) / np.linalg.norm(exact)
    assert err < 1e-10


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_flat_interface_matches_continuum(axis):
    """phi = s - 0.37 along one wall-bounded axis, point sources +/-S at two
    cells: the flux between them is S, the continuum pressure rises by
    S * integral of rho ds, and the two-layer face coefficient reproduces
    that at every cell centre exactly (piecewise-linear continuum solution)."""
    n, m = 32, 4
    h = 1.0 / n
    bc = [P, P, P]
    bc[axis] = N
    bc = tuple(bc)
    shape = [m, m, m]
    shape[2 - axis] = n
    shape = tuple(shape)
    x, y, z = centres(shape, h)
    s = (x, y, z)[axis]
    phi = s - 0.37
    rho_l, rho_g = 1.0, 1e-3
    k1, k2, S = 4, 24, 2.5
    idx = np.arange(n)
    rhs1 = np.zeros(n)
    rhs1[k1], rhs1[k2] = S / h, -S / h
    rhs = np.broadcast_to(np.moveaxis(rhs1[None, None, :], 2, 2 - axis), shape).copy()
    res = oracle.solve(phi, rhs, h, rho_l, rho_g, 0.0, bc, tol=1e-13)
    # continuum: p(s) = S * integral_{s1}^{s} rho(t) dt between the sources
    sc = (idx + 0.5) * h
    s1, s2, zi = sc[k1], sc[k2], 0.37

    def rho_int(a, b):  # integral of rho over [a, b], liquid below zi
        lo_l = max(a, -1.0)
        liq = max(0.0, min(b, zi) - lo_l)
        gas = max(0.0, b - max(a, zi))
        return rho_l * liq + rho_g * gas

    p1 = np.array([S * rho_int(s1, min(max(t, s1), s2)) for t in sc])
    p1 -= p1.mean()
    got = np.moveaxis(res["p"], 2 - axis, 2)[0, 0, :]
    assert np.allclose(np.moveaxis(res["p"], 2 - axis, 2), got[None, None, :], atol=1e-12)
    assert np.max(np.abs(got - p1)) <= 1e-10 * np.max(np.abs(p1))


def test_dense_direct_solve_8cubed():
    """8^3 with a bubble and surface tension: CG equals the dense direct
    solution of (-A + 11^T/n) x = -b, which is the mean-free solution."""
    shape, h = (8, 8, 8), 1.0 / 8
    bc = (P, P, N)
    phi = synth.level_set(shape, h, [((0.5, 0.5, 0.45), 0.3)], bc=bc)
    rhs = rng(4).standard_normal(shape)
    res = oracle.solve(phi, rhs, h, 1.0, 1e-3, 0.05, bc, tol=1e-13)
    n = phi.size
    M = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        M[:, c] = oracle.apply(res["faces"], e.reshape(shape), h, bc).ravel()
    x = np.linalg.solve(-M + np.ones((n, n)) / n, -res["b"].ravel())
    assert abs(x.mean()) < 1e-9 * np.abs(x).max()
    x -= x.mean()
    err = np.linalg.norm(res["p"].ravel() - x) / np.linalg.norm(x)
    assert err < 1e-9
    xg, sweeps, rel = oracle.gs(res["faces"], res["b"], h, bc, tol=1e-12)
    assert sweeps >= 0
    assert np.linalg.norm(xg.ravel() - x) / np.linalg.norm(x) < 1e-7


def _static_bubble_dp(n, rho_g, sigma, R=0.25, c=(0.5, 0.5, 0.4)):
    h = 1.0 / n
    shape = (n, n, n)
    x, y, z = centres(shape, h)
    d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    phi = synth.level_set(shape, h, [(c, R)])
    res = oracle.solve(phi, np.zeros(shape), h, 1.0, rho_g, sigma, (P, P, N), tol=1e-12)
    p = res["p"]
    return p[d < R - 2 * h].mean() - p[d > R + 2 * h].mean()


def test_static_bubble_laplace_pressure():
    """rhs = 0: the pressure is piecewise constant with p_in - p_out = 2 sigma/R
    (Laplace); the discrete difference converges at second order.  Density
    ratio and sigma are the paper's runtime parameters."""
    rho_g, sigma = paper_params()
    R = 0.25
    exact = 2.0 * sigma / R
    errs = [abs(_static_bubble_dp(n, rho_g, sigma, R) - exact) / exact for n in (16, 32, 64)]
    assert errs[2] < 1e-3
    for a, b in zip(errs, errs[1:]):
        assert np.log2(a / b) > 1.7


def _manufactured_error(n, rho_g, amp, sigma=0.01, R=0.25, R1=0.375, c=(0.5, 0.5, 0.4)):
    """p = amp*q(r) + (2 sigma/R) 1[r<R] with q = Q(r^2), Q'(s) =
    (s - R1^2)^2 (s - R^2)^3: q' and q'' vanish on the bubble surface (no
    flux jump, continuous rhs) and q is C^2 at R1 where it meets zero."""
    h = 1.0 / n
    shape = (n, n, n)
    x, y, z = centres(shape, h)
    d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    s = d * d
    Qp = Poly([-R1 ** 2, 1.0]) ** 2 * Poly([-R ** 2, 1.0]) ** 3
    Q = Qp.integ()
    Q = Q - Q(R1 ** 2)
    Qpp = Qp.deriv()
    inside = d < R1
    # radial Laplacian of Q(r^2): q'' + 2 q'/r = 6 Q'(s) + 4 s Q''(s)
    lap = np.where(inside, amp * (6.0 * Qp(s) + 4.0 * s * Qpp(s)), 0.0)
    beta = np.where(d < R, 1.0 / rho_g, 1.0)
    p_exact = np.where(inside, amp * Q(s), 0.0) + np.where(d < R, 2.0 * sigma / R, 0.0)
    p_exact -= p_exact.mean()
    phi = synth.level_set(shape, h, [(c, R)])
    res = oracle.solve(phi, beta * lap, h, 1.0, rho_g, sigma, (P, P, N), tol=1e-12)
    return np.linalg.norm(res["p"] - p_exact) / np.linalg.norm(p_exact)


def test_manufactured_jump_solution_second_order():
    """Second-order convergence towards an exact solution with a pressure
    jump (density ratio 10: clean rates; ratio 1000: overall rate)."""
    e = [_manufactured_error(n, 0.1, 1e5) for n in (16, 32, 64)]
    assert e[2] < 1e-3
    for a, b in zip(e, e[1:]):
        assert np.log2(a / b) > 1.8
    e1000 = [_manufactured_error(n, 1e-3, 1e5) for n in (16, 64)]
    assert np.log2(e1000[0] / e1000[1]) / 2.0 > 1.8


def test_curvature_closed_forms():
    """Sphere: kappa = 2/r (gas inside, phi = R - r); cylinder: 1/r;
    plane: 0; second-order convergence; clamp |kappa| <= 1/h."""
    c = np.array([0.5, 0.5, 0.5])
    errs = []
    for n in (32, 64):
        h = 1.0 / n
        shape = (n, n, n)
        x, y, z = centres(shape, h)
        r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
        k = oracle.curvature(0.3 - r, h, (P, P, N))
        band = (r > 0.2) & (r < 0.35)
        errs.append(np.max(np.abs(k[band] - 2.0 / r[band]) * r[band] / 2.0))
        assert np.all(np.abs(k) <= 1.0 / h + 1e-12)
        assert k[r < 0.5 * h].size == 0 or np.all(k[r < h] <= 1.0 / h + 1e-12)
        rc = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2)
        kc = oracle.curvature(0.3 - rc, h, (P, P, N))
        bandc = (rc > 0.15) & (rc < 0.35)
        assert np.max(np.abs(kc[bandc] - 1.0 / rc[bandc]) * rc[bandc]) < 0.01
        kp = oracle.curvature(z - 0.37, h, (P, P, N))
        assert np.all(kp == 0.0)
    assert errs[1] < 0.01
    assert np.log2(errs[0] / errs[1]) > 1.8


def test_jump_source_properties():
    """J telescopes (sums to zero), vanishes without surface tension, and
    pushes pressure up on the gas side: positive on liquid cells next to a
    bubble, negative on gas cells."""
    n, h = 24, 1.0 / 24
    shape = (n, n, n)
    phi = synth.level_set(shape, h, [((0.5, 0.5, 0.45), 0.27)])
    kappa = oracle.curvature(phi, h, (P, P, N))
    f = oracle.faces(phi, 1.0, 1e-3, (P, P, N))
    J = oracle.jump(phi, kappa, f, h, 0.07, (P, P, N))
    assert abs(J.sum()) <= 1e-12 * np.abs(J).sum()
    assert np.all(J[phi > 0] <= 0.0) and np.all(J[phi <= 0] >= 0.0)
    assert np.abs(J).max() > 0.0
    assert np.all(oracle.jump(phi, kappa, f, h, 0.0, (P, P, N)) == 0.0)


def test_faces_special_cases():
    """Equal densities give 1/rho everywhere; single-fluid regions give
    1/rho of that fluid; wall faces are zero; periodic faces 0 and n agree."""
    shape, h = (8, 10, 12), 1.0 / 12
    bc = (P, P, N)
    phi = synth.level_set(shape, h, [((0.5, 0.5, 0.5), 0.25)], bc=bc)
    f = oracle.faces(phi, 0.5, 0.5, bc)
    assert np.allclose(f.fx, 2.0, rtol=0, atol=1e-15)
    assert np.allclose(f.fy, 2.0, rtol=0, atol=1e-15)
    assert np.all(f.fz[0] == 0.0) and np.all(f.fz[-1] == 0.0)
    assert np.allclose(f.fz[1:-1], 2.0, rtol=0, atol=1e-15)
    f = oracle.faces(-np.ones(shape), 1.0, 1e-3, bc)
    assert np.all(f.fx == 1.0) and np.all(f.fz[1:-1] == 1.0)
    f = oracle.faces(np.ones(shape), 1.0, 1e-3, bc)
    assert np.allclose(f.fx, 1e3) and np.allclose(f.fz[1:-1], 1e3)
    f = oracle.faces(phi, 1.0, 1e-3, bc)
    assert np.array_equal(f.fx[:, :, 0], f.fx[:, :, -1])
    assert np.array_equal(f.fy[:, 0, :], f.fy[:, -1, :])
    # an interface face lies strictly between the two one-fluid values
    mixed = (phi[:, :, 1:] > 0) != (phi[:, :, :-1] > 0)
    vals = f.fx[:, :, 1:-1][mixed]
    assert vals.size > 0 and np.all(vals > 1.0) and np.all(vals < 1e3)


def test_divergence_closed_form():
    """u_x = sin(2 pi x) on x-faces: (div u)_i = 2 sin(pi h) cos(2 pi x_i) / h."""
    shape, h = (4, 6, 16), 1.0 / 16
    xf = np.arange(16) * h
    ux = np.broadcast_to(np.sin(2 * np.pi * xf)[None, None, :], shape).copy()
    zero = np.zeros(shape)
    d = oracle.divergence(ux, zero, zero, h)
    xc = (np.arange(16) + 0.5) * h
    exact = 2.0 * np.sin(np.pi * h) * np.cos(2 * np.pi * xc) / h
    assert np.allclose(d, exact[None, None, :], rtol=0, atol=1e-12)


def test_projection_makes_velocity_divergence_free():
    """After the solve, u = u* - beta (grad p - jump) has discrete divergence
    b - A p (the residual), i.e. ~1e-12 of div u*; wall normal velocity
    stays zero (bubble workload of the 32^3 config)."""
    phi, u, prm = synth.workload("bubble32")
    h, bc = prm["h"], prm["bc"]
    rhs = oracle.divergence(*u, h)
    res = oracle.solve(phi, rhs, h, prm["rho_l"], prm["rho_g"], prm["sigma"], bc, tol=1e-12)
    fx, fy, fz = oracle.project(phi, res["kappa"], res["faces"], res["p"], *u, h, prm["sigma"], bc)
    div = oracle.divergence_full(fx, fy, fz, h)
    assert np.linalg.norm(div) <= 1e-10 * np.linalg.norm(rhs)
    assert np.all(fz[0] == 0.0) and np.all(fz[-1] == 0.0)


# ---------------------------------------------------- outflow (p = 0) sides
D, ND, DN = oracle.DIRICHLET, oracle.NEUMANN_DIRICHLET, oracle.DIRICHLET_NEUMANN
OUT_BCS = [(P, P, D), (D, N, P), (ND, P, DN), (D, D, D), (N, DN, ND)]


def _eig_axis_any(n, kind):
    """_eig_axis plus the outflow kinds, from the closed forms of the 1-D
    cell-centred second difference with p = 0 on a boundary face (ghost
    -p): both sides sin(pi m (i+1/2)/n), m = 1..n; wall low / outflow high
    cos(a (i+1/2)), outflow low / wall high sin(a (i+1/2)), a = (2m+1) pi/(2n)."""
    if kind in (P, N):
        return _eig_axis(n, kind)
    i = np.arange(n) + 0.5
    if kind == D:
        m = np.arange(1, n + 1)
        lam = 2.0 * np.cos(np.pi * m / n) - 2.0
        V = np.sin(np.pi * np.outer(i, m) / n)
    else:
        a = (2 * np.arange(n) + 1) * np.pi / (2 * n)
        lam = 2.0 * np.cos(a) - 2.0
        V = np.cos(np.outer(i, a)) if kind == ND else np.sin(np.outer(i, a))
    return lam, V / np.linalg.norm(V, axis=0)


def spectral_solve_any(b, h, beta, bc):
    """Exact discrete solution of beta * L p = b by diagonalisation (no mean
    removal: with an outflow side L has no null space)."""
    nz, ny, nx = b.shape
    lx, Vx = _eig_axis_any(nx, bc[0])
    ly, Vy = _eig_axis_any(ny, bc[1])
    lz, Vz = _eig_axis_any(nz, bc[2])
    bh = np.einsum("kji,ia,jb,kc->cba", b.astype(complex), Vx.conj(), Vy.conj(), Vz.conj())
    lam = (lz[:, None, None] + ly[None, :, None] + lx[None, None, :]) * beta / (h * h)
    assert np.abs(lam).min() > 0.0
    return np.einsum("cba,ia,jb,kc->kji", bh / lam, Vx, Vy, Vz).real


@pytest.mark.parametrize("bc", OUT_BCS)
def test_outflow_constant_coefficient_matches_spectral(bc):
    """rho_l = rho_g: beta times the 7-point Laplacian with p = 0 on the
    outflow faces, solved exactly by sine/cosine bases; b keeps its mean."""
    shape, h = (8, 12, 16), 1.0 / 16
    phi = synth.level_set(shape, h, [((0.5, 0.4, 0.3), 0.2)], bc=(N, N, N))
    rhs = rng(4).standard_normal(shape)
    res = oracle.solve(phi, rhs, h, 0.5, 0.5, 0.0, bc, tol=1e-13)
    assert res["iters"] >= 0 and np.array_equal(res["b"], rhs)
    exact = spectral_solve_any(rhs, h, 2.0, bc)
    assert np.linalg.norm(res["p"] - exact) / np.linalg.norm(exact) < 1e-10


@pytest.mark.parametrize("bc", OUT_BCS[:3])
def test_outflow_operator_symmetric_negative_definite(bc):
    """With an outflow side the operator stays symmetric and becomes
    negative definite: constants are no longer in its null space and the
    smallest eigenvalue of -A (dense, 6x4x8 cells) is positive."""
    shape, h = (6, 4, 8), 1.0 / 8
    phi = synth.level_set(shape, h, [((0.4, 0.5, 0.45), 0.3)], bc=(N, N, N))
    f = oracle.faces(phi, 1.0, 1e-3, bc)
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = oracle.apply(f, e.reshape(shape), h, bc).ravel()
    assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(-A).min() > 0.0
    assert np.abs(oracle.apply(f, np.ones(shape), h, bc)).max() > 0.0


def test_outflow_flux_problem_converges_second_order():
    """1-D in z: wall at z = 0, outflow p = 0 at z = 1, liquid below the flat
    interface z0 and gas above, uniform source f.  Continuum: the flux
    beta p' = f z is continuous, p(z) = -int_z^1 f s / beta(s) ds.  The
    discrete solution (ghost-fluid faces, outflow ghost) converges at second
    order; a p = 0 placed at the last cell centre instead of the face would
    be first order."""
    z0, f, rl, rg = 0.37, 1.0, 1.0, 1e-3
    errs = []
    for nz in (16, 32, 64):
        h = 1.0 / nz
        shape = (nz, 4, 4)
        zc = (np.arange(nz) + 0.5) * h
        phi = np.broadcast_to((zc - z0)[:, None, None], shape).copy()
        rhs = np.full(shape, f)
        res = oracle.solve(phi, rhs, h, rl, rg, 0.0, (P, P, ND), tol=1e-13)
        # exact: p(z) = -int_z^1 f s beta(s)^-1 ds, beta = 1/rho
        def P_exact(z):
            if z >= z0:
                return -f * rg * (1.0 - z * z) / 2.0
            return -f * rg * (1.0 - z0 * z0) / 2.0 - f * rl * (z0 * z0 - z * z) / 2.0
        ex = np.array([P_exact(z) for z in zc])
        errs.append(np.max(np.abs(res["p"][:, 0, 0] - ex)) / np.max(np.abs(ex)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.8, (errs, orders)


def test_outflow_solvers_agree_and_projection_is_divergence_free():
    """A bubble under an outflow top: Jacobi-PCG, Gauss-Seidel and a dense
    direct solve give one pressure; the velocity correction, outflow faces
    included, leaves a divergence equal to the residual (~1e-12 of div u*)."""
    shape, h = (8, 8, 8), 1.0 / 8
    bc = (P, P, ND)
    phi = synth.level_set(shape, h, [((0.5, 0.5, 0.5), 0.3)], bc=bc)
    u = synth.velocity(3, shape, h, bc=(P, P, N))
    rhs = oracle.divergence(*u, h)
    res = oracle.solve(phi, rhs, h, 1.0, 1e-3, 0.02, bc, tol=1e-13)
    xg, sweeps, rel = oracle.gs(res["faces"], res["b"], h, bc, tol=1e-11, maxsweeps=200000)
    assert sweeps >= 0
    assert np.linalg.norm(xg - res["p"]) / np.linalg.norm(res["p"]) < 1e-9
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = oracle.apply(res["faces"], e.reshape(shape), h, bc).ravel()
    xd = np.linalg.solve(A, res["b"].ravel()).reshape(shape)
    assert np.linalg.norm(xd - res["p"]) / np.linalg.norm(xd) < 1e-10
    fx, fy, fz = oracle.project(phi, res["kappa"], res["faces"], res["p"], *u, h, 0.02, bc)
    div = oracle.divergence_full(fx, fy, fz, h)
    assert np.linalg.norm(div) <= 1e-10 * np.linalg.norm(rhs)
    assert np.all(fz[0] == 0.0)          # wall bottom keeps u* = 0
    assert np.abs(fz[-1]).max() > 0.0    # the outflow top carries the flux out


# ------------------------------------------- phase change: the flux jump
def _layer(orient, n=24, s0=0.37):
    """A planar interface across one axis, the gas side open (outflow) and
    the liquid side closed (wall); mdot = 0.5 + 0.3 s (s the coordinate
    along that axis), so the interface value is 0.5 + 0.3 s0 exactly."""
    h = 1.0 / n
    if orient == "x":
        shape, bc, ax = (4, 4, n), (ND, P, P), 0
    else:
        shape, bc, ax = (n, 4, 4), ((P, P, ND) if orient == "z_up" else (P, P, DN)), 2
    x, y, z = centres(shape, h)
    s = x if ax == 0 else z
    phi = s0 - s if orient == "z_down" else s - s0
    mdot = 0.5 + 0.3 * s
    return shape, h, bc, ax, s, np.ascontiguousarray(phi), np.ascontiguousarray(mdot)


@pytest.mark.parametrize("orient", ["z_up", "z_down", "x"])
def test_flux_jump_planar_layer_is_exact(orient):
    """Evaporation from a flat liquid layer, u* = 0.  The liquid (closed by a
    wall) stays at rest with uniform pressure; the gas leaves through the
    outflow side with the velocity jump mdot_G [1/rho] and a linear pressure
    falling to 0 on the outflow face.  That piecewise-linear pressure is
    reproduced by the ghost-fluid flux-jump discretisation to rounding (both
    sides linear, jumps imposed at the interface point), and so are the
    velocities: 0 on every liquid face and on the interface face (stored
    liquid side), the jump on every gas face."""
    rho_l, rho_g, s0 = 1.0, 1e-3, 0.37
    shape, h, bc, ax, s, phi, mdot = _layer(orient, s0=s0)
    jinv = 1.0 / rho_g - 1.0 / rho_l
    mg = 0.5 + 0.3 * s0
    res = oracle.solve(phi, np.zeros(shape), h, rho_l, rho_g, 0.07, bc, tol=1e-14, mdot=mdot)
    # gas velocity along +s (z_up, x) or -s (z_down); p = 0 on the outflow face
    if orient == "z_down":
        exact = np.where(phi > 0, rho_g * mg * jinv * s, rho_g * mg * jinv * s0)
    else:
        exact = np.where(phi > 0, rho_g * mg * jinv * (1.0 - s), rho_g * mg * jinv * (1.0 - s0))
    assert np.abs(res["p"] - exact).max() < 1e-10 * np.abs(exact).max()
    zero = [np.zeros(shape)] * 3
    fx, fy, fz = oracle.project(phi, res["kappa"], res["faces"], res["p"], *zero, h, 0.07, bc,
                                mdot=mdot, rho_l=rho_l, rho_g=rho_g)
    un = fx if ax == 0 else fz
    # face f sits at s = f h; the gas faces (outflow face included) carry the jump
    fcoord = np.arange(un.shape[2 - ax]) * h
    shp = [1, 1, 1]
    shp[2 - ax] = -1
    fcoord = fcoord.reshape(shp)
    # a gas face has gas on both sides; the interface face stores the liquid side
    gasface = (fcoord + 0.5 * h < s0) if orient == "z_down" else (fcoord - 0.5 * h > s0)
    want = np.where(gasface, (-mg if orient == "z_down" else mg) * jinv, 0.0)
    want = np.broadcast_to(want, un.shape)
    assert np.abs(un - want).max() < 1e-9 * mg * jinv
    for other in ((fy, fz) if ax == 0 else (fx, fy)):
        assert np.abs(other).max() < 1e-9 * mg * jinv


def _crossing_faces(gas, bc):
    """Faces whose two cells lie in different fluids (periodic wrap faces
    included, boundary faces of other axes excluded)."""
    count = 0
    for ax in range(3):
        npax = 2 - ax
        d = np.diff(gas.astype(np.int8), axis=npax) != 0
        count += int(d.sum())
        if bc[ax] == P:
            first = np.take(gas, [0], axis=npax)
            last = np.take(gas, [-1], axis=npax)
            count += int((first != last).sum())
    return count


@pytest.mark.parametrize("bc", [(P, P, N), (P, P, ND), (D, D, D)])
def test_flux_jump_source_is_the_created_volume(bc):
    """Uniform mdot: every interface face adds B / h = -mdot [1/rho] / h to
    the right-hand side in total (split between its two rows), so the source
    sums to -mdot [1/rho] (interface faces) / h; each row's share is
    positive (B < 0 for evaporation) and the gas row carries almost all of
    it (its share is 1 / (1 + theta_l rho_l / (theta_g rho_g)))."""
    shape, h = (12, 10, 8), 1.0 / 12
    rho_l, rho_g, md = 1.0, 1e-3, 0.3
    phi = synth.level_set(shape, h, [((0.3, 0.4, 0.5), 0.2), ((0.45, 0.4, 0.2), 0.12)],
                          bc=(P, P, N) if bc[0] == P else (N, N, N))
    f = oracle.faces(phi, rho_l, rho_g, bc)
    Jf = oracle.flux_jump(phi, np.full(shape, md), f, h, rho_l, rho_g, bc)
    B = -md * (1.0 / rho_g - 1.0 / rho_l)
    ncross = _crossing_faces(phi > 0, bc)
    assert ncross > 20
    assert abs(Jf.sum() - B * ncross / h) < 1e-12 * abs(B) * ncross / h
    band = Jf != 0.0
    assert np.all(Jf[band] * B > 0)
    gas_part = Jf[(phi > 0) & band].sum() / Jf[band].sum()
    assert gas_part > 0.9


def test_flux_jump_projection_keeps_liquid_divergence_free():
    """An evaporating bubble under an outflow top with a smooth u*: after the
    solve and the correction (liquid-side velocity on interface faces) every
    liquid cell is divergence-free to the solve's tolerance, while the
    phase change's volume leaves through the outflow face."""
    shape, h = (16, 12, 12), 1.0 / 16
    bc = (P, P, ND)
    rho_l, rho_g = 1.0, 1e-3
    phi = synth.level_set(shape, h, [((0.4, 0.5, 0.45), 0.2)], bc=bc)
    x, y, z = centres(shape, h)
    mdot = np.ascontiguousarray(0.02 * (1.0 + x + 0.5 * y * z))
    u = synth.velocity(4, shape, h, bc=(P, P, N))
    rhs = oracle.divergence(*u, h)
    res = oracle.solve(phi, rhs, h, rho_l, rho_g, 0.02, bc, tol=1e-13, mdot=mdot)
    fx, fy, fz = oracle.project(phi, res["kappa"], res["faces"], res["p"], *u, h, 0.02, bc,
                                mdot=mdot, rho_l=rho_l, rho_g=rho_g)
    div = oracle.divergence_full(fx, fy, fz, h)
    liquid = phi <= 0
    scale = np.linalg.norm(res["b"])
    assert np.abs(div[liquid]).max() < 1e-9 * scale
    assert np.abs(div[~liquid]).max() > 1e-3 * scale  # gas cells hold the created volume
    # the outflow face carries the created volume plus nothing else (div u* = 0 in total)
    created = -oracle.flux_jump(phi, mdot, res["faces"], h, rho_l, rho_g, bc).sum() * h ** 3
    out = fz[-1].sum() * h * h
    assert created > 0 and abs(out - created) < 1e-8 * created
