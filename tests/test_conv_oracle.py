"""Pins of the FP64 conv-net oracle (oracle/conv.py).

Forward convolution against scipy's n-D correlation (an independent
library routine), gradients against the adjoint identities and central
finite differences, pooling/upsampling against their definitions, and the
whole U-Net gradient against a directional finite difference.
"""
import numpy as np
import pytest

from oracle import conv

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3d_matches_scipy_correlate():
    g = rng(1)
    x = g.standard_normal((6, 5, 7, 3))
    w = g.standard_normal((4, 3, 3, 3, 3))
    b = g.standard_normal(4)
    y = conv.conv3d(x, w, b)
    for co in range(4):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            ref += scipy_ndimage.correlate(x[..., ci], w[co, :, :, :, ci], mode="constant", cval=0.0)
        assert np.allclose(y[..., co], ref, rtol=0, atol=1e-12)


def test_conv3d_identity_and_shift_kernels():
    x = rng(2).standard_normal((4, 4, 4, 2))
    w = np.zeros((2, 3, 3, 3, 2))
    w[:, 1, 1, 1, :] = np.eye(2)
    assert np.array_equal(conv.conv3d(x, w), x)
    w = np.zeros((1, 3, 3, 3, 1))
    w[0, 1, 1, 2, 0] = 1.0  # tap (0, 0, +1): y[z, y, x] = x[z, y, x + 1]
    y = conv.conv3d(x[..., :1], w)
    assert np.array_equal(y[:, :, :-1, 0], x[:, :, 1:, 0]) and np.all(y[:, :, -1, 0] == 0)


def test_dgrad_wgrad_adjoint_identities():
    g = rng(3)
    x = g.standard_normal((5, 6, 4, 3))
    w = g.standard_normal((2, 3, 3, 3, 3))
    gy = g.standard_normal((5, 6, 4, 2))
    lhs = (conv.conv3d(x, w) * gy).sum()
    assert lhs == pytest.approx((x * conv.conv3d_dgrad(gy, w)).sum(), rel=1e-12)
    assert lhs == pytest.approx((w * conv.conv3d_wgrad(x, gy)).sum(), rel=1e-12)
    assert np.allclose(conv.bias_grad(gy), gy.sum(axis=(0, 1, 2)))


def test_gradients_match_finite_differences():
    g = rng(4)
    x = g.standard_normal((4, 4, 4, 2))
    w = g.standard_normal((3, 3, 3, 3, 2))
    b = g.standard_normal(3)
    gy = g.standard_normal((4, 4, 4, 3))

    def loss(x_, w_, b_):
        return (conv.conv3d(x_, w_, b_) * gy).sum()

    eps = 1e-6
    for idx in [(0, 0, 0, 1), (1, 2, 3, 0), (3, 3, 3, 1)]:
        e = np.zeros_like(x)
        e[idx] = eps
        fd = (loss(x + e, w, b) - loss(x - e, w, b)) / (2 * eps)
        assert fd == pytest.approx(conv.conv3d_dgrad(gy, w)[idx], rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 0, 0, 0), (2, 1, 2, 0, 1), (1, 2, 2, 2, 0)]:
        e = np.zeros_like(w)
        e[idx] = eps
        fd = (loss(x, w + e, b) - loss(x, w - e, b)) / (2 * eps)
        assert fd == pytest.approx(conv.conv3d_wgrad(x, gy)[idx], rel=1e-6, abs=1e-8)


def test_pool_and_upsample_and_their_adjoints():
    g = rng(5)
    x = g.standard_normal((4, 6, 8, 3))
    p = conv.avgpool2(x)
    assert p[1, 2, 3, 1] == pytest.approx(x[2:4, 4:6, 6:8, 1].mean())
    u = conv.upsample2(p)
    assert np.array_equal(u[3, 5, 7], p[1, 2, 3])
    gp = g.standard_normal(p.shape)
    assert (p * gp).sum() == pytest.approx((x * conv.avgpool2_adjoint(gp)).sum(), rel=1e-12)
    gu = g.standard_normal(u.shape)
    assert (u * gu).sum() == pytest.approx((p * conv.upsample2_adjoint(gu)).sum(), rel=1e-12)


def test_unet_gradient_directional_finite_difference():
    g = rng(6)
    params = conv.init_params(g)
    for k in params:
        if k.endswith(".b"):
            params[k] = 0.1 * g.standard_normal(params[k].shape)
    x = g.standard_normal((8, 8, 8, conv.IN_CH))
    target = g.standard_normal((8, 8, 8))

    def loss(p):
        out, _ = conv.unet_forward(p, x)
        return conv.gauge_mse(out, target)[0]

    out, cache = conv.unet_forward(params, x)
    L, gout = conv.gauge_mse(out, target)
    grads, gin = conv.unet_backward(params, cache, gout)
    d = {k: g.standard_normal(v.shape) for k, v in params.items()}
    eps = 1e-6
    plus = {k: params[k] + eps * d[k] for k in params}
    minus = {k: params[k] - eps * d[k] for k in params}
    fd = (loss(plus) - loss(minus)) / (2 * eps)
    an = sum((grads[k] * d[k]).sum() for k in params)
    assert fd == pytest.approx(an, rel=1e-5)
    # input gradient too
    dx = g.standard_normal(x.shape)
    fdx = (conv.gauge_mse(conv.unet_forward(params, x + eps * dx)[0], target)[0] -
           conv.gauge_mse(conv.unet_forward(params, x - eps * dx)[0], target)[0]) / (2 * eps)
    assert fdx == pytest.approx((gin * dx).sum(), rel=1e-5)


def test_gauge_mse_and_adam():
    t = rng(7).standard_normal((4, 4, 4))
    L, g = conv.gauge_mse(t + 3.0, t)
    assert L == pytest.approx(0.0, abs=1e-24) and np.allclose(g, 0.0)
    p, m, v = conv.adam(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, lr=0.1)
    # first bias-corrected step moves by lr * sign(grad)
    assert p[0] == pytest.approx(0.9, rel=1e-6)


# ------------------------------------------- learned guess on a coarser grid
def test_restrict8_matches_uniform_filter():
    """Mean of the 8 children = scipy's 2-wide box mean sampled at the odd
    cells (an independent library routine)."""
    a = rng(11).standard_normal((6, 8, 10))
    ref = scipy_ndimage.uniform_filter(a, size=2, mode="constant")[1::2, 1::2, 1::2]
    assert np.allclose(conv.restrict8(a), ref, rtol=0, atol=1e-14)


def test_features_closed_form():
    """A linear level set restricts exactly to its value at the coarse
    centres; f0 is that value over 4 coarse cells, clipped to [-1, 1]; f1 has
    rms 1, keeps the sign of b and ignores its scale."""
    n, h = 16, 1.0 / 16
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = 0.3 * x - 0.2 * y + 0.9 * z - 0.41
    b = rng(12).standard_normal((n, n, n))
    f0, f1 = conv.half_res_features(phi, b, h)
    H = 2.0 * h
    cc = (np.arange(n // 2) + 0.5) * H
    Z, Y, X = np.meshgrid(cc, cc, cc, indexing="ij")
    phic = 0.3 * X - 0.2 * Y + 0.9 * Z - 0.41
    assert np.allclose(f0, np.clip(phic / (4 * H), -1, 1), rtol=0, atol=1e-14)
    assert 0 < np.mean(np.abs(f0) == 1.0) < 1  # both clipped and unclipped cells
    assert np.sqrt(np.mean(f1 * f1)) == pytest.approx(1.0, rel=1e-14)
    g0, g1 = conv.half_res_features(phi, -7.5 * b, h)
    assert np.allclose(g1, -f1, rtol=0, atol=1e-14) and np.array_equal(g0, f0)
    assert np.all(conv.features(phi, np.zeros_like(b), h)[1] == 0)


@pytest.mark.parametrize("per", [(True, True, False), (False, False, False), (True, True, True),
                                 (False, True, False)])
def test_prolongation_matches_scipy_zoom(per):
    """Cell-centred linear interpolation onto the grid twice as fine is
    scipy's order-1 zoom with grid-aligned cells, wrapping periodic axes and
    repeating the end cell of wall axes; axes taken one at a time."""
    q = rng(13).standard_normal((4, 6, 8))
    ref = q
    for ax_np, p in ((2, per[0]), (1, per[1]), (0, per[2])):
        zf = [1, 1, 1]
        zf[ax_np] = 2
        ref = scipy_ndimage.zoom(ref, zf, order=1, grid_mode=True,
                                 mode="grid-wrap" if p else "nearest")
    out = conv.prolong_trilinear2(q, per)
    assert out.shape == (8, 12, 16)
    assert np.allclose(out, ref, rtol=0, atol=1e-13)


def test_prolongation_exact_on_linear_fields_and_constants():
    """Away from wall ends the interpolation reproduces any linear field at
    the fine centres; every row's weights sum to 1 (constants are kept)."""
    n, H = 8, 1.0 / 8
    c = (np.arange(n) + 0.5) * H
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    q = 1.5 * X - 0.25 * Y + 2.0 * Z + 0.125
    out = conv.prolong_trilinear2(q, (False, False, False))
    f = (np.arange(2 * n) + 0.5) * (H / 2)
    z, y, x = np.meshgrid(f, f, f, indexing="ij")
    exact = 1.5 * x - 0.25 * y + 2.0 * z + 0.125
    inner = (slice(1, -1),) * 3
    assert np.allclose(out[inner], exact[inner], rtol=0, atol=1e-13)
    assert np.allclose(conv.prolong_trilinear2(np.full((4, 4, 4), 2.5), (True, False, True)), 2.5,
                       rtol=0, atol=1e-15)


@pytest.mark.parametrize("per", [(True, True, False), (False, False, False)])
def test_prolongation_adjoint_identity(per):
    g = rng(14)
    q = g.standard_normal((4, 6, 8))
    v = g.standard_normal((8, 12, 16))
    lhs = np.sum(conv.prolong_trilinear2(q, per) * v)
    assert lhs == pytest.approx(np.sum(q * conv.prolong_trilinear2_adjoint(v, per)), rel=1e-12)


def _energy_case(seed, n=8, bc=(0, 0, 1)):
    import synth
    h = 1.0 / n
    phi = synth.level_set((n, n, n), h, [((0.5, 0.45, 0.4), 0.27)], pool_z0=0.8, bc=bc)
    f0 = np.clip(phi / (4 * h), -1, 1)
    g = rng(seed)
    return g.standard_normal((n, n, n)), g.standard_normal((n, n, n)), f0, bc


def test_energy_loss_invariants():
    """0 <= L <= 1 (A is positive semidefinite); L = 0 when q is a multiple
    of t; L does not change when q is scaled (by either sign), so the
    gradient is orthogonal to q; L is unchanged when a constant is added
    (constants are the operator's null space with periodic and wall axes)."""
    q, t, f0, bc = _energy_case(15)
    L, gq = conv.energy_loss(q, t, f0, 1.0, 1e-3, bc)
    assert 0.0 < L < 1.0
    for lam in (3.0, -0.5):
        L2, g2 = conv.energy_loss(lam * q, t, f0, 1.0, 1e-3, bc)
        assert L2 == pytest.approx(L, rel=1e-12)
        assert np.allclose(lam * g2, gq, rtol=1e-10, atol=1e-14 * np.abs(gq).max())
    assert abs(np.sum(gq * q)) <= 1e-12 * np.linalg.norm(gq) * np.linalg.norm(q)
    assert conv.energy_loss(q + 4.0, t, f0, 1.0, 1e-3, bc)[0] == pytest.approx(L, rel=1e-10)
    L0, g0 = conv.energy_loss(-2.0 * t, t, f0, 1.0, 1e-3, bc)
    assert abs(L0) < 1e-14 and np.abs(g0).max() < 1e-12 * np.abs(gq).max() * 1e3


def test_energy_loss_is_best_multiple_error():
    """L is the squared A-norm error of the best multiple of q relative to
    the A-norm of t: the quadratic N(alpha) = |alpha q - t|_A^2, fitted
    through three values, has minimum L * |t|_A^2.  |x|_A^2 here comes from a
    dense matrix assembled column by column from the oracle's operator."""
    import oracle
    q, t, f0, bc = _energy_case(16, n=6)
    n = q.size
    f = oracle.faces(f0, 1.0, 1e-3, bc)
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = -oracle.apply(f, e.reshape(q.shape), 1.0, bc).ravel()

    def N(alpha):
        e = (alpha * q - t).ravel()
        return e @ A @ e

    fit = np.polyfit([-1.0, 0.0, 1.0], [N(-1.0), N(0.0), N(1.0)], 2)
    nmin = fit[2] - fit[1] ** 2 / (4.0 * fit[0])
    L, _ = conv.energy_loss(q, t, f0, 1.0, 1e-3, bc)
    assert L == pytest.approx(nmin / N(0.0), rel=1e-10)


def test_energy_gradient_finite_difference():
    """Central differences of L along random directions and single entries;
    q is t plus noise so that L sits well inside (0, 1) and its derivatives
    stand clear of the rounding of L itself."""
    q, t, f0, bc = _energy_case(17)
    q = t + 0.5 * q
    L, gq = conv.energy_loss(q, t, f0, 1.0, 1e-3, bc)
    assert 0.05 < L < 0.95
    eps = 1e-5
    g = rng(18)
    for _ in range(3):
        d = g.standard_normal(q.shape)
        fd = (conv.energy_loss(q + eps * d, t, f0, 1.0, 1e-3, bc)[0] -
              conv.energy_loss(q - eps * d, t, f0, 1.0, 1e-3, bc)[0]) / (2 * eps)
        assert fd == pytest.approx(np.sum(gq * d), rel=1e-6)
    for idx in [(0, 0, 0), (3, 4, 5), (7, 7, 7)]:
        e = np.zeros_like(q)
        e[idx] = eps
        fd = (conv.energy_loss(q + e, t, f0, 1.0, 1e-3, bc)[0] -
              conv.energy_loss(q - e, t, f0, 1.0, 1e-3, bc)[0]) / (2 * eps)
        assert fd == pytest.approx(gq[idx], rel=1e-5, abs=1e-9)


def test_adam_two_steps_closed_form():
    """Two bias-corrected Adam steps written out for scalars: after the
    first, m = 0.1 g1, v = 0.001 g1^2; the second combines both gradients."""
    p0, g1, g2, lr = 0.7, 0.3, -0.05, 0.01
    p1, m1, v1 = conv.adam(np.array([p0]), np.array([g1]), np.zeros(1), np.zeros(1), 1, lr=lr)
    p2, _, _ = conv.adam(p1, np.array([g2]), m1, v1, 2, lr=lr)
    mhat = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vhat = (0.999 * 0.001 * g1 * g1 + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    assert p1[0] == pytest.approx(p0 - lr * g1 / (abs(g1) + 1e-8), rel=1e-14)
    assert p2[0] == pytest.approx(p1[0] - lr * mhat / (np.sqrt(vhat) + 1e-8), rel=1e-14)


# ------------------------------------------- the deflated energy loss
def _bfs_components(gas, bc):
    """Brute-force flood fill with face neighbours (periodic axes wrapped):
    the partition of the gas cells, as a set of frozensets of flat indices."""
    nz, ny, nx = gas.shape
    seen = np.zeros_like(gas, dtype=bool)
    comps = set()
    for start in zip(*np.nonzero(gas)):
        if seen[start]:
            continue
        stack, members = [start], []
        seen[start] = True
        while stack:
            k, j, i = stack.pop()
            members.append((k * ny + j) * nx + i)
            for ax, n in ((2, nx), (1, ny), (0, nz)):
                for s in (-1, 1):
                    c = [k, j, i]
                    c[ax] += s
                    axis = 2 - ax
                    if not 0 <= c[ax] < n:
                        if bc[axis] != 0:
                            continue
                        c[ax] %= n
                    c = tuple(c)
                    if gas[c] and not seen[c]:
                        seen[c] = True
                        stack.append(c)
        comps.add(frozenset(members))
    return comps


def _defl_case(seed=3, n=8):
    import synth
    h = 1.0 / n
    bc = (0, 0, 1)
    # a bubble across the periodic x boundary, one inside, one touching the z wall
    phi = synth.level_set((n, n, n), h, [((0.02, 0.5, 0.5), 0.2), ((0.5, 0.4, 0.45), 0.18),
                                         ((0.6, 0.75, 0.12), 0.15)], bc=bc)
    g = rng(seed)
    return phi, h, bc, g.standard_normal(phi.shape), g.standard_normal(phi.shape)


def test_gas_components_match_flood_fill():
    phi, h, bc, _, _ = _defl_case()
    lab, m = conv.gas_components(phi, bc)
    ours = {frozenset(np.flatnonzero(lab.ravel() == j)) for j in range(m)}
    assert m >= 2 and ours == _bfs_components(phi > 0, bc)
    # numbered by each component's lowest cell
    firsts = [np.flatnonzero(lab.ravel() == j)[0] for j in range(m)]
    assert firsts == sorted(firsts)


def test_deflated_energy_invariances_and_plain_limit():
    """D annihilates the component indicators (and constants), so adding any
    Z c + const to q changes nothing; scaling q changes nothing; with no gas
    the loss is the plain energy loss."""
    phi, h, bc, q, t = _defl_case(5)
    L, _ = conv.deflated_energy_loss(q, t, phi, h, 1.0, 1e-3, bc)
    lab, m = conv.gas_components(phi, bc)
    shift = sum(float(c) * (lab == j) for j, c in enumerate(rng(6).standard_normal(m))) + 0.7
    assert conv.deflated_energy_loss(q + shift, t, phi, h, 1.0, 1e-3, bc)[0] == pytest.approx(L, rel=1e-9)
    assert conv.deflated_energy_loss(-3.5 * q, t, phi, h, 1.0, 1e-3, bc)[0] == pytest.approx(L, rel=1e-12)
    liquid = -np.ones_like(phi)
    Ld, gd = conv.deflated_energy_loss(q, t, liquid, h, 1.0, 1e-3, bc)
    Lp, gp = conv.energy_loss(q, t, liquid, 1.0, 1e-3, bc)
    # (the gradient does not depend on the scale of the operator)
    assert Ld == pytest.approx(Lp, rel=1e-12) and np.allclose(gd, gp, rtol=1e-9, atol=1e-12)


def test_deflated_energy_is_the_best_correction_by_brute_force():
    """L = min over (alpha, c) of ||alpha q - t - Z c||_A^2 / min over c of
    ||t - Z c||_A^2, both minima found by a general-purpose optimiser (no E)."""
    from scipy.optimize import minimize
    from oracle import apply, faces
    phi, h, bc, q, t = _defl_case(7)
    L, _ = conv.deflated_energy_loss(q, t, phi, h, 1.0, 1e-3, bc)
    f = faces(phi, 1.0, 1e-3, bc)
    lab, m = conv.gas_components(phi, bc)
    Z = [(lab == j).astype(float) for j in range(m)]

    def en(v):
        return float(np.sum(v * -apply(f, v, h, bc)))

    def num(x):
        return en(x[0] * q - t - sum(c * z for c, z in zip(x[1:], Z)))

    def den(x):
        return en(t - sum(c * z for c, z in zip(x, Z)))

    top = minimize(num, np.zeros(m + 1), method="BFGS", options={"gtol": 1e-10}).fun
    bot = minimize(den, np.zeros(m), method="BFGS", options={"gtol": 1e-10}).fun
    assert top / bot == pytest.approx(L, rel=1e-6)


def test_deflated_energy_gradient_finite_difference():
    phi, h, bc, q, t = _defl_case(9)
    q = t + 0.5 * q
    L, gq = conv.deflated_energy_loss(q, t, phi, h, 1.0, 1e-3, bc)
    assert 0.05 < L < 0.95
    eps = 1e-5
    g = rng(10)
    for _ in range(3):
        d = g.standard_normal(q.shape)
        fd = (conv.deflated_energy_loss(q + eps * d, t, phi, h, 1.0, 1e-3, bc)[0] -
              conv.deflated_energy_loss(q - eps * d, t, phi, h, 1.0, 1e-3, bc)[0]) / (2 * eps)
        assert fd == pytest.approx(np.sum(gq * d), rel=1e-6)
