"""FP64 numpy oracle of the learned warm-start network.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
baseline; the product library never imports it, and it shares no code with
the CUDA kernels.

Layouts: activations (nz, ny, nx, C) (channels last, "NDHWC" without N);
3x3x3 weights (Cout, 3, 3, 3, Cin) indexed [co, dz, dy, dx, ci] with tap
offset (dz-1, dy-1, dx-1); zero padding outside the volume.

The network is a 4-level U-Net (channels 16/32/64/64): per level two 3x3x3
convolutions with ReLU, 2x2x2 average pooling down, nearest-neighbour
upsampling plus concatenation with the same-level encoder output on the
way up, and a 1x1x1 head to one output channel.  Every function below
follows the definition of its operation directly: a sum over the 27 taps of
channel contractions, with no blocking or reordering.
"""
from __future__ import annotations

import numpy as np

CH = (16, 32, 64, 64)
IN_CH = 2


def _shifted(xp, dz, dy, dx, shape):
    nz, ny, nx = shape
    return xp[dz:dz + nz, dy:dy + ny, dx:dx + nx, :]


def conv3d(x, w, b=None):
    """y[v, co] = b[co] + sum_{taps t, ci} x[v + off_t, ci] * w[co, t, ci]."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    nz, ny, nx, cin = x.shape
    cout = w.shape[0]
    assert w.shape == (cout, 3, 3, 3, cin)
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((nz, ny, nx, cout))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                y += _shifted(xp, dz, dy, dx, (nz, ny, nx)) @ w[:, dz, dy, dx, :].T
    if b is not None:
        y += np.asarray(b, dtype=np.float64)
    return y


def conv3d_dgrad(g, w):
    """Gradient w.r.t. the input of conv3d for output gradient g:
    dx[v, ci] = sum_{t, co} g[v - off_t, co] * w[co, t, ci]."""
    g = np.asarray(g, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    nz, ny, nx, cout = g.shape
    cin = w.shape[4]
    gp = np.pad(g, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dx_ = np.zeros((nz, ny, nx, cin))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                # output v' = v - off_t  <=>  padded index v + (2 - d)
                dx_ += _shifted(gp, 2 - dz, 2 - dy, 2 - dx, (nz, ny, nx)) @ w[:, dz, dy, dx, :]
    return dx_


def conv3d_wgrad(x, g):
    """Gradient w.r.t. the weights: dw[co, t, ci] = sum_v x[v + off_t, ci] g[v, co]."""
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    nz, ny, nx, cin = x.shape
    cout = g.shape[3]
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dw = np.zeros((cout, 3, 3, 3, cin))
    g2 = g.reshape(-1, cout)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dw[:, dz, dy, dx, :] = g2.T @ _shifted(xp, dz, dy, dx, (nz, ny, nx)).reshape(-1, cin)
    return dw


def bias_grad(g):
    return np.asarray(g, dtype=np.float64).reshape(-1, g.shape[-1]).sum(axis=0)


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    """2x2x2 mean of each block of children."""
    nz, ny, nx, c = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def avgpool2_adjoint(g):
    """Adjoint of avgpool2: every child receives g/8."""
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def upsample2(x):
    """Nearest-neighbour x2: each fine cell takes its parent's value."""
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def upsample2_adjoint(g):
    """Adjoint of upsample2: a parent receives the sum over its 8 children."""
    nz, ny, nx, c = g.shape
    return g.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(1, 3, 5))


# ------------------------------------------------------------------ U-Net
def layer_shapes():
    """(name, cout, cin) of every 3x3x3 conv in forward order, plus the head."""
    c0, c1, c2, c3 = CH
    return [("e0a", c0, IN_CH), ("e0b", c0, c0),
            ("e1a", c1, c0), ("e1b", c1, c1),
            ("e2a", c2, c1), ("e2b", c2, c2),
            ("e3a", c3, c2), ("e3b", c3, c3),
            ("d2a", c2, c3 + c2), ("d2b", c2, c2),
            ("d1a", c1, c2 + c1), ("d1b", c1, c1),
            ("d0a", c0, c1 + c0), ("d0b", c0, c0)]


def init_params(rng):
    """He-normal conv weights, zero biases, small head."""
    p = {}
    for name, co, ci in layer_shapes():
        p[name + ".w"] = rng.standard_normal((co, 3, 3, 3, ci)) * np.sqrt(2.0 / (27 * ci))
        p[name + ".b"] = np.zeros(co)
    p["head.w"] = rng.standard_normal((1, CH[0])) * np.sqrt(1.0 / CH[0])
    p["head.b"] = np.zeros(1)
    return p


def unet_forward(p, x, rnd=None):
    """Returns (output (nz, ny, nx), cache of every activation).

    rnd (optional) is applied to every stored activation (convolution
    outputs after ReLU and pooled tensors): a test can pass a rounding to
    the kernels' storage format to compare on identically rounded operands.
    """
    rnd = (lambda a: a) if rnd is None else rnd
    cache = {"in": x}

    def cr(name, inp):
        z = conv3d(inp, p[name + ".w"], p[name + ".b"])
        y = rnd(relu(z))
        cache[name + ".in"] = inp
        cache[name + ".out"] = y
        return y

    e0 = cr("e0b", cr("e0a", x))
    e1 = cr("e1b", cr("e1a", rnd(avgpool2(e0))))
    e2 = cr("e2b", cr("e2a", rnd(avgpool2(e1))))
    e3 = cr("e3b", cr("e3a", rnd(avgpool2(e2))))
    d2 = cr("d2b", cr("d2a", np.concatenate([upsample2(e3), e2], axis=-1)))
    d1 = cr("d1b", cr("d1a", np.concatenate([upsample2(d2), e1], axis=-1)))
    d0 = cr("d0b", cr("d0a", np.concatenate([upsample2(d1), e0], axis=-1)))
    out = d0 @ p["head.w"].T + p["head.b"]
    cache["d0"] = d0
    return out[..., 0], cache


def unet_backward(p, cache, gout, rnd=None):
    """Gradients of sum(out * gout) w.r.t. every parameter (and the input).

    rnd (optional) is applied where activation gradients are stored (the
    head's output gradient, every input gradient, the upsampling adjoint and
    the merged skip + pooling gradient), to compare with kernels that keep
    those tensors in a narrower format.
    """
    rnd = (lambda a: a) if rnd is None else rnd
    g = {}
    d0 = cache["d0"]
    gout = np.asarray(gout, dtype=np.float64)[..., None]
    g["head.w"] = (gout.reshape(-1, 1).T @ d0.reshape(-1, d0.shape[-1]))
    g["head.b"] = gout.reshape(-1, 1).sum(axis=0)
    gd0 = rnd(gout @ p["head.w"])

    def back(name, gy):
        y = cache[name + ".out"]
        gz = gy * (y > 0)
        g[name + ".w"] = conv3d_wgrad(cache[name + ".in"], gz)
        g[name + ".b"] = bias_grad(gz)
        return rnd(conv3d_dgrad(gz, p[name + ".w"]))

    c0, c1, c2, c3 = CH
    gcat0 = back("d0a", back("d0b", gd0))
    gd1 = rnd(upsample2_adjoint(gcat0[..., :c1]))
    ge0 = gcat0[..., c1:]
    gcat1 = back("d1a", back("d1b", gd1))
    gd2 = rnd(upsample2_adjoint(gcat1[..., :c2]))
    ge1 = gcat1[..., c2:]
    gcat2 = back("d2a", back("d2b", gd2))
    ge3 = rnd(upsample2_adjoint(gcat2[..., :c3]))
    ge2 = gcat2[..., c3:]
    gp2 = back("e3a", back("e3b", ge3))
    ge2 = rnd(ge2 + avgpool2_adjoint(gp2))
    gp1 = back("e2a", back("e2b", ge2))
    ge1 = rnd(ge1 + avgpool2_adjoint(gp1))
    gp0 = back("e1a", back("e1b", ge1))
    ge0 = rnd(ge0 + avgpool2_adjoint(gp0))
    gin = back("e0a", back("e0b", ge0))
    return g, gin


def gauge_mse(pred, target):
    """Mean squared error after removing each field's mean (the pressure is
    defined up to a constant); returns (loss, d loss / d pred)."""
    e = (pred - pred.mean()) - (target - target.mean())
    n = e.size
    return float((e * e).sum() / n), 2.0 * e / n


def adam(param, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), returns (param, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------- learned guess on a coarser grid
def restrict8(a):
    """Grid half as fine in every axis: each coarse cell takes the mean of its
    8 children (2 x 2 x 2 blocks of the fine grid), arrays (nz, ny, nx)."""
    a = np.asarray(a, dtype=np.float64)
    nz, ny, nx = a.shape
    return a.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))


def features(phi, b, h):
    """The two network input channels on a grid of cell size h:
    f0 = clip(phi / (4h), -1, 1) (the level set in units of 4 cells, cut off
    away from the interface) and f1 = b / rms(b) (rms 1; b = 0 gives 0).
    Returns (f0, f1), each (nz, ny, nx) float64."""
    phi = np.asarray(phi, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    f0 = np.clip(phi / (4.0 * h), -1.0, 1.0)
    rms = np.sqrt(np.mean(b * b))
    f1 = b / rms if rms > 0.0 else b.copy()
    return f0, f1


def half_res_features(phi, b, h):
    """Input of a network whose grid is half as fine as the solver's (cell
    size 2h): the features of the child means of phi and of b."""
    return features(restrict8(phi), restrict8(b), 2.0 * h)


def _interp_matrix(n, periodic):
    """(2n, n) matrix of linear interpolation from n cell centres to the 2n
    cell centres of the grid twice as fine along one axis.  Fine centre f sits
    at coarse coordinate x = (f + 1/2)/2 - 1/2 (coarse centres at integers);
    it takes (1 - w) of coarse cell floor(x) and w of floor(x) + 1, w = x -
    floor(x).  Out-of-range coarse cells wrap on a periodic axis and are
    replaced by the nearest end cell on a wall axis."""
    P = np.zeros((2 * n, n))
    for f in range(2 * n):
        x = (f + 0.5) / 2.0 - 0.5
        lo = int(np.floor(x))
        w = x - lo
        for idx, wt in ((lo, 1.0 - w), (lo + 1, w)):
            idx = idx % n if periodic else min(max(idx, 0), n - 1)
            P[f, idx] += wt
    return P


def prolong_trilinear2(q, periodic):
    """Cell-centred trilinear interpolation of q (nz, ny, nx) onto the grid
    twice as fine: the 1-D interpolation of _interp_matrix applied along
    x, y and z in turn.  periodic = (x, y, z) booleans."""
    out = np.asarray(q, dtype=np.float64)
    for ax_np, per in ((2, periodic[0]), (1, periodic[1]), (0, periodic[2])):
        P = _interp_matrix(out.shape[ax_np], per)
        out = np.moveaxis(np.tensordot(P, out, axes=([1], [ax_np])), 0, ax_np)
    return out


def prolong_trilinear2_adjoint(g, periodic):
    """Adjoint of prolong_trilinear2, written as a scatter: every fine value
    g[f] is distributed to the coarse cells it was interpolated from, with the
    same weights (one axis at a time)."""
    out = np.asarray(g, dtype=np.float64)
    for ax_np, per in ((2, periodic[0]), (1, periodic[1]), (0, periodic[2])):
        m = np.moveaxis(out, ax_np, 0)
        n = m.shape[0] // 2
        acc = np.zeros((n,) + m.shape[1:])
        for f in range(2 * n):
            x = (f + 0.5) / 2.0 - 0.5
            lo = int(np.floor(x))
            w = x - lo
            for idx, wt in ((lo, 1.0 - w), (lo + 1, w)):
                idx = idx % n if per else min(max(idx, 0), n - 1)
                acc[idx] += wt * m[f]
        out = np.moveaxis(acc, 0, ax_np)
    return out


# ------------------------------------------------------- energy-norm loss
def energy_loss(q, t, f0, rho_l, rho_g, bc):
    """Energy-norm training loss of a predicted pressure shape q for the
    target t, and its gradient with respect to q.

    A is the positive semidefinite ghost-fluid operator, minus the C oracle's
    operator, with the face coefficients that the oracle builds from the
    level set f0 (the network's input channel phi / 4h: the interface
    fraction theta = |f0_a| / (|f0_a| + |f0_b|) does not depend on the scale
    of phi, and the scale of A cancels in the loss).  With a = q.At,
    c = q.Aq, d = t.At:

        L = 1 - a^2 / (c d),

    the squared A-norm error of the best multiple alpha q (alpha = a / c),
    relative to the A-norm of t.  A is symmetric, so

        dL/dq = -2 a At / (c d) + 2 a^2 Aq / (c^2 d).

    Returns (L, dL/dq)."""
    from . import apply, faces
    q = np.asarray(q, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    f = faces(np.asarray(f0, dtype=np.float64), rho_l, rho_g, bc)
    Aq = -apply(f, q, 1.0, bc)
    At = -apply(f, t, 1.0, bc)
    a = float(np.sum(q * At))
    c = float(np.sum(q * Aq))
    d = float(np.sum(t * At))
    L = 1.0 - a * a / (c * d)
    grad = -2.0 * a * At / (c * d) + 2.0 * a * a * Aq / (c * c * d)
    return L, grad


def gas_components(phi, bc):
    """Connected gas regions (phi > 0) with face neighbours, periodic axes
    wrapped: (labels, m), labels -1 in liquid and 0..m-1 in gas, numbered in
    the order of each component's lowest cell index (C order).  The labelling
    is scipy.ndimage.label (6-connectivity); components that touch across a
    periodic boundary are merged with a small union-find over label pairs."""
    from scipy import ndimage
    gas = np.asarray(phi) > 0.0
    lab, m = ndimage.label(gas)
    parent = list(range(m + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for axis in range(3):
        if bc[axis] != 0:  # not periodic
            continue
        ax = 2 - axis
        lo, hi = np.take(lab, 0, axis=ax), np.take(lab, -1, axis=ax)
        for a, b in zip(lo[(lo > 0) & (hi > 0)], hi[(lo > 0) & (hi > 0)]):
            ra, rb = find(int(a)), find(int(b))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(int(v)) for v in range(m + 1)])
    flat = np.where(lab.ravel() > 0, roots[lab.ravel()], 0)
    order, first = [], {}
    for c, r in enumerate(flat):
        if r and r not in first:
            first[r] = len(order)
            order.append(r)
    out = np.full(flat.shape, -1, dtype=np.int64)
    for r, k in first.items():
        out[flat == r] = k
    return out.reshape(lab.shape), len(order)


def deflated_energy_loss(q, t, phi, h, rho_l, rho_g, bc):
    """The training loss of a guess for the deflated solver: deflated CG
    corrects any start exactly along the gas components' indicator vectors Z,
    so what it inherits is the error's energy in D = A - A Z E^-1 Z^T A,
    E = Z^T A Z (A the positive semidefinite ghost-fluid operator, minus the
    C oracle's).  With a = q.Dt, c = q.Dq, d = t.Dt:

        L = 1 - a^2 / (c d),   dL/dq = -2 a Dt / (c d) + 2 a^2 Dq / (c^2 d),

    the relative D-energy error of the best multiple of q.  The component
    projection is formed with a dense solve of the small E.  Returns (L, dL/dq)."""
    from . import apply, faces
    q = np.asarray(q, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    f = faces(np.asarray(phi, dtype=np.float64), rho_l, rho_g, bc)
    A = lambda v: -apply(f, v, h, bc)  # noqa: E731
    lab, m = gas_components(phi, bc)
    Z = np.stack([(lab == j).astype(np.float64) for j in range(m)]) if m else np.zeros((0,) + q.shape)
    AZ = np.stack([A(z) for z in Z]) if m else Z
    E = np.einsum("ixyz,jxyz->ij", Z, AZ) if m else np.zeros((0, 0))

    def D(v):
        Av = A(v)
        if not m:
            return Av
        c = np.linalg.solve(E, np.einsum("ixyz,xyz->i", AZ, v))
        return Av - np.einsum("i,ixyz->xyz", c, AZ)

    Dq, Dt = D(q), D(t)
    a, c, d = float(np.sum(q * Dt)), float(np.sum(q * Dq)), float(np.sum(t * Dt))
    L = 1.0 - a * a / (c * d)
    grad = -2.0 * a * Dt / (c * d) + 2.0 * a * a * Dq / (c * c * d)
    return L, grad
