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
