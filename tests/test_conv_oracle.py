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
