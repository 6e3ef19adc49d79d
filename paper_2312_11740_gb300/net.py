"""Argument marshalling for the learned-warm-start C-ABI (include/mp_net.h).

Every operation runs in the CUDA library (tcgen05 BF16 convolutions and
their helpers); this module only converts torch tensors to pointers.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _lib
from .poisson import MPError, _check, _ptr, _stream_ptr

# network trained at 128^3 on 1-16-bubble problems with the energy loss
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                               "unet128_energy.npz")


def _lib_():
    return _lib.load()


def mp_conv3d_fwd(xa, w, cout, xb=None, bias=None, up_a=False, relu=False, out32=False):
    """xa: (nz, ny, nx, ca) bf16 (half-res grid when up_a); xb: (nz, ny, nx, cb) bf16;
    w: (cout, 27, ca+cb) bf16; bias: (cout,) f32.  Returns (nz, ny, nx, cout)."""
    if up_a:
        nz, ny, nx = (2 * xa.shape[0], 2 * xa.shape[1], 2 * xa.shape[2])
    else:
        nz, ny, nx = xa.shape[:3]
    ca = xa.shape[3]
    cb = 0 if xb is None else xb.shape[3]
    dev = xa.device
    y = torch.empty((nz, ny, nx, cout), dtype=torch.float32 if out32 else torch.bfloat16,
                    device=dev)
    st = _lib_().mp_conv3d_fwd(
        nx, ny, nz, _ptr(xa, torch.bfloat16), ca, int(up_a),
        None if xb is None else _ptr(xb, torch.bfloat16), cb, _ptr(w, torch.bfloat16),
        None if bias is None else _ptr(bias, torch.float32), cout, int(relu),
        None if out32 else _ptr(y, torch.bfloat16), _ptr(y, torch.float32) if out32 else None,
        None)
    _check(st, "mp_conv3d_fwd")
    return y


def mp_conv3d_wgrad(xa, g, xb=None, up_a=False):
    """Weight gradient (cout, 27, ca+cb) f32 of mp_conv3d_fwd for output gradient g."""
    nz, ny, nx, cout = g.shape
    ca = xa.shape[3]
    cb = 0 if xb is None else xb.shape[3]
    dw = torch.empty((cout, 27, ca + cb), dtype=torch.float32, device=g.device)
    st = _lib_().mp_conv3d_wgrad(
        nx, ny, nz, _ptr(xa, torch.bfloat16), ca, int(up_a),
        None if xb is None else _ptr(xb, torch.bfloat16), cb, _ptr(g, torch.bfloat16), cout,
        _ptr(dw, torch.float32), None)
    _check(st, "mp_conv3d_wgrad")
    return dw


class Net:
    """U-Net handle.  Parameters: one FP32 vector (see include/mp_net.h)."""

    def __init__(self, nx, ny, nz, stream=None):
        h = ctypes.c_void_p()
        _check(_lib_().mp_net_create(ctypes.byref(h), nx, ny, nz, _stream_ptr(stream)),
               "mp_net_create")
        self.handle = h
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz

    def param_count(self):
        return int(_lib_().mp_net_param_count(self.handle))

    def set_params(self, p):
        _check(_lib_().mp_net_set_params(self.handle, _ptr(p, torch.float32,
                                                           self.param_count())),
               "mp_net_set_params")

    def get_params(self):
        p = torch.empty(self.param_count(), dtype=torch.float32, device="cuda")
        _check(_lib_().mp_net_get_params(self.handle, _ptr(p, torch.float32)), "mp_net_get_params")
        return p

    def get_adam(self):
        """Adam's moment estimates (m, v), device FP32 copies."""
        m = torch.empty(self.param_count(), dtype=torch.float32, device="cuda")
        v = torch.empty_like(m)
        _check(_lib_().mp_net_get_adam(self.handle, _ptr(m, torch.float32),
                                       _ptr(v, torch.float32)), "mp_net_get_adam")
        return m, v

    def set_adam(self, m, v):
        """Restore Adam's moments (after set_params, which zeroes them)."""
        n = self.param_count()
        _check(_lib_().mp_net_set_adam(self.handle, _ptr(m, torch.float32, n),
                                       _ptr(v, torch.float32, n)), "mp_net_set_adam")

    def set_input(self, x16):
        _check(_lib_().mp_net_set_input(self.handle, _ptr(x16, torch.bfloat16, self.n * 16)),
               "mp_net_set_input")

    def features(self, phi, b, h, b_scale):
        """Input features from phi and the mean-free rhs b; returns s = rms(b_scale * b)."""
        s = ctypes.c_double(0.0)
        _check(_lib_().mp_net_features(self.handle, _ptr(phi), _ptr(b), float(h), float(b_scale),
                                       ctypes.byref(s)), "mp_net_features")
        return s.value

    def get_input2(self):
        x2 = torch.empty(self.shape + (2,), dtype=torch.bfloat16, device="cuda")
        _check(_lib_().mp_net_get_input2(self.handle, _ptr(x2, torch.bfloat16, self.n * 2)),
               "mp_net_get_input2")
        return x2

    def set_input2(self, x2):
        _check(_lib_().mp_net_set_input2(self.handle, _ptr(x2, torch.bfloat16, self.n * 2)),
               "mp_net_set_input2")

    def forward(self):
        q = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        _check(_lib_().mp_net_forward(self.handle, _ptr(q, torch.float32)), "mp_net_forward")
        return q

    def pressure(self, s):
        p = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        _check(_lib_().mp_net_pressure(self.handle, float(s), _ptr(p)), "mp_net_pressure")
        return p

    def make_target(self, p):
        """q = (p - mean) / rms for training (FP32)."""
        q = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        _check(_lib_().mp_net_make_target(self.handle, _ptr(p, numel=self.n),
                                          _ptr(q, torch.float32)), "mp_net_make_target")
        return q

    def backward(self, gq):
        g = torch.empty(self.param_count(), dtype=torch.float32, device="cuda")
        _check(_lib_().mp_net_backward(self.handle, _ptr(gq, torch.float32, self.n),
                                       _ptr(g, torch.float32)), "mp_net_backward")
        return g

    def launches(self):
        """Kernels launched by the network's inference paths so far."""
        return int(_lib_().mp_net_launches(self.handle))

    def load(self, path=None):
        """Parameters from an .npz written by learn.py (default: the packaged
        network trained at 128^3 with the energy loss); returns its metadata."""
        import json
        import numpy as np
        d = np.load(path or DEFAULT_WEIGHTS)
        self.set_params(torch.from_numpy(d["params"].astype(np.float32)).cuda())
        return json.loads(str(d["meta"])) if "meta" in d.files else {}

    def features_at(self, factor, phi, b, h, b_scale):
        """features() for fields on a grid `factor` (1, 2) times finer."""
        s = ctypes.c_double(0.0)
        nf = self.n * factor ** 3
        _check(_lib_().mp_net_features_at(self.handle, int(factor), _ptr(phi, numel=nf),
                                          _ptr(b, numel=nf), float(h), float(b_scale),
                                          ctypes.byref(s)), "mp_net_features_at")
        return s.value

    def pressure_at(self, factor, bc, s):
        """pressure() interpolated onto a grid `factor` (1, 2) times finer."""
        shape = tuple(factor * d for d in self.shape)
        p = torch.empty(shape, dtype=torch.float64, device="cuda")
        arr = (ctypes.c_int * 3)(*[int(v) for v in bc])
        _check(_lib_().mp_net_pressure_at(self.handle, int(factor), arr, float(s), _ptr(p)),
               "mp_net_pressure_at")
        return p

    def set_loss(self, kind, rho_l=1.0, rho_g=1e-3, bc=(0, 0, 1)):
        """Training loss: 0 = gauge-free MSE, 1 = energy norm of the
        best-scaled guess under the ghost-fluid operator of the input's phi."""
        arr = (ctypes.c_int * 3)(*[int(b) for b in bc])
        _check(_lib_().mp_net_set_loss(self.handle, int(kind), float(rho_l), float(rho_g), arr),
               "mp_net_set_loss")

    def loss_grad(self, target):
        """Forward pass, the training loss against target and dL/dq (no
        update); returns (loss, gq) with gq FP32 on the device."""
        loss = ctypes.c_double(0.0)
        gq = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        _check(_lib_().mp_net_loss_grad(self.handle, _ptr(target, torch.float32, self.n),
                                        _ptr(gq, torch.float32), ctypes.byref(loss)),
               "mp_net_loss_grad")
        return loss.value, gq

    def train_step(self, target, lr, step):
        loss = ctypes.c_double(0.0)
        _check(_lib_().mp_net_train_step(self.handle, _ptr(target, torch.float32, self.n),
                                         ctypes.c_float(lr), int(step), ctypes.byref(loss)),
               "mp_net_train_step")
        return loss.value

    def train_step_grad(self, gq, lr, step):
        """One Adam step from an externally formed gradient dL/dq (FP32, device)."""
        _check(_lib_().mp_net_train_step_grad(self.handle, _ptr(gq, torch.float32, self.n),
                                              ctypes.c_float(lr), int(step)),
               "mp_net_train_step_grad")

    def close(self):
        if getattr(self, "handle", None):
            _lib_().mp_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_poisson_set_net(handle, net):
    return _check(_lib_().mp_poisson_set_net(handle, None if net is None else net.handle),
                  "mp_poisson_set_net")


__all__ = ["Net", "mp_conv3d_fwd", "mp_conv3d_wgrad", "mp_poisson_set_net", "MPError"]
