"""Argument marshalling for the mp_poisson C-ABI (torch tensors <-> pointers)."""
from __future__ import annotations

import ctypes

import torch

from . import _lib

PERIODIC = _lib.MP_BC_PERIODIC
NEUMANN = _lib.MP_BC_NEUMANN
DIRICHLET = _lib.MP_BC_DIRICHLET                  # outflow (p = 0) on both sides
NEUMANN_DIRICHLET = _lib.MP_BC_NEUMANN_DIRICHLET  # wall/inflow low, outflow high
DIRICHLET_NEUMANN = _lib.MP_BC_DIRICHLET_NEUMANN  # outflow low, wall/inflow high


class MPError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, mp_status_str(status), status))


def _lib_():
    return _lib.load()


def mp_status_str(status: int) -> str:
    return _lib_().mp_status_str(int(status)).decode()


def _ptr(t: torch.Tensor, dtype=torch.float64, numel=None, device=True) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError("expected a contiguous %s tensor" % dtype)
    if device and not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError("expected a host tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d elements, got %d" % (numel, t.numel()))
    return t.data_ptr()


def _check(status: int, where: str, ok=(0,)):
    if status not in ok:
        raise MPError(status, where)
    return status


def mp_opts_default(**overrides) -> _lib.mp_opts:
    o = _lib.mp_opts()
    _lib_().mp_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "stream":
            v = _stream_ptr(v)
        setattr(o, k, v)
    return o


def _stream_ptr(s):
    if s is None:
        return None
    if isinstance(s, torch.cuda.Stream):
        return s.cuda_stream
    return int(s)


def mp_poisson_setup(grid, h, bc, phi, rho_l, rho_g, sigma, opts=None):
    nx, ny, nz = grid
    handle = ctypes.c_void_p()
    bcs = (ctypes.c_int * 3)(*bc)
    st = _lib_().mp_poisson_setup(
        ctypes.byref(handle), _lib.mp_grid(nx, ny, nz), float(h), bcs,
        _ptr(phi, numel=nx * ny * nz), float(rho_l), float(rho_g), float(sigma),
        ctypes.byref(opts) if opts is not None else None)
    _check(st, "mp_poisson_setup")
    return handle


def mp_poisson_set_geometry(handle, phi, rho_l, rho_g, sigma):
    return _check(_lib_().mp_poisson_set_geometry(handle, _ptr(phi), float(rho_l), float(rho_g),
                                                  float(sigma)), "mp_poisson_set_geometry")


def mp_poisson_set_mass_flux(handle, mdot):
    """Phase-change mass flux per cell (device f64 tensor), or None to clear."""
    ptr = None if mdot is None else _ptr(mdot)
    return _check(_lib_().mp_poisson_set_mass_flux(handle, ptr), "mp_poisson_set_mass_flux")


def mp_poisson_deflated_energy(handle, q, t, gq=None):
    """Deflated energy loss of q against t (FP32 device tensors) and, into gq, its
    gradient; returns the loss."""
    loss = ctypes.c_double(0.0)
    n = q.numel()
    _check(_lib_().mp_poisson_deflated_energy(
        handle, _ptr(q, torch.float32), _ptr(t, torch.float32, n),
        None if gq is None else _ptr(gq, torch.float32, n), ctypes.byref(loss)),
        "mp_poisson_deflated_energy")
    return loss.value


def mp_poisson_set_opts(handle, opts):
    return _check(_lib_().mp_poisson_set_opts(handle, ctypes.byref(opts)), "mp_poisson_set_opts")


def mp_poisson_solve(handle, rhs, p, tol, hist_cap=4096, allow_not_converged=False):
    it = ctypes.c_int(0)
    hist = (ctypes.c_double * max(1, hist_cap))()
    hlen = ctypes.c_int(0)
    st = _lib_().mp_poisson_solve(handle, _ptr(rhs), _ptr(p), float(tol), ctypes.byref(it), hist,
                                  hist_cap, ctypes.byref(hlen))
    ok = (0, _lib.MP_ERR_NOT_CONVERGED) if allow_not_converged else (0,)
    _check(st, "mp_poisson_solve", ok)
    return it.value, [hist[i] for i in range(hlen.value)], st


def mp_poisson_project_step(handle, ux, uy, uz, p, tol):
    it = ctypes.c_int(0)
    _check(_lib_().mp_poisson_project_step(handle, _ptr(ux), _ptr(uy), _ptr(uz), _ptr(p),
                                           float(tol), ctypes.byref(it)),
           "mp_poisson_project_step")
    return it.value


def mp_poisson_project_step_host(handle, ux, uy, uz, p, tol):
    it = ctypes.c_int(0)
    _check(_lib_().mp_poisson_project_step_host(
        handle, _ptr(ux, device=False), _ptr(uy, device=False), _ptr(uz, device=False),
        _ptr(p, device=False), float(tol), ctypes.byref(it)), "mp_poisson_project_step_host")
    return it.value


def mp_poisson_apply(handle, x, y):
    return _check(_lib_().mp_poisson_apply(handle, _ptr(x), _ptr(y)), "mp_poisson_apply")


def mp_poisson_divergence(handle, ux, uy, uz, div):
    return _check(_lib_().mp_poisson_divergence(handle, _ptr(ux), _ptr(uy), _ptr(uz), _ptr(div)),
                  "mp_poisson_divergence")


def mp_poisson_rhs(handle, rhs, b):
    return _check(_lib_().mp_poisson_rhs(handle, _ptr(rhs), _ptr(b)), "mp_poisson_rhs")


def mp_poisson_rhs_noalloc(rhs, J, b, stream=None):
    """b = rhs + J - mean(rhs + J) without any device allocation (enqueued on
    `stream`; the call does not wait for the work).  The library uses the
    current device's scratch and launches there, so the three tensors must
    share one device, which is made current for the call."""
    n = rhs.numel()
    if not (rhs.device == J.device == b.device):
        raise ValueError("rhs, J and b must be on one device")
    with torch.cuda.device(rhs.device):
        return _check(_lib_().mp_poisson_rhs_noalloc(n, _ptr(rhs, numel=n), _ptr(J, numel=n),
                                                     _ptr(b, numel=n), _stream_ptr(stream)),
                      "mp_poisson_rhs_noalloc")


def mp_poisson_project(handle, p, ux, uy, uz):
    return _check(_lib_().mp_poisson_project(handle, _ptr(p), _ptr(ux), _ptr(uy), _ptr(uz)),
                  "mp_poisson_project")


def mp_poisson_get_fields(handle, kappa=None, bx=None, by=None, bz=None, J=None):
    def p(t):
        return None if t is None else _ptr(t)
    return _check(_lib_().mp_poisson_get_fields(handle, p(kappa), p(bx), p(by), p(bz), p(J)),
                  "mp_poisson_get_fields")


def mp_poisson_get_stats(handle):
    s = _lib.mp_stats()
    _check(_lib_().mp_poisson_get_stats(handle, ctypes.byref(s)), "mp_poisson_get_stats")
    return {k: getattr(s, k) for k, _ in _lib.mp_stats._fields_}


def mp_poisson_get_components(handle, n):
    """(comp, m): each cell's gas-component id (-1 liquid; int32 device tensor of n cells)
    and the component count used for deflation."""
    comp = torch.empty(n, dtype=torch.int32, device="cuda")
    m = ctypes.c_int(0)
    _check(_lib_().mp_poisson_get_components(handle, ctypes.c_void_p(comp.data_ptr()),
                                             ctypes.byref(m)), "mp_poisson_get_components")
    return comp, m.value


def mp_poisson_set_profiling(handle, enable):
    return _check(_lib_().mp_poisson_set_profiling(handle, int(bool(enable))),
                  "mp_poisson_set_profiling")


def mp_poisson_get_profile(handle):
    n = ctypes.c_int(0)
    _check(_lib_().mp_poisson_get_profile(handle, None, 0, ctypes.byref(n)), "mp_poisson_get_profile")
    arr = (_lib.mp_kernel_prof * max(1, n.value))()
    _check(_lib_().mp_poisson_get_profile(handle, arr, n.value, ctypes.byref(n)),
           "mp_poisson_get_profile")
    return [dict(name=a.name.decode(), level=a.level, cells=a.cells, launches=a.launches,
                 total_ms=a.total_ms, alg_bytes=a.alg_bytes) for a in arr[:n.value]]


def mp_poisson_destroy(handle):
    if handle:
        _lib_().mp_poisson_destroy(handle)


class Poisson:
    """Owns one solver handle.  Arrays are torch tensors of shape (nz, ny, nx)."""

    def __init__(self, phi, h, bc=(PERIODIC, PERIODIC, NEUMANN), rho_l=1.0, rho_g=1e-3,
                 sigma=0.0, **opts):
        nz, ny, nx = phi.shape
        self.shape = (nz, ny, nx)
        self.h = float(h)
        self.opts = mp_opts_default(**opts)
        self.handle = mp_poisson_setup((nx, ny, nz), h, bc, phi.contiguous(), rho_l, rho_g, sigma,
                                       self.opts)

    def set_opts(self, **opts):
        for k, v in opts.items():
            setattr(self.opts, k, _stream_ptr(v) if k == "stream" else v)
        mp_poisson_set_opts(self.handle, self.opts)

    def set_geometry(self, phi, rho_l, rho_g, sigma):
        mp_poisson_set_geometry(self.handle, phi.contiguous(), rho_l, rho_g, sigma)

    def deflated_energy(self, q, t, grad=True):
        """(loss, dL/dq) of the deflated energy loss (mp_poisson_deflated_energy)."""
        gq = torch.empty_like(q) if grad else None
        loss = mp_poisson_deflated_energy(self.handle, q.contiguous(), t.contiguous(), gq)
        return loss, gq

    def set_mass_flux(self, mdot):
        if mdot is not None and tuple(mdot.shape) != tuple(self.shape):
            raise ValueError("mass flux must have the grid's shape %s" % (tuple(self.shape),))
        mp_poisson_set_mass_flux(self.handle, None if mdot is None else mdot.contiguous())

    def solve(self, rhs, p=None, tol=1e-10, allow_not_converged=False):
        if p is None:
            p = torch.zeros_like(rhs)
        it, hist, st = mp_poisson_solve(self.handle, rhs, p, tol,
                                        allow_not_converged=allow_not_converged)
        return p, it, hist

    def project_step(self, ux, uy, uz, p, tol=1e-10):
        return mp_poisson_project_step(self.handle, ux, uy, uz, p, tol)

    def apply(self, x):
        y = torch.empty_like(x)
        mp_poisson_apply(self.handle, x, y)
        return y

    def divergence(self, ux, uy, uz):
        d = torch.empty_like(ux)
        mp_poisson_divergence(self.handle, ux, uy, uz, d)
        return d

    def rhs(self, rhs):
        b = torch.empty_like(rhs)
        mp_poisson_rhs(self.handle, rhs, b)
        return b

    def project(self, p, ux, uy, uz):
        mp_poisson_project(self.handle, p, ux, uy, uz)

    def fields(self):
        z = lambda: torch.empty(self.shape, dtype=torch.float64, device="cuda")  # noqa: E731
        k, bx, by, bz, J = z(), z(), z(), z(), z()
        mp_poisson_get_fields(self.handle, k, bx, by, bz, J)
        return dict(kappa=k, bx=bx, by=by, bz=bz, J=J)

    def stats(self):
        return mp_poisson_get_stats(self.handle)

    def components(self):
        comp, m = mp_poisson_get_components(self.handle, self.shape[0] * self.shape[1] * self.shape[2])
        return comp.view(self.shape), m

    def set_profiling(self, enable=True):
        mp_poisson_set_profiling(self.handle, enable)

    def profile(self):
        return mp_poisson_get_profile(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            mp_poisson_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
