"""FP64 CPU oracle for the multiphase pressure-Poisson solve.

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the CPU
baseline leg of the benchmark use it; the product library never imports it.
It shares no code with the CUDA path (only the seeded generators in
``synth.py``).  See ``mp_oracle.c`` for the discretisation and the passages
it follows; ``conv.py`` holds the conv-net oracle.

Arrays are numpy float64 of shape (nz, ny, nx).  Internally the oracle keeps
n+1 faces per axis; ``owned_to_full`` converts the low-face-owned layout of
the generators (n faces per axis, wrapped) into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmp_oracle.so")
_lib = None

PERIODIC = 0
NEUMANN = 1            # wall or inflow on both sides (zero normal pressure gradient)
DIRICHLET = 2          # outflow on both sides (p = 0 on the boundary face)
NEUMANN_DIRICHLET = 3  # wall/inflow on the low side, outflow on the high side
DIRICHLET_NEUMANN = 4  # outflow on the low side, wall/inflow on the high side


def singular(bc):
    """True when the operator annihilates constants (no outflow side)."""
    return not any(b in (DIRICHLET, NEUMANN_DIRICHLET, DIRICHLET_NEUMANN) for b in bc)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, -O2, portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.POINTER(ctypes.c_double)
        I3 = ctypes.POINTER(ctypes.c_int)
        i, d = ctypes.c_int, ctypes.c_double
        lib.oracle_curvature.argtypes = [i, i, i, d, I3, D, D]
        lib.oracle_faces.argtypes = [i, i, i, I3, D, d, d, D, D, D]
        lib.oracle_jump.argtypes = [i, i, i, d, I3, D, D, D, D, D, d, D]
        lib.oracle_apply.argtypes = [i, i, i, d, I3, D, D, D, D, D]
        lib.oracle_residual.argtypes = [i, i, i, d, I3, D, D, D, D, D, D]
        lib.oracle_residual.restype = d
        lib.oracle_cg.argtypes = [i, i, i, d, I3, D, D, D, D, D, d, i, D]
        lib.oracle_cg.restype = i
        lib.oracle_gs.argtypes = [i, i, i, d, I3, D, D, D, D, D, d, i, D]
        lib.oracle_gs.restype = i
        lib.oracle_divergence.argtypes = [i, i, i, d, D, D, D, D]
        lib.oracle_project.argtypes = [i, i, i, d, I3, D, D, D, D, D, d, D, D, D, D]
        lib.oracle_flux_jump.argtypes = [i, i, i, d, I3, D, D, D, D, D, d, d, D]
        lib.oracle_project_flux.argtypes = [i, i, i, I3, D, D, D, D, D, d, d, D, D, D]
        _lib = lib
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _per(bc):
    """Boundary codes per axis, as the C oracle takes them."""
    return (ctypes.c_int * 3)(*[int(b) for b in bc])


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Faces:
    """Face coefficients with n+1 faces per axis (fx, fy, fz)."""

    def __init__(self, fx, fy, fz):
        self.fx, self.fy, self.fz = fx, fy, fz


def curvature(phi, h, bc):
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    out = np.empty_like(phi)
    _load().oracle_curvature(nx, ny, nz, h, _per(bc), _p(phi), _p(out))
    return out


def faces(phi, rho_l, rho_g, bc):
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    fx = np.empty((nz, ny, nx + 1))
    fy = np.empty((nz, ny + 1, nx))
    fz = np.empty((nz + 1, ny, nx))
    _load().oracle_faces(nx, ny, nz, _per(bc), _p(phi), rho_l, rho_g, _p(fx), _p(fy), _p(fz))
    return Faces(fx, fy, fz)


def jump(phi, kappa, f, h, sigma, bc):
    phi, kappa = _f64(phi), _f64(kappa)
    nz, ny, nx = phi.shape
    out = np.empty_like(phi)
    _load().oracle_jump(nx, ny, nz, h, _per(bc), _p(phi), _p(kappa), _p(f.fx), _p(f.fy),
                        _p(f.fz), sigma, _p(out))
    return out


def apply(f, x, h, bc):
    x = _f64(x)
    nz, ny, nx = x.shape
    y = np.empty_like(x)
    _load().oracle_apply(nx, ny, nz, h, _per(bc), _p(f.fx), _p(f.fy), _p(f.fz), _p(x), _p(y))
    return y


def residual(f, b, x, h, bc):
    b, x = _f64(b), _f64(x)
    nz, ny, nx = x.shape
    r = np.empty_like(x)
    n = _load().oracle_residual(nx, ny, nz, h, _per(bc), _p(f.fx), _p(f.fy), _p(f.fz),
                                _p(b), _p(x), _p(r))
    return r, n


def cg(f, b, h, bc, tol=1e-12, maxit=200000, x0=None):
    """Jacobi-PCG solve of A x = b (b mean-free unless an axis has an outflow
    side). Returns (x, iters, relres)."""
    b = _f64(b)
    nz, ny, nx = b.shape
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    rel = ctypes.c_double(0.0)
    it = _load().oracle_cg(nx, ny, nz, h, _per(bc), _p(f.fx), _p(f.fy), _p(f.fz), _p(b), _p(x),
                           tol, maxit, ctypes.byref(rel))
    return x, it, rel.value


def gs(f, b, h, bc, tol=1e-10, maxsweeps=100000, x0=None):
    """Lexicographic Gauss-Seidel solve (small grids). Returns (x, sweeps, relres)."""
    b = _f64(b)
    nz, ny, nx = b.shape
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    rel = ctypes.c_double(0.0)
    it = _load().oracle_gs(nx, ny, nz, h, _per(bc), _p(f.fx), _p(f.fy), _p(f.fz), _p(b), _p(x),
                           tol, maxsweeps, ctypes.byref(rel))
    return x, it, rel.value


def owned_to_full(u, axis):
    """n faces per axis (face 0 = the face below cell 0, wrapped) -> n+1 faces.

    Face n is the same physical face as face 0 (periodic) or the top wall,
    which the owned layout stores in the same slot as the bottom wall.
    """
    u = _f64(u)
    ax = 2 - axis  # numpy axis of x/y/z
    first = np.take(u, [0], axis=ax)
    return np.ascontiguousarray(np.concatenate([u, first], axis=ax))


def divergence(ux, uy, uz, h):
    """Divergence of owned-layout face velocities."""
    fx, fy, fz = owned_to_full(ux, 0), owned_to_full(uy, 1), owned_to_full(uz, 2)
    nz, ny, nx = ux.shape
    out = np.empty((nz, ny, nx))
    _load().oracle_divergence(nx, ny, nz, h, _p(fx), _p(fy), _p(fz), _p(out))
    return out


def divergence_full(fx, fy, fz, h):
    nz, ny, nx = fx.shape[0], fx.shape[1], fx.shape[2] - 1
    out = np.empty((nz, ny, nx))
    _load().oracle_divergence(nx, ny, nz, h, _p(_f64(fx)), _p(_f64(fy)), _p(_f64(fz)), _p(out))
    return out


def flux_jump(phi, mdot, f, h, rho_l, rho_g, bc):
    """Phase-change source: the flux jump B = -mdot [1/rho] of every interface
    face split between its two rows (see mp_oracle.c).  mdot: cell values."""
    phi, mdot = _f64(phi), _f64(mdot)
    nz, ny, nx = phi.shape
    out = np.zeros_like(phi)
    _load().oracle_flux_jump(nx, ny, nz, h, _per(bc), _p(phi), _p(mdot), _p(f.fx), _p(f.fy),
                             _p(f.fz), rho_l, rho_g, _p(out))
    return out


def project(phi, kappa, f, p, ux, uy, uz, h, sigma, bc, mdot=None, rho_l=1.0, rho_g=1e-3):
    """Corrected face velocities (n+1 faces per axis) u = u* - beta (grad p - jump);
    with a phase-change mass flux mdot, interface faces get the liquid-side
    velocity."""
    fx, fy, fz = owned_to_full(ux, 0), owned_to_full(uy, 1), owned_to_full(uz, 2)
    phi, kappa, p = _f64(phi), _f64(kappa), _f64(p)
    nz, ny, nx = phi.shape
    _load().oracle_project(nx, ny, nz, h, _per(bc), _p(phi), _p(kappa), _p(f.fx), _p(f.fy),
                           _p(f.fz), sigma, _p(p), _p(fx), _p(fy), _p(fz))
    if mdot is not None:
        _load().oracle_project_flux(nx, ny, nz, _per(bc), _p(phi), _p(_f64(mdot)), _p(f.fx),
                                    _p(f.fy), _p(f.fz), rho_l, rho_g, _p(fx), _p(fy), _p(fz))
    return fx, fy, fz


def assemble(phi, rhs, h, rho_l, rho_g, sigma, bc, mdot=None):
    """kappa, faces, J and the right-hand side b = rhs + J, minus its mean
    when the operator is singular (no outflow side).  With a phase-change
    mass flux mdot, J includes its flux-jump source."""
    kappa = curvature(phi, h, bc)
    f = faces(phi, rho_l, rho_g, bc)
    J = jump(phi, kappa, f, h, sigma, bc)
    if mdot is not None:
        J = J + flux_jump(phi, mdot, f, h, rho_l, rho_g, bc)
    b = _f64(rhs) + J
    if singular(bc):
        b = b - b.mean()
    return kappa, f, J, b


def solve(phi, rhs, h, rho_l, rho_g, sigma, bc, tol=1e-12, maxit=200000, mdot=None):
    """Full oracle solve: returns dict with p (mean-free when singular), b, kappa,
    faces, iters, relres."""
    kappa, f, J, b = assemble(phi, rhs, h, rho_l, rho_g, sigma, bc, mdot=mdot)
    x, it, rel = cg(f, b, h, bc, tol=tol, maxit=maxit)
    return dict(p=x, b=b, kappa=kappa, faces=f, J=J, iters=it, relres=rel)
