"""Seeded synthetic inputs for the pressure-Poisson projection step.

This module is the only code shared by the CPU oracle and the CUDA path. It
draws geometry and velocity fields; it holds none of the solver's arithmetic
(no curvature, no face coefficients, no jump, no divergence, no operator).

Conventions (the layout the C-ABI documents):
  * grid nx*ny*nz cubic cells of edge h, cell (i,j,k) centred at ((i+1/2)h, ...);
  * arrays are numpy float64 of shape (nz, ny, nx): x fastest, C order;
  * face arrays use "each cell owns its low face": ux[k,j,i] sits on the face
    between cells i-1 and i (x = i*h), wrapped so that face 0 of a periodic
    axis is the face between cell n-1 and cell 0; on a wall (Neumann) axis
    face 0 is the wall itself, shared by the bottom and top wall.

The level set follows the paper's sign convention: phi > 0 in gas, phi < 0
in liquid, phi = 0 on the interface (Section 2, Fig. 2 caption).
"""
from __future__ import annotations

import numpy as np

PERIODIC = 0
NEUMANN = 1

# Workload recipes (grid, geometry, fluid parameters) of the benchmark configs.
# rho_g / rho_l = 0.001 is the paper's example gas/liquid density ratio
# (the runtime-parameter TOML figure of Section 4, mph_rhoGas); sigma is the surface tension.
WORKLOADS = {
    "bubble32": dict(n=32, bubbles=[((0.5, 0.5, 0.4), 0.25)], pool_z0=None,
                     rho_l=1.0, rho_g=1e-3, sigma=0.01, useed=1),
    "bubble256": dict(n=256, bubbles=[((0.5, 0.5, 0.4), 0.15)], pool_z0=None,
                      rho_l=1.0, rho_g=1e-3, sigma=0.07, useed=2),
    "bubbles512": dict(n=512, nbubbles=64, rmin=0.02, rmax=0.06, pool_z0=None,
                       rho_l=1.0, rho_g=1e-3, sigma=0.07, gseed=3, useed=3),
    "pool256": dict(n=256, nbubbles=32, rmin=0.02, rmax=0.06, pool_z0=0.3,
                    rho_l=1.0, rho_g=1e-3, sigma=0.07, gseed=5, useed=5),
}


def cell_centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def _min_image(d: np.ndarray, length: float, periodic: bool) -> np.ndarray:
    if not periodic:
        return d
    return d - length * np.round(d / length)


def level_set(shape, h, bubbles, pool_z0=None, bc=(PERIODIC, PERIODIC, NEUMANN), device=None):
    """Gas-positive signed distance of a union of spherical bubbles and an
    optional gas layer above a liquid pool (gas for z > pool_z0).

    phi = max(z - pool_z0, max_b (R_b - |x - c_b|)), distances taken with the
    minimum-image convention along periodic axes.  Returns (nz, ny, nx) f64
    (a torch tensor on `device` when given; same formula).
    """
    if device is not None:
        return _level_set_torch(shape, h, bubbles, pool_z0, bc, device)
    nz, ny, nx = shape
    x = cell_centres(nx, h)[None, None, :]
    y = cell_centres(ny, h)[None, :, None]
    z = cell_centres(nz, h)[:, None, None]
    lx, ly, lz = nx * h, ny * h, nz * h
    phi = np.full(shape, -np.inf)
    if pool_z0 is not None:
        phi = np.maximum(phi, np.broadcast_to(z - pool_z0, shape))
    for (cx, cy, cz), r in bubbles:
        dx = _min_image(x - cx, lx, bc[0] == PERIODIC)
        dy = _min_image(y - cy, ly, bc[1] == PERIODIC)
        dz = _min_image(z - cz, lz, bc[2] == PERIODIC)
        phi = np.maximum(phi, r - np.sqrt(dx * dx + dy * dy + dz * dz))
    return np.ascontiguousarray(phi)


def _level_set_torch(shape, h, bubbles, pool_z0, bc, device):
    import torch
    nz, ny, nx = shape
    f64 = torch.float64
    x = ((torch.arange(nx, dtype=f64, device=device) + 0.5) * h)[None, None, :]
    y = ((torch.arange(ny, dtype=f64, device=device) + 0.5) * h)[None, :, None]
    z = ((torch.arange(nz, dtype=f64, device=device) + 0.5) * h)[:, None, None]
    lx, ly, lz = nx * h, ny * h, nz * h
    phi = torch.full(shape, -float("inf"), dtype=f64, device=device)
    if pool_z0 is not None:
        phi = torch.maximum(phi, (z - pool_z0).expand(shape))

    def mi(d, length, periodic):
        return d - length * torch.round(d / length) if periodic else d

    for (cx, cy, cz), r in bubbles:
        dx = mi(x - cx, lx, bc[0] == PERIODIC)
        dy = mi(y - cy, ly, bc[1] == PERIODIC)
        dz = mi(z - cz, lz, bc[2] == PERIODIC)
        phi = torch.maximum(phi, r - torch.sqrt(dx * dx + dy * dy + dz * dz))
    return phi.contiguous()


def random_bubbles(seed, count, rmin, rmax, n, h=None, pool_z0=None, max_tries=200000):
    """Non-overlapping bubbles by rejection sampling (PCG64(seed)).

    Radii ~ U[rmin, rmax]; centres uniform in the unit cube with wall clearance
    R + 2h <= c_z <= top - R - 2h (top = 1, or pool_z0 - 4h under a pool);
    gap |c_a - c_b|_minimage >= R_a + R_b + 4h.
    """
    h = 1.0 / n if h is None else h
    rng = np.random.Generator(np.random.PCG64(seed))
    top = 1.0 if pool_z0 is None else pool_z0 - 2.0 * h
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place bubbles")
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(0.0, 1.0, size=3)
        lo, hi = r + 2.0 * h, top - r - 2.0 * h
        if hi <= lo:
            continue
        c[2] = lo + (hi - lo) * rng.uniform()
        ok = True
        for (c2, r2) in out:
            d = np.array(c) - np.array(c2)
            d[:2] -= np.round(d[:2])
            if np.sqrt((d * d).sum()) < r + r2 + 4.0 * h:
                ok = False
                break
        if ok:
            out.append(((float(c[0]), float(c[1]), float(c[2])), float(r)))
    return out


def _draw_modes(rng, modes, kmax):
    """Mode list [(k (3 ints), psi, a)]: k in [-kmax, kmax]^3 minus 0,
    psi ~ U[0, 2pi), a ~ N(0, 1), drawn in that order per mode."""
    out = []
    while len(out) < modes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            continue
        psi = rng.uniform(0.0, 2.0 * np.pi)
        a = rng.standard_normal()
        out.append((k, psi, a))
    return out


def _eval_modes_numpy(mode_list, shape, h, origin):
    """sum_m a_m cos(2 pi k_m . x + psi_m) at points origin + h*index,
    evaluated separably through complex exponentials along each axis."""
    nz, ny, nx = shape
    xs = origin[0] + h * np.arange(nx)
    ys = origin[1] + h * np.arange(ny)
    zs = origin[2] + h * np.arange(nz)
    acc = np.zeros(shape, dtype=np.complex128)
    for k, psi, a in mode_list:
        ex = np.exp(2j * np.pi * k[0] * xs)[None, None, :]
        ey = np.exp(2j * np.pi * k[1] * ys)[None, :, None]
        ez = np.exp(2j * np.pi * k[2] * zs)[:, None, None]
        acc += (a * np.exp(1j * psi)) * (ez * ey) * ex
    return acc.real


def _eval_modes_torch(mode_list, shape, h, origin, device):
    import torch
    nz, ny, nx = shape
    f64 = torch.float64
    xs = origin[0] + h * torch.arange(nx, dtype=f64, device=device)
    ys = origin[1] + h * torch.arange(ny, dtype=f64, device=device)
    zs = origin[2] + h * torch.arange(nz, dtype=f64, device=device)
    acc = torch.zeros(shape, dtype=f64, device=device)
    tp = 2.0 * np.pi
    for k, psi, a in mode_list:
        # cos(A + B + C + psi) with A, B, C the per-axis phases, expanded separably
        ph_x = tp * float(k[0]) * xs
        ph_y = tp * float(k[1]) * ys
        ph_z = tp * float(k[2]) * zs + psi
        cz, sz = torch.cos(ph_z)[:, None], torch.sin(ph_z)[:, None]
        cy, sy = torch.cos(ph_y)[None, :], torch.sin(ph_y)[None, :]
        czy = (cz * cy - sz * sy)[:, :, None]
        szy = (sz * cy + cz * sy)[:, :, None]
        acc += a * (czy * torch.cos(ph_x)[None, None, :] - szy * torch.sin(ph_x)[None, None, :])
    return acc


def velocity(seed, shape, h, modes=16, kmax=4, bc=(PERIODIC, PERIODIC, NEUMANN), device=None):
    """Seeded smooth face velocity u* = (ux, uy, uz), each max-normalised to 1.

    Each component is a 16-mode random Fourier series evaluated on its own
    faces (low-face ownership, see module doc); the normal component vanishes
    on wall faces.  Returns three (nz, ny, nx) float64 numpy arrays, or torch
    tensors on `device` when given (same modes; values agree to rounding).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    comps = []
    origins = [(0.0, 0.5 * h, 0.5 * h), (0.5 * h, 0.0, 0.5 * h), (0.5 * h, 0.5 * h, 0.0)]
    for axis in range(3):
        ml = _draw_modes(rng, modes, kmax)
        if device is None:
            u = _eval_modes_numpy(ml, shape, h, origins[axis])
        else:
            u = _eval_modes_torch(ml, shape, h, origins[axis], device)
        if bc[axis] == NEUMANN:
            if axis == 0:
                u[:, :, 0] = 0.0
            elif axis == 1:
                u[:, 0, :] = 0.0
            else:
                u[0, :, :] = 0.0
        u /= abs(u).max()
        comps.append(u if device is not None else np.ascontiguousarray(u))
    return tuple(comps)


def perturbed_velocity(u0, seed, amp=0.05, shape=None, h=None, bc=(PERIODIC, PERIODIC, NEUMANN)):
    """u0 + amp * xi with xi a fresh max-normalised 16-mode field (seed)."""
    shape = u0[0].shape if shape is None else shape
    h = 1.0 / shape[2] if h is None else h
    xi = velocity(seed, shape, h, bc=bc)
    return tuple(np.ascontiguousarray(a + amp * b) for a, b in zip(u0, xi))


def workload(name: str):
    """(phi, (ux, uy, uz), params) for a named workload recipe."""
    w = WORKLOADS[name]
    n = w["n"]
    h = 1.0 / n
    shape = (n, n, n)
    if "bubbles" in w:
        bubbles = w["bubbles"]
    else:
        bubbles = random_bubbles(w["gseed"], w["nbubbles"], w["rmin"], w["rmax"], n,
                                 pool_z0=w["pool_z0"])
    phi = level_set(shape, h, bubbles, w["pool_z0"])
    u = velocity(w["useed"], shape, h)
    params = dict(h=h, rho_l=w["rho_l"], rho_g=w["rho_g"], sigma=w["sigma"],
                  bc=(PERIODIC, PERIODIC, NEUMANN), bubbles=bubbles, pool_z0=w["pool_z0"])
    return phi, u, params
