"""Seeded synthetic workloads: grid descriptions and initial states.

This module is the one place both the CUDA path and the FP64 oracle take
their inputs from. It holds no arithmetic of the stage update itself: only
case descriptions (grid, boundary conditions, jets) and the initial
conserved state of each workload, written from its stated primitive fields
(rho, u, p) with E = p / (gamma - 1) + rho |u|^2 / 2.

Sharp edges in the initial data are smoothed with a tanh of width dx:
unlimited 5th-order linear reconstruction turns a sharp 1 -> 0.1 step into
negative face densities, so the paper's plumes are seeded smoothly too.

Random numbers come from numpy's Philox counter-based generator, keyed by
the case seed, and are drawn once on the host; both sides consume the same
bytes.

Workloads:
  density_wave  3D periodic cube, rho = 1 + 0.2 sin(2 pi x) + noise, u = (1,0,0), p = 1
  blast         unit cube, outflow, sphere r < 0.2 at (1,1)/(0.125,0.1) in (rho,p), u = 0
  plume         1024 x 1024 x 2048 box, 33 Mach-3 inflow jets on z = 0, outflow elsewhere
  jets4         128^3 box, 4 Mach-2 inflow jets on z = 0
  sod           quasi-1D shock tube along x
  tgv           periodic Taylor-Green vortex at Mach 0.5 with density noise
                (tgv_batch: 64 of them with edges drawn from {48,64,80,96,128})
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

PERIODIC, OUTFLOW, INFLOW = 0, 1, 2
NVAR = 5


@dataclass
class Case:
    """Grid, physics constants and boundary conditions of one workload."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    gamma: float = 1.4
    alpha: float = 0.0          # IGR alpha; set to dx^2 by the constructors
    cfl: float = 0.4
    sweeps: int = 5
    bc: Tuple[int, ...] = (PERIODIC,) * 6   # faces -x,+x,-y,+y,-z,+z
    jets: List[Tuple[float, ...]] = field(default_factory=list)  # (cx,cy,R,rho,w,p,edge)
    steps: int = 1
    seed: int = 0
    noise: float = 0.0
    mach: float = 0.0           # Mach number of the Taylor-Green initial state
    order: int = 5              # face reconstruction: 5th (default) or 3rd order
    sigma_solver: int = 0       # Sigma sweeps: 0 Jacobi, 1 red-black Gauss-Seidel
    mu: float = 0.0             # shear viscosity (0: Euler)
    zeta: float = 0.0           # bulk viscosity

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def resized(self, nx: int, ny: int, nz: int) -> "Case":
        """Same case on another box, dx unchanged (jets keep their positions)."""
        return replace(self, nx=nx, ny=ny, nz=nz)


def _e(p, rho, u2, gamma):
    return p / (gamma - 1.0) + 0.5 * rho * u2


def _centres(case: Case, window):
    k0, k1, j0, j1, i0, i1 = window
    dx = case.dx
    x = (np.arange(i0, i1) + 0.5) * dx
    y = (np.arange(j0, j1) + 0.5) * dx
    z = (np.arange(k0, k1) + 0.5) * dx
    return z[:, None, None], y[None, :, None], x[None, None, :]


def _full(case):
    return (0, case.nz, 0, case.ny, 0, case.nx)


def _noise(case: Case, shape):
    if case.noise == 0.0:
        return 0.0
    rng = np.random.Generator(np.random.Philox(case.seed))
    return rng.uniform(-case.noise, case.noise, size=shape)


# ------------------------------------------------------------------ cases

def density_wave(n: int = 32, seed: int = 1, noise: float = 1e-3, ny: Optional[int] = None,
                 nz: Optional[int] = None, steps: int = 100, sweeps: int = 5) -> Case:
    """Periodic cube of side 1 (n cells along x), rho = 1 + 0.2 sin(2 pi x)."""
    dx = 1.0 / n
    return Case("density_wave", n, ny or n, nz or n, dx, alpha=dx * dx, sweeps=sweeps,
                bc=(PERIODIC,) * 6, steps=steps, seed=seed, noise=noise)


def blast(n: int = 256, seed: int = 2, noise: float = 1e-4, steps: int = 500,
          sweeps: int = 10) -> Case:
    """Sod-type spherical blast in the unit cube with outflow boundaries."""
    dx = 1.0 / n
    return Case("blast", n, n, n, dx, alpha=dx * dx, sweeps=sweeps, bc=(OUTFLOW,) * 6,
                steps=steps, seed=seed, noise=noise)


def _jet(case_dx, cx, cy, radius_cells, mach, p_j, rho_j, jitter, gamma=1.4, edge=1.0):
    w = mach * math.sqrt(gamma * p_j / rho_j) * (1.0 + 0.05 * jitter)
    return (cx, cy, radius_cells * case_dx, rho_j, w, p_j, edge)


def plume(nx: int = 1024, ny: int = 1024, nz: int = 2048, seed: int = 3, steps: int = 2000,
          sweeps: int = 5) -> Case:
    """Many-jet plume: 33 Mach-3 jets of radius 8 cells on the z = 0 face, in
    rings of 3, 10 and 20 at radii 24, 60, 100 cells around the face centre
    of the 1024 x 1024 reference box (angular offsets 0, pi/10, 0), pressure
    ratio 2, rho_jet = 1, +-5% seeded velocity jitter per jet. dx = 1/1024.
    A smaller box keeps the same dx and jet positions relative to its centre."""
    dx = 1.0 / 1024
    rng = np.random.Generator(np.random.Philox(seed))
    xi = rng.uniform(-1.0, 1.0, size=33)
    cx0, cy0 = 0.5 * nx * dx, 0.5 * ny * dx
    jets = []
    n = 0
    for count, radius, offset in ((3, 24, 0.0), (10, 60, math.pi / 10), (20, 100, 0.0)):
        for m in range(count):
            th = offset + 2.0 * math.pi * m / count
            jets.append(_jet(dx, cx0 + radius * dx * math.cos(th), cy0 + radius * dx * math.sin(th),
                             8, 3.0, 2.0, 1.0, xi[n]))
            n += 1
    bc = (OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW, INFLOW, OUTFLOW)
    return Case("plume", nx, ny, nz, dx, alpha=dx * dx, sweeps=sweeps, bc=bc, jets=jets,
                steps=steps, seed=seed)


def jets4(n: int = 128, steps: int = 300, sweeps: int = 5, mach: float = 2.0) -> Case:
    """Four Mach-2 jets at (0.5 +- 0.125, 0.5 +- 0.125) of the unit box, radius
    6/128 (6 cells at 128^3; the same geometry on other grids), edges smoothed
    over 2 cells (with 1 cell the start-up loses positivity near t = 0.126 at
    128^3)."""
    dx = 1.0 / n
    jets = [_jet(dx, 0.5 + sx * 0.125, 0.5 + sy * 0.125, 6.0 * n / 128.0, mach, 2.0, 1.0, 0.0, edge=2.0)
            for sy in (-1, 1) for sx in (-1, 1)]
    bc = (OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW, INFLOW, OUTFLOW)
    return Case("jets4", n, n, n, dx, alpha=dx * dx, sweeps=sweeps, bc=bc, jets=jets, steps=steps)


def sod(n: int, transverse: int = 4, sweeps: int = 5) -> Case:
    """Quasi-1D shock tube along x on [0, 1]: outflow in x, periodic in y, z."""
    dx = 1.0 / n
    bc = (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    return Case("sod", n, transverse, transverse, dx, alpha=dx * dx, sweeps=sweeps, bc=bc)


def tgv(n: int, seed: int = 4, instance: int = 0, steps: int = 200, sweeps: int = 5,
        mach: float = 0.5, noise: float = 0.05) -> Case:
    """Periodic cube of side 1 with a Taylor-Green vortex (k = 2 pi, V0 = 1,
    rho0 = 1, p0 = 1 / (gamma M^2)) and density noise U(-noise, noise)."""
    dx = 1.0 / n
    return Case("tgv", n, n, n, dx, alpha=dx * dx, sweeps=sweeps, bc=(PERIODIC,) * 6, steps=steps,
                seed=seed * 1000 + instance, noise=noise, mach=mach)


def tgv_batch(count: int = 64, seed: int = 4, steps: int = 200):
    """count Taylor-Green instances whose edges are drawn from {48,64,80,96,128}."""
    rng = np.random.Generator(np.random.Philox(seed))
    edges = rng.choice([48, 64, 80, 96, 128], size=count)
    return [tgv(int(e), seed=seed, instance=i, steps=steps) for i, e in enumerate(edges)]


# --------------------------------------------------------- initial states

def initial_state(case: Case, window=None, cell_average: bool = False) -> np.ndarray:
    """Initial conserved state (5, nz, ny, nx) in float64 (or the sub-box
    window = (k0, k1, j0, j1, i0, i1) of it). cell_average=True returns exact
    cell averages for the density wave (used by the order-of-accuracy test)."""
    window = window or _full(case)
    z, y, x = _centres(case, window)
    shape = (window[1] - window[0], window[3] - window[2], window[5] - window[4])
    g = case.gamma
    ones = np.ones(shape)
    if case.name == "density_wave":
        amp = 0.2
        if cell_average:
            h = case.dx
            amp = 0.2 * math.sin(math.pi * h) / (math.pi * h)
        rho = (1.0 + amp * np.sin(2.0 * math.pi * x)) * ones
        if window != _full(case) and case.noise:
            raise ValueError("noisy cases are generated whole")
        rho = rho + _noise(case, shape)
        u = ones
        p = ones
        # E = p/(g-1) + rho u^2/2 is affine in rho, so cell averages carry over
        return np.stack([rho, rho * u, 0 * ones, 0 * ones, _e(p, rho, u * u, g)])
    if case.name == "blast":
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        s = 0.5 * (1.0 - np.tanh((r - 0.2) / case.dx))
        rho = 0.125 + (1.0 - 0.125) * s
        p = 0.1 + (1.0 - 0.1) * s
        if window != _full(case) and case.noise:
            raise ValueError("noisy cases are generated whole")
        rho = rho + _noise(case, shape)
        return np.stack([rho, 0 * ones, 0 * ones, 0 * ones, _e(p, rho, 0.0, g) * ones])
    if case.name == "sod":
        s = 0.5 * (1.0 - np.tanh((x - 0.5) / case.dx)) * ones
        rho = 0.125 + (1.0 - 0.125) * s
        p = 0.1 + (1.0 - 0.1) * s
        return np.stack([rho, 0 * ones, 0 * ones, 0 * ones, _e(p, rho, 0.0, g)])
    if case.name in ("plume", "jets4"):
        return jet_initial_state(case, window, np)
    if case.name == "tgv":
        k = 2.0 * math.pi
        m = case.mach
        p0 = 1.0 / (g * m * m)
        u = np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
        v = -np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
        p = p0 + (1.0 / 16.0) * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * k * z) + 2.0)
        if window != _full(case) and case.noise:
            raise ValueError("noisy cases are generated whole")
        rho = 1.0 + _noise(case, shape)
        return np.stack([rho * ones, rho * u, rho * v, 0 * ones, _e(p, rho, u * u + v * v, g)])
    raise ValueError(f"no initial state for case {case.name!r}")


def _jet_plane_fields(case: Case, y, x, xp):
    """Sum over jets of s_n (q_jet_n - q_ambient) on the (y, x) plane."""
    g = case.gamma
    amb_e = _e(1.0, 1.0, 0.0, g)
    d_rho = 0.0 * (x + y)
    d_mz = 0.0 * (x + y)
    d_e = 0.0 * (x + y)
    for (cx, cy, R, rho_j, w_j, p_j, edge) in case.jets:
        r = xp.sqrt((x - cx) ** 2 + (y - cy) ** 2)
        s = 0.5 * (1.0 - xp.tanh((r - R) / (edge * case.dx)))
        d_rho = d_rho + s * (rho_j - 1.0)
        d_mz = d_mz + s * (rho_j * w_j)
        d_e = d_e + s * (_e(p_j, rho_j, w_j * w_j, g) - amb_e)
    return d_rho, d_mz, d_e


def jet_initial_state(case: Case, window=None, xp=np, device=None, dtype=None):
    """Quiescent ambient (rho = 1, p = 1, u = 0) plus a short plug of jet gas
    at the inflow face: q = q_amb + f(z) sum_n s_n(r) (q_jet_n - q_amb), with
    s_n the same tanh radial profile as the inflow boundary and
    f(z) = (1 - tanh((z - 4 dx) / dx)) / 2. xp is numpy or torch (then the
    state is built on `device` in `dtype` without a host copy)."""
    window = window or _full(case)
    k0, k1, j0, j1, i0, i1 = window
    dx = case.dx
    if xp is np:
        x = ((np.arange(i0, i1) + 0.5) * dx)[None, :]
        y = ((np.arange(j0, j1) + 0.5) * dx)[:, None]
        z = ((np.arange(k0, k1) + 0.5) * dx)[:, None, None]
    else:
        f64 = xp.float64
        x = ((xp.arange(i0, i1, dtype=f64, device=device) + 0.5) * dx)[None, :]
        y = ((xp.arange(j0, j1, dtype=f64, device=device) + 0.5) * dx)[:, None]
        z = ((xp.arange(k0, k1, dtype=f64, device=device) + 0.5) * dx)[:, None, None]
    d_rho, d_mz, d_e = _jet_plane_fields(case, y, x, xp)
    f = 0.5 * (1.0 - xp.tanh((z - 4.0 * dx) / dx))
    amb_e = _e(1.0, 1.0, 0.0, case.gamma)
    rho = 1.0 + f * d_rho[None]
    mz = f * d_mz[None]
    e = amb_e + f * d_e[None]
    zero = 0.0 * rho
    q = xp.stack([rho, zero, zero, mz, e])
    if xp is not np and dtype is not None:
        q = q.to(dtype)
    return q
