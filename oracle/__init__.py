"""FP64 CPU oracle of the IGR Euler stage (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. It shares no code with the CUDA path; the two
meet only in the seeded initial states that both consume.

The arithmetic lives in ``igr_oracle.c`` (plain loops over ghost-cell
arrays, double precision, no contraction). This module only marshals numpy
arrays through ctypes. A grid description is any object with the attributes
``nx, ny, nz, dx, gamma, alpha, cfl, sweeps, bc`` (6 ints: 0 periodic,
1 outflow, 2 inflow, faces -x,+x,-y,+y,-z,+z) and ``jets`` (list of
``(cx, cy, radius, rho, w, p, edge_width)``), and optionally ``order`` (5 or 3)
``sigma_solver`` (0 Jacobi, 1 red-black Gauss-Seidel) and the viscosities
``mu``, ``zeta`` (0: Euler).
"""
import ctypes as C

import numpy as np

from .build import build

_lib = None


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("gamma", C.c_double), ("alpha", C.c_double),
                ("cfl", C.c_double), ("sweeps", C.c_int), ("bc", C.c_int * 6),
                ("njets", C.c_int), ("jets", C.POINTER(C.c_double)),
                ("order", C.c_int), ("sigma_solver", C.c_int),
                ("mu", C.c_double), ("zeta", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, p, g = C.c_double, C.c_void_p, C.POINTER(_Grid)
        sig = {
            "orc_fill_ghosts": (None, [g, p, p]),
            "orc_source": (None, [g, p, p]),
            "orc_apply_A": (None, [g, p, p, p]),
            "orc_jacobi": (None, [g, p, p, p, C.c_int]),
            "orc_rhs": (None, [g, p, p, p]),
            "orc_max_speed": (d, [g, p]),
            "orc_stage": (None, [g, p, p, p, p, d, d]),
            "orc_step": (d, [g, p, p, d]),
            "orc_run": (d, [g, p, p, C.c_int, d]),
            "orc_adjoint_step": (None, [g, p, p, d, p, p, p, p, p]),
            "orc_rhs_vjp": (None, [g, p, p, p, p, p]),
            "orc_source_vjp": (None, [g, p, p, p]),
            "orc_jacobi_vjp": (None, [g, p, p, p, C.c_int, p, p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


class Grid:
    """ctypes view of a grid description (keeps the jet table alive)."""

    def __init__(self, cfg):
        jets = np.ascontiguousarray(np.asarray(list(cfg.jets), dtype=np.float64).reshape(-1, 7))
        self._jets = jets
        self.nx, self.ny, self.nz = int(cfg.nx), int(cfg.ny), int(cfg.nz)
        self.s = _Grid(self.nx, self.ny, self.nz, float(cfg.dx), float(cfg.gamma),
                       float(cfg.alpha), float(cfg.cfl), int(cfg.sweeps),
                       (C.c_int * 6)(*[int(b) for b in cfg.bc]), int(jets.shape[0]),
                       jets.ctypes.data_as(C.POINTER(C.c_double)),
                       int(getattr(cfg, "order", 5)), int(getattr(cfg, "sigma_solver", 0)),
                       float(getattr(cfg, "mu", 0.0)), float(getattr(cfg, "zeta", 0.0)))

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def ptr(self):
        return C.byref(self.s)


def _grid(cfg):
    return cfg if isinstance(cfg, Grid) else Grid(cfg)


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != int(np.prod(shape)):
        raise ValueError(f"array of {a.size} values where {shape} was expected")
    return a


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def fill_ghosts(cfg, q):
    """Conserved state with 3 ghost layers: (5, nz+6, ny+6, nx+6)."""
    g = _grid(cfg)
    q = _f64(q, (5, g.n))
    out = np.empty((5, g.nz + 6, g.ny + 6, g.nx + 6))
    lib().orc_fill_ghosts(g.ptr, _p(q), _p(out))
    return out


def source(cfg, q):
    """IGR source b = alpha [tr((grad u)^2) + tr^2(grad u)], (nz, ny, nx)."""
    g = _grid(cfg)
    q = _f64(q, (5, g.n))
    b = np.empty((g.nz, g.ny, g.nx))
    lib().orc_source(g.ptr, _p(q), _p(b))
    return b


def apply_A(cfg, q, s):
    """The discrete elliptic operator applied to s: (A s), (nz, ny, nx)."""
    g = _grid(cfg)
    q = _f64(q, (5, g.n))
    s = _f64(s, (g.n,))
    out = np.empty((g.nz, g.ny, g.nx))
    lib().orc_apply_A(g.ptr, _p(q), _p(s), _p(out))
    return out


def jacobi(cfg, q, b, sigma, sweeps):
    """Jacobi sweeps on A sigma = b from the warm start sigma; returns a new array."""
    g = _grid(cfg)
    q = _f64(q, (5, g.n))
    b = _f64(b, (g.n,))
    s = np.array(_f64(sigma, (g.n,)), copy=True).reshape(g.nz, g.ny, g.nx)
    lib().orc_jacobi(g.ptr, _p(q), _p(b), _p(s), int(sweeps))
    return s


def rhs(cfg, q, sigma):
    """Spatial operator L(q; Sigma) with Sigma given, (5, nz, ny, nx)."""
    g = _grid(cfg)
    q = _f64(q, (5, g.n))
    s = _f64(sigma, (g.n,))
    out = np.empty((5, g.nz, g.ny, g.nx))
    lib().orc_rhs(g.ptr, _p(q), _p(s), _p(out))
    return out


def max_speed(cfg, q):
    g = _grid(cfg)
    return float(lib().orc_max_speed(g.ptr, _p(_f64(q, (5, g.n)))))


def stage(cfg, qs, qn, sigma, w, dt):
    """One RK stage; returns (out, sigma_after_solve)."""
    g = _grid(cfg)
    qs = _f64(qs, (5, g.n))
    qn = _f64(qn, (5, g.n))
    s = np.array(_f64(sigma, (g.n,)), copy=True).reshape(g.nz, g.ny, g.nx)
    out = np.empty((5, g.nz, g.ny, g.nx))
    lib().orc_stage(g.ptr, _p(qs), _p(qn), _p(s), _p(out), float(w), float(dt))
    return out, s


def run(cfg, q, sigma=None, nsteps=1, fixed_dt=0.0):
    """nsteps SSP-RK3 steps from (q, sigma); returns (q, sigma, t) as new arrays."""
    g = _grid(cfg)
    q = np.array(_f64(q, (5, g.n)), copy=True).reshape(5, g.nz, g.ny, g.nx)
    s = (np.zeros((g.nz, g.ny, g.nx)) if sigma is None
         else np.array(_f64(sigma, (g.n,)), copy=True).reshape(g.nz, g.ny, g.nx))
    t = lib().orc_run(g.ptr, _p(q), _p(s), int(nsteps), float(fixed_dt))
    return q, s, float(t)


def _jacobi5(cfg):
    """The adjoint is written for the default scheme: 5th-order faces, Jacobi."""
    if (getattr(cfg, "order", 5) != 5 or getattr(cfg, "sigma_solver", 0) != 0
            or getattr(cfg, "mu", 0.0) != 0.0 or getattr(cfg, "zeta", 0.0) != 0.0):
        raise ValueError("the adjoint covers the inviscid scheme with 5th-order faces and Jacobi sweeps only")


def adjoint_step(cfg, q, sigma, dt, lq, ls):
    """Adjoint of one SSP-RK3 step with fixed dt: given the adjoints (lq, ls)
    of the step's outputs (q', Sigma'), returns (lq_in, ls_in, gw) — the
    adjoints of (q, Sigma) and the gradient with respect to the jet
    velocities w_n of <lq, q'> + <ls, Sigma'>."""
    _jacobi5(cfg)
    g = _grid(cfg)
    if g.s.sweeps > 63:
        raise ValueError("at most 63 sweeps")
    q = _f64(q, (5, g.n))
    sig = _f64(sigma, (g.n,))
    lq = _f64(lq, (5, g.n))
    ls = _f64(ls, (g.n,))
    lq_out = np.empty((5, g.nz, g.ny, g.nx))
    ls_out = np.empty((g.nz, g.ny, g.nx))
    gw = np.zeros(max(1, g.s.njets))
    lib().orc_adjoint_step(g.ptr, _p(q), _p(sig), float(dt), _p(lq), _p(ls), _p(lq_out), _p(ls_out), _p(gw))
    return lq_out, ls_out, gw[:g.s.njets]


def rhs_vjp(cfg, q, sigma, Lb):
    """(dL/dq)^T Lb and (dL/dSigma)^T Lb of the spatial operator."""
    _jacobi5(cfg)
    g = _grid(cfg)
    qb = np.zeros((5, g.nz, g.ny, g.nx))
    sb = np.zeros((g.nz, g.ny, g.nx))
    lib().orc_rhs_vjp(g.ptr, _p(_f64(q, (5, g.n))), _p(_f64(sigma, (g.n,))), _p(_f64(Lb, (5, g.n))),
                      _p(qb), _p(sb))
    return qb, sb


def source_vjp(cfg, q, bb):
    """(db/dq)^T bb of the IGR source."""
    _jacobi5(cfg)
    g = _grid(cfg)
    qb = np.zeros((5, g.nz, g.ny, g.nx))
    lib().orc_source_vjp(g.ptr, _p(_f64(q, (5, g.n))), _p(_f64(bb, (g.n,))), _p(qb))
    return qb


def jacobi_vjp(cfg, q, b, sigma0, sweeps, sb):
    """Adjoints of (sigma0, b, rho) of `sweeps` Jacobi sweeps given the
    adjoint sb of their result."""
    _jacobi5(cfg)
    g = _grid(cfg)
    s = np.array(_f64(sb, (g.n,)), copy=True)
    bb = np.zeros(g.n)
    rb = np.zeros(g.n)
    lib().orc_jacobi_vjp(g.ptr, _p(_f64(q, (5, g.n))), _p(_f64(b, (g.n,))), _p(_f64(sigma0, (g.n,))),
                         int(sweeps), _p(s), _p(bb), _p(rb))
    shp = (g.nz, g.ny, g.nx)
    return s.reshape(shp), bb.reshape(shp), rb.reshape(shp)
