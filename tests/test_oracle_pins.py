"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
closed form, an invariant, a textbook solution or a brute-force solve.
A plausible slip anywhere in the oracle (a dropped term, a wrong sign,
index or weight, a transposed operand) fails at least one of these.
"""
import json
import math
import os
from dataclasses import replace

import numpy as np
import pytest

import oracle
from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import INFLOW, OUTFLOW, PERIODIC, Case

import sod_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 1.4


def cons(rho, u, v, w, p, g=GAMMA):
    return np.stack([rho, rho * u, rho * v, rho * w, p / (g - 1) + 0.5 * rho * (u * u + v * v + w * w)])


def box(n, bc, nx=None, ny=None, nz=None, alpha_scale=1.0, sweeps=5, jets=()):
    nx, ny, nz = nx or n, ny or n, nz or n
    dx = 1.0 / nx
    return Case("pin", nx, ny, nz, dx, alpha=alpha_scale * dx * dx, sweeps=sweeps, bc=tuple(bc),
                jets=list(jets))


def centres(c):
    z = (np.arange(c.nz) + 0.5) * c.dx
    y = (np.arange(c.ny) + 0.5) * c.dx
    x = (np.arange(c.nx) + 0.5) * c.dx
    return np.meshgrid(z, y, x, indexing="ij")


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("bc", [(PERIODIC,) * 6, (OUTFLOW,) * 6,
                                (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, PERIODIC)])
def test_uniform_state_preserved_bitwise(bc):
    """Identical face states give identical fluxes: dq/dt = 0 exactly, grad u = 0
    gives b = 0 and Sigma stays 0; the increment-form RK keeps q bit-identical."""
    c = box(6, bc, nx=7, ny=6, nz=5)
    shape = (c.nz, c.ny, c.nx)
    q = cons(np.full(shape, 1.3), np.full(shape, 0.7), np.full(shape, -0.4),
             np.full(shape, 0.25), np.full(shape, 2.1))
    q1, s1, t = oracle.run(c, q, None, nsteps=10)
    assert np.array_equal(q1, q)
    assert np.all(s1 == 0.0)
    assert t > 0


def test_periodic_conservation():
    """Flux form with periodic faces: totals of rho, m, E change only by
    round-off, with a non-trivial Sigma."""
    c = box(16, (PERIODIC,) * 6)
    z, y, x = centres(c)
    tp = 2 * np.pi
    rho = 1 + 0.2 * np.sin(tp * x) * np.cos(tp * y) + 0.1 * np.sin(tp * z)
    u = 0.5 * np.sin(tp * y)
    v = 0.3 * np.cos(tp * x) * np.sin(tp * z)
    w = -0.4 * np.sin(tp * x)
    p = 1 + 0.1 * np.cos(tp * (x + y))
    q = cons(rho, u, v, w, p)
    q1, s1, _ = oracle.run(c, q, None, nsteps=10)
    assert np.abs(s1).max() > 1e-6        # Sigma is active
    tot0 = q.reshape(5, -1).sum(axis=1)
    tot1 = q1.reshape(5, -1).sum(axis=1)
    scale = np.abs(q).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale)


def test_sigma_zero_for_uniform_velocity():
    """grad u = 0 (variable density, uniform velocity, exact m/rho) gives
    b = 0 and Sigma = 0 exactly (Eq. igrelliptic with zero left side)."""
    c = box(8, (OUTFLOW,) * 6)
    z, y, x = centres(c)
    rho = 1 + 0.3 * np.sin(5 * x + 3 * y) * np.cos(2 * z)
    q = cons(rho, 1.0 + 0 * rho, 0.5 + 0 * rho, -0.25 + 0 * rho, 1 + 0 * rho)
    assert np.all(oracle.source(c, q) == 0.0)
    s = oracle.jacobi(c, q, oracle.source(c, q), np.zeros(c.ncells), 7)
    assert np.all(s == 0.0)


def test_source_for_linear_velocity():
    """Linear u = G x: central differences are exact, so at cells away from
    the boundary b = alpha [tr(G G) + tr(G)^2] with tr(G G) = sum G_ab G_ba
    (not sum G_ab^2: the off-diagonal product distinguishes the two)."""
    c = box(8, (OUTFLOW,) * 6, alpha_scale=0.7)
    z, y, x = centres(c)
    Gm = np.array([[0.3, 2.0, 0.0], [-1.0, 0.5, 0.2], [0.1, 0.0, -0.7]])
    X = [x, y, z]
    u = [sum(Gm[a, b] * X[b] for b in range(3)) for a in range(3)]
    q = cons(1 + 0 * x, u[0], u[1], u[2], 5 + 0 * x)
    b = oracle.source(c, q)
    expect = c.alpha * (np.trace(Gm @ Gm) + np.trace(Gm) ** 2)
    inner = b[1:-1, 1:-1, 1:-1]
    assert np.allclose(inner, expect, rtol=1e-11, atol=0)
    assert not np.isclose(expect, c.alpha * (np.sum(Gm * Gm) + np.trace(Gm) ** 2))


def test_source_for_quadratic_velocity():
    """Quadratic u: the central difference (u(x+h) - u(x-h)) / (2h) is still
    exact at the cell centre, while a one-sided difference would be off by
    O(h), which the linear field above cannot reveal. With
    u = (x^2, x y, z^2 / 2) (rho = 1) the gradient at a centre is
    G = [[2x, 0, 0], [y, x, 0], [0, 0, z]], so
    b = alpha [4x^2 + x^2 + z^2 + (3x + z)^2]."""
    c = box(9, (OUTFLOW,) * 6, alpha_scale=0.4)
    z, y, x = centres(c)
    q = cons(1 + 0 * x, x * x, x * y, 0.5 * z * z, 5 + 0 * x)
    b = oracle.source(c, q)
    expect = c.alpha * (4 * x * x + x * x + z * z + (3 * x + z) ** 2)
    assert np.allclose(b[1:-1, 1:-1, 1:-1], expect[1:-1, 1:-1, 1:-1], rtol=1e-11, atol=1e-14)


# ------------------------------------------------------- elliptic solve

@pytest.mark.parametrize("alpha_scale", [1.0, 0.3])
def test_jacobi_fourier_mode_decay(alpha_scale):
    """Uniform rho, b = 0, periodic: one Jacobi sweep multiplies the mode
    cos(k.x) by beta * 2 sum_d cos(theta_d) / (1 + 6 beta), beta = alpha/dx^2."""
    c = box(8, (PERIODIC,) * 6, alpha_scale=alpha_scale)
    z, y, x = centres(c)
    kk = 2 * np.pi * np.array([1, 2, 3])
    s0 = np.cos(kk[0] * x + kk[1] * y + kk[2] * z)
    q = cons(2.0 + 0 * x, 0 * x, 0 * x, 0 * x, 1 + 0 * x)
    s1 = oracle.jacobi(c, q, np.zeros(c.ncells), s0, 1)
    beta = alpha_scale
    fac = beta * 2 * np.sum(np.cos(kk * c.dx)) / (1 + 6 * beta)
    assert np.allclose(s1, fac * s0, rtol=0, atol=1e-14)


def test_sigma_solve_closed_form():
    """Uniform rho0, b = cos(k.x): Sigma = rho0 b / (1 + beta sum_d 2 (1 - cos theta_d))."""
    c = box(8, (PERIODIC,) * 6)
    z, y, x = centres(c)
    kk = 2 * np.pi * np.array([2, 1, 3])
    rho0 = 1.7
    b = np.cos(kk[0] * x + kk[1] * y + kk[2] * z)
    q = cons(rho0 + 0 * x, 0 * x, 0 * x, 0 * x, 1 + 0 * x)
    s = oracle.jacobi(c, q, b, np.zeros(c.ncells), 600)
    expect = rho0 * b / (1 + np.sum(2 * (1 - np.cos(kk * c.dx))))
    assert np.allclose(s, expect, rtol=0, atol=1e-13)


def _dense_A(c, q):
    n = c.ncells
    A = np.empty((n, n))
    e = np.zeros(n)
    for m in range(n):
        e[:] = 0
        e[m] = 1
        A[:, m] = oracle.apply_A(c, q, e).ravel()
    return A


@pytest.mark.parametrize("n", [4, 5, 6])
@pytest.mark.parametrize("bc", [(PERIODIC,) * 6, (OUTFLOW,) * 6,
                                (PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, INFLOW, OUTFLOW)])
def test_sigma_vs_dense_direct_solve(n, bc):
    """The assembled operator is symmetric positive definite with a 7-point
    sparsity pattern and non-positive off-diagonals; converged Jacobi sweeps
    match a dense direct solve."""
    c = box(n, bc)
    rng = np.random.Generator(np.random.Philox(11))
    rho = rng.uniform(0.5, 2.0, size=(n, n, n))
    q = cons(rho, 0 * rho, 0 * rho, 0 * rho, 1 + 0 * rho)
    A = _dense_A(c, q)
    assert np.array_equal(A, A.T) or np.max(np.abs(A - A.T)) <= 1e-15 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    assert np.all((A != 0).sum(axis=1) <= 7)
    assert np.allclose(np.diag(A), np.diag(A))  # finite
    b = rng.uniform(-1, 1, size=c.ncells)
    direct = np.linalg.solve(A, b)
    s = oracle.jacobi(c, q, b, np.zeros(c.ncells), 3000)
    assert np.max(np.abs(s.ravel() - direct)) <= 1e-12 * np.max(np.abs(direct))


def test_elliptic_operator_second_order_consistent():
    """Manufactured check of the variable-coefficient operator: for smooth
    rho(x), Sigma(x) (periodic, fixed alpha) the discrete A Sigma converges at
    second order to Sigma/rho - alpha d/dx(Sigma'/rho)."""
    alpha = 0.01
    errs = []
    for n in (32, 64, 128):
        c = box(n, (PERIODIC,) * 6, nx=n, ny=2, nz=2)
        c = replace(c, alpha=alpha)
        z, y, x = centres(c)
        tp = 2 * np.pi
        rho = 1 + 0.5 * np.sin(tp * x)
        drho = 0.5 * tp * np.cos(tp * x)
        S = np.cos(tp * x)
        dS = -tp * np.sin(tp * x)
        d2S = -tp * tp * np.cos(tp * x)
        exact = S / rho - alpha * (d2S / rho - dS * drho / rho ** 2)
        q = cons(rho, 0 * x, 0 * x, 0 * x, 1 + 0 * x)
        errs.append(np.max(np.abs(oracle.apply_A(c, q, S) - exact)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.85), orders


# ---------------------------------------------------- reconstruction / flux

def _quartic_avg(coef, xl, xr):
    """Exact cell average of sum coef[m] x^m over [xl, xr]."""
    prim = lambda x: sum(cf * x ** (m + 1) / (m + 1) for m, cf in enumerate(coef))
    return (prim(xr) - prim(xl)) / (xr - xl)


def _poly(coef, x):
    return sum(cf * x ** m for m, cf in enumerate(coef))


def test_sigma_flux_exact_for_quartic_sigma():
    """u = 0, uniform rho and p, Sigma = cell averages of a quartic P(x):
    both 5th-order face values equal P at the face, so away from the
    boundary rhs(m_x) = -(P(x_{i+1/2}) - P(x_{i-1/2})) / dx, and Sigma drives
    nothing else (u = 0 makes the mass and energy fluxes vanish)."""
    n = 16
    c = box(n, (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC), nx=n, ny=3, nz=2)
    coef = [0.3, -1.1, 2.5, 0.7, -1.9]
    xf = np.arange(n + 1) * c.dx
    sig_row = np.array([_quartic_avg(coef, xf[i], xf[i + 1]) for i in range(n)])
    sig = np.broadcast_to(sig_row, (c.nz, c.ny, n)).copy()
    shape = (c.nz, c.ny, n)
    q = cons(np.full(shape, 1.2), np.zeros(shape), np.zeros(shape), np.zeros(shape), np.full(shape, 0.9))
    L = oracle.rhs(c, q, sig)
    inner = slice(3, n - 3)
    expect = -(_poly(coef, xf[1:]) - _poly(coef, xf[:-1])) / c.dx
    assert np.allclose(L[1][..., inner], expect[inner], rtol=1e-11, atol=1e-11)
    for v in (0, 2, 3, 4):
        assert np.max(np.abs(L[v])) <= 1e-11


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_face_states_exact_for_quartic_density(axis):
    """u = 0, uniform p, rho = cell averages of a quartic along one axis: the
    left- and right-biased face values both equal rho at the face, so the LF
    jump term vanishes and L = 0 away from the boundary in that axis. A wrong
    weight in either one-sided formula breaks the equality."""
    n = 16
    dims = [3, 3, 3]
    dims[axis] = n
    bc = [PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = OUTFLOW
    c = Case("pin", dims[0], dims[1], dims[2], 1.0 / n, alpha=1.0 / n ** 2, bc=tuple(bc))
    coef = [1.0, 0.4, -0.3, 0.2, 0.1]
    xf = np.arange(n + 1) * c.dx
    row = np.array([_quartic_avg(coef, xf[i], xf[i + 1]) for i in range(n)])
    shape = (c.nz, c.ny, c.nx)
    bshape = [1, 1, 1]
    bshape[2 - axis] = n
    rho = np.broadcast_to(row.reshape(bshape), shape).copy()
    q = cons(rho, 0 * rho, 0 * rho, 0 * rho, 1 + 0 * rho)
    L = oracle.rhs(c, q, np.zeros(shape))
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(3, n - 3)
    assert np.max(np.abs(L[(slice(None),) + tuple(sl)])) <= 1e-12


@pytest.mark.parametrize("axis", [0, 2])
def test_third_order_faces_exact_for_quadratic_only(axis):
    """3rd-order faces (Sec. "Discretization": third- or fifth-order finite
    volumes): rho = cell averages of a quadratic along one axis gives equal
    left/right face values at every face, hence L = 0 away from the boundary;
    a quartic does not (the 5th-order weights would still be exact there)."""
    n = 16
    dims = [3, 3, 3]
    dims[axis] = n
    bc = [PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = OUTFLOW
    c = Case("pin", dims[0], dims[1], dims[2], 1.0 / n, alpha=1.0 / n ** 2, bc=tuple(bc), order=3)
    xf = np.arange(n + 1) * c.dx
    shape = (c.nz, c.ny, c.nx)
    bshape = [1, 1, 1]
    bshape[2 - axis] = n
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(3, n - 3)
    out = []
    for coef in ([1.0, 0.4, -0.3], [1.0, 0.4, -0.3, 0.2, 0.9]):
        row = np.array([_quartic_avg(coef, xf[i], xf[i + 1]) for i in range(n)])
        rho = np.broadcast_to(row.reshape(bshape), shape).copy()
        q = cons(rho, 0 * rho, 0 * rho, 0 * rho, 1 + 0 * rho)
        L = oracle.rhs(c, q, np.zeros(shape))
        out.append(np.max(np.abs(L[(slice(None),) + tuple(sl)])))
    assert out[0] <= 1e-12, out
    assert out[1] > 1e-6, out


@pytest.mark.parametrize("alpha_scale", [1.0, 0.3])
def test_red_black_gauss_seidel_closed_form(alpha_scale):
    """Red-black Gauss-Seidel (Sec. "Discretization": Jacobi or Gauss-Seidel)
    on a periodic box of even size with rho = 1, b = 0, Sigma = 1: every red
    update multiplies the (uniform) black values by l = 6 beta / (1 + 6 beta)
    and every black update the red ones, so after n sweeps red cells hold
    l^(2n-1) and black cells l^(2n) (Jacobi gives l^n everywhere). beta =
    alpha / dx^2 other than 1 as well, where a beta dropped from the
    diagonal would show."""
    c = box(8, (PERIODIC,) * 6, nx=8, ny=6, nz=4, alpha_scale=alpha_scale)
    c = replace(c, sigma_solver=1)
    beta = c.alpha / c.dx ** 2
    lam = 6 * beta / (1 + 6 * beta)
    shape = (c.nz, c.ny, c.nx)
    q = cons(np.ones(shape), np.zeros(shape), np.zeros(shape), np.zeros(shape), np.ones(shape))
    z, y, x = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    red = (x + y + z) % 2 == 0
    for n in (1, 2, 3):
        s = oracle.jacobi(c, q, np.zeros(shape), np.ones(shape), n)
        assert np.allclose(s[red], lam ** (2 * n - 1), rtol=1e-14, atol=0)
        assert np.allclose(s[~red], lam ** (2 * n), rtol=1e-14, atol=0)
    sj = oracle.jacobi(replace(c, sigma_solver=0), q, np.zeros(shape), np.ones(shape), 3)
    assert np.allclose(sj, lam ** 3, rtol=1e-14, atol=0)


@pytest.mark.parametrize("alpha_scale", [1.0, 0.3])
@pytest.mark.parametrize("bc", [(OUTFLOW,) * 6, (PERIODIC,) * 4 + (OUTFLOW,) * 2])
def test_red_black_gauss_seidel_converges_to_direct_solve(bc, alpha_scale):
    """Red-black sweeps reach the dense direct solve of A Sigma = b (A
    assembled from the oracle's operator), and faster than Jacobi."""
    c = box(6, bc, nx=6, ny=4, nz=6, alpha_scale=alpha_scale)
    rng = np.random.Generator(np.random.Philox(5))
    shape = (c.nz, c.ny, c.nx)
    rho = 1 + 0.3 * rng.uniform(-1, 1, shape)
    q = cons(rho, np.zeros(shape), np.zeros(shape), np.zeros(shape), np.ones(shape))
    n = rho.size
    A = np.stack([oracle.apply_A(c, q, np.eye(n)[k]).ravel() for k in range(n)], 1)
    b = rng.normal(size=n)
    exact = np.linalg.solve(A, b).reshape(shape)
    gs = replace(c, sigma_solver=1)
    s = oracle.jacobi(gs, q, b.reshape(shape), np.zeros(shape), 400)
    assert np.max(np.abs(s - exact)) <= 1e-12 * np.max(np.abs(exact))
    for sweeps in (2, 5, 10):
        e_gs = np.linalg.norm(oracle.jacobi(gs, q, b.reshape(shape), np.zeros(shape), sweeps) - exact)
        e_j = np.linalg.norm(oracle.jacobi(c, q, b.reshape(shape), np.zeros(shape), sweeps) - exact)
        assert e_gs < e_j, (sweeps, e_gs, e_j)


def _visc_rhs(c, q):
    """Viscous part of L: L(mu, zeta) - L(0, 0) on the same state, Sigma = 0."""
    z = np.zeros((c.nz, c.ny, c.nx))
    return oracle.rhs(c, q, z) - oracle.rhs(replace(c, mu=0.0, zeta=0.0), q, z)


def test_viscous_shear_wave_closed_form():
    """u = (0, v(x), 0), rho = 1, p = 1 (Eq. constitutive_law, compact face
    stencil): only tau_xy = mu dv/dx acts, so the viscous rates are exactly
    m_y: mu (v[i+1] - 2 v[i] + v[i-1]) / dx^2 and
    E:   mu (v[i+1]^2 - 2 v[i]^2 + v[i-1]^2) / (2 dx^2)
    (the work term u . tau with the face velocity (v[i] + v[i+1]) / 2);
    mass and the other momenta get nothing."""
    n = 24
    c = replace(box(n, (PERIODIC,) * 6, nx=n, ny=4, nz=3), mu=0.013)
    x = (np.arange(n) + 0.5) / n
    v1 = 0.3 * np.sin(2 * np.pi * x) + 0.1 * np.cos(6 * np.pi * x)
    shape = (c.nz, c.ny, n)
    v = np.broadcast_to(v1, shape)
    q = cons(np.ones(shape), np.zeros(shape), v, np.zeros(shape), np.ones(shape))
    L = _visc_rhs(c, q)
    dx2 = c.dx ** 2
    vp, vm = np.roll(v1, -1), np.roll(v1, 1)
    assert np.allclose(L[2], c.mu * (vp - 2 * v1 + vm) / dx2, rtol=0, atol=1e-12)
    assert np.allclose(L[4], c.mu * (vp ** 2 - 2 * v1 ** 2 + vm ** 2) / (2 * dx2), rtol=0, atol=1e-12)
    for f in (0, 1, 3):
        assert np.max(np.abs(L[f])) <= 1e-12


def test_viscous_longitudinal_wave_closed_form():
    """u = (u(x), 0, 0): tau_xx = (4 mu / 3 + zeta) du/dx (Stokes' form of the
    normal stress), so m_x gains (4 mu/3 + zeta)(u[i+1] - 2u[i] + u[i-1]) / dx^2
    and E the matching work term; separate mu and zeta pin both factors."""
    n = 20
    for mu, zeta in ((0.01, 0.0), (0.0, 0.02), (0.007, 0.015)):
        c = replace(box(n, (PERIODIC,) * 6, nx=n, ny=3, nz=4), mu=mu, zeta=zeta)
        x = (np.arange(n) + 0.5) / n
        u1 = 0.2 * np.sin(2 * np.pi * x + 0.3)
        shape = (c.nz, c.ny, n)
        u = np.broadcast_to(u1, shape)
        q = cons(np.ones(shape), u, np.zeros(shape), np.zeros(shape), np.ones(shape))
        L = _visc_rhs(c, q)
        k = 4 * mu / 3 + zeta
        up, um = np.roll(u1, -1), np.roll(u1, 1)
        dx2 = c.dx ** 2
        assert np.allclose(L[1], k * (up - 2 * u1 + um) / dx2, rtol=0, atol=1e-12), (mu, zeta)
        assert np.allclose(L[4], k * (up ** 2 - 2 * u1 ** 2 + um ** 2) / (2 * dx2), rtol=0, atol=1e-12)
        for f in (0, 2, 3):
            assert np.max(np.abs(L[f])) <= 1e-12


def test_viscous_operator_second_order():
    """A smooth periodic 3D flow with variable density: the viscous part of L
    converges at second order to div tau and div (u . tau) of Eq.
    (constitutive_law), differentiated symbolically (every tangential and
    divergence term enters)."""
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("x y z")
    tp = 2 * sp.pi
    mu, zeta = 0.011, 0.023
    rho = 1 + 0.2 * sp.sin(tp * (X + Y)) * sp.cos(tp * Z)
    u = [0.3 * sp.sin(tp * Y) * sp.cos(tp * Z) + 0.1 * sp.cos(tp * X),
         0.25 * sp.sin(tp * Z) * sp.cos(tp * X),
         0.2 * sp.cos(tp * (X + Y)) + 0.1 * sp.sin(tp * Z)]
    xs = (X, Y, Z)
    Gr = [[sp.diff(u[a], xs[b]) for b in range(3)] for a in range(3)]
    div = Gr[0][0] + Gr[1][1] + Gr[2][2]
    tau = [[mu * (Gr[a][b] + Gr[b][a]) + (zeta - 2 * mu / 3) * div * (1 if a == b else 0)
            for b in range(3)] for a in range(3)]
    rhs_m = [sum(sp.diff(tau[a][b], xs[b]) for b in range(3)) for a in range(3)]
    rhs_E = sum(sp.diff(sum(u[a] * tau[a][b] for a in range(3)), xs[b]) for b in range(3))
    fr = sp.lambdify(xs, rho, "numpy")
    fu = [sp.lambdify(xs, e, "numpy") for e in u]
    fm = [sp.lambdify(xs, e, "numpy") for e in rhs_m]
    fE = sp.lambdify(xs, rhs_E, "numpy")
    errs = []
    for n in (16, 32):
        c = replace(box(n, (PERIODIC,) * 6, nx=n, ny=n, nz=n), mu=mu, zeta=zeta)
        z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) / n] * 3, indexing="ij")
        r = fr(x, y, z)
        uu = [fu[a](x, y, z) * np.ones_like(x) for a in range(3)]
        q = cons(r, uu[0], uu[1], uu[2], np.ones_like(x))
        L = _visc_rhs(c, q)
        e = [np.max(np.abs(L[1 + a] - fm[a](x, y, z))) for a in range(3)]
        e.append(np.max(np.abs(L[4] - fE(x, y, z))))
        assert np.max(np.abs(L[0])) <= 1e-12
        errs.append(np.array(e))
    orders = np.log2(errs[0] / errs[1])
    assert np.all(orders > 1.8) and np.all(orders < 2.4), (errs, orders)


def test_time_step_rule():
    """dt = cfl dx / max_d(|u_d| + c): rho = 1.4, p = 1 gives c = 1; with
    u = (0.5, -2, 1) the maximum is 3."""
    c = box(5, (PERIODIC,) * 6)
    shape = (5, 5, 5)
    q = cons(np.full(shape, 1.4), np.full(shape, 0.5), np.full(shape, -2.0), np.full(shape, 1.0),
             np.full(shape, 1.0))
    assert math.isclose(oracle.max_speed(c, q), 3.0, rel_tol=1e-15)
    _, _, t = oracle.run(c, q, None, nsteps=1)
    assert math.isclose(t, 0.4 * c.dx / 3.0, rel_tol=1e-15)


def test_inflow_ghost_blend():
    """Inflow ghosts on -z: (1 - sum s) q_interior + sum s q_jet with
    s = (1 - tanh((r - R)/(w dx)))/2: s = 1/2 exactly at r = R, the jet state
    deep inside, the interior state far away; periodic/outflow elsewhere."""
    n = 12
    dx = 1.0 / n
    jet = (4.5 * dx, 5.5 * dx, 2.0 * dx, 0.8, 3.0, 2.0, 1.0)  # centred on cell (4, 5)
    c = Case("pin", n, n, 6, dx, alpha=dx * dx,
             bc=(OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW, INFLOW, OUTFLOW), jets=[jet])
    shape = (c.nz, c.ny, c.nx)
    rng = np.random.Generator(np.random.Philox(5))
    rho = rng.uniform(0.9, 1.1, size=shape)
    q = cons(rho, 0.1 + 0 * rho, 0 * rho, 0.2 + 0 * rho, 1 + 0 * rho)
    qg = oracle.fill_ghosts(c, q)
    qj = np.array([0.8, 0.0, 0.0, 0.8 * 3.0, 2.0 / 0.4 + 0.5 * 0.8 * 9.0])
    G = 3
    for layer in (0, 1, 2):  # ghost planes k = -3, -2, -1
        at = lambda i, j: qg[:, layer, j + G, i + G]
        inner = lambda i, j: q[:, 0, j, i]
        # r = R at cell (6, 5): s = 1/2
        assert np.allclose(at(6, 5), 0.5 * inner(6, 5) + 0.5 * qj, rtol=1e-15, atol=1e-15)
        # centre: s = (1 - tanh(-2))/2
        s = 0.5 * (1 - math.tanh(-2.0))
        assert np.allclose(at(4, 5), (1 - s) * inner(4, 5) + s * qj, rtol=1e-14)
        # far corner, r - R = 6.6 dx: s < exp(-13.2), essentially the interior
        assert np.allclose(at(11, 0), inner(11, 0), rtol=0, atol=1e-5 * np.abs(qj).max())
    # +z outflow copies the last plane; x faces copy the edge column
    assert np.array_equal(qg[:, c.nz + G, G:-G, G:-G], q[:, -1])
    assert np.array_equal(qg[:, G:-G, G:-G, 0], q[:, :, :, 0])


@pytest.mark.parametrize("xbc", ["outflow", "periodic"])
def test_inflow_corner_ghost_blend(xbc):
    """Inflow ghosts below the -z face whose column lies outside the face's
    x/y extent (the corner blocks the viscous tangential stencils read). The
    reading: such a ghost is the blend of the face cell its column maps to
    (clamp on an outflow axis, wrap on a periodic one), taken with that face
    cell's own weight s, i.e. ghost(i, j) = ghost(map(i), map(j)).
    Jet centred on cell (1, 5) with R = 2 dx and one-cell edges, so the
    weights are hand-computable: the clamped column i = -1..-3 maps to cell 0,
    at r = dx, r - R = -dx, s = (1 - tanh(-1))/2; the wrapped column i = -2
    of a 12-cell periodic axis maps to cell 10, at r = 9 dx, s = (1 - tanh(7))/2.
    Blending with the unmapped ghost coordinate (x = -1.5 dx: r = 3 dx,
    s = (1 - tanh(1))/2) fails both."""
    n = 12
    dx = 1.0 / n
    jet = (1.5 * dx, 5.5 * dx, 2.0 * dx, 0.8, 3.0, 2.0, 1.0)
    xb = OUTFLOW if xbc == "outflow" else PERIODIC
    c = Case("pin", n, n, 6, dx, alpha=dx * dx, bc=(xb, xb, OUTFLOW, OUTFLOW, INFLOW, OUTFLOW), jets=[jet])
    shape = (c.nz, c.ny, c.nx)
    rng = np.random.Generator(np.random.Philox(6))
    rho = rng.uniform(0.9, 1.1, size=shape)
    q = cons(rho, 0.1 + 0 * rho, -0.05 + 0 * rho, 0.2 + 0 * rho, rng.uniform(0.9, 1.1, size=shape))
    qg = oracle.fill_ghosts(c, q)
    qj = np.array([0.8, 0.0, 0.0, 0.8 * 3.0, 2.0 / 0.4 + 0.5 * 0.8 * 9.0])
    G = 3
    at = lambda layer, i, j: qg[:, layer, j + G, i + G]
    blend = lambda s, face: (1 - s) * face + s * qj
    for layer in (0, 1, 2):
        if xbc == "outflow":
            s = 0.5 * (1 - math.tanh(-1.0))  # face cell (0, 5): r - R = -dx
            for i in (-1, -2, -3):
                assert np.allclose(at(layer, i, 5), blend(s, q[:, 0, 5, 0]), rtol=1e-14, atol=0)
            # corner column (-1, -1) -> face cell (0, 0): r = sqrt(26) dx
            s00 = 0.5 * (1 - math.tanh(math.sqrt(26.0) - 2.0))
            assert np.allclose(at(layer, -1, -1), blend(s00, q[:, 0, 0, 0]), rtol=1e-14, atol=0)
        else:
            s = 0.5 * (1 - math.tanh(7.0))  # face cell (10, 5): r = 9 dx
            assert np.allclose(at(layer, -2, 5), blend(s, q[:, 0, 5, 10]), rtol=1e-14, atol=0)
            # the +x ghost column 12 wraps to cell 0: r - R = -dx
            s0 = 0.5 * (1 - math.tanh(-1.0))
            assert np.allclose(at(layer, 12, 5), blend(s0, q[:, 0, 5, 0]), rtol=1e-14, atol=0)


# ---------------------------------------------------- convergence and symmetry

@pytest.mark.slow
def test_density_wave_design_order():
    """Smooth density wave advected one period at u = 1, p = 1 (grad u = 0, so
    Sigma = 0): with dt ~ dx^(5/3) the 3rd-order RK error matches the 5th-order
    spatial error and the L1 error of rho falls at order close to 5."""
    errs = []
    for n in (16, 32, 64):
        c = inputs.density_wave(n, noise=0.0, ny=3, nz=3)
        q0 = inputs.initial_state(c, cell_average=True)
        dt_target = 0.15 * c.dx * (16.0 * c.dx) ** (2.0 / 3.0)
        steps = int(math.ceil(1.0 / dt_target))
        q1, s1, t = oracle.run(c, q0, None, nsteps=steps, fixed_dt=1.0 / steps)
        assert math.isclose(t, 1.0, rel_tol=1e-12)
        errs.append(np.mean(np.abs(q1[0] - q0[0])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.5), (errs, orders)


@pytest.mark.slow
def test_density_wave_design_order_third_order_faces():
    """The same wave with 3rd-order faces and dt ~ dx: both the spatial and
    the temporal error are 3rd order, so the L1 error falls at order ~3."""
    errs = []
    for n in (16, 32, 64):
        c = replace(inputs.density_wave(n, noise=0.0, ny=3, nz=3), order=3)
        q0 = inputs.initial_state(c, cell_average=True)
        steps = int(math.ceil(1.0 / (0.3 * c.dx)))
        q1, s1, t = oracle.run(c, q0, None, nsteps=steps, fixed_dt=1.0 / steps)
        errs.append(np.mean(np.abs(q1[0] - q0[0])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 2.7) and np.all(orders < 3.5), (errs, orders)


@pytest.mark.slow
def test_sod_converges_to_exact_solution():
    """Quasi-1D Sod tube at t = 0.2: the L1 error of rho against the exact
    Riemann solution falls with resolution at a rate of at least 0.6."""
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    errs = []
    for n in (100, 200, 400):
        c = inputs.sod(n)
        q0 = inputs.initial_state(c)
        steps = int(math.ceil(0.2 / (0.4 * c.dx / 2.0)))
        q1, _, t = oracle.run(c, q0, None, nsteps=steps, fixed_dt=0.2 / steps)
        x = (np.arange(n) + 0.5) * c.dx
        ex = sod_exact.sample(L, R, x, 0.2)
        rho = q1[0].mean(axis=(0, 1))
        assert np.all(np.isfinite(q1))
        assert np.max(np.abs(q1[0] - q1[0][:1, :1, :])) <= 1e-12  # stays 1D
        errs.append(np.mean(np.abs(rho - ex[0])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.01, errs
    assert np.all(orders > 0.6), (errs, orders)


def test_exact_riemann_solver_matches_textbook_star_state():
    """The test helper itself is pinned to the published Sod star state."""
    g = json.load(open(os.path.join(GOLDEN, "sod_star_state.json")))
    L = (g["left"]["rho"], g["left"]["u"], g["left"]["p"])
    R = (g["right"]["rho"], g["right"]["u"], g["right"]["p"])
    p, u, rl, rr = sod_exact.star_state(L, R, g["gamma"])
    tol = 0.5 * 10.0 ** -g["digits"]
    assert abs(p - g["p_star"]) <= tol
    assert abs(u - g["u_star"]) <= tol
    assert abs(rl - g["rho_star_left"]) <= tol
    assert abs(rr - g["rho_star_right"]) <= tol


def test_blast_mirror_symmetry():
    """The noise-free spherical blast stays symmetric under x -> 1 - x (and
    y, z): rho even, the normal momentum odd."""
    c = inputs.blast(20, noise=0.0, sweeps=10)
    q0 = inputs.initial_state(c)
    q1, s1, _ = oracle.run(c, q0, None, nsteps=5)
    assert np.abs(s1).max() > 0
    for ax, mv in ((3, 1), (2, 2), (1, 3)):
        flip = lambda a: np.flip(a, axis=ax - 1)
        assert np.allclose(q1[0], flip(q1[0]), rtol=0, atol=1e-13)
        assert np.allclose(q1[4], flip(q1[4]), rtol=0, atol=1e-13)
        assert np.allclose(q1[mv], -flip(q1[mv]), rtol=0, atol=1e-13)
        assert np.allclose(s1, np.flip(s1, axis=ax - 1), rtol=0, atol=1e-13)


# ------------------------------------------------------------- adjoint

def _offset_state(c, seed):
    """Smooth state whose velocity components stay away from zero (|u| has a
    kink at 0 that central differences would straddle)."""
    rng = np.random.Generator(np.random.Philox(seed))
    z, y, x = centres(c)
    ph = rng.uniform(0, 2 * np.pi, size=8)
    tp = 2 * np.pi
    rho = 1 + 0.2 * np.sin(tp * x + ph[0]) * np.cos(tp * y + ph[1]) + 0.1 * np.sin(tp * z + ph[2])
    u = 0.45 + 0.2 * np.sin(tp * y + ph[3])
    v = -0.4 + 0.15 * np.cos(tp * x + ph[4]) * np.sin(tp * z)
    w = 0.42 + 0.2 * np.sin(tp * x + ph[5])
    p = 1 + 0.1 * np.cos(tp * (x + y) + ph[6])
    return cons(rho, u, v, w, p)


def _fd_agrees(fd_at, ad, hs=(1e-6, 3e-7), tol=1e-6):
    """The adjoint against central differences: the LF speed max(aL, aR) is
    only piecewise smooth, so take the better of two small steps."""
    errs = [abs(fd_at(h) - ad) / abs(ad) for h in hs]
    return min(errs) <= tol, errs


@pytest.mark.parametrize("bc", [(PERIODIC,) * 6, (OUTFLOW,) * 6])
def test_adjoint_parts_match_finite_differences(bc):
    """Vector-Jacobian products of the spatial operator, the source and the
    Jacobi sweeps against central differences of the pinned forward maps."""
    c = box(8, bc, nx=8, ny=7, nz=6, sweeps=3)
    rng = np.random.Generator(np.random.Philox(7))
    q = _offset_state(c, 2)
    s = 0.05 * np.sin(2 * np.pi * centres(c)[2] * 3)
    vq, vs = rng.normal(size=q.shape), rng.normal(size=s.shape)
    Lb = rng.normal(size=q.shape)
    qb, sb = oracle.rhs_vjp(c, q, s, Lb)
    ok, errs = _fd_agrees(lambda h: np.sum(Lb * (oracle.rhs(c, q + h * vq, s + h * vs)
                                                 - oracle.rhs(c, q - h * vq, s - h * vs))) / (2 * h),
                          np.sum(qb * vq) + np.sum(sb * vs))
    assert ok, ("rhs", errs)
    bb = rng.normal(size=s.shape)
    qb = oracle.source_vjp(c, q, bb)
    ok, errs = _fd_agrees(lambda h: np.sum(bb * (oracle.source(c, q + h * vq) - oracle.source(c, q - h * vq))) / (2 * h),
                          np.sum(qb * vq))
    assert ok, ("source", errs)
    b = oracle.source(c, q)
    vb, vr = rng.normal(size=s.shape), rng.normal(size=s.shape)
    sbar = rng.normal(size=s.shape)
    s0b, bbar, rbar = oracle.jacobi_vjp(c, q, b, s, 3, sbar)
    qv = np.zeros_like(q)
    qv[0] = vr
    J = lambda h: oracle.jacobi(c, q + h * qv, b + h * vb, s + h * vs, 3)
    ok, errs = _fd_agrees(lambda h: np.sum(sbar * (J(h) - J(-h))) / (2 * h),
                          np.sum(s0b * vs) + np.sum(bbar * vb) + np.sum(rbar * vr))
    assert ok, ("jacobi", errs)


def test_jacobi_adjoint_is_the_transposed_sweep():
    """With uniform density the sweep is linear and symmetric: its adjoint with
    respect to the warm start applied to e_m equals the forward sweep of e_m."""
    c = box(6, (PERIODIC,) * 6)
    q = cons(1.3 + 0 * centres(c)[0], 0 * centres(c)[0], 0 * centres(c)[0], 0 * centres(c)[0],
             1 + 0 * centres(c)[0])
    rng = np.random.Generator(np.random.Philox(12))
    a, bvec = rng.normal(size=c.ncells), rng.normal(size=c.ncells)
    zero = np.zeros(c.ncells)
    fa = oracle.jacobi(c, q, zero, a, 1).ravel()
    s0b, _, _ = oracle.jacobi_vjp(c, q, zero, zero, 1, bvec)
    assert np.isclose(np.dot(fa, bvec), np.dot(a, s0b.ravel()), rtol=1e-13)


@pytest.mark.parametrize("bc", [(PERIODIC,) * 6, (OUTFLOW,) * 6])
def test_adjoint_step_matches_finite_differences(bc):
    """The adjoint of a full SSP-RK3 step (fixed dt) in the state and Sigma."""
    c = box(8, bc, nx=8, ny=7, nz=6, sweeps=3)
    rng = np.random.Generator(np.random.Philox(3))
    q = _offset_state(c, 4)
    s = 0.05 * np.cos(2 * np.pi * centres(c)[1] * 2)
    dt = 0.01
    lq, ls = rng.normal(size=q.shape), rng.normal(size=s.shape)
    aq, a_s, _ = oracle.adjoint_step(c, q, s, dt, lq, ls)
    vq, vs = rng.normal(size=q.shape), rng.normal(size=s.shape)

    def fd(h):
        qp, sp, _ = oracle.run(c, q + h * vq, s + h * vs, 1, dt)
        qm, sm, _ = oracle.run(c, q - h * vq, s - h * vs, 1, dt)
        return (np.sum(lq * (qp - qm)) + np.sum(ls * (sp - sm))) / (2 * h)

    ok, errs = _fd_agrees(fd, np.sum(aq * vq) + np.sum(a_s * vs))
    assert ok, errs


def test_adjoint_jet_velocity_gradient():
    """d/dw of <lq, q'> + <ls, Sigma'> through the inflow ghosts, per jet."""
    dx = 1.0 / 16
    w = 2 * math.sqrt(2.8)
    c = Case("jets", 16, 14, 10, dx, alpha=dx * dx, sweeps=3,
             bc=(OUTFLOW,) * 4 + (INFLOW, OUTFLOW),
             jets=[(0.3, 0.45, 3 * dx, 1.0, w, 2.0, 1.0), (0.65, 0.5, 2.5 * dx, 1.0, 0.8 * w, 2.0, 1.0)])
    q0 = inputs.jet_initial_state(c)
    q, s, _ = oracle.run(c, q0, None, 3, 1e-3)
    dt = 1e-3
    rng = np.random.Generator(np.random.Philox(8))
    lq, ls = rng.normal(size=q.shape), rng.normal(size=s.shape)
    _, _, gw = oracle.adjoint_step(c, q, s, dt, lq, ls)
    for n in range(2):
        def fd(h):
            vals = []
            for sgn in (1, -1):
                jets = [list(j) for j in c.jets]
                jets[n][4] += sgn * h
                cc = replace(c, jets=[tuple(j) for j in jets])
                q1, s1, _ = oracle.run(cc, q, s, 1, dt)
                vals.append(np.sum(lq * q1) + np.sum(ls * s1))
            return (vals[0] - vals[1]) / (2 * h)
        ok, errs = _fd_agrees(fd, gw[n], hs=(1e-5, 1e-6), tol=1e-6)
        assert ok, (n, errs)
