"""Viscous stresses (igr_config.mu, zeta; Eq. constitutive_law in the
Navier-Stokes form of the IGR system) on the GPU against the FP64 oracle with
the same viscosities. The inviscid scheme is a separate kernel instantiation,
so the other parity tests cover it unchanged."""
import math
from dataclasses import replace

import numpy as np
import pytest

import oracle
from metrics import field_errors, sigma_error
from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import INFLOW, OUTFLOW, PERIODIC, Case

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_07392_gb300 import build
    build.build()
    yield


def gpu_run(case, q0, precision, nsteps, tiles=None):
    import torch
    from paper_2505_07392_gb300 import igr
    with igr.Solver(case, precision) as s:
        s.set_state(torch.from_numpy(np.ascontiguousarray(q0)).cuda())
        if tiles:
            s.set_tiles(*tiles)
        t = s.step(nsteps)
        q, sig = s.get_state(torch.float64)
        return q.cpu().numpy(), sig.cpu().numpy(), t


def smooth_state(case, seed):
    rng = np.random.Generator(np.random.Philox(seed))
    ph = rng.uniform(0, 2 * np.pi, size=8)
    L = np.array([case.nx, case.ny, case.nz]) * case.dx
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) * case.dx / l for n, l in
                            zip((case.nz, case.ny, case.nx), (L[2], L[1], L[0]))], indexing="ij")
    tp = 2 * np.pi
    rho = 1 + 0.2 * np.sin(tp * x + ph[0]) * np.cos(tp * y + ph[1]) + 0.1 * np.sin(tp * z + ph[2])
    u = 0.3 * np.sin(tp * y + ph[3]) * np.cos(tp * z)
    v = 0.25 * np.cos(tp * x + ph[4]) * np.sin(tp * z + ph[5])
    w = -0.3 * np.sin(tp * x + ph[6]) * np.cos(tp * y)
    p = 1 + 0.1 * np.cos(tp * (x + y) + ph[7])
    return np.stack([rho, rho * u, rho * v, rho * w, p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)])


@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_viscous_blast(precision):
    c = replace(inputs.blast(32, steps=20, sweeps=4), mu=2e-3, zeta=1e-3)
    q0 = inputs.initial_state(c)
    qo, so, to = oracle.run(c, q0, None, nsteps=20)
    qg, sg, tg = gpu_run(c, q0, precision, 20)
    err = field_errors(qg, qo)
    assert max(err.values()) <= TOL[precision], err
    assert sigma_error(sg, so, 0) <= 10 * TOL[precision]
    # the viscous terms change the answer beyond the tolerance
    qi, _, _ = oracle.run(replace(c, mu=0.0, zeta=0.0), q0, None, nsteps=20)
    assert max(field_errors(qi, qo).values()) > 100 * TOL["f32"]


SHAPES = [
    ((7, 13, 33), (PERIODIC,) * 6),
    ((33, 7, 13), (OUTFLOW,) * 6),
    ((13, 33, 7), (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, OUTFLOW)),
    ((65, 9, 5), (PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, PERIODIC, PERIODIC)),
]


@pytest.mark.parametrize("shape,bc", SHAPES)
def test_viscous_odd_shapes_fp64(shape, bc):
    """Tiles cut anywhere, boundary corners (the tangential neighbours reach
    one cell diagonally past the tile interior)."""
    nx, ny, nz = shape
    dx = 1.0 / max(shape)
    c = Case("odd", nx, ny, nz, dx, alpha=dx * dx, sweeps=3, bc=bc, mu=5e-3, zeta=2e-3)
    q0 = smooth_state(c, seed=nx)
    qo, so, to = oracle.run(c, q0, None, nsteps=4)
    qg, sg, tg = gpu_run(c, q0, "f64", 4)
    err = field_errors(qg, qo)
    assert max(err.values()) <= TOL["f64"], err


def test_viscous_jets_fp64():
    n = 24
    dx = 1.0 / n
    w = 2 * math.sqrt(2.8)
    c = Case("jets", n, n - 4, n + 4, dx, alpha=dx * dx, sweeps=4, mu=1e-3, zeta=0.0,
             bc=(OUTFLOW,) * 4 + (INFLOW, OUTFLOW),
             jets=[(0.3, 0.45, 3 * dx, 1.0, w, 2.0, 1.0), (0.65, 0.5, 2.5 * dx, 1.0, 0.8 * w, 2.0, 1.0)])
    q0 = inputs.jet_initial_state(c)
    qo, so, to = oracle.run(c, q0, None, nsteps=8)
    qg, sg, tg = gpu_run(c, q0, "f64", 8)
    err = field_errors(qg, qo)
    assert max(err.values()) <= TOL["f64"], err


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_viscous_rhs(precision):
    import torch
    from paper_2505_07392_gb300 import igr
    c = Case("rhs", 36, 20, 24, 1.0 / 36, alpha=1.0 / 36 ** 2, mu=4e-3, zeta=3e-3,
             bc=(PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW))
    q0 = smooth_state(c, seed=5)
    rng = np.random.Generator(np.random.Philox(9))
    sig = 0.05 * smooth_state(c, seed=6)[0] + 0.01 * rng.uniform(-1, 1, size=(c.nz, c.ny, c.nx))
    Lo = oracle.rhs(c, q0, sig)
    dt = igr.storage_torch_dtype(precision)
    with igr.Solver(c, precision) as s:
        Lg = s.rhs(torch.from_numpy(q0).to(dt).cuda(), torch.from_numpy(sig).to(dt).cuda()).double().cpu().numpy()
    rel = np.linalg.norm((Lg - Lo).reshape(5, -1), axis=1) / np.linalg.norm(Lo.reshape(5, -1), axis=1)
    assert np.all(rel <= 10 * TOL[precision]), rel


def test_viscous_launch_shape_invariant():
    c = replace(inputs.blast(20, sweeps=3), mu=2e-3, zeta=1e-3)
    q0 = inputs.initial_state(c)
    ref = gpu_run(c, q0, "f32", 4, tiles=(20, 20, 20))
    for tiles in ((4, 4, 4), (8, 16, 5), (7, 13, 11)):
        out = gpu_run(c, q0, "f32", 4, tiles=tiles)
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), tiles


def test_adjoint_refuses_viscous():
    import torch
    from paper_2505_07392_gb300 import igr
    c = replace(inputs.blast(8, sweeps=2), mu=1e-3)
    with igr.Solver(c, "f64") as s:
        q = torch.from_numpy(inputs.initial_state(c)).cuda()
        sig = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(igr.IGRError) as e:
            s.adjoint_step(q, sig, torch.zeros_like(q), torch.zeros_like(sig), 1e-3)
        assert e.value.status == igr.ERR_UNSUPPORTED
