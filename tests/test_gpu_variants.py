"""The scheme's alternatives on the GPU (Sec. "Discretization": third- or
fifth-order finite volumes; Jacobi or Gauss-Seidel sweeps) against the FP64
oracle taking the same options: 3rd-order faces (igr_config.order = 3) and
red-black Gauss-Seidel sweeps in place (sigma_solver = IGR_SOLVER_RBGS)."""
import math
from dataclasses import replace

import numpy as np
import pytest

import oracle
from metrics import field_errors, sigma_error
from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import INFLOW, OUTFLOW, PERIODIC, Case

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 2e-3, "bf16": 1.6e-2}


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


def _jets(n=24):
    dx = 1.0 / n
    w = 2 * math.sqrt(2.8)
    return Case("jets", n, n - 4, n - 6, dx, alpha=dx * dx, sweeps=4,
                bc=(OUTFLOW,) * 4 + (INFLOW, OUTFLOW),
                jets=[(0.3, 0.45, 3 * dx, 1.0, w, 2.0, 1.0), (0.65, 0.5, 2.5 * dx, 1.0, 0.8 * w, 2.0, 1.0)])


VARIANTS = {"order3": dict(order=3), "rbgs": dict(sigma_solver=1), "order3+rbgs": dict(order=3, sigma_solver=1)}


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_blast_variants(variant, precision):
    c = replace(inputs.blast(32, steps=20, sweeps=4), **VARIANTS[variant])
    q0 = inputs.initial_state(c)
    qo, so, to = oracle.run(c, q0, None, nsteps=20)
    qg, sg, tg = gpu_run(c, q0, precision, 20)
    err = field_errors(qg, qo)
    assert max(err.values()) <= TOL[precision], err
    assert sigma_error(sg, so, 0) <= 10 * TOL[precision]
    assert math.isclose(tg, to, rel_tol=max(TOL[precision], 1e-13))


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_inflow_and_periodic_variants_fp64(variant):
    for c in (replace(_jets(), **VARIANTS[variant]), replace(inputs.tgv(16), **VARIANTS[variant])):
        q0 = inputs.jet_initial_state(c) if c.jets else inputs.initial_state(c)
        qo, so, to = oracle.run(c, q0, None, nsteps=6)
        qg, sg, tg = gpu_run(c, q0, "f64", 6)
        err = field_errors(qg, qo)
        assert max(err.values()) <= TOL["f64"], (c.name, err)
        assert sigma_error(sg, so, 1e-300) <= 1e-11, c.name


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("sweeps", [1, 3])
def test_solve_sigma_rbgs(precision, sweeps):
    """igr_solve_sigma with red-black sweeps against the oracle's sweeps."""
    import torch
    from paper_2505_07392_gb300 import igr
    c = Case("sig", 28, 18, 22, 1.0 / 28, alpha=1.0 / 28 ** 2, sweeps=sweeps, sigma_solver=1,
             bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, OUTFLOW))
    rng = np.random.Generator(np.random.Philox(3))
    shape = (c.nz, c.ny, c.nx)
    z, y, x = np.meshgrid(*[(np.arange(m) + 0.5) / m for m in shape], indexing="ij")
    rho = 1 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    u = 0.3 * np.sin(2 * np.pi * y)
    v = 0.2 * np.cos(2 * np.pi * z)
    w = -0.25 * np.sin(2 * np.pi * x)
    q0 = np.stack([rho, rho * u, rho * v, rho * w, 2.5 + 0.5 * rho * (u * u + v * v + w * w)])
    s0 = 0.05 * rng.uniform(-1, 1, shape)
    so = oracle.jacobi(c, q0, oracle.source(c, q0), s0, sweeps)
    dt = igr.storage_torch_dtype(precision)
    with igr.Solver(c, precision) as s:
        sg = s.solve_sigma(torch.from_numpy(q0).to(dt).cuda(), torch.from_numpy(s0).to(dt).cuda(), sweeps)
        sg = sg.double().cpu().numpy()
    assert sigma_error(sg, so, 0) <= 10 * TOL[precision]


def test_rbgs_closed_form_on_gpu():
    """rho = 1, b = 0, Sigma = 1 on a periodic box: after n red-black sweeps
    red cells hold l^(2n-1), black l^(2n), l = 6 beta / (1 + 6 beta)."""
    import torch
    from paper_2505_07392_gb300 import igr
    c = Case("cf", 16, 8, 12, 1 / 16, alpha=1 / 256, sweeps=1, sigma_solver=1, bc=(PERIODIC,) * 6)
    beta = c.alpha / c.dx ** 2
    lam = 6 * beta / (1 + 6 * beta)
    shape = (c.nz, c.ny, c.nx)
    q = np.stack([np.ones(shape), np.zeros(shape), np.zeros(shape), np.zeros(shape), np.ones(shape)])
    z, y, x = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    red = (x + y + z) % 2 == 0
    with igr.Solver(c, "f64") as s:
        for n in (1, 2, 3):
            sg = s.solve_sigma(torch.from_numpy(q).cuda(), torch.ones(shape, dtype=torch.float64).cuda(), n)
            sg = sg.cpu().numpy()
            # b = 0: the velocity is zero
            assert np.allclose(sg[red], lam ** (2 * n - 1), rtol=1e-14, atol=0)
            assert np.allclose(sg[~red], lam ** (2 * n), rtol=1e-14, atol=0)


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_variants_do_not_depend_on_launch_shape(variant):
    """Bitwise the same results for every z-chunking (red-black sweeps update
    each cell from neighbours no thread writes during the half-sweep)."""
    import torch
    c = replace(inputs.blast(20, sweeps=3), **VARIANTS[variant])
    q0 = inputs.initial_state(c)
    ref = gpu_run(c, q0, "f32", 4, tiles=(20, 20, 20))
    for tiles in ((4, 4, 4), (8, 16, 5), (7, 13, 11)):
        out = gpu_run(c, q0, "f32", 4, tiles=tiles)
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), tiles


def test_adjoint_refuses_variants():
    import torch
    from paper_2505_07392_gb300 import igr
    for v in VARIANTS.values():
        c = replace(inputs.blast(8, sweeps=2), **v)
        with igr.Solver(c, "f64") as s:
            q = torch.from_numpy(inputs.initial_state(c)).cuda()
            sig = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
            with pytest.raises(igr.IGRError) as e:
                s.adjoint_step(q, sig, torch.zeros_like(q), torch.zeros_like(sig), 1e-3)
            assert e.value.status == igr.ERR_UNSUPPORTED
