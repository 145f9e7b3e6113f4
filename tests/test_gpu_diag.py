"""igr_diagnose: FP64 totals, extrema and the residual of the elliptic
equation (Eq. igrelliptic) against the oracle's operator and source.

Every stored value converts to double exactly, so the device evaluation and
the oracle see the same numbers; they differ only in summation order (1e-12)
and, where an inflow face is present in FP32/16-bit modes, in the inflow
tables, which the device holds in the arithmetic type (1e-6).
"""
import numpy as np
import pytest

import oracle
from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import INFLOW, OUTFLOW, PERIODIC, Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_07392_gb300 import build
    build.build()
    yield


def _expected(c, q, sig):
    q = np.asarray(q, dtype=np.float64)
    sig = np.asarray(sig, dtype=np.float64)
    A = oracle.apply_A(c, q, sig)
    b = oracle.source(c, q)
    vol = c.dx ** 3
    p = (c.gamma - 1) * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])
    bn = np.linalg.norm(b)
    # momentum totals cancel (symmetric flows): compared on the scale sum |m| dx^3
    mscale = np.abs(q[1:4]).sum() * vol
    return {"mass": q[0].sum() * vol, "momentum": (mscale,) + tuple(q[1 + a].sum() * vol for a in range(3)),
            "energy": q[4].sum() * vol, "rho_min": q[0].min(), "p_min": p.min(),
            "sigma_absmax": np.abs(sig).max(), "b_norm": bn,
            "sigma_residual": np.linalg.norm(A - b) / bn if bn > 0 else np.linalg.norm(A)}


def _check(got, exp, tol):
    for k, v in exp.items():
        g = got[k]
        if isinstance(v, tuple):
            scale, v = v[0], v[1:]
            for a, b in zip(g, v):
                assert abs(a - b) <= tol * scale, (k, g, v)
        else:
            assert abs(g - v) <= tol * max(abs(v), 1e-300), (k, g, v)


def _jets(n=16):
    dx = 1.0 / n
    w = 2 * np.sqrt(2.8)
    return Case("jets", n, n - 2, n - 4, dx, alpha=dx * dx, sweeps=3,
                bc=(OUTFLOW,) * 4 + (INFLOW, OUTFLOW),
                jets=[(0.3, 0.45, 3 * dx, 1.0, w, 2.0, 1.0), (0.65, 0.5, 2.5 * dx, 1.0, 0.8 * w, 2.0, 1.0)])


CASES = [
    ("blast-f64", lambda: inputs.blast(12, sweeps=4), "f64", 1e-12),
    ("blast-f32", lambda: inputs.blast(14, sweeps=4), "f32", 1e-12),
    ("tgv-f16", lambda: inputs.tgv(16), "f16", 1e-12),
    ("tgv-bf16", lambda: inputs.tgv(12), "bf16", 1e-12),
    ("jets-f64", _jets, "f64", 1e-12),
    ("jets-f32", _jets, "f32", 1e-6),
    ("blast-f16inc", lambda: inputs.blast(14, sweeps=4), "f16inc", 1e-12),
]


@pytest.mark.parametrize("name,make,precision,tol", CASES, ids=[c[0] for c in CASES])
def test_diagnose_matches_oracle(name, make, precision, tol):
    import torch
    from paper_2505_07392_gb300 import igr
    c = make()
    q0 = inputs.jet_initial_state(c) if c.jets else inputs.initial_state(c)
    with igr.Solver(c, precision) as s:
        s.set_state(torch.from_numpy(q0).cuda())
        s.step(3)
        got = s.diagnose()
        q, sig = s.get_state(torch.float64)
    _check(got, _expected(c, q.cpu().numpy(), sig.cpu().numpy()), tol)
    assert 0 < got["sigma_residual"] < 1


def test_residual_of_exact_solve_vanishes():
    """Sigma from a dense direct solve of A Sigma = b (A assembled column by
    column from the oracle's operator on a 6^3 outflow box): the device
    residual is at round-off; Jacobi sweeps from Sigma = 0 lower it
    monotonically toward that."""
    import torch
    from paper_2505_07392_gb300 import igr
    c = Case("o", 6, 6, 6, 1 / 6, alpha=1 / 36, sweeps=1, bc=(OUTFLOW,) * 6)
    rng = np.random.Generator(np.random.Philox(11))
    z, y, x = np.meshgrid(*[(np.arange(6) + 0.5) / 6] * 3, indexing="ij")
    rho = 1 + 0.3 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.1 * rng.uniform(-1, 1, x.shape)
    u = 0.3 * np.sin(2 * np.pi * y + 0.4)
    v = -0.2 * np.cos(2 * np.pi * z)
    w = 0.25 * np.sin(2 * np.pi * x)
    q = np.stack([rho, rho * u, rho * v, rho * w, 2.5 + 0.5 * rho * (u * u + v * v + w * w)])
    n = 216
    A = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = oracle.apply_A(c, q, e).ravel()
    b = oracle.source(c, q).ravel()
    sig_exact = np.linalg.solve(A, b).reshape(6, 6, 6)
    with igr.Solver(c, "f64") as s:
        s.set_state(torch.from_numpy(q).cuda(), torch.from_numpy(sig_exact).cuda())
        assert s.diagnose()["sigma_residual"] <= 1e-12
        res = []
        for sweeps in (1, 2, 4, 8, 16):
            sig = oracle.jacobi(c, q, b.reshape(6, 6, 6), np.zeros((6, 6, 6)), sweeps)
            s.set_state(torch.from_numpy(q).cuda(), torch.from_numpy(sig).cuda())
            res.append(s.diagnose()["sigma_residual"])
    assert all(r1 < r0 for r0, r1 in zip(res, res[1:])), res
    assert res[0] < 1


def test_totals_conserved_periodic():
    """Under periodic boundaries the FP64 totals stay at their initial values
    to round-off over many steps (FP64 storage)."""
    import torch
    from paper_2505_07392_gb300 import igr
    c = inputs.tgv(16)
    with igr.Solver(c, "f64") as s:
        s.set_state(torch.from_numpy(inputs.initial_state(c)).cuda())
        d0 = s.diagnose()
        s.step(20)
        d1 = s.diagnose()
    for k in ("mass", "energy"):
        assert abs(d1[k] - d0[k]) <= 1e-13 * abs(d0[k]), k
    for a in range(3):
        assert abs(d1["momentum"][a] - d0["momentum"][a]) <= 1e-13 * d0["mass"]
