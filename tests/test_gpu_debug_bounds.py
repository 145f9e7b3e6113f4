"""The bounds-checking debug build (libigr_debug.so, IGR_DEBUG_BOUNDS): every
global index the forward kernels form is checked against its array's length.
Run over odd shapes (the one- and four-cell kernel forms), boundary
kinds, inflow jets, the scheme alternatives, viscous terms, the increment
storage forms, the host RK base, batches (grouped launches), the
allocation-free solve and the adjoint kernels, no index may fall outside
its array;
the self-test shows that a single out-of-range index is counted (and not
dereferenced). This stands in for a memory checker."""
import ctypes as C
import gc
import math
from dataclasses import replace

import numpy as np
import pytest

from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import INFLOW, OUTFLOW, PERIODIC, Case

pytestmark = pytest.mark.gpu


@pytest.fixture
def debug_lib(monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_07392_gb300 import build, igr
    path = build.build(debug_bounds=True)
    gc.collect()  # no handle of the normal library may reach the debug one
    monkeypatch.setattr(igr, "LIB_PATH", path)
    monkeypatch.setattr(igr, "_lib", None)  # restored to the normal library afterwards
    yield igr.lib()
    gc.collect()


def _hits(L, clear=0):
    h = C.c_ulonglong()
    from paper_2505_07392_gb300 import igr
    assert L.igr_debug_bounds_hits(C.byref(h), clear) == igr.OK
    return h.value


def test_selftest_counts_one(debug_lib):
    from paper_2505_07392_gb300 import igr
    _hits(debug_lib, clear=1)
    assert debug_lib.igr_debug_bounds_selftest() == igr.OK
    assert _hits(debug_lib, clear=1) == 1


def _state(c, seed):
    rng = np.random.Generator(np.random.Philox(seed))
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in (c.nz, c.ny, c.nx)], indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, size=4)
    rho = 1 + 0.2 * np.sin(2 * np.pi * x + ph[0]) * np.cos(2 * np.pi * y + ph[1])
    u = 0.3 * np.sin(2 * np.pi * z + ph[2])
    v = -0.2 * np.cos(2 * np.pi * x + ph[3])
    w = 0.25 * np.sin(2 * np.pi * y)
    return np.stack([rho, rho * u, rho * v, rho * w, 2.5 + 0.5 * rho * (u * u + v * v + w * w)])


def _jets(n=20):
    dx = 1.0 / n
    wv = 2 * math.sqrt(2.8)
    return Case("jets", n, n - 1, n + 3, dx, alpha=dx * dx, sweeps=3, bc=(OUTFLOW,) * 4 + (INFLOW, OUTFLOW),
                jets=[(0.3, 0.45, 3 * dx, 1.0, wv, 2.0, 1.0), (0.65, 0.5, 2.5 * dx, 1.0, 0.8 * wv, 2.0, 1.0)])


def test_no_index_out_of_bounds(debug_lib):
    import torch
    from paper_2505_07392_gb300 import igr
    L = debug_lib
    _hits(L, clear=1)
    shapes = [((7, 13, 33), (PERIODIC,) * 6), ((33, 7, 13), (OUTFLOW,) * 6),
              ((13, 33, 7), (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, OUTFLOW)),
              ((65, 9, 5), (PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, PERIODIC, PERIODIC)),
              ((4, 4, 4), (PERIODIC,) * 6), ((36, 12, 8), (OUTFLOW,) * 6),
              ((132, 5, 6), (PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW))]
    cases = []
    for (nx, ny, nz), bc in shapes:
        dx = 1.0 / max(nx, ny, nz)
        cases.append((Case("odd", nx, ny, nz, dx, alpha=dx * dx, sweeps=2, bc=bc), "f64"))
    cases += [(_jets(), "f32"), (_jets(24), "f16"),
              (replace(inputs.blast(20, sweeps=2), order=3, sigma_solver=1), "f32"),
              (replace(Case("v", 13, 8, 11, 1 / 13, alpha=1 / 169, sweeps=2, bc=(OUTFLOW,) * 6), mu=1e-3), "f64"),
              (replace(_jets(16), mu=1e-3, zeta=1e-3), "bf16"), (_jets(24), "f16inc"),
              (Case("odd", 36, 12, 8, 1 / 36, alpha=1 / 36 ** 2, sweeps=2, bc=(OUTFLOW,) * 6), "bf16inc"),
              # rows of 128 cells, 16 rows: the full-tile sweep and source kernels
              (Case("full", 128, 16, 6, 1 / 128, alpha=1 / 128 ** 2, sweeps=2, bc=(PERIODIC,) * 6), "f16inc"),
              (replace(Case("full", 128, 16, 6, 1 / 128, alpha=1 / 128 ** 2, sweeps=2,
                            bc=(OUTFLOW,) * 4 + (PERIODIC,) * 2), sigma_solver=1), "f32")]
    for c, prec in cases:
        q0 = inputs.jet_initial_state(c) if c.jets else _state(c, c.nx)
        dt, st = igr.state_torch_dtype(prec), igr.storage_torch_dtype(prec)
        for forms in ((0, 0), (1, 1)) if c.nx % 4 == 0 else ((0, 0),):
            with igr.Solver(c, prec) as s:
                s.set_kernel_forms(*forms)
                q = torch.from_numpy(q0).to(dt).cuda()
                s.set_state(q)
                s.step(2)
                sig = torch.zeros(s.shape, dtype=st, device="cuda")
                s.solve_sigma(q, sig, 2)
                s.rhs(q, sig)
                s.diagnose()
            assert _hits(L) == 0, (c.name, c.nx, c.ny, c.nz, prec, forms)
    # RK base in host memory, batches, allocation-free solve
    c = inputs.blast(16, sweeps=2)
    with igr.Solver(c, "f16", host_rk_base=True) as s:
        s.set_state(torch.from_numpy(inputs.initial_state(c)).half().cuda())
        s.step(2)
    cases = [inputs.tgv(12), inputs.tgv(16, instance=1), replace(inputs.blast(10, sweeps=2), order=3),
             replace(inputs.tgv(128, instance=2), ny=16, nz=6)]  # grouped full-tile source and sweep
    with igr.Batch(cases, "f16") as b:
        for inst, cc in zip(b.instances, cases):
            inst.set_state(torch.from_numpy(inputs.initial_state(cc)).half().cuda())
        b.step(3, sync=True)
    c = Case("na", 12, 10, 8, 1 / 12, alpha=1 / 144, sweeps=3, bc=(OUTFLOW,) * 6)
    cfg, _j = igr.make_config(c, "f32")
    q = torch.from_numpy(_state(c, 3)).float().cuda()
    sig = torch.zeros((c.nz, c.ny, c.nx), dtype=torch.float32, device="cuda")
    assert L.igr_solve_sigma_noalloc(C.byref(cfg), C.c_void_p(q.data_ptr()), C.c_void_p(sig.data_ptr()), 3,
                                     None) == igr.OK
    torch.cuda.synchronize()
    assert _hits(L) == 0
    # the adjoint kernels (scatter through the boundary mapping and the jet
    # blend, the transposed sweeps' neighbour gathers, the jet reduction)
    for c, prec in ((_jets(), "f64"), (Case("a", 13, 9, 7, 1 / 13, alpha=1 / 169, sweeps=2,
                                            bc=(PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, PERIODIC, PERIODIC)), "f32")):
        q0 = inputs.jet_initial_state(c) if c.jets else _state(c, 5)
        dt, ct = igr.storage_torch_dtype(prec), igr.compute_torch_dtype(prec)
        rng = np.random.Generator(np.random.Philox(11))
        with igr.Solver(c, prec) as s:
            q = torch.from_numpy(q0).to(dt).cuda()
            sig = torch.zeros(s.shape, dtype=dt, device="cuda")
            lq = torch.from_numpy(rng.normal(size=q0.shape)).to(ct).cuda()
            ls = torch.from_numpy(rng.normal(size=s.shape)).to(ct).cuda()
            s.adjoint_step(q, sig, lq, ls, 1e-3)
            s.sync()
        assert _hits(L) == 0, (c.name, prec)


def test_normal_library_has_no_counter():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_07392_gb300 import build, igr
    build.build()
    h = C.c_ulonglong()
    assert igr.lib().igr_debug_bounds_hits(C.byref(h), 0) == igr.ERR_UNSUPPORTED
