"""igr_solve_sigma_noalloc, the allocation-free Sigma solve, against the
context-based igr_solve_sigma.

The allocation-free entry point serves callers that cannot allocate device
memory where they need the solve (inside another framework's fixed memory
budget, in allocation-free real-time loops, in hooks that may not call
cudaMalloc). Its scratch lives in a static device array of the library. The
tests call it through the C ABI twice in a row (the second call reuses the
array the first one left behind), in every storage precision, and require
the context solve's bits: both run the same kernels on the same inputs. This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import OUTFLOW, PERIODIC, Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_07392_gb300 import build
    build.build()
    yield


def _state(case, seed):
    rng = np.random.Generator(np.random.Philox(seed))
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in (case.nz, case.ny, case.nx)], indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, size=6)
    tp = 2 * np.pi
    rho = 1 + 0.2 * np.sin(tp * x + ph[0]) * np.cos(tp * y + ph[1]) + 0.1 * np.cos(tp * z)
    u = 0.3 * np.sin(tp * y + ph[2])
    v = 0.2 * np.cos(tp * z + ph[3])
    w = 0.25 * np.sin(tp * x + ph[4])
    p = 1 + 0.1 * np.cos(tp * (x + z) + ph[5])
    E = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


# Rows of 44 cells take the 4-cell kernel forms (nx % 4 == 0), rows of 42 the
# 1-cell forms; the second buffer of the scratch starts n values after the
# first, which lands differently for every storage width.
GRIDS = [(44, 36, 28), (42, 30, 20)]


@pytest.mark.parametrize("precision", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", GRIDS)
def test_noalloc_solve_matches_context_solve_twice(precision, shape):
    """Two calls in a row (different states and sweep counts, the second
    reusing the array the first left behind) give the context solve's bits."""
    import torch
    from paper_2505_07392_gb300 import igr
    L = igr.lib()
    nx, ny, nz = shape
    case = Case("noalloc", nx, ny, nz, 1.0 / nx, alpha=1.0 / nx ** 2, sweeps=5,
                bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, OUTFLOW))
    cfg, _jets = igr.make_config(case, precision)
    st = igr.storage_torch_dtype(precision)
    stream = torch.cuda.current_stream()
    results = []
    for call, (seed, sweeps) in enumerate(((1, 5), (2, 4))):
        q = torch.from_numpy(_state(case, seed)).to(st).cuda()
        s0 = (0.05 * torch.from_numpy(_state(case, seed + 10)[0])).to(st).cuda()
        with igr.Solver(case, precision) as s:
            ref = s.solve_sigma(q, s0.clone(), sweeps)
            torch.cuda.synchronize()
            ref = ref.cpu()
        sig = s0.clone()
        rc = L.igr_solve_sigma_noalloc(C.byref(cfg), C.c_void_p(q.data_ptr()), C.c_void_p(sig.data_ptr()),
                                       sweeps, C.c_void_p(stream.cuda_stream))
        assert rc == igr.OK, L.igr_noalloc_last_error().decode()
        torch.cuda.synchronize()
        got = sig.cpu()
        assert ref.abs().max() > 0
        assert torch.equal(got, ref), (call, (got.double() - ref.double()).abs().max().item())
        results.append(got)
    assert not torch.equal(results[0], results[1])


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_noalloc_unaligned_caller_buffers(precision):
    """Caller tensors that start one element into their storage (aligned to
    the element, not to the 4-cell vector width) take the 1-cell forms and
    give the bits of the aligned call."""
    import torch
    from paper_2505_07392_gb300 import igr
    L = igr.lib()
    case = Case("noalloc", 44, 36, 28, 1.0 / 44, alpha=1.0 / 44 ** 2, sweeps=3,
                bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, OUTFLOW))
    cfg, _jets = igr.make_config(case, precision)
    st = igr.storage_torch_dtype(precision)
    stream = torch.cuda.current_stream()
    n = case.nx * case.ny * case.nz
    q = torch.from_numpy(_state(case, 4)).to(st).cuda()
    s0 = (0.05 * torch.from_numpy(_state(case, 14)[0])).to(st).cuda()
    qa = torch.empty(5 * n + 1, dtype=st, device="cuda")
    qa[1:] = q.reshape(-1)
    sa = torch.empty(n + 1, dtype=st, device="cuda")
    sa[1:] = s0.reshape(-1)
    qu, su = qa[1:], sa[1:]
    assert qu.data_ptr() % 8 != 0
    ref = s0.clone()
    for qq, ss in ((q, ref), (qu, su)):
        rc = L.igr_solve_sigma_noalloc(C.byref(cfg), C.c_void_p(qq.data_ptr()), C.c_void_p(ss.data_ptr()),
                                       3, C.c_void_p(stream.cuda_stream))
        assert rc == igr.OK, L.igr_noalloc_last_error().decode()
    torch.cuda.synchronize()
    assert torch.equal(su.cpu(), ref.reshape(-1).cpu())


def test_noalloc_red_black_sweeps():
    """With red-black Gauss-Seidel sweeps (in place, no second Sigma buffer)
    the allocation-free solve gives the context solve's bits."""
    import torch
    from dataclasses import replace
    from paper_2505_07392_gb300 import igr
    L = igr.lib()
    case = Case("noalloc", 40, 36, 28, 1.0 / 40, alpha=1.0 / 40 ** 2, sweeps=3, sigma_solver=1,
                bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, OUTFLOW))
    cfg, _jets = igr.make_config(case, "f32")
    stream = torch.cuda.current_stream()
    q = torch.from_numpy(_state(case, 3)).float().cuda()
    s0 = (0.05 * torch.from_numpy(_state(case, 13)[0])).float().cuda()
    with igr.Solver(case, "f32") as s:
        ref = s.solve_sigma(q, s0.clone(), 3)
        torch.cuda.synchronize()
        ref = ref.cpu()
    sig = s0.clone()
    st = L.igr_solve_sigma_noalloc(C.byref(cfg), C.c_void_p(q.data_ptr()), C.c_void_p(sig.data_ptr()),
                                   3, C.c_void_p(stream.cuda_stream))
    assert st == igr.OK, L.igr_noalloc_last_error().decode()
    torch.cuda.synchronize()
    assert torch.equal(sig.cpu(), ref)
    with igr.Solver(replace(case, sigma_solver=0), "f32") as s:
        jac = s.solve_sigma(q, s0.clone(), 3).cpu()
    assert not torch.equal(jac, ref)  # the red-black path really ran


def test_noalloc_rejects_what_it_cannot_hold():
    from paper_2505_07392_gb300 import igr
    L = igr.lib()
    L.igr_noalloc_max_cells.restype = C.c_size_t
    L.igr_noalloc_max_cells.argtypes = [C.c_int]
    L.igr_noalloc_last_error.restype = C.c_char_p
    cap = L.igr_noalloc_max_cells(igr.F32)
    assert cap >= 100_000
    n = int(round(cap ** (1 / 3))) + 8
    big = Case("big", n, n, n, 1.0 / n, alpha=1.0 / n ** 2, bc=(PERIODIC,) * 6)
    cfg, _ = igr.make_config(big, "f32")
    dummy = C.c_void_p(256)  # never dereferenced: the size check comes first
    st = L.igr_solve_sigma_noalloc(C.byref(cfg), dummy, dummy, 3, None)
    assert st == igr.ERR_INVALID_ARG
    assert b"scratch" in L.igr_noalloc_last_error()
    jets = inputs.jets4(16)
    cfg2, _j = igr.make_config(jets, "f32")
    st = L.igr_solve_sigma_noalloc(C.byref(cfg2), dummy, dummy, 3, None)
    assert st == igr.ERR_UNSUPPORTED
