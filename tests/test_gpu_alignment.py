"""Caller pointer alignment at the C ABI.

A device pointer must be aligned to its element size; the calls reject one
that is not before any launch (IGR_ERR_INVALID_ARG), so no kernel ever sees
it. A pointer aligned to the element but not to the 4-cell vector width of
the source and Jacobi kernels' 4-cell forms (a tensor sliced one element
into its storage) makes igr_solve_sigma take the 1-cell forms, which give
the same bits.
"""
import ctypes as C

import numpy as np
import pytest

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
    ph = rng.uniform(0, 2 * np.pi, size=4)
    tp = 2 * np.pi
    rho = 1 + 0.2 * np.sin(tp * x + ph[0]) * np.cos(tp * y)
    u = 0.3 * np.sin(tp * y + ph[1])
    v = 0.2 * np.cos(tp * z + ph[2])
    w = 0.25 * np.sin(tp * x + ph[3])
    p = 1 + 0.1 * np.cos(tp * (x + z))
    return np.stack([rho, rho * u, rho * v, rho * w, p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)])


CASE = Case("align", 64, 20, 12, 1.0 / 64, alpha=1.0 / 64 ** 2, sweeps=3,
            bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, OUTFLOW, OUTFLOW))


def _shifted(t, shift):
    """A copy of t that starts `shift` elements into a larger buffer."""
    import torch
    buf = torch.empty(t.numel() + shift, dtype=t.dtype, device=t.device)
    v = buf[shift:]
    v.copy_(t.reshape(-1))
    return v.view(t.shape)


@pytest.mark.parametrize("precision", ["f64", "f32", "f16", "bf16"])
def test_solve_sigma_with_sliced_tensors_takes_the_one_cell_forms(precision):
    import torch
    from paper_2505_07392_gb300 import igr
    st = igr.storage_torch_dtype(precision)
    q = torch.from_numpy(_state(CASE, 1)).to(st).cuda()
    s0 = (0.05 * torch.from_numpy(_state(CASE, 2)[0])).to(st).cuda()
    with igr.Solver(CASE, precision) as s:
        s.set_kernel_forms(1, 1)  # the 4-cell forms (rows of 64 default to the 1-cell forms)
        ref = s.solve_sigma(q, s0.clone(), 3).cpu()
        qu, su = _shifted(q, 1), _shifted(s0, 1)
        assert qu.data_ptr() % 16 != 0 and su.data_ptr() % 16 != 0
        got = s.solve_sigma(qu, su, 3).cpu()
        assert torch.equal(got, ref)
        # only one of the two unaligned
        got2 = s.solve_sigma(qu, s0.clone(), 3).cpu()
        assert torch.equal(got2, ref)


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_byte_misaligned_pointers_are_rejected_before_any_launch(precision):
    import torch
    from paper_2505_07392_gb300 import igr
    L = igr.lib()
    st = igr.storage_torch_dtype(precision)
    n = CASE.nx * CASE.ny * CASE.nz
    buf = torch.zeros(6 * n + 64, dtype=st, device="cuda")
    lam = torch.zeros(6 * n + 64, dtype=igr.compute_torch_dtype(precision), device="cuda")
    good = C.c_void_p(buf.data_ptr())
    bad = C.c_void_p(buf.data_ptr() + 1)  # an odd byte address: never a valid element
    lgood, lbad = C.c_void_p(lam.data_ptr()), C.c_void_p(lam.data_ptr() + 2)
    code = {"f32": igr.DT_F32, "f16": igr.DT_F16}[precision]
    with igr.Solver(CASE, precision) as s:
        h = s.h
        assert L.igr_solve_sigma(h, bad, good, 3, code) == igr.ERR_INVALID_ARG
        assert L.igr_solve_sigma(h, good, bad, 3, code) == igr.ERR_INVALID_ARG
        assert L.igr_rhs(h, bad, good, lgood, code) == igr.ERR_INVALID_ARG
        assert L.igr_rhs(h, good, good, lbad, code) == igr.ERR_INVALID_ARG
        assert L.igr_rk_combine(h, bad, good, lgood, good, 16, 1, 1e-3) == igr.ERR_INVALID_ARG
        assert L.igr_set_state(h, bad, None, code, 1) == igr.ERR_INVALID_ARG
        assert L.igr_get_state(h, bad, None, code, 1) == igr.ERR_INVALID_ARG
        assert L.igr_adjoint_step(h, good, good, lbad, lgood, lgood, lgood, None, 1e-3, code) == igr.ERR_INVALID_ARG
        cfg, _j = igr.make_config(CASE, precision)
        assert L.igr_solve_sigma_noalloc(C.byref(cfg), bad, good, 3, None) == igr.ERR_INVALID_ARG
        s.sync()  # nothing was launched, nothing failed asynchronously
