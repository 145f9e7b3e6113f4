"""RK base in host memory (igr_config.host_rk_base): the same kernels read
q^n over the CPU-GPU link instead of from a third device buffer, so every
result must equal the in-core run's bit for bit."""
import math

import numpy as np
import pytest

from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import INFLOW, OUTFLOW, Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_07392_gb300 import build
    build.build()
    yield


def _jets(n=24):
    dx = 1.0 / n
    w = 2 * math.sqrt(2.8)
    return Case("jets", n, n - 4, n + 8, dx, alpha=dx * dx, sweeps=4,
                bc=(OUTFLOW,) * 4 + (INFLOW, OUTFLOW),
                jets=[(0.3, 0.45, 3 * dx, 1.0, w, 2.0, 1.0), (0.65, 0.5, 2.5 * dx, 1.0, 0.8 * w, 2.0, 1.0)])


def _run(case, q0, precision, steps, host):
    import torch
    from paper_2505_07392_gb300 import igr
    with igr.Solver(case, precision, host_rk_base=host) as s:
        s.set_state(torch.from_numpy(q0).to(igr.storage_torch_dtype(precision)).cuda())
        t = s.step(steps)
        q, sig = s.get_state()
        d = s.diagnose()
    return q, sig, t, d


@pytest.mark.parametrize("name,make,precision", [
    ("blast-f32", lambda: inputs.blast(24, sweeps=6), "f32"),
    ("blast-f16", lambda: inputs.blast(24, sweeps=6), "f16"),
    ("jets-f64", _jets, "f64"),
    ("jets-bf16", _jets, "bf16"),
])
def test_host_rk_base_bitwise(name, make, precision):
    import torch
    c = make()
    q0 = inputs.jet_initial_state(c) if c.jets else inputs.initial_state(c)
    a = _run(c, q0, precision, 7, False)
    b = _run(c, q0, precision, 7, True)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[2] == b[2]  # the same dt sequence
    assert a[3] == b[3]


def test_batches_refuse_host_rk_base():
    from paper_2505_07392_gb300 import igr
    cases = [inputs.tgv(12), inputs.tgv(16)]
    cfgs = [igr.make_config(c, "f32", host_rk_base=(i == 1)) for i, c in enumerate(cases)]
    import ctypes
    arr = (igr.Config * 2)(*[cf for cf, _ in cfgs])
    h = ctypes.c_void_p()
    assert igr.lib().igr_create_batch(arr, 2, None, None, ctypes.byref(h)) == igr.ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", ["f32", "f16"])
@pytest.mark.parametrize("host_rk_base", [False, True])
def test_set_conserved_round_trip_is_bitwise(precision, host_rk_base):
    """A host-driven loop (igr_get_state of q alone into host memory, then
    igr_set_conserved of it) keeps Sigma on the device and gives the bits of
    uninterrupted stepping, q and Sigma."""
    import torch
    from paper_2505_07392_gb300 import igr
    c = _jets()
    q0 = torch.from_numpy(inputs.jet_initial_state(c)).to(igr.storage_torch_dtype(precision)).cuda()
    with igr.Solver(c, precision, host_rk_base=host_rk_base) as s:
        s.set_state(q0)
        s.step(4)
        qa, sa = s.get_state()
    npdt = {"f32": np.float32, "f16": np.float16}[precision]
    with igr.Solver(c, precision, host_rk_base=host_rk_base) as s:
        s.set_state(q0)
        for _ in range(2):
            s.step(2)
            _, sig_before = s.get_state()
            qh = np.empty((5,) + s.shape, dtype=npdt)
            s.get_state_host(qh)
            s.set_conserved(qh)
            _, sig_after = s.get_state()
            assert torch.equal(sig_before, sig_after)
        # a device tensor in another dtype is converted on the device
        qd, _ = s.get_state(torch.float64)
        s.set_conserved(qd)
        qb, sb = s.get_state()
    assert torch.equal(qa, qb)
    assert torch.equal(sa, sb)


@pytest.mark.parametrize("precision", ["f32", "f16", "f16inc"])
@pytest.mark.parametrize("host_rk_base", [False, True])
def test_step_host_equals_separate_calls(precision, host_rk_base):
    """igr_step_host (q in from host memory, the energy field's copy
    overlapped with stage 1's source and sweeps, steps, q out with the
    read-back overlapped with the last stage's z-slabs) gives the bits of
    igr_set_conserved + igr_step + igr_get_state, with several slabs (short
    z-chunks), in place or into another buffer, for one or several steps;
    the increment form moves its FP32 state."""
    import torch
    from paper_2505_07392_gb300 import igr
    if host_rk_base and precision.endswith("inc"):
        pytest.skip("the increment forms keep the RK base on the device")
    c = _jets()
    npdt = {"f32": np.float32, "f16": np.float16, "f16inc": np.float32}[precision]
    q0 = inputs.jet_initial_state(c).astype(npdt)
    with igr.Solver(c, precision, host_rk_base=host_rk_base) as s:
        s.set_tiles(4, 4, 4)  # nz = 32: eight flux chunks, so several slabs
        s.set_state(torch.from_numpy(q0).cuda())
        s.step(1)
        ref = []
        for n in (1, 3):
            s.step(n)
            qh = np.empty((5,) + s.shape, dtype=npdt)
            s.get_state_host(qh)
            ref.append(qh)
        _, sig_ref = s.get_state()
    with igr.Solver(c, precision, host_rk_base=host_rk_base) as s:
        s.set_tiles(4, 4, 4)
        s.set_state(torch.from_numpy(q0).cuda())
        s.step(1)
        qh = np.empty((5,) + s.shape, dtype=npdt)
        s.get_state_host(qh)
        s.step_host(qh)  # in place
        assert np.array_equal(qh.view(np.uint8), ref[0].view(np.uint8))
        out = np.empty_like(qh)
        s.step_host(qh, out, nsteps=3)
        assert np.array_equal(out.view(np.uint8), ref[1].view(np.uint8))
        _, sig = s.get_state()
    assert torch.equal(sig, sig_ref)


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_step_host_ragged_slabs(precision):
    """igr_step_host with nz not a multiple of the chunk (29 planes in chunks
    of 4: eight chunks, the last one short, in eight slabs), through raw
    pinned host tensors (BF16 has no numpy type), against separate calls."""
    import ctypes
    import torch
    from dataclasses import replace
    from paper_2505_07392_gb300 import igr
    c = replace(_jets(), nz=29)
    dt = igr.storage_torch_dtype(precision)
    code = {"bf16": igr.DT_BF16, "f16": igr.DT_F16}[precision]
    q0 = torch.from_numpy(inputs.jet_initial_state(c)).to(dt)
    L = igr.lib()
    with igr.Solver(c, precision) as s:
        s.set_tiles(4, 4, 4)
        s.set_state(q0.cuda())
        s.step(2)
        ref, _ = s.get_state()
    with igr.Solver(c, precision) as s:
        s.set_tiles(4, 4, 4)
        s.set_state(q0.cuda())
        s.step(1)
        h = torch.empty((5,) + s.shape, dtype=dt, pin_memory=True)
        assert L.igr_get_state(s.h, ctypes.c_void_p(h.data_ptr()), None, code, 0) == igr.OK
        assert L.igr_step_host(s.h, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(h.data_ptr()), 1,
                               code) == igr.OK
    assert torch.equal(h.cuda(), ref)
