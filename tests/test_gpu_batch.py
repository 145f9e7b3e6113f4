"""Batches and launch shapes on the GPU.

A batch of independent instances (igr_create_batch / igr_step_batch) must
give, instance by instance, the bits a lone context gives: the kernels are
the same and nothing is shared between instances. The launch shape must not
change a bit either: the z-chunk length of every kernel class
(igr_set_tiles / igr_autotune; no atomics, and every face flux comes out of
the same instructions whatever the chunking) and the one- or four-cell form
of the source and Jacobi kernels (igr_set_kernel_forms; both evaluate the
same sequence of rounded operations).
"""
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


def _alone(case, q0, precision, steps, tiles=None, forms=None):
    import torch
    from paper_2505_07392_gb300 import igr
    with igr.Solver(case, precision) as s:
        s.set_state(q0)
        if tiles:
            s.set_tiles(*tiles)
        if forms:
            s.set_kernel_forms(*forms)
            assert s.kernel_forms() == forms
        s.step(steps)
        q, sig = s.get_state()
    return q, sig


@pytest.mark.parametrize("precision", ["f32", "f16", "f16inc"])
def test_batch_equals_single_bitwise(precision):
    import torch
    from paper_2505_07392_gb300 import igr
    from dataclasses import replace
    # uneven sizes, different sweep counts, red-black sweeps, 3rd-order
    # faces and an inflow face in one batch: the grouped launches split by
    # kernel form and scheme, every instance keeps its own buffers
    # 128 x 128 x 12 and 128 x 16 x 12 (red-black): every 4-cell tile inside,
    # the full-tile source and sweep bodies in their own grouped launches
    cases = [inputs.tgv(16, instance=0), inputs.tgv(24, instance=1), inputs.tgv(20, instance=2),
             inputs.blast(12, sweeps=4), replace(inputs.tgv(16, instance=3), sigma_solver=1),
             replace(inputs.blast(12, sweeps=3), order=3), _jets_case(20),
             replace(inputs.tgv(128, instance=4), nz=12),
             replace(inputs.tgv(128, instance=5), ny=16, nz=12, sigma_solver=1)]
    dt = igr.state_torch_dtype(precision)
    q0 = [torch.from_numpy(inputs.jet_initial_state(c) if c.jets else inputs.initial_state(c)).to(dt).cuda()
          for c in cases]
    torch.cuda.synchronize()
    steps = 6  # first step direct, then captured graphs of grouped launches replayed
    with igr.Batch(cases, precision) as b:
        for inst, q in zip(b.instances, q0):
            inst.set_state(q)
        b.step(2)
        b.step(steps - 2, sync=True)
        got = [inst.get_state() for inst in b.instances]
    for c, q, (qb, sb) in zip(cases, q0, got):
        qa, sa = _alone(c, q, precision, steps)
        assert torch.equal(qa, qb), c.name
        assert torch.equal(sa, sb), c.name
        assert torch.isfinite(qb.float()).all()


def test_batch_autotune_keeps_state_and_bits():
    """igr_autotune_batch writes only scratch (states and Sigma unchanged),
    gives every instance z-chunks within [4, nz], and the batch then steps
    to the bits of lone contexts (uneven sizes, red-black sweeps, an inflow
    face, instances given largest last)."""
    import torch
    from paper_2505_07392_gb300 import igr
    from dataclasses import replace
    cases = [inputs.tgv(16, instance=0), replace(inputs.tgv(16, instance=3), sigma_solver=1), _jets_case(20),
             inputs.tgv(24, instance=1), inputs.tgv(32, instance=2)]
    precision = "f16inc"
    dt = igr.state_torch_dtype(precision)
    q0 = [torch.from_numpy(inputs.jet_initial_state(c) if c.jets else inputs.initial_state(c)).to(dt).cuda()
          for c in cases]
    torch.cuda.synchronize()
    with igr.Batch(cases, precision) as b:
        for inst, q in zip(b.instances, q0):
            inst.set_state(q)
        before = [inst.get_state() for inst in b.instances]
        tiles = b.autotune(reps=1)
        after = [inst.get_state() for inst in b.instances]
        for (qa, sa), (qb, sb) in zip(before, after):
            assert torch.equal(qa, qb) and torch.equal(sa, sb)
        for c, t in zip(cases, tiles):
            assert all(min(4, c.nz) <= z <= c.nz for z in t), (c.name, t)
        b.step(2)
        b.step(3, sync=True)
        got = [inst.get_state() for inst in b.instances]
    for c, q, (qb, sb) in zip(cases, q0, got):
        qa, sa = _alone(c, q, precision, 5)
        assert torch.equal(qa, qb), c.name
        assert torch.equal(sa, sb), c.name


def test_results_do_not_depend_on_z_chunks():
    import torch
    from paper_2505_07392_gb300 import igr
    dx = 1.0 / 40
    w = 2.0 * np.sqrt(1.4 * 2.0)
    case = Case("jets", 40, 36, 44, dx, alpha=dx * dx, sweeps=5,
                bc=(OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW, INFLOW, OUTFLOW),
                jets=[(0.3, 0.45, 4 * dx, 1.0, w, 2.0, 1.0), (0.7, 0.55, 3 * dx, 1.0, 0.9 * w, 2.0, 1.0)])
    q0 = torch.from_numpy(inputs.jet_initial_state(case)).float().cuda()
    ref = _alone(case, q0, "f32", 4, tiles=(44, 44, 44))
    for tiles in ((4, 4, 4), (8, 16, 32), (32, 8, 5), (7, 13, 11)):
        q, s = _alone(case, q0, "f32", 4, tiles=tiles)
        assert torch.equal(q, ref[0]), tiles
        assert torch.equal(s, ref[1]), tiles
    with igr.Solver(case, "f32") as s:
        s.set_state(q0)
        tiles = s.autotune(reps=2)
        assert all(4 <= t <= case.nz for t in tiles)
        s.step(4)
        q, sig = s.get_state()
    assert torch.equal(q, ref[0])


def _jets_case(n=40):
    dx = 1.0 / n
    w = 2.0 * np.sqrt(1.4 * 2.0)
    return Case("jets", n, n - 4, n + 4, dx, alpha=dx * dx, sweeps=5,
                bc=(OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW, INFLOW, OUTFLOW),
                jets=[(0.3, 0.45, 4 * dx, 1.0, w, 2.0, 1.0), (0.7, 0.55, 3 * dx, 1.0, 0.9 * w, 2.0, 1.0)])


@pytest.mark.parametrize("precision", ["f64", "f32", "f16", "bf16", "f16inc", "bf16inc"])
@pytest.mark.parametrize("kind", ["jets", "tgv_rbgs", "wide", "wide_rbgs", "full", "full_rbgs"])
def test_kernel_forms_give_the_same_bits(precision, kind):
    """Every combination of the one- and four-cell forms of the source and
    Jacobi kernels gives the same bits. Rows of 40 and 24 cells: the default
    rule picks the one-cell forms there, the four-cell forms are forced, and
    every block of the four-cell forms is an edge block. Rows of 260 cells
    and 20 rows: blocks of 128 x 8 cells inside the grid (no mapped loads)
    beside edge blocks in x and y. Rows of 128 cells and 16 rows: every
    block inside, the sweep launched as the full-tile kernel alone."""
    import torch
    from dataclasses import replace
    from paper_2505_07392_gb300 import igr
    if kind in ("jets", "wide", "full"):
        case = _jets_case()
        if kind == "wide":
            case = replace(case, nx=260, ny=20, nz=12)
        if kind == "full":
            case = replace(case, nx=128, ny=16, nz=12)
        q0 = torch.from_numpy(inputs.jet_initial_state(case))
    else:
        case = replace(inputs.tgv(24, instance=3), sigma_solver=1)
        if kind == "wide_rbgs":
            case = replace(case, nx=260, ny=20, nz=12)
        if kind == "full_rbgs":
            case = replace(case, nx=128, ny=16, nz=12)
        q0 = torch.from_numpy(inputs.initial_state(case))
    q0 = q0.to(igr.state_torch_dtype(precision)).cuda()
    if kind in ("jets", "tgv_rbgs"):
        with igr.Solver(case, precision) as s:
            assert s.kernel_forms() == (0, 0)
    ref = _alone(case, q0, precision, 3, forms=(0, 0))
    for forms in ((1, 1), (1, 0), (0, 1)):
        q, sig = _alone(case, q0, precision, 3, forms=forms)
        assert torch.equal(q, ref[0]), forms
        assert torch.equal(sig, ref[1]), forms
    assert torch.isfinite(ref[0].double()).all()


def test_kernel_form_rule_and_checks():
    """The default rule (four cells where the busy-lane share is at least the
    instruction ratio) and the argument checks of igr_set_kernel_forms."""
    from paper_2505_07392_gb300 import igr
    expect = {48: (0, 0), 64: (0, 0), 80: (1, 0), 96: (1, 0), 128: (1, 1), 130: (0, 0), 256: (1, 1),
              1024: (1, 1)}
    for nx, forms in expect.items():
        c = Case("box", nx, 8, 8, 1.0 / nx, alpha=1.0 / nx ** 2, sweeps=1, bc=(OUTFLOW,) * 6)
        with igr.Solver(c, "f32") as s:
            assert s.kernel_forms() == forms, nx
            if nx % 4 == 0:
                s.set_kernel_forms(1, 1)
                assert s.kernel_forms() == (1, 1)
            else:
                with pytest.raises(igr.IGRError):
                    s.set_kernel_forms(1, 1)
            s.set_kernel_forms(0, 0)
            assert s.kernel_forms() == (0, 0)
            s.set_kernel_forms(-1, -1)
            assert s.kernel_forms() == forms
    c = Case("odd", 30, 8, 8, 1.0 / 30, alpha=1.0 / 900, sweeps=1, bc=(OUTFLOW,) * 6)
    with igr.Solver(c, "f32") as s:
        with pytest.raises(igr.IGRError):
            s.set_kernel_forms(1, 0)
        with pytest.raises(igr.IGRError):
            s.set_kernel_forms(0, 2)



def test_autotune_cache(tmp_path, monkeypatch):
    """A tuned launch shape is stored under its problem and GPU; a second
    context for the same problem takes it from the file; another precision
    is tuned and stored apart."""
    import torch
    from paper_2505_07392_gb300 import igr
    path = str(tmp_path / "tiles.json")
    monkeypatch.setenv("IGR_AUTOTUNE_CACHE", path)
    c = inputs.tgv(32)
    q0 = torch.from_numpy(inputs.initial_state(c))
    with igr.Solver(c, "f16") as s:
        s.set_state(q0.half().cuda())
        tiles = s.autotune(reps=2)
        forms = s.kernel_forms()
    stored = igr.autotune_cache_load(path)
    assert len(stored) == 1
    (entry,) = stored.values()
    assert entry == {"tiles": list(tiles), "forms": list(forms)}
    with igr.Solver(c, "f16") as s:
        s.set_state(q0.half().cuda())
        s.set_tiles(5, 5, 5)
        assert s.autotune(reps=2) == tiles and s.kernel_forms() == forms
    with igr.Solver(c, "f32") as s:
        s.set_state(q0.float().cuda())
        s.autotune(reps=2)
    assert len(igr.autotune_cache_load(path)) == 2
