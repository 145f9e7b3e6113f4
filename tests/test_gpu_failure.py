"""Failure detection made on the host: an allocation that the caller's
allocator refuses. igr_create asks the allocator for every device buffer;
when any one request fails it must return IGR_ERR_OOM, hand back everything
it did get, and leave the device usable (nothing faults)."""
import ctypes as C

import pytest

from paper_2505_07392_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_07392_gb300 import build
    build.build()
    yield


def _allocator(fail_at):
    """An allocator over torch's caching allocator that refuses request
    number fail_at (0-based; None: never) and records what is live."""
    import torch
    live, count = {}, [0]
    dev = torch.cuda.current_device()

    @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
    def alloc(nbytes, user):
        n = count[0]
        count[0] += 1
        if fail_at is not None and n == fail_at:
            return None
        p = int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))
        live[p] = nbytes
        return p

    @C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)
        live.pop(ptr)

    from paper_2505_07392_gb300 import igr
    return igr.Allocator(alloc, free, None), live, count, (alloc, free)


@pytest.mark.parametrize("host_rk_base", [False, True])
def test_refused_allocation_returns_oom_and_frees(host_rk_base):
    import torch
    from paper_2505_07392_gb300 import igr
    L = igr.lib()
    case = inputs.blast(16, sweeps=2)
    cfg, _jets = igr.make_config(case, "f16", host_rk_base=host_rk_base)
    # how many requests a successful create makes
    a, live, count, keep = _allocator(None)
    h = C.c_void_p()
    assert L.igr_create(C.byref(cfg), C.byref(a), None, C.byref(h)) == igr.OK
    n = count[0]
    assert n >= 5 and live
    assert L.igr_destroy(h) == igr.OK
    assert not live
    for k in range(n):
        a, live, count, keep = _allocator(k)
        h = C.c_void_p()
        st = L.igr_create(C.byref(cfg), C.byref(a), None, C.byref(h))
        assert st == igr.ERR_OOM, (k, st)
        assert not h.value
        assert not live, k  # every buffer it got was handed back
    # the device is still usable
    with igr.Solver(case, "f16") as s:
        s.set_state(torch.from_numpy(inputs.initial_state(case)).half().cuda())
        s.step(1)
