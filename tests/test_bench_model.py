"""The algorithmic byte model behind bench.py's roofline (CPU only): words
per cell of each kernel class, counted from the fields each kernel reads and
writes, and the step totals they add up to."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2505_07392_gb300 import inputs  # noqa: E402


def _words(sweeps):
    # per stage: source reads rho, m (4) and writes b (1); a sweep reads
    # Sigma, rho, b (3) and writes Sigma (1); the flux kernel reads q (5) and
    # Sigma (1) and writes q (5), and from stage 2 on also reads the RK base (5)
    source = 3 * (4 + 1)
    jacobi = 3 * sweeps * (3 + 1)
    flux = (5 + 1 + 5) + 2 * (5 + 1 + 5 + 5)
    return source, jacobi, flux


def test_one_storage_type():
    for prec, w in (("f64", 8), ("f32", 4), ("f16", 2), ("bf16", 2)):
        for sweeps in (5, 10):
            s, j, f = _words(sweeps)
            assert bench.bytes_per_cell(sweeps, prec) == {"source": s * w, "jacobi": j * w, "flux": f * w}
            assert s + j + f == 58 + 12 * sweeps
    assert sum(bench.bytes_per_cell(5, "f16").values()) == 236
    assert sum(bench.bytes_per_cell(5, "f32").values()) == 472


def test_increment_forms():
    # FP32 state (4 B), 16-bit increments, Sigma, b and stage density (2 B)
    source = (4 * 4 + 2 * 2) + 2 * (4 * 4 + 4 * 2 + 2 * 2)  # stage 1 reads rho, m; 2, 3 also their increments
    jacobi = 3 * 5 * (3 * 2 + 2)
    flux = (5 * 4 + 2 + 5 * 2) + (5 * 4 + 5 * 2 + 2 + 5 * 2) + (5 * 4 + 5 * 2 + 2 + 5 * 4)
    for prec in ("f16inc", "bf16inc"):
        assert bench.bytes_per_cell(5, prec) == {"source": source, "jacobi": jacobi, "flux": flux}
    assert source + jacobi + flux == 322


def test_state_bytes():
    c = inputs.density_wave(8)
    n = c.ncells
    assert bench.igr_state_bytes(c, "f64") == n * 6 * 8
    assert bench.igr_state_bytes(c, "f32") == n * 6 * 4
    assert bench.igr_state_bytes(c, "f16") == n * 6 * 2
    assert bench.igr_state_bytes(c, "f16inc") == n * (5 * 4 + 2)
