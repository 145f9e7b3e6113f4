"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a copy
of igr_oracle.c built with -fsanitize=address,undefined (no recovery) runs
the oracle's entry points on tiny grids (every boundary kind, inflow jets,
3rd-order faces, red-black sweeps, viscous terms, the adjoint) in a
subprocess that preloads the ASan runtime. Any out-of-bounds access or
undefined behaviour aborts it."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
import oracle
oracle.build = lambda force=False: LIB
from dataclasses import replace
from paper_2505_07392_gb300 import inputs
from paper_2505_07392_gb300.inputs import Case, INFLOW, OUTFLOW, PERIODIC

def state(c, seed):
    rng = np.random.Generator(np.random.Philox(seed))
    rho = 1 + 0.1 * rng.uniform(-1, 1, (c.nz, c.ny, c.nx))
    m = 0.2 * rng.uniform(-1, 1, (3, c.nz, c.ny, c.nx))
    E = 2.5 + 0.5 * (m ** 2).sum(0) / rho
    return np.concatenate([rho[None], m, E[None]])

dx = 1 / 8
jets = [(0.5, 0.5, 2 * dx, 1.0, 2.0, 2.0, 1.0)]
cases = [Case("p", 6, 5, 7, dx, alpha=dx * dx, sweeps=2, bc=(PERIODIC,) * 6),
         Case("o", 7, 4, 5, dx, alpha=dx * dx, sweeps=2, bc=(OUTFLOW,) * 6),
         Case("j", 8, 8, 6, dx, alpha=dx * dx, sweeps=2, bc=(OUTFLOW,) * 4 + (INFLOW, OUTFLOW), jets=jets)]
cases += [replace(cases[0], order=3, sigma_solver=1), replace(cases[1], mu=1e-3, zeta=2e-3),
          replace(cases[2], order=3, mu=1e-3)]
for n, c in enumerate(cases):
    q = inputs.jet_initial_state(c) if c.jets else state(c, n)
    sig = 0.01 * state(c, n + 7)[0]
    oracle.fill_ghosts(c, q)
    b = oracle.source(c, q)
    oracle.apply_A(c, q, sig)
    oracle.jacobi(c, q, b, sig, 2)
    oracle.rhs(c, q, sig)
    oracle.max_speed(c, q)
    oracle.run(c, q, sig, nsteps=2, fixed_dt=1e-3)
    if c.order == 5 and c.sigma_solver == 0 and c.mu == 0:
        lq = state(c, n + 3)
        oracle.adjoint_step(c, q, sig, 1e-3, lq, 0.1 * lq[0])
print("sanitized oracle ok")
'''


def test_oracle_under_asan_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    asan = subprocess.run([gcc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime")
    lib = str(tmp_path / "libigr_oracle_san.so")
    src = os.path.join(ROOT, "oracle", "igr_oracle.c")
    subprocess.run([gcc, "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fno-omit-frame-pointer",
                    "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fPIC", "-shared",
                    "-o", lib, src, "-lm"], check=True)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    code = "ROOT = %r\nLIB = %r\n" % (ROOT, lib) + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "sanitized oracle ok" in r.stdout
