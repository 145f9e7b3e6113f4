"""The oracle's pins catch plausible mistakes. Each entry below plants one
mistake (a wrong weight, sign, index or coefficient, a dropped or
transposed term) in a copy of igr_oracle.c, builds it, and runs the pins
of tests/test_oracle_pins.py against it in a subprocess: at least one pin
must fail. The mistakes are planted in throw-away copies of the oracle on
the CPU; nothing here touches the CUDA path."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "igr_oracle.c")

# name: (text in igr_oracle.c, replacement, how many occurrences to replace (0: all))
MUTATIONS = {
    "left face weight 47 -> 46": (
        "return (2.0 * v[0] - 13.0 * v[1] + 47.0 * v[2]", "return (2.0 * v[0] - 13.0 * v[1] + 46.0 * v[2]", 1),
    "right face stencil shifted by one cell": (
        "return (-3.0 * v[1] + 27.0 * v[2] + 47.0 * v[3] - 13.0 * v[4] + 2.0 * v[5]) / 60.0;",
        "return (-3.0 * v[0] + 27.0 * v[1] + 47.0 * v[2] - 13.0 * v[3] + 2.0 * v[4]) / 60.0;", 1),
    "LF dissipation sign": (
        "- 0.5 * lam * (qR[v] - qL[v]);", "+ 0.5 * lam * (qR[v] - qL[v]);", 1),
    "LF speed: min instead of max": (
        "double lam = aL > aR ? aL : aR;", "double lam = aL < aR ? aL : aR;", 1),
    "Sigma enters the flux with a minus sign": (
        "    double P = p + sig;\n    F[0] = rho * u[d];", "    double P = p - sig;\n    F[0] = rho * u[d];", 1),
    "kinetic energy without the 1/2": (
        "double ke = 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);",
        "double ke = 1.0 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);", 1),
    "energy flux without the pressure work": (
        "F[4] = (E + P) * u[d];", "F[4] = E * u[d];", 1),
    "sound speed without gamma": (
        "return fabs(u[d]) + sqrt(g->gamma * p / rho);", "return fabs(u[d]) + sqrt(p / rho);", 1),
    "flux divergence sign": (
        "L[v * N + I(g, i, j, k)] += F[v * NF + hi] - F[v * NF + lo];",
        "L[v * N + I(g, i, j, k)] += F[v * NF + lo] - F[v * NF + hi];", 1),
    "source without tr(G)^2": (
        "b[I(g, i, j, k)] = g->alpha * (trG2 + trG * trG);", "b[I(g, i, j, k)] = g->alpha * trG2;", 1),
    "source with G_ac G_ac instead of G_ac G_ca": (
        "trG2 += Gm[a][c] * Gm[c][a];", "trG2 += Gm[a][c] * Gm[a][c];", 1),
    "one-sided velocity gradient": (
        "Gm[a][c] = (up - um) / (2.0 * g->dx);", "Gm[a][c] = (up - m[a][GI(g, i, j, k)] / rho[GI(g, i, j, k)]) / g->dx;", 1),
    "face coefficient r_i instead of (r_i + r_nb)/2": (
        "double cf = 0.5 * (ri + 1.0 / rho[nb]);", "double cf = ri;", 0),
    "Jacobi diagonal without beta": (
        "                            diag += beta * cf;\n", "                            diag += cf;\n", 1),
    "RK stage-2 weight 1/4 -> 1/3": (
        "orc_stage(g, q1, q, sigma, q2, 0.25, dt);", "orc_stage(g, q1, q, sigma, q2, 1.0 / 3.0, dt);", 1),
    "RK increment without (qs - qn)": (
        "out[n] = qn[n] + w * ((qs[n] - qn[n]) + dt * L[n]);", "out[n] = qn[n] + w * dt * L[n];", 1),
    "dt rule without dx": (
        "g->cfl * g->dx / orc_max_speed(g, q)", "g->cfl / orc_max_speed(g, q)", 1),
    "outflow ghost copies the second-nearest cell": (
        "int shi = g->bc[1] == BC_PERIODIC ? hi % nx : nx - 1;", "int shi = g->bc[1] == BC_PERIODIC ? hi % nx : nx - 2;", 1),
    "jet blend weight inverted": (
        "double sn = 0.5 * (1.0 - tanh((r - J[2]) / (J[6] * g->dx)));",
        "double sn = 0.5 * (1.0 + tanh((r - J[2]) / (J[6] * g->dx)));", 1),
    "viscous stress without the transpose term": (
        "double tau = g->mu * (Gr[a][d] + Gr[d][a])", "double tau = g->mu * (Gr[a][d] + Gr[a][d])", 1),
    "viscous work at one cell instead of the face mean": (
        "work += 0.5 * (uA[a] + uB[a]) * tau;", "work += uA[a] * tau;", 1),
    "bulk viscosity coefficient zeta + 2 mu / 3": (
        "(g->zeta - 2.0 * g->mu / 3.0) * div", "(g->zeta + 2.0 * g->mu / 3.0) * div", 1),
    "viscous normal derivative without 1/dx": (
        "Gr[a][d] = (uB[a] - uA[a]) / g->dx;", "Gr[a][d] = (uB[a] - uA[a]);", 1),
    "viscous tangential derivative over 2 dx": (
        "Gr[a][t] = ((uAp[a] - uAm[a]) + (uBp[a] - uBm[a])) / (4.0 * g->dx);",
        "Gr[a][t] = ((uAp[a] - uAm[a]) + (uBp[a] - uBm[a])) / (2.0 * g->dx);", 1),
    "3rd-order left face weights (-1, 4, 3)/6": (
        "return (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;", "return (-v[1] + 4.0 * v[2] + 3.0 * v[3]) / 6.0;", 1),
    "jet energy without the kinetic term": (
        "qj[4] = p / (g->gamma - 1.0) + 0.5 * rho * w * w;", "qj[4] = p / (g->gamma - 1.0);", 1),
    "inflow corner ghost blended at its own (unmapped) column": (
        "double x = (mi + 0.5) * g->dx, y = (mj + 0.5) * g->dx;",
        "double x = (i + 0.5) * g->dx, y = (j + 0.5) * g->dx;", 1),
    "Sigma ghosts blended with the jet state": (
        "    fill_axis_z(g, sg, -1);\n}", "    fill_axis_z(g, sg, 0);\n}", 1),
    "periodic z-ghost wrapped one cell too far": (
        "int shi = g->bc[5] == BC_PERIODIC ? hi % nz : nz - 1;", "int shi = g->bc[5] == BC_PERIODIC ? (hi + 1) % nz : nz - 1;", 1),
    "CFL speed without gamma": (
        "        double c = sqrt(g->gamma * p / rho);\n        for (int d = 0; d < 3; d++) {",
        "        double c = sqrt(p / rho);\n        for (int d = 0; d < 3; d++) {", 1),
    "adjoint: LF dissipation sign": (
        "qLb[v] += 0.5 * lam * Fh_b[v];", "qLb[v] -= 0.5 * lam * Fh_b[v];", 1),
    "adjoint: left face weight 47 -> 46": (
        "static const double cl[6] = {2.0 / 60, -13.0 / 60, 47.0 / 60,",
        "static const double cl[6] = {2.0 / 60, -13.0 / 60, 46.0 / 60,", 1),
    "adjoint: stage-2 weight": (
        "const double wst[3] = {1.0, 0.25, 2.0 / 3.0};", "const double wst[3] = {1.0, 0.3, 2.0 / 3.0};", 1),
    "adjoint: Jacobi mu without the diagonal": (
        "mu[c] = sb[c] / diag;", "mu[c] = sb[c];", 1),
    "adjoint: Jacobi density term sign": (
        "rhob[c] -= rb[c] / (rho[c] * rho[c]);", "rhob[c] += rb[c] / (rho[c] * rho[c]);", 1),
    "adjoint: pressure work into the energy": (
        "    Eb += Fb[4] * u[d];\n    Pb += Fb[4] * u[d];", "    Eb += Fb[4] * u[d];\n    Pb += 0.0 * Fb[4] * u[d];", 1),
    "adjoint: sound-speed derivative in p": (
        "pb += ab * gm / (2.0 * c * rho);", "pb += ab * gm / (c * rho);", 1),
}

RUNNER = r'''
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import oracle
oracle.build = lambda force=False: LIB
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", ROOT + "/tests/test_oracle_pins.py"]))
'''


def _survives(name, gcc, tmp):
    """True when every pin passes with mistake `name` planted."""
    old, new, count = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, "the mutation no longer matches the oracle source: " + name
    mutated = src.replace(old, new) if count == 0 else src.replace(old, new, count)
    assert mutated != src
    d = os.path.join(tmp, "m%d" % list(MUTATIONS).index(name))
    os.makedirs(d)
    c_file = os.path.join(d, "igr_oracle_mutant.c")
    with open(c_file, "w") as f:
        f.write(mutated)
    lib = os.path.join(d, "libigr_oracle_mutant.so")
    subprocess.run([gcc, "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                    "-shared", "-o", lib, c_file, "-lm"], check=True)
    code = "ROOT = %r\nLIB = %r\n" % (ROOT, lib) + RUNNER
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    return r.returncode == 0


def test_pins_catch_every_planted_mistake(tmp_path):
    import concurrent.futures as cf
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    with cf.ThreadPoolExecutor(4) as ex:
        alive = dict(zip(MUTATIONS, ex.map(lambda n: _survives(n, gcc, str(tmp_path)), MUTATIONS)))
    survivors = [n for n, a in alive.items() if a]
    assert not survivors, "no pin fails with: " + "; ".join(survivors)
