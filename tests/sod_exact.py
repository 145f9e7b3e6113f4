"""Exact solution of the 1D Riemann problem for an ideal gas.

Written from the textbook pressure-function formulation (Toro, Riemann
Solvers and Numerical Methods for Fluid Dynamics, Ch. 4): the star pressure
p* solves f_L(p) + f_R(p) + u_R - u_L = 0, with f_K the shock (Rankine-
Hugoniot) branch for p > p_K and the rarefaction (isentropic) branch
otherwise; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2. The solution is then
sampled along x/t. Used only as a test pin of the oracle's shock behaviour.
"""
import math

import numpy as np


def _f(p, rho, pk, g):
    """f_K(p) and its derivative."""
    c = math.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (g - 1.0) / (2.0 * g)
    f = 2.0 * c / (g - 1.0) * ((p / pk) ** e - 1.0)
    df = 1.0 / (rho * c) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(L, R, g=1.4):
    rl, ul, pl = L
    rr, ur, pr = R
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _f(p, rl, pl, g)
        fr, dr = _f(p, rr, pr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-15 * p:
            break
    fl, _ = _f(p, rl, pl, g)
    fr, _ = _f(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    # densities either side of the contact
    def rho_star(rho, pk):
        if p > pk:
            r = p / pk
            gg = (g - 1.0) / (g + 1.0)
            return rho * (r + gg) / (gg * r + 1.0)
        return rho * (p / pk) ** (1.0 / g)
    return p, u, rho_star(rl, pl), rho_star(rr, pr)


def sample(L, R, x, t, x0=0.5, g=1.4):
    """(rho, u, p) at positions x (array) and time t > 0."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us, rsl, rsr = star_state(L, R, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    out = np.empty((3, len(x)))
    for n, xx in enumerate(x):
        s = (xx - x0) / t
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                w = (rl, ul, pl) if s <= sl else (rsl, us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - cl:
                    w = (rl, ul, pl)
                elif s >= us - csl:
                    w = (rsl, us, ps)
                else:
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    w = (rl * (c / cl) ** (2 / (g - 1)), u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                w = (rr, ur, pr) if s >= sr else (rsr, us, ps)
            else:
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + cr:
                    w = (rr, ur, pr)
                elif s <= us + csr:
                    w = (rsr, us, ps)
                else:
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    w = (rr * (c / cr) ** (2 / (g - 1)), u, pr * (c / cr) ** (2 * g / (g - 1)))
        out[:, n] = w
    return out
