"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

Textbook method (Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4): Newton iteration on the pressure function for the star
pressure, then sampling of the self-similar wave fan. Written for the tests;
independent of both the oracle and the CUDA library.
"""
import math

import numpy as np


def _fk(p, rk, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    pr = p / pk
    f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    d = 1.0 / (rk * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, d


def star_state(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum generated")
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _fk(p, rl, pl, cl, g)
        fr, dr = _fk(p, rr, pr, cr, g)
        f = fl + fr + (ur - ul)
        pn = max(1e-14, p - f / (dl + dr))
        if abs(pn - p) <= 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, g=1.4):
    """Density, velocity, pressure at similarity coordinates xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    xi = np.asarray(xi, dtype=float)
    out = np.zeros((3,) + xi.shape)
    gm = (g - 1.0) / (g + 1.0)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1.0) / (2 * g) * ps / pl + (g - 1.0) / (2 * g))
                if s <= sl:
                    v = (rl, ul, pl)
                else:
                    v = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1.0) / (2 * g))
                if s <= ul - cl:
                    v = (rl, ul, pl)
                elif s >= us - csl:
                    v = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * (ul - s))
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    v = (r, u, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1.0) / (2 * g) * ps / pr + (g - 1.0) / (2 * g))
                if s >= sr:
                    v = (rr, ur, pr)
                else:
                    v = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:
                csr = cr * (ps / pr) ** ((g - 1.0) / (2 * g))
                if s >= ur + cr:
                    v = (rr, ur, pr)
                elif s <= us + csr:
                    v = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2.0 * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - (g - 1.0) / 2.0 * (ur - s))
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    v = (r, u, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        out[(slice(None),) + idx] = v
    return out
