"""Shared test utilities (no scheme arithmetic: norms, fixtures, admissibility)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table1():
    """{(limiter, N): (L1, L2, Linf)} from the printed Table 1 fixture."""
    out = {}
    with open(os.path.join(GOLDEN, "table1_entropy_wave.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lim, n, a, b, c = line.split()
            out[(lim, int(n))] = (float(a), float(b), float(c))
    return out


def rel_norms(x, ref):
    e = np.abs(np.asarray(x) - np.asarray(ref))
    r = np.abs(np.asarray(ref))
    return (e.sum() / r.sum(), np.sqrt((e ** 2).sum() / (r ** 2).sum()), e.max() / r.max())


def internal_energy(u):
    """rho e = E - |m|^2 / (2 rho) for a (4, ...) conserved array."""
    return u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0]


def admissible(u):
    """Membership of the convex set G: rho > 0 and E - |m|^2/(2 rho) > 0."""
    return (u[0] > 0) & (internal_energy(u) > 0)


def euler_flux_x(u, gamma=1.4):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (v1 * v1 + v2 * v2))
    return np.array([rho * v1, rho * v1 * v1 + p, rho * v1 * v2, (E + p) * v1])


def euler_flux_y(u, gamma=1.4):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (v1 * v1 + v2 * v2))
    return np.array([rho * v2, rho * v1 * v2, rho * v2 * v2 + p, (E + p) * v2])


def transpose_state(s):
    """Swap x and y in a (20, ny, nx) state: m1 <-> m2, u_1 <-> u_3, u_2 <-> u_4."""
    t = np.swapaxes(s, 1, 2).copy()
    out = t.copy()
    for k in range(5):
        out[4 * k + 1] = t[4 * k + 2]
        out[4 * k + 2] = t[4 * k + 1]
    out[4:8], out[12:16] = out[12:16].copy(), out[4:8].copy()
    out[8:12], out[16:20] = out[16:20].copy(), out[8:12].copy()
    return out
