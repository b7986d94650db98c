"""Seeded synthetic initial data for the blended D2Q5 vectorial LBM.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle. It holds only problem definitions: analytic or seeded initial states in
primitive variables (rho, v1, v2, p), turned into the conserved variables
(rho, rho*v1, rho*v2, E) of the problem statement with the ideal-gas law
p = (gamma-1)(E - rho|v|^2/2) (paper, Sec. 1, the Euler system and its
equation of state). None of the scheme's arithmetic (equilibria, intermediate
states, limiters, collide-and-stream) lives here.

Conventions: every field is a float64 array of shape (ny, nx), x fastest,
cell (i, j) centred at (x0 + (i + 1/2) dx, y0 + (j + 1/2) dx).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4


@dataclass
class Problem:
    """One initial-value problem on a uniform Cartesian grid."""

    name: str
    nx: int
    ny: int
    dx: float
    x0: float
    y0: float
    rho: np.ndarray
    m1: np.ndarray
    m2: np.ndarray
    E: np.ndarray
    bc: tuple = (0, 0, 0, 0)  # west, east, south, north: 0 periodic, 1 zero-gradient, 2 reflective,
    #                           3 prescribed (Dirichlet) state
    gamma: float = GAMMA
    meta: dict = field(default_factory=dict)
    # a side that switches type along its length: ghost cells with index along the
    # side (column for south/north, row for west/east) >= split[s] take bc_hi[s]
    bc_hi: tuple | None = None
    split: tuple = (0, 0, 0, 0)
    bfield: "BoundaryField | None" = None

    def conserved(self) -> np.ndarray:
        """(4, ny, nx) float64 stack of rho, m1, m2, E."""
        return np.stack([self.rho, self.m1, self.m2, self.E])


@dataclass
class BoundaryField:
    """State prescribed on the Dirichlet parts of the boundary: at time t, the cell
    with centre (x, y) holds the conserved state `inside` if
    nx x + ny y >= c0 + c1 t for each half-plane (nx, ny, c0, c1), else `outside`."""

    inside: tuple
    outside: tuple
    planes: tuple = ()

    def state_at(self, x, y, t: float = 0.0) -> np.ndarray:
        """(4, *x.shape) conserved field; the half-plane test in the operation order
        of the library and the oracle (products, then the sums)."""
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        inside = np.ones(x.shape, dtype=bool)
        for (a, b, c0, c1) in self.planes:
            inside &= (a * x + b * y) >= (c0 + c1 * t)
        out = np.empty((4,) + x.shape)
        for q in range(4):
            out[q] = np.where(inside, self.inside[q], self.outside[q])
        return out


def cell_centres(nx: int, ny: int, dx: float, x0: float = 0.0, y0: float = 0.0):
    x = x0 + (np.arange(nx) + 0.5) * dx
    y = y0 + (np.arange(ny) + 0.5) * dx
    return np.meshgrid(x, y)  # each (ny, nx)


def primitive_to_conserved(rho, v1, v2, p, gamma=GAMMA):
    """Ideal-gas conserved variables of the Euler system (paper Sec. 1)."""
    rho = np.asarray(rho, dtype=np.float64)
    v1 = np.broadcast_to(np.asarray(v1, dtype=np.float64), rho.shape)
    v2 = np.broadcast_to(np.asarray(v2, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    m1 = rho * v1
    m2 = rho * v2
    E = p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)
    return rho.copy(), m1.copy(), m2.copy(), E.copy()


def _make(name, nx, ny, dx, x0, y0, prim, bc, gamma=GAMMA, **meta) -> Problem:
    rho, m1, m2, E = primitive_to_conserved(*prim, gamma=gamma)
    return Problem(name, nx, ny, dx, x0, y0, rho, m1, m2, E, tuple(bc), gamma, dict(meta))


# --------------------------------------------------------------------------
# Sinusoidal entropy wave (paper Sec. 4.1, Table 1)
# --------------------------------------------------------------------------
def entropy_wave(n: int, t: float = 0.0) -> Problem:
    """[0,1]^2 periodic, rho = 1 + 0.1 sin(2 pi (x+y)), v = (1, 1), p = 1.

    The exact solution at time t is the initial state translated by (t, t).
    """
    dx = 1.0 / n
    X, Y = cell_centres(n, n, dx)
    rho = 1.0 + 0.1 * np.sin(2.0 * math.pi * ((X - t) + (Y - t)))
    return _make("entropy_wave", n, n, dx, 0.0, 0.0, (rho, 1.0, 1.0, 1.0), (0, 0, 0, 0))


# --------------------------------------------------------------------------
# Isentropic vortex (smooth periodic workload; not in the paper)
# --------------------------------------------------------------------------
def isentropic_vortex(n: int, t: float = 0.0, strength: float = 5.0, L: float = 10.0,
                      uinf=(1.0, 1.0), gamma: float = GAMMA) -> Problem:
    """Shu-Yee isentropic vortex on [0,L]^2, periodic, centred at (L/2, L/2) at t=0.

    rho_inf = p_inf = 1 (T = p/rho = 1), free stream uinf. The exact Euler
    solution at time t is the vortex translated by uinf*t; distances use the
    periodic minimum image, so the box edge carries an O(exp(-12)) mismatch.
    """
    dx = L / n
    X, Y = cell_centres(n, n, dx)
    xc = (0.5 * L + uinf[0] * t) % L
    yc = (0.5 * L + uinf[1] * t) % L
    xb = (X - xc + 0.5 * L) % L - 0.5 * L
    yb = (Y - yc + 0.5 * L) % L - 0.5 * L
    r2 = xb * xb + yb * yb
    du = strength / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    v1 = uinf[0] - du * yb
    v2 = uinf[1] + du * xb
    dT = -(gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return _make("isentropic_vortex", n, n, dx, 0.0, 0.0, (rho, v1, v2, p), (0, 0, 0, 0), gamma,
                 strength=strength, L=L, t=t)


def vortex_with_bumps(n: int, seed: int = 2, nbumps: int = 8, amp: float = 0.05,
                      width: float = 0.3, L: float = 10.0) -> Problem:
    """Isentropic vortex whose density carries `nbumps` seeded Gaussian bumps.

    Centres ~ U[0,L]^2 from default_rng(seed); periodic minimum-image distance;
    velocity and pressure are those of the vortex, so E is recomputed.
    """
    base = isentropic_vortex(n, L=L)
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, L, size=(nbumps, 2))
    X, Y = cell_centres(n, n, base.dx)
    rho = base.rho.copy()
    for cx, cy in centres:
        xb = (X - cx + 0.5 * L) % L - 0.5 * L
        yb = (Y - cy + 0.5 * L) % L - 0.5 * L
        rho += amp * np.exp(-(xb * xb + yb * yb) / (2.0 * width * width))
    v1 = base.m1 / base.rho
    v2 = base.m2 / base.rho
    p = (base.gamma - 1.0) * (base.E - 0.5 * base.rho * (v1 * v1 + v2 * v2))
    return _make("vortex_with_bumps", n, n, base.dx, 0.0, 0.0, (rho, v1, v2, p), (0, 0, 0, 0),
                 centres=centres)


# --------------------------------------------------------------------------
# Seeded four-quadrant Riemann problems
# --------------------------------------------------------------------------
def quadrant_states(rng: np.random.Generator) -> np.ndarray:
    """(4, 4) array: rows SW, SE, NW, NE; columns rho, v1, v2, p.

    rho, p ~ U[0.1, 2]; v1, v2 ~ U[-1, 1]; drawn in that row/column order.
    """
    u = rng.uniform(size=(4, 4))
    s = np.empty((4, 4))
    s[:, 0] = 0.1 + 1.9 * u[:, 0]
    s[:, 1] = -1.0 + 2.0 * u[:, 1]
    s[:, 2] = -1.0 + 2.0 * u[:, 2]
    s[:, 3] = 0.1 + 1.9 * u[:, 3]
    return s


def quadrant_riemann(nx: int, ny: int | None = None, seed: int = 0,
                     states: np.ndarray | None = None, bc=(1, 1, 1, 1)) -> Problem:
    """Four constant states split at the domain centre; dx = 1/nx (x-extent 1)."""
    ny = nx if ny is None else ny
    if states is None:
        states = quadrant_states(np.random.default_rng(seed))
    dx = 1.0 / nx
    X, Y = cell_centres(nx, ny, dx)
    xm, ym = 0.5 * nx * dx, 0.5 * ny * dx
    q = (X > xm).astype(int) + 2 * (Y > ym).astype(int)  # 0 SW, 1 SE, 2 NW, 3 NE
    prim = [states[q, k] for k in range(4)]
    return _make("quadrant_riemann", nx, ny, dx, 0.0, 0.0, prim, bc, states=states)


def lax_liu_config3(n: int) -> Problem:
    """2D Riemann problem, configuration 3 of Lax-Liu (paper Sec. 4.7), split at 0.8."""
    dx = 1.0 / n
    X, Y = cell_centres(n, n, dx)
    st = np.array([[0.138, 1.206, 1.206, 0.029],   # x<=0.8, y<=0.8
                   [0.5323, 0.0, 1.206, 0.3],      # x>0.8,  y<=0.8
                   [0.5323, 1.206, 0.0, 0.3],      # x<=0.8, y>0.8
                   [1.5, 0.0, 0.0, 1.5]])          # x>0.8,  y>0.8
    q = (X > 0.8).astype(int) + 2 * (Y > 0.8).astype(int)
    prim = [st[q, k] for k in range(4)]
    return _make("lax_liu_config3", n, n, dx, 0.0, 0.0, prim, (1, 1, 1, 1))


def batch_instances(count: int = 256, seed: int = 1, sides=tuple(64 * k for k in range(1, 17))):
    """Seeded batch of uneven quadrant Riemann problems.

    Grid sides nx, ny are drawn independently from {64, 128, 192, ..., 1024}
    (multiples of 64) with default_rng(seed); each instance then draws its own
    quadrant states from the same stream. Zero-gradient boundaries on all sides.
    """
    rng = np.random.default_rng(seed)
    sides = np.array(sides)
    nxs = rng.choice(sides, size=count)
    nys = rng.choice(sides, size=count)
    out = []
    for k in range(count):
        st = quadrant_states(rng)
        out.append(quadrant_riemann(int(nxs[k]), int(nys[k]), states=st))
    return out


# --------------------------------------------------------------------------
# Near-vacuum blast (Sedov-type) and 1D-on-2D shock tubes
# --------------------------------------------------------------------------
def blast(n: int, p_ambient: float = 1e-6, energy: float = 1.0, half_width: float = 1.1,
          bc=(2, 2, 2, 2)) -> Problem:
    """[-1.1,1.1]^2, rho = 1, v = 0, p = p_ambient; total energy `energy` put into the
    2x2 centre cells as internal energy (E = energy / (4 dx^2) there). Needs even n."""
    if n % 2:
        raise ValueError("blast needs an even grid")
    dx = 2.0 * half_width / n
    rho = np.ones((n, n))
    p = np.full((n, n), p_ambient)
    r, m1, m2, E = primitive_to_conserved(rho, 0.0, 0.0, p)
    c = n // 2
    E[c - 1:c + 1, c - 1:c + 1] = energy / (4.0 * dx * dx)
    return Problem("blast", n, n, dx, -half_width, -half_width, r, m1, m2, E, tuple(bc), GAMMA,
                   {"p_ambient": p_ambient, "energy": energy})


def shock_tube(nx: int, left, right, x_split: float = 0.5, length: float = 1.0, ny: int = 4,
               gamma: float = GAMMA, bc=(1, 1, 0, 0)) -> Problem:
    """x-only Riemann data (rho, v1, p) on nx x ny cells, periodic in y (paper Sec. 4)."""
    dx = length / nx
    X, _ = cell_centres(nx, ny, dx)
    L = X <= x_split
    rho = np.where(L, left[0], right[0])
    v1 = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    return _make("shock_tube", nx, ny, dx, 0.0, 0.0, (rho, v1, 0.0, p), bc, gamma,
                 left=tuple(left), right=tuple(right), x_split=x_split)


def sod(nx: int, ny: int = 4) -> Problem:
    return shock_tube(nx, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), ny=ny)


def leblanc(nx: int, ny: int = 4) -> Problem:
    """LeBlanc shock tube (Sec. 4.5): [0, 9], split at x = 3, gamma = 5/3,
    (rho, v1, p) = (1, 0, 0.1 (gamma - 1)) left, (1e-3, 0, 1e-7 (gamma - 1)) right."""
    g = 5.0 / 3.0
    return shock_tube(nx, (1.0, 0.0, 0.1 * (g - 1.0)), (1e-3, 0.0, 1e-7 * (g - 1.0)), x_split=3.0,
                      length=9.0, ny=ny, gamma=g)


def near_vacuum_wave(nx: int, ny: int = 4, amp: float = 0.9999995) -> Problem:
    """Near-vacuum smooth isentropic wave (Sec. 4.4): periodic [-1, 1], gamma = 3,
    rho = 1 + amp sin(pi x), v1 = 0, p = rho^gamma (rho down to 5e-7)."""
    g = 3.0
    dx = 2.0 / nx
    X, _ = cell_centres(nx, ny, dx, x0=-1.0)
    rho = 1.0 + amp * np.sin(np.pi * X)
    return _make("near_vacuum_wave", nx, ny, dx, -1.0, 0.0, (rho, 0.0, 0.0, rho ** g), (0, 0, 0, 0), g,
                 amp=amp)


def random_cells(nx: int, ny: int, seed: int, bc=(0, 0, 0, 0), rho_range=(0.1, 2.0),
                 p_range=(0.1, 2.0), v_range=(-1.0, 1.0), gamma=GAMMA) -> Problem:
    """Independent random admissible state in every cell (a discontinuity at every face)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(*rho_range, size=(ny, nx))
    v1 = rng.uniform(*v_range, size=(ny, nx))
    v2 = rng.uniform(*v_range, size=(ny, nx))
    p = rng.uniform(*p_range, size=(ny, nx))
    return _make("random_cells", nx, ny, 1.0 / max(nx, ny), 0.0, 0.0, (rho, v1, v2, p), bc, gamma)


# --------------------------------------------------------------------------
# Prescribed-state boundaries: double Mach reflection (Sec. 4.7) and
# astrophysical jets (Sec. 4.8)
# --------------------------------------------------------------------------
def _conserved_state(rho, v1, v2, p, gamma):
    r, m1, m2, E = primitive_to_conserved(np.array(rho), v1, v2, p, gamma=gamma)
    return (float(r), float(m1), float(m2), float(E))


def double_mach_reflection(ny: int) -> Problem:
    """[0, 3] x [0, 1], gamma = 1.4, a Mach 10 shock through (1/6, 0) at 60 degrees
    to the x-axis moving right: pre-shock (rho, v1, v2, p) = (1.4, 0, 0, 1) where
    x >= 1/6 + (y + 20 t) / sqrt(3), post-shock (8, 8.25 cos(pi/6), -8.25 sin(pi/6),
    116.5) elsewhere. Every side holds that exact moving-shock field (Maxwellian
    populations), except the bottom for x >= 1/6, a reflective wall. nx = 3 ny;
    the paper's grids are 1500 x 500 and 3000 x 1000 to t = 0.2."""
    g = 1.4
    nx = 3 * ny
    dx = 1.0 / ny
    pre = _conserved_state(1.4, 0.0, 0.0, 1.0, g)
    post = _conserved_state(8.0, 8.25 * math.cos(math.pi / 6), -8.25 * math.sin(math.pi / 6), 116.5, g)
    s3 = math.sqrt(3.0)
    bf = BoundaryField(pre, post, ((1.0, -1.0 / s3, 1.0 / 6.0, 20.0 / s3),))
    X, Y = cell_centres(nx, ny, dx)
    u = bf.state_at(X, Y, 0.0)
    xc = (np.arange(nx) + 0.5) * dx
    split = int(np.count_nonzero(xc < 1.0 / 6.0))      # bottom cells left of the wall
    return Problem("double_mach_reflection", nx, ny, dx, 0.0, 0.0, u[0], u[1], u[2], u[3],
                   (3, 3, 3, 3), g, {"t_end": 0.2}, bc_hi=(3, 3, 2, 3), split=(0, 0, split, 0), bfield=bf)


def astro_jet(ny: int, mach: int = 80) -> Problem:
    """High Mach number jet: gamma = 5/3, ambient (rho, v1, v2, p) = (0.5, 0, 0, 0.4127);
    through |y| < 0.05 of the left side the state (5, 30, 0, 0.4127) enters (Mach 80,
    domain [0, 2] x [-0.5, 0.5], t = 0.07) or (5, 800, 0, 0.4127) (Mach 2000, domain
    [0, 1] x [-0.25, 0.25], t = 0.001); elsewhere on the left side the ambient state,
    zero gradient on the other sides. nx = 2 ny (the paper: 800 x 400)."""
    g = 5.0 / 3.0
    if mach == 80:
        length, v_jet, t_end = 2.0, 30.0, 0.07
    elif mach == 2000:
        length, v_jet, t_end = 1.0, 800.0, 0.001
    else:
        raise ValueError("mach is 80 or 2000")
    nx = 2 * ny
    dx = length / nx
    y0 = -length / 4.0
    amb = _conserved_state(0.5, 0.0, 0.0, 0.4127, g)
    jet = _conserved_state(5.0, v_jet, 0.0, 0.4127, g)
    bf = BoundaryField(jet, amb, ((0.0, 1.0, -0.05, 0.0), (0.0, -1.0, -0.05, 0.0)))
    rho = np.full((ny, nx), amb[0])
    return Problem(f"astro_jet_mach{mach}", nx, ny, dx, 0.0, y0, rho, np.zeros_like(rho), np.zeros_like(rho),
                   np.full((ny, nx), amb[3]), (3, 1, 1, 1), g, {"t_end": t_end}, bfield=bf)
