"""Pins of the per-face limiter bounds (Sec. 3.3-3.4) by brute force (no GPU).

The closed-form spectral radius is checked against a dense generalized eigen-solve
of the printed matrices A and B and against sampling of phi; every bound is checked
to be the largest theta that keeps the convex-decomposition states inside the
bounds, found by bisection on the definition (density bounds, membership of G).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W


def _pair(rng):
    """A random intermediate state u* in G and a random correction dF."""
    rho = rng.uniform(0.05, 3.0)
    v = rng.uniform(-3, 3, 2)
    p = 10 ** rng.uniform(-4, 1)
    us = np.array([rho, rho * v[0], rho * v[1], p / 0.4 + 0.5 * rho * v @ v])
    df = rng.normal(size=4) * 10 ** rng.uniform(-3, 1, size=4)
    return us, df


def _A_B(us, df):
    A = np.array([[df[0], 0, -df[1]], [0, df[0], -df[2]], [-df[1], -df[2], 2 * df[3]]])
    B = np.array([[us[0], 0, -us[1]], [0, us[0], -us[2]], [-us[1], -us[2], 2 * us[3]]])
    return A, B


def _in_G(u):
    return u[0] > 0 and u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0] > 0


def test_gql_radius_matches_generalized_eigensolve():
    rng = np.random.default_rng(0)
    for _ in range(500):
        us, df = _pair(rng)
        A, B = _A_B(us, df)
        lam = scipy.linalg.eigh(A, B, eigvals_only=True)
        ref = np.abs(lam).max()
        got = O.gql_radius(us, df)
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-300)


def test_gql_radius_is_min_of_phi():
    """min over w of phi(w) = 1 / radius (Sec. 3.4), by sampling w and at the eigenvector."""
    rng = np.random.default_rng(1)
    for _ in range(60):
        us, df = _pair(rng)
        A, B = _A_B(us, df)
        r = O.gql_radius(us, df)
        w = rng.normal(size=(20000, 2)) * 5
        ww = (w ** 2).sum(1)
        num = us[0] * ww - 2 * us[1] * w[:, 0] - 2 * us[2] * w[:, 1] + 2 * us[3]
        den = np.abs(df[0] * ww - 2 * df[1] * w[:, 0] - 2 * df[2] * w[:, 1] + 2 * df[3])
        assert np.all(num / den >= (1.0 / r) * (1 - 1e-9))
        lam, Z = scipy.linalg.eigh(A, B)
        z = Z[:, np.argmax(np.abs(lam))]
        phi = (z @ B @ z) / abs(z @ A @ z)
        assert phi == pytest.approx(1.0 / r, rel=1e-8)


def _largest(pred, hi=1e6):
    """Largest theta in [0, hi] with pred(theta), pred monotone (an interval from 0)."""
    lo = 0.0
    if pred(hi):
        return hi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if pred(mid):
            lo = mid
        else:
            hi = mid
    return lo


def test_theta_p_is_largest_admissible():
    """theta_p = largest theta with u* -/+ theta dF / kappa in G (eq. GQL)."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        us, df = _pair(rng)
        kappa = rng.uniform(0.5, 5.0)
        tp = O.theta_p(kappa, 0.0, us, df)
        ref = _largest(lambda t: _in_G(us - t / kappa * df) and _in_G(us + t / kappa * df))
        assert tp == pytest.approx(ref, rel=1e-7)
        # the epsilon of Sec. 3.4 only ever lowers the bound
        assert O.theta_p(kappa, 1e-16, us, df) <= tp


def test_theta_rho_pp_is_largest_positive():
    rng = np.random.default_rng(3)
    for _ in range(300):
        rs = rng.uniform(0.01, 2)
        dfr = rng.normal() * 10 ** rng.uniform(-3, 1)
        kappa = rng.uniform(0.5, 5)
        got = O.theta_rho_pp(kappa, 0.0, rs, dfr)
        ref = _largest(lambda t: rs - t / kappa * dfr > 0 and rs + t / kappa * dfr > 0)
        assert got == pytest.approx(ref, rel=1e-9)
    assert O.theta_rho_pp(1.0, 1e-16, 1.0, 0.0) == 1.0


def test_theta_rho_lmp_is_largest_within_bounds():
    """The three printed cases of Sec. 3.3.1: u^(1) stays in the bounds of the left cell
    and u^(2) in those of the right cell."""
    rng = np.random.default_rng(4)
    for _ in range(500):
        rs = rng.uniform(0.5, 2)
        mu_l, mu_r = rs - rng.uniform(0, 0.5, 2) * (rng.uniform() > 0.2)
        nu_l, nu_r = rs + rng.uniform(0, 0.5, 2) * (rng.uniform() > 0.2)
        dfr = rng.normal() * (rng.uniform() > 0.05)
        kappa = rng.uniform(0.5, 5)
        got = O.theta_rho_lmp(kappa, rs, dfr, mu_l, nu_l, mu_r, nu_r)
        if dfr == 0.0:
            assert got == 1.0
            continue
        ref = _largest(lambda t: mu_l <= rs - t / kappa * dfr <= nu_l
                       and mu_r <= rs + t / kappa * dfr <= nu_r)
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("lim", [O.LIM_PP, O.LIM_LMP, O.LIM_RLMP])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 2, 2, 1)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bruteforce_theta_on_4x4(lim, bc, seed):
    """On a 4x4 grid, every face's theta is the largest value in [0, 1] that keeps both
    convex-decomposition states of the face (eq. convex_decomposition_blending) in G and,
    for (R)LMP, inside the density bounds of the cell they belong to. The bounds are
    enumerated here from the face states."""
    nx = ny = 4
    p = W.random_cells(nx, ny, 100 + seed, bc=bc, rho_range=(0.05, 2.0), p_range=(0.01, 2.0),
                       v_range=(-2.0, 2.0))
    cfg = O.Config(nx, ny, bc, lim)
    s = O.new_state(p.conserved())
    a = O.kinetic_speed(O.max_speed(cfg, s), 0.5)
    s = O.init_populations(cfg, s, a)
    for _ in range(2):
        s = O.step(O.Config(nx, ny, bc, O.LIM_FIRST), s, a)  # non-equilibrium populations
        a = O.kinetic_speed(O.max_speed(cfg, s), 0.5)
    _, d = O.step(cfg, s, a, debug=True)
    kappa = a / 4.0
    usx, usy, dfx, dfy = d["ustar_x"], d["ustar_y"], d["dflux_x"], d["dflux_y"]

    # density bounds of interior cells by enumeration (eq. LMP_minmax)
    def bounds(j, i):
        vals = [s[0, j, i], usx[j, i, 0], usx[j, i + 1, 0], usy[j, i, 0], usy[j + 1, i, 0]]
        lo, hi = min(vals), max(vals)
        if lim == O.LIM_RLMP:
            lo, hi = 0.999 * lo, 1.001 * hi
        return lo, hi

    checked = 0
    for j in range(ny):
        for i in range(nx + 1):  # x-faces i-1/2
            if not (1 <= i <= nx - 1):
                continue  # bounds of ghost cells are not enumerated here
            us, df = usx[j, i], dfx[j, i]
            bl, br = bounds(j, i - 1), bounds(j, i)
            checked += _check_face(lim, kappa, us, df, bl, br, d["theta_x"][j, i])
        for i in range(nx):
            for jj in range(1, ny):  # y-faces jj-1/2 between rows jj-1 and jj
                us, df = usy[jj, i], dfy[jj, i]
                bl, br = bounds(jj - 1, i), bounds(jj, i)
                checked += _check_face(lim, kappa, us, df, bl, br, d["theta_y"][jj, i])
    assert checked > 0


def _check_face(lim, kappa, us, df, bl, br, theta):
    def ok(t):
        u1 = us - t / kappa * df      # belongs to the left / lower cell
        u2 = us + t / kappa * df      # belongs to the right / upper cell
        if not (_in_G(u1) and _in_G(u2)):
            return False
        if lim in (O.LIM_LMP, O.LIM_RLMP):
            return bl[0] <= u1[0] <= bl[1] and br[0] <= u2[0] <= br[1]
        return True
    if df[0] == 0.0:
        return 0
    ref = min(1.0, _largest(ok, hi=1.0))
    assert theta == pytest.approx(ref, rel=1e-7, abs=1e-12), (theta, ref)
    return 1
