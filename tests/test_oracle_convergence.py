"""Whole-scheme pins: convergence orders on the isentropic vortex and the exact
Riemann solution for x-only data (no GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W
from tests.exact_riemann import sample

LAM_FIXED = 3.7  # above lambda of the strength-5 vortex (3.34), held constant on every grid


def _vortex_error(n, lim):
    p = W.isentropic_vortex(n)
    cfg = O.Config(n, n, (0, 0, 0, 0), lim)
    a = O.kinetic_speed(LAM_FIXED, 0.5)
    nst = int(round(1.0 * a / p.dx))
    r = O.run(cfg, p.conserved(), p.dx, nsteps=nst, lam_fixed=LAM_FIXED)
    exact = W.isentropic_vortex(n, t=nst * p.dx / a)
    return np.abs(r["state"][0] - exact.rho).mean()


@pytest.mark.parametrize("lim,lo,hi", [(O.LIM_PP, 1.9, 2.1), (O.LIM_SECOND, 1.9, 2.1),
                                        (O.LIM_FIRST, 0.6, 1.1)])
def test_vortex_convergence_order(lim, lo, hi):
    """Second order for the blended scheme with the PP limiter (theta = 1 on smooth
    data), first order for theta = 0 (Sec. 2.1, 2.2)."""
    O.set_threads(4)
    e64, e128, e256 = (_vortex_error(n, lim) for n in (64, 128, 256))
    order = np.log2(e128 / e256)
    assert lo <= order <= hi, (e64, e128, e256, order)
    assert e64 > e128 > e256


@pytest.mark.parametrize("lim", [O.LIM_LMP, O.LIM_RLMP])
def test_sod_against_exact_riemann(lim):
    """Sec. 4.2 setup (1D on 2D, 4 cells periodic in y, zero-gradient x ends, t = 0.2):
    the L1 density error against the exact solution is small and, for LMP, falls with N
    (RLMP trades a little monotonicity for less dissipation, Sec. 4.2)."""
    errs = []
    for n in (100, 200, 400):
        p = W.sod(n)
        r = O.run(O.Config(n, 4, p.bc, lim), p.conserved(), p.dx, t_end=0.2)
        assert r["t"] == pytest.approx(0.2, abs=1e-14)
        x = (np.arange(n) + 0.5) / n
        ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / 0.2)
        errs.append(np.abs(r["state"][0, 0] - ex[0]).mean())
    assert max(errs) < 0.008 and errs[2] < 0.005
    if lim == O.LIM_LMP:
        assert errs[0] > errs[1] > errs[2]
        assert np.log2(errs[0] / errs[2]) / 2 > 0.3


def test_riemann_random_x_rows_against_exact():
    """Random left/right states, LMP, N = 400: density L1 error below 1.5% of the range."""
    rng = np.random.default_rng(12)
    for _ in range(3):
        L = (rng.uniform(0.2, 2), rng.uniform(-0.5, 0.5), rng.uniform(0.2, 2))
        R = (rng.uniform(0.2, 2), rng.uniform(-0.5, 0.5), rng.uniform(0.2, 2))
        n = 400
        p = W.shock_tube(n, L, R)
        r = O.run(O.Config(n, 4, p.bc, O.LIM_LMP), p.conserved(), p.dx, t_end=0.1)
        x = (np.arange(n) + 0.5) / n
        ex = sample(L, R, (x - 0.5) / 0.1)
        err = np.abs(r["state"][0, 0] - ex[0]).mean()
        assert err < 0.015 * (max(L[0], R[0]) - min(L[0], R[0]) + 0.1), (L, R, err)


def test_sod_pp_oscillates_but_stays_positive():
    """Sec. 4.2: PP keeps theta ~ 1 (oscillatory second order) yet rho, p > 0."""
    n = 200
    p = W.sod(n)
    cfg = O.Config(n, 4, p.bc, O.LIM_PP)
    r = O.run(cfg, p.conserved(), p.dx, t_end=0.2)
    s = r["state"]
    e = s[3] - 0.5 * (s[1] ** 2 + s[2] ** 2) / s[0]
    assert (s[0] > 0).all() and (e > 0).all()
    a = O.kinetic_speed(O.max_speed(cfg, s), 0.5)
    _, d = O.step(cfg, s, a, debug=True)
    assert np.mean(d["theta_x"] > 0.99) > 0.9
