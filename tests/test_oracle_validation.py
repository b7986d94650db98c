"""Oracle on the paper's 1D validation cases with exact solutions (1D-on-2D: 4 cells
periodic in y, Sec. 4 preamble): the near-vacuum smooth isentropic wave with
gamma = 3 (Sec. 4.4; exact by characteristics, the Riemann invariants obey two
Burgers equations) and the LeBlanc shock tube with gamma = 5/3 (Sec. 4.5; exact
by the textbook Riemann solver). Pins: admissibility at every step, first-order
convergence of theta = 0, the blended schemes several times more accurate, and
errors falling with the grid.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W
from tests import exact_riemann as ER
from tests.exact_wave import near_vacuum_wave_exact


def _run_checked(cfg, p, t_end):
    """Run to t_end, asserting every step's state in G."""
    def check(n, st):
        rho = st[0]
        rhoe = st[3] - 0.5 * (st[1] ** 2 + st[2] ** 2) / rho
        assert rho.min() > 0.0 and rhoe.min() > 0.0, n
    return O.run(cfg, p.conserved(), p.dx, t_end=t_end, callback=check)


def _l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_near_vacuum_exact_solution_is_the_initial_state_at_t0():
    x = np.linspace(-1, 1, 17)
    assert np.allclose(near_vacuum_wave_exact(x, 0.0), 1.0 + 0.9999995 * np.sin(np.pi * x), atol=1e-14)


def test_near_vacuum_wave():
    errs = {}
    for N in (50, 100, 200):
        p = W.near_vacuum_wave(N)
        x = -1.0 + (np.arange(N) + 0.5) * p.dx
        ex = near_vacuum_wave_exact(x, 0.1)
        for lim in (O.LIM_FIRST, O.LIM_PP, O.LIM_RLMP):
            cfg = O.Config(N, 4, p.bc, lim, 3.0, 0.5, 1e-16)
            r = _run_checked(cfg, p, 0.1)
            assert r["t"] == pytest.approx(0.1, abs=1e-14)
            errs[N, lim] = _l1(r["state"][0, 0], ex)
    for N in (50, 100, 200):
        assert errs[N, O.LIM_PP] < 0.3 * errs[N, O.LIM_FIRST]
        assert errs[N, O.LIM_RLMP] < 0.3 * errs[N, O.LIM_FIRST]
    for lim in (O.LIM_FIRST, O.LIM_PP, O.LIM_RLMP):
        assert errs[200, lim] < errs[100, lim] < errs[50, lim]
    # theta = 0 converges at first order
    assert 1.7 < errs[50, O.LIM_FIRST] / errs[100, O.LIM_FIRST] < 2.3


@pytest.mark.parametrize("lim", [O.LIM_FIRST, O.LIM_PP, O.LIM_RLMP])
def test_leblanc_tube(lim):
    g = 5.0 / 3.0
    left, right = (1.0, 0.0, 0.1 * (g - 1.0)), (1e-3, 0.0, 1e-7 * (g - 1.0))
    errs = []
    for N in (200, 400):
        p = W.leblanc(N)
        x = (np.arange(N) + 0.5) * p.dx
        ex = ER.sample(left, right, (x - 3.0) / 6.0, g)[0]
        cfg = O.Config(N, 4, p.bc, lim, g, 0.5, 1e-16, 5)   # zero-gradient ends, 5-cell sponge
        r = _run_checked(cfg, p, 6.0)
        errs.append(_l1(r["state"][0, 0], ex))
    assert errs[1] < errs[0]
    bound = {O.LIM_FIRST: 0.06, O.LIM_PP: 0.02, O.LIM_RLMP: 0.015}[lim]
    assert errs[0] < bound
