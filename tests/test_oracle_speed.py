"""The kinetic speed lambda^n of the numerical section (Sec. 4 preamble): the
maximum over the cells of the Euclidean flow speed sqrt(v1^2 + v2^2) plus the
sound speed sqrt(gamma p / rho).

Prop. convex_preservation_O1 bounds the spectral radii of f' and g' by
max(|v1|, |v2|) + c, which is smaller whenever both velocity components are
non-zero; every other oracle test either holds a fixed or moves along one axis,
so these states, with v1 and v2 both non-zero, are what tells the two norms
apart. Expected values are worked out by hand from the formula.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _uniform(nx, ny, rho, v1, v2, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)
    c = np.empty((4, ny, nx))
    c[0], c[1], c[2], c[3] = rho, rho * v1, rho * v2, E
    return c


def test_lambda_is_the_euclidean_speed_plus_sound_speed():
    # (rho, v1, v2, p) = (1, 3, 4, 1), gamma = 1.4: |v| = 5, c = sqrt(1.4)
    cons = _uniform(6, 5, 1.0, 3.0, 4.0, 1.0, 1.4)
    lam = O.max_speed(O.Config(6, 5, (0, 0, 0, 0), O.LIM_PP, 1.4), O.new_state(cons))
    assert lam == pytest.approx(5.0 + math.sqrt(1.4), rel=1e-14)
    # the max-norm reading would give 4 + sqrt(1.4), 16 % smaller
    assert abs(lam - (4.0 + math.sqrt(1.4))) > 0.9


@pytest.mark.parametrize("v1, v2", [(-3.0, 4.0), (3.0, -4.0), (-4.0, -3.0), (0.6, 0.8)])
def test_lambda_depends_on_the_norm_of_v_only(v1, v2):
    # rho = 2, p = 0.9, gamma = 1.4: c = sqrt(1.4 * 0.9 / 2) = sqrt(0.63)
    cons = _uniform(5, 4, 2.0, v1, v2, 0.9, 1.4)
    lam = O.max_speed(O.Config(5, 4, (1, 1, 1, 1), O.LIM_LMP, 1.4), O.new_state(cons))
    assert lam == pytest.approx(math.hypot(v1, v2) + math.sqrt(0.63), rel=1e-14)


def test_maximum_is_taken_at_the_cell_with_the_largest_euclidean_speed():
    # cell A moves at (3, 4) (|v| = 5, max-norm 4), cell B at (4.6, 0) (|v| = 4.6,
    # max-norm 4.6), same rho = 1 and p = 1: lambda = 5 + c; the max-norm reading
    # would pick cell B and give 4.6 + c
    gamma = 1.4
    cons = _uniform(6, 6, 1.0, 0.0, 0.0, 1.0, gamma)
    a = _uniform(1, 1, 1.0, 3.0, 4.0, 1.0, gamma)[:, 0, 0]
    b = _uniform(1, 1, 1.0, 4.6, 0.0, 1.0, gamma)[:, 0, 0]
    cons[:, 1, 2] = a
    cons[:, 4, 3] = b
    lam = O.max_speed(O.Config(6, 6, (0, 0, 0, 0), O.LIM_PP, gamma), O.new_state(cons))
    assert lam == pytest.approx(5.0 + math.sqrt(1.4), rel=1e-14)


def test_first_kinetic_speed_of_a_run_is_four_lambda():
    # alpha = 1/2: a^0 = 2 lambda / (1 - alpha) = 4 lambda (Sec. 4 preamble)
    cons = _uniform(6, 6, 1.0, 3.0, 4.0, 1.0, 1.4)
    r = O.run(O.Config(6, 6, (0, 0, 0, 0), O.LIM_PP, 1.4), cons, 0.1, nsteps=1)
    assert r["a"][0] == pytest.approx(4.0 * (5.0 + math.sqrt(1.4)), rel=1e-14)
