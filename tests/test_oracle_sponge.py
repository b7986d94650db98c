"""Sponge layer of Sec. 4.2 in the oracle: theta = 0 on every face of the cells
within `sponge` cells of a zero-gradient side.

Pins: a cell all of whose faces are in the sponge is updated exactly as by the
first-order scheme (theta = 0 on every face it reads), a cell none of whose faces
is in the sponge exactly as without it, and periodic sides get no layer.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W


def _stepped(p, nsteps=3):
    """A state out of equilibrium: `nsteps` plain PP steps from u_0."""
    cfg = O.Config(p.nx, p.ny, p.bc, O.LIM_PP, p.gamma, 0.5, 1e-16)
    r = O.run(cfg, p.conserved(), p.dx, nsteps=nsteps)
    return r["state"], r["a"][-1]


@pytest.mark.parametrize("bc,s", [((1, 1, 1, 1), 3), ((0, 0, 1, 1), 2), ((1, 2, 2, 1), 4)])
def test_sponge_cells_update_first_order_and_others_unchanged(bc, s):
    p = W.quadrant_riemann(26, 22, seed=4, bc=bc)
    st, a = _stepped(p)
    nx, ny = p.nx, p.ny
    out = {}
    for name, lim, sp in (("sponge", O.LIM_PP, s), ("plain", O.LIM_PP, 0), ("first", O.LIM_FIRST, 0)):
        cfg = O.Config(nx, ny, bc, lim, p.gamma, 0.5, 1e-16, sp)
        out[name] = O.step(cfg, st, a)

    def layer(i, j):
        return ((bc[0] == 1 and i < s) or (bc[1] == 1 and i >= nx - s) or
                (bc[2] == 1 and j < s) or (bc[3] == 1 and j >= ny - s))

    n_first = n_plain = 0
    for j in range(ny):
        for i in range(nx):
            near = [layer(i + di, j + dj) for di, dj in ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1))]
            if near[0]:
                # every face of a layer cell has theta = 0: the first-order update
                assert np.array_equal(out["sponge"][:, j, i], out["first"][:, j, i]), (i, j)
                n_first += 1
            elif not any(near):
                assert np.array_equal(out["sponge"][:, j, i], out["plain"][:, j, i]), (i, j)
                n_plain += 1
    assert n_first > 0 and n_plain > 0
    # periodic sides carry no layer: with bc (0, 0, 1, 1) the x-extent is free
    if bc[0] == 0:
        assert not layer(0, ny // 2)


def test_sponge_theta_faces():
    """The debug theta is 0 exactly on faces touching a layer cell (s = 2, all sides)."""
    p = W.quadrant_riemann(12, 10, seed=5, bc=(1, 1, 1, 1))
    st, a = _stepped(p)
    cfg = O.Config(12, 10, (1, 1, 1, 1), O.LIM_PP, p.gamma, 0.5, 1e-16, 2)
    _, dbg = O.step(cfg, st, a, debug=True)
    cfg0 = O.Config(12, 10, (1, 1, 1, 1), O.LIM_PP, p.gamma, 0.5, 1e-16, 0)
    _, dbg0 = O.step(cfg0, st, a, debug=True)
    # x-faces i+1/2, i = -1..11, rows 0..9: in the layer iff i < 2 or i + 1 >= 10 or the row is
    for j in range(10):
        for f in range(13):
            i = f - 1
            inl = i < 2 or i + 1 >= 10 or j < 2 or j >= 8
            want = 0.0 if inl else dbg0["theta_x"][j, f]
            assert dbg["theta_x"][j, f] == want, (j, f)


def test_sponge_rejects_negative_width():
    cfg = O.Config(8, 8, (1, 1, 1, 1), O.LIM_PP, 1.4, 0.5, 1e-16, -1)
    st = O.new_state(W.quadrant_riemann(8, 8, seed=1, bc=(1, 1, 1, 1)).conserved())
    with pytest.raises(ValueError):
        O.step(cfg, O.init_populations(O.Config(8, 8, (1, 1, 1, 1)), st, 4.0), 4.0)
