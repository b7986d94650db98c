"""Oracle pins for prescribed-state (Dirichlet) boundaries and sides that switch
type along their length (partial walls), as the double Mach reflection (Sec. 4.7)
and the astrophysical jets (Sec. 4.8) use them.

- The ghost fill equals an independent construction from numpy.pad (modes
  'wrap', 'edge', 'symmetric' for periodic, zero-gradient and mirror ghosts, with
  the mirror's sign change and population swap) plus the field's states with
  equilibrium populations, x ghosts first and then y ghosts of every column.
- A flow at the prescribed state everywhere stays exactly at rest in time.
- Dirichlet ends hold the same states as zero-gradient ends while no wave has
  reached them (fixed a), to round-off.
- A split side acts like the uniform side of each type away from the switch.
- The prescribed fields match the paper's formulas: the double Mach reflection's
  shock moves along x = 1/6 + (y + 20 t)/sqrt(3), and the Rankine-Hugoniot
  conditions hold across it (to the printed 3 digits); the jet enters only
  through |y| < 0.05.
- lambda covers the prescribed states; bad configurations are rejected.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W
from tests.gpu_helpers import oracle_cfg

PER, ZG, MIR, DIR = 0, 1, 2, 3
PAD_MODE = {PER: "wrap", ZG: "edge", MIR: "symmetric"}


def _random_state(nx, ny, seed, a=4.0, gamma=1.4):
    """Admissible random conserved fields with non-equilibrium populations."""
    p = W.random_cells(nx, ny, seed)
    st = O.new_state(p.conserved())
    st = O.init_populations(O.Config(nx, ny), st, a)
    rng = np.random.default_rng(seed + 100)
    st[4:] *= 1.0 + 0.05 * rng.standard_normal(st[4:].shape)
    return st


def _mirror(v, axis):
    """Mirror transform of 20-plane values across an x-wall (axis 0) or y-wall (axis 1)."""
    v = v.copy()
    if axis == 0:
        v[[4, 5, 6, 7, 8, 9, 10, 11]] = v[[8, 9, 10, 11, 4, 5, 6, 7]]
        v[1::4] *= -1.0
    else:
        v[[12, 13, 14, 15, 16, 17, 18, 19]] = v[[16, 17, 18, 19, 12, 13, 14, 15]]
        v[2::4] *= -1.0
    return v


def _expected_ext(st, cfg, bf, a, t):
    """Ghost fill built from numpy.pad, one side type at a time."""
    nx, ny = cfg.nx, cfg.ny
    hi = cfg.bc if cfg.bc_hi is None else cfg.bc_hi

    def side_type(s, k):
        return cfg.bc[s] if k < cfg.split[s] else hi[s]

    def dirichlet(i, j):
        x = cfg.x0 + (i + 0.5) * cfg.dx
        y = cfg.y0 + (j + 0.5) * cfg.dx
        u = np.asarray(bf.state_at(x, y, t), dtype=np.float64).reshape(4)
        M = O.maxwellians(u, a, cfg.gamma, cfg.alpha)
        return np.concatenate([u, M[0], M[1], M[2], M[3]])

    img = st.reshape(20, ny, nx)
    # x pass on interior rows
    xp = {t_: np.pad(img, ((0, 0), (0, 0), (2, 2)), mode=PAD_MODE[t_]) for t_ in PAD_MODE}
    ext = np.zeros((20, ny + 4, nx + 4))
    ext[:, 2:ny + 2, :] = xp[PER]
    for j in range(ny):
        for s, cols in ((0, (0, 1)), (1, (nx + 2, nx + 3))):
            ty = side_type(s, j)
            for I in cols:
                i = I - 2
                if ty == DIR:
                    ext[:, j + 2, I] = dirichlet(i, j)
                else:
                    v = xp[ty][:, j, I]
                    ext[:, j + 2, I] = _mirror(v, 0) if ty == MIR else v
    # y pass on every column, from the x-filled rows
    yp = {t_: np.pad(ext[:, 2:ny + 2, :], ((0, 0), (2, 2), (0, 0)), mode=PAD_MODE[t_]) for t_ in PAD_MODE}
    for I in range(nx + 4):
        i = I - 2
        for s, rows in ((2, (0, 1)), (3, (ny + 2, ny + 3))):
            ty = side_type(s, i)
            for J in rows:
                j = J - 2
                if ty == DIR:
                    ext[:, J, I] = dirichlet(i, j)
                else:
                    v = yp[ty][:, J, I]
                    ext[:, J, I] = _mirror(v, 1) if ty == MIR else v
    return ext


FIELD = W.BoundaryField(inside=W._conserved_state(1.2, 0.3, -0.2, 0.9, 1.4),
                        outside=W._conserved_state(0.7, -0.1, 0.25, 0.4, 1.4),
                        planes=((1.0, -0.6, 0.35, 0.8), (-0.2, 1.0, -0.4, 0.0)))

CASES = [
    ((DIR, DIR, DIR, DIR), None, (0, 0, 0, 0)),
    ((DIR, ZG, MIR, DIR), None, (0, 0, 0, 0)),
    ((PER, PER, DIR, MIR), None, (0, 0, 0, 0)),
    ((DIR, DIR, DIR, DIR), (DIR, DIR, MIR, DIR), (0, 0, 3, 0)),      # double Mach reflection's sides
    ((ZG, MIR, DIR, ZG), (DIR, ZG, MIR, MIR), (2, 4, 5, 3)),         # every side switches
    ((MIR, DIR, ZG, DIR), (MIR, MIR, DIR, ZG), (0, 2, 2, 5)),
]


@pytest.mark.parametrize("bc,bc_hi,split", CASES)
def test_ghost_fill_matches_numpy_pad(bc, bc_hi, split):
    nx, ny, a, t = 9, 7, 5.0, 0.13
    st = _random_state(nx, ny, 3)
    cfg = O.Config(nx, ny, bc, O.LIM_PP, bc_hi=bc_hi, split=split, x0=-0.3, y0=0.1, dx=0.1,
                   field=O.Field(FIELD.inside, FIELD.outside, FIELD.planes))
    got = O.fill_ghosts(cfg, st, a, t)
    want = _expected_ext(st, cfg, FIELD, a, t)
    assert np.array_equal(got, want)


def test_field_states_differ_across_the_planes():
    """The test field really puts both states on the ghosts used above."""
    nx, ny = 9, 7
    x = -0.3 + (np.arange(-2, nx + 2) + 0.5) * 0.1
    y = 0.1 + (np.arange(-2, ny + 2) + 0.5) * 0.1
    X, Y = np.meshgrid(x, y)
    u = FIELD.state_at(X, Y, 0.13)
    assert (u[0] == FIELD.inside[0]).any() and (u[0] == FIELD.outside[0]).any()


@pytest.mark.parametrize("lim", [O.LIM_PP, O.LIM_LMP, O.LIM_RLMP])
def test_uniform_prescribed_flow_stays_put(lim):
    g = 1.4
    u = W._conserved_state(1.3, 0.4, -0.3, 0.8, g)
    bf = W.BoundaryField(u, u, ())
    nx, ny = 12, 10
    cons = np.stack([np.full((ny, nx), u[q]) for q in range(4)])
    cfg = O.Config(nx, ny, (DIR,) * 4, lim, g, x0=0.0, y0=0.0, dx=0.1, field=O.Field(u, u, ()))
    r = O.run(cfg, cons, 0.1, nsteps=30)
    np.testing.assert_allclose(r["state"][:4], cons, rtol=1e-14, atol=0)


@pytest.mark.parametrize("lim", [O.LIM_PP, O.LIM_LMP])
def test_dirichlet_ends_equal_zero_gradient_before_the_waves_arrive(lim):
    """Sod tube on [0, 1] with the initial states prescribed at both ends."""
    nx = 80
    p = W.sod(nx)
    left = tuple(float(v) for v in p.conserved()[:, 0, 0])
    right = tuple(float(v) for v in p.conserved()[:, 0, -1])
    fld = O.Field(left, right, ((-1.0, 0.0, -0.5, 0.0),))   # x <= 0.5: left state
    lam = 2.5                                                # fixed a = 4 lam, above every wave speed
    steps = 12                                               # waves travel < 0.5 - 4 dx
    cz = O.Config(nx, 4, (ZG, ZG, PER, PER), lim, p.gamma)
    cd = O.Config(nx, 4, (DIR, DIR, PER, PER), lim, p.gamma, x0=p.x0, y0=p.y0, dx=p.dx, field=fld)
    rz = O.run(cz, p.conserved(), p.dx, nsteps=steps, lam_fixed=lam)
    rd = O.run(cd, p.conserved(), p.dx, nsteps=steps, lam_fixed=lam)
    np.testing.assert_allclose(rd["state"], rz["state"], rtol=0, atol=1e-14)
    assert not np.allclose(rz["state"][0, 0, 30:50], p.rho[0, 30:50])   # the waves did move


def test_split_side_acts_like_each_uniform_side_away_from_the_switch():
    nx, ny, a, k = 24, 8, 6.0, 12
    st = _random_state(nx, ny, 5, a)
    fld = O.Field(FIELD.inside, FIELD.outside, FIELD.planes)
    kw = dict(x0=0.0, y0=0.0, dx=0.05, field=fld)
    for lim in (O.LIM_PP, O.LIM_LMP):
        split = O.step(O.Config(nx, ny, (ZG, ZG, DIR, ZG), lim, bc_hi=(ZG, ZG, MIR, ZG), split=(0, 0, k, 0), **kw),
                       st, a, t=0.05)
        lo = O.step(O.Config(nx, ny, (ZG, ZG, DIR, ZG), lim, **kw), st, a, t=0.05)
        hi = O.step(O.Config(nx, ny, (ZG, ZG, MIR, ZG), lim, **kw), st, a, t=0.05)
        assert np.array_equal(split[:, :, :k - 3], lo[:, :, :k - 3])
        assert np.array_equal(split[:, :, k + 3:], hi[:, :, k + 3:])
        assert not np.array_equal(split[:, 0, :], lo[:, 0, :])
        assert not np.array_equal(split[:, 0, :], hi[:, 0, :])


def test_double_mach_shock_position_and_jump():
    p = W.double_mach_reflection(30)
    bf = p.bfield
    cfg = oracle_cfg(p, O.LIM_LMP)
    st = O.init_populations(cfg, O.new_state(p.conserved()), 40.0)
    for t in (0.0, 0.01, 0.05):
        ext = O.fill_ghosts(cfg, st, 40.0, t)
        for J, j in ((p.ny + 2, p.ny), (p.ny + 3, p.ny + 1)):        # top ghost rows
            y = (j + 0.5) * p.dx
            x = (np.arange(-2, p.nx + 2) + 0.5) * p.dx
            pre = x - (1.0 / 6.0 + (y + 20.0 * t) / math.sqrt(3.0)) > 1e-9
            post = x - (1.0 / 6.0 + (y + 20.0 * t) / math.sqrt(3.0)) < -1e-9
            assert np.all(ext[0, J, pre] == 1.4) and np.all(ext[0, J, post] == 8.0)
    # bottom: prescribed left of x = 1/6, mirror of the first row right of it
    ext = O.fill_ghosts(cfg, st, 40.0, 0.0)
    k = p.split[2]
    assert (k - 0.5) * p.dx < 1.0 / 6.0 < (k + 0.5) * p.dx
    assert np.all(ext[0, 1, 2:k + 2] == 8.0)
    np.testing.assert_array_equal(ext[0, 1, k + 2:p.nx + 2], ext[0, 2, k + 2:p.nx + 2])
    np.testing.assert_array_equal(ext[2, 1, k + 2:p.nx + 2], -ext[2, 2, k + 2:p.nx + 2])
    # Rankine-Hugoniot across a shock moving at 10 (Mach 10 into c = 1), normal (cos 30, -sin 30)
    g, s = 1.4, 10.0
    n = np.array([math.cos(math.pi / 6), -math.sin(math.pi / 6)])

    def flux_n(u):
        r, m, E = u[0], np.array(u[1:3]), u[3]
        v = m / r
        pr = (g - 1) * (E - 0.5 * r * v @ v)
        vn = v @ n
        return np.array([r * vn, *(m * vn + pr * n), (E + pr) * vn])

    ua, ub = np.array(bf.inside), np.array(bf.outside)
    jump = flux_n(ub) - flux_n(ua) - s * (ub - ua)
    assert np.all(np.abs(jump) <= 2e-3 * np.abs(flux_n(ub)).max())


def test_jet_enters_only_through_the_nozzle():
    p = W.astro_jet(40)
    cfg = oracle_cfg(p, O.LIM_RLMP)
    st = O.init_populations(cfg, O.new_state(p.conserved()), 130.0)
    ext = O.fill_ghosts(cfg, st, 130.0, 0.0)
    y = p.y0 + (np.arange(-2, p.ny + 2) + 0.5) * p.dx
    inside = np.abs(y[2:p.ny + 2]) < 0.05
    assert inside.sum() == 4
    for I in (0, 1):
        assert np.all(ext[1, 2:p.ny + 2, I][inside] == 150.0)
        assert np.all(ext[1, 2:p.ny + 2, I][~inside] == 0.0)
    # the other sides are zero-gradient copies
    np.testing.assert_array_equal(ext[:, 2:p.ny + 2, p.nx + 2], ext[:, 2:p.ny + 2, p.nx + 1])


def test_lambda_covers_the_prescribed_states():
    p = W.astro_jet(20)
    lam = O.max_speed(oracle_cfg(p, O.LIM_PP), O.new_state(p.conserved()))
    g = 5.0 / 3.0
    assert lam == pytest.approx(30.0 + math.sqrt(g * 0.4127 / 5.0), rel=1e-14)
    lam0 = O.max_speed(O.Config(p.nx, p.ny, (1, 1, 1, 1), O.LIM_PP, g), O.new_state(p.conserved()))
    assert lam0 == pytest.approx(math.sqrt(g * 0.4127 / 0.5), rel=1e-14)


@pytest.mark.parametrize("kw", [
    dict(bc=(DIR, ZG, ZG, ZG)),                                           # no field
    dict(bc=(ZG, ZG, MIR, ZG), bc_hi=(ZG, ZG, DIR, ZG), split=(0, 0, 1, 0)),   # split too close to a corner
    dict(bc=(ZG, ZG, MIR, ZG), bc_hi=(ZG, ZG, DIR, ZG), split=(0, 0, 9, 0)),
    dict(bc=(PER, PER, ZG, ZG), bc_hi=(PER, ZG, ZG, ZG), split=(0, 4, 0, 0)),  # periodic side split
    dict(bc=(ZG, ZG, ZG, ZG), bc_hi=(ZG, ZG, MIR, ZG)),                   # types differ without a split
])
def test_bad_boundary_configurations_are_rejected(kw):
    nx, ny = 10, 8
    fld = None if kw.get("bc", (0,))[0] == DIR else O.Field(FIELD.inside, FIELD.outside, FIELD.planes)
    cfg = O.Config(nx, ny, kw["bc"], O.LIM_PP, bc_hi=kw.get("bc_hi"), split=kw.get("split", (0, 0, 0, 0)),
                   dx=0.1, field=fld)
    with pytest.raises(ValueError):
        O.step(cfg, _random_state(nx, ny, 1), 5.0)


@pytest.mark.parametrize("lim", [O.LIM_LMP, O.LIM_RLMP])
def test_double_mach_and_jet_stay_admissible(lim):
    def check(n, st):
        rho = st[0]
        rhoe = st[3] - 0.5 * (st[1] ** 2 + st[2] ** 2) / rho
        assert rho.min() > 0.0 and rhoe.min() > 0.0, n
    for p, steps in ((W.double_mach_reflection(24), 60), (W.astro_jet(24), 60)):
        r = O.run(oracle_cfg(p, lim), p.conserved(), p.dx, nsteps=steps, callback=check)
        assert r["n"] == steps
