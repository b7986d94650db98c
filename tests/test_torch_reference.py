"""The PyTorch restatement used to check the adjoint against autograd, pinned to
the oracle: same forward map to round-off, and autograd equal to central
differences of the oracle on smooth data."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W

torch = pytest.importorskip("torch")

from tests import torch_reference as TR  # noqa: E402


@pytest.mark.parametrize("lim", [O.LIM_FIRST, O.LIM_SECOND, O.LIM_PP, O.LIM_LMP, O.LIM_RLMP])
def test_forward_matches_oracle(lim):
    p = W.vortex_with_bumps(24)
    cfg = O.Config(24, 24, (0, 0, 0, 0), lim, 1.4, 0.5, 1e-16)
    lam = 1.05 * O.max_speed(cfg, O.new_state(p.conserved()))
    ref = O.run(cfg, p.conserved(), p.dx, nsteps=25, lam_fixed=lam)["state"]
    got = TR.rollout(torch.tensor(p.conserved()), 25, O.kinetic_speed(lam, 0.5), lim).numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_forward_matches_oracle_with_active_limiter():
    """Random admissible cells (periodic): theta < 1 and theta = 0 occur."""
    p = W.random_cells(16, 12, seed=3)
    cfg = O.Config(16, 12, (0, 0, 0, 0), O.LIM_PP, 1.4, 0.5, 1e-13)
    lam = 1.05 * O.max_speed(cfg, O.new_state(p.conserved()))
    a = O.kinetic_speed(lam, 0.5)
    st = O.run(cfg, p.conserved(), p.dx, nsteps=2, lam_fixed=lam)["state"]
    _, dbg = O.step(cfg, st, a, debug=True)
    assert (dbg["theta_x"] < 1).sum() + (dbg["theta_y"] < 1).sum() > 10
    ref = O.run(cfg, p.conserved(), p.dx, nsteps=6, lam_fixed=lam)["state"]
    got = TR.rollout(torch.tensor(p.conserved()), 6, a, O.LIM_PP, eps=1e-13).numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_autograd_matches_oracle_differences():
    p = W.vortex_with_bumps(20)
    cfg = O.Config(20, 20, (0, 0, 0, 0), O.LIM_PP, 1.4, 0.5, 1e-16)
    lam = 1.05 * O.max_speed(cfg, O.new_state(p.conserved()))
    a = O.kinetic_speed(lam, 0.5)
    rng = np.random.default_rng(1)
    w = rng.uniform(0.5, 1.5, size=(4, 20, 20))
    c0 = p.conserved()
    u0 = torch.tensor(c0, requires_grad=True)
    sN = TR.rollout(u0, 15, a, O.LIM_PP)
    (0.5 * (torch.tensor(w) * sN[:4] ** 2).sum()).backward()
    g = u0.grad.numpy()
    for (j, i, c) in [(3, 4, 0), (10, 17, 1), (15, 2, 2), (8, 8, 3)]:
        h = 1e-5 * max(1.0, abs(c0[c, j, i]))
        up, dn = c0.copy(), c0.copy()
        up[c, j, i] += h
        dn[c, j, i] -= h
        A = O.run(cfg, up, p.dx, nsteps=15, lam_fixed=lam)["state"][:4]
        B = O.run(cfg, dn, p.dx, nsteps=15, lam_fixed=lam)["state"][:4]
        fd = 0.5 * float((w * (A - B) * (A + B)).sum()) / (2 * h)
        assert abs(fd - g[c, j, i]) <= 1e-6 * abs(g[c, j, i]), (j, i, c, fd, g[c, j, i])


def test_dynamic_speed_rollout_matches_oracle_and_its_differences():
    """The dynamic kinetic speed a^n = 4 lambda(s^n): the forward map equals the
    oracle's dynamic run, and autograd through the max equals central differences
    of the oracle's run (smooth data, a unique argmax that stays put within h)."""
    p = W.vortex_with_bumps(20)
    cfg = O.Config(20, 20, (0, 0, 0, 0), O.LIM_PP, 1.4, 0.5, 1e-16)
    nsteps = 8
    ref = O.run(cfg, p.conserved(), p.dx, nsteps=nsteps)["state"]
    u0 = torch.tensor(p.conserved(), requires_grad=True)
    sN = TR.rollout_dynamic(u0, nsteps, O.LIM_PP)
    assert np.abs(sN.detach().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    rng = np.random.default_rng(4)
    w = rng.uniform(0.5, 1.5, size=(4, 20, 20))
    (torch.tensor(w) * sN[:4]).sum().backward()
    g = u0.grad.numpy()
    # the gradient of the max reaches the state: holding a^n fixed gives another gradient
    a_seq = O.run(cfg, p.conserved(), p.dx, nsteps=nsteps)["a"]
    u0h = torch.tensor(p.conserved(), requires_grad=True)
    s = TR.init_populations(u0h, a_seq[0], 0.5, 1.4)
    for a in a_seq:
        s = TR.step(s, a, O.LIM_PP)
    (torch.tensor(w) * s[:4]).sum().backward()
    assert np.abs(u0h.grad.numpy() - g).max() > 1e-6 * np.abs(g).max()
    for k in range(6):
        d = rng.standard_normal((4, 20, 20)) * np.abs(p.conserved()) * 1e-2
        h = 1e-4

        def L(x):
            return float((w * O.run(cfg, p.conserved() + x * d, p.dx, nsteps=nsteps)["state"][:4]).sum())

        fd = (4.0 * (L(h) - L(-h)) / (2 * h) - (L(2 * h) - L(-2 * h)) / (4 * h)) / 3.0
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-7 * abs(ad), (k, fd, ad)


def _waves(n=24):
    """Smooth periodic waves with no flat region: the LMP bound is active on 240-310
    faces per step, and theta moves smoothly with the data (a flat region puts dF^rho
    at 0 where rho* sits on a bound, and LMP's theta jumps there between 1 and 0)."""
    X, Y = np.meshgrid((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n)
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * X + 0.4) * np.cos(2 * np.pi * Y + 0.7) + 0.1 * np.sin(4 * np.pi * (X + 2 * Y))
    v1 = 0.5 * np.cos(2 * np.pi * Y + 0.2)
    v2 = 0.3 * np.sin(2 * np.pi * X + 1.1)
    p = 1.0 + 0.2 * np.cos(2 * np.pi * (X - Y))
    return np.stack(W.primitive_to_conserved(rho, v1, v2, p)), 1.0 / n


@pytest.mark.parametrize("lim", [O.LIM_LMP, O.LIM_RLMP])
def test_lmp_restatement_matches_oracle_theta_and_differences(lim):
    """LMP / RLMP: the step equals the oracle's with the bound active on hundreds of
    faces, and autograd equals central differences (Richardson) of the oracle's run
    along random directions."""
    cons, dx = _waves()
    n = cons.shape[1]
    cfg = O.Config(n, n, (0, 0, 0, 0), lim, 1.4, 0.5, 1e-16)
    lam = 1.05 * O.max_speed(cfg, O.new_state(cons))
    a = O.kinetic_speed(lam, 0.5)
    st = O.run(cfg, cons, dx, nsteps=3, lam_fixed=lam)["state"]
    _, dbg = O.step(cfg, st, a, debug=True)
    assert (dbg["theta_x"] < 1.0).sum() + (dbg["theta_y"] < 1.0).sum() > 200
    got = TR.step(torch.tensor(st), a, lim).numpy()
    ref = O.step(cfg, st, a)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    nsteps = 6
    rng = np.random.default_rng(5)
    w = rng.uniform(0.5, 1.5, size=(4, n, n))
    u0 = torch.tensor(cons, requires_grad=True)
    (torch.tensor(w) * TR.rollout(u0, nsteps, a, lim)[:4]).sum().backward()
    g = u0.grad.numpy()
    for k in range(4):
        d = rng.standard_normal((4, n, n)) * np.abs(cons) * 1e-2
        h = 1e-5

        def L(x):
            return float((w * O.run(cfg, cons + x * d, dx, nsteps=nsteps, lam_fixed=lam)["state"][:4]).sum())

        fd = (4.0 * (L(h) - L(-h)) / (2 * h) - (L(2 * h) - L(-2 * h)) / (4 * h)) / 3.0
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (k, fd, ad)


def boxed_waves(case, nx=24, ny=20):
    """Smooth waves (nowhere flat) in a box with the sides of `case`: zero-gradient
    and mirror walls ("zg-mirror"); zero-gradient sides with a 3-cell sponge layer,
    periodic in y ("sponge"); prescribed states on two sides and a south side that
    switches from mirror to zero gradient at column 15 ("dirichlet-split").
    Returns (oracle Config without limiter, conserved fields, dx, boundary kwargs)."""
    dx = 1.0 / nx
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * X + 0.4) * np.cos(2 * np.pi * Y + 0.7) + 0.1 * np.sin(4 * np.pi * (X + 2 * Y))
    v1 = 0.4 * np.cos(2 * np.pi * Y + 0.2)
    v2 = 0.3 * np.sin(2 * np.pi * X + 1.1)
    p = 1.0 + 0.2 * np.cos(2 * np.pi * (X - Y))
    cons = np.stack(W.primitive_to_conserved(rho, v1, v2, p))
    kw = {"bc": (1, 1, 2, 2), "sponge": 0}
    if case == "sponge":
        kw = {"bc": (1, 1, 0, 0), "sponge": 3}
    elif case == "dirichlet-split":
        st = W._conserved_state(1.0, 0.3, 0.15, 1.0, 1.4)
        kw = {"bc": (3, 1, 2, 3), "sponge": 0, "bc_hi": (3, 1, 1, 3), "split": (0, 0, 15, 0),
              "field": O.Field(st, st, ())}
    return cons, dx, kw


def _box_cfg(nx, ny, lim, kw, dx):
    return O.Config(nx, ny, kw["bc"], lim, 1.4, 0.5, 1e-16, kw["sponge"], bc_hi=kw.get("bc_hi"),
                    split=kw.get("split", (0, 0, 0, 0)), dx=dx, field=kw.get("field"))


@pytest.mark.parametrize("case", ["zg-mirror", "sponge", "dirichlet-split"])
def test_frame_restatement_matches_oracle_step(case):
    """The step inside the oracle's ghost frame (gathered from the oracle's own fill)
    equals the oracle's step for every limiter."""
    cons, dx, kw = boxed_waves(case)
    ny, nx = cons.shape[1:]
    for lim in range(5):
        cfg = _box_cfg(nx, ny, lim, kw, dx)
        lam = 1.05 * O.max_speed(cfg, O.new_state(cons))
        a = O.kinetic_speed(lam, 0.5)
        st = O.run(cfg, cons, dx, nsteps=3, lam_fixed=lam)["state"]
        fr = TR.ghost_frame(cfg, a, sponge=kw["sponge"])
        got = TR.step_frame(torch.tensor(st), a, lim, fr).numpy()
        ref = O.step(cfg, st, a)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (case, lim)


@pytest.mark.parametrize("case", ["zg-mirror", "dirichlet-split"])
def test_frame_restatement_gradient_matches_differences(case):
    """LMP in a box: autograd through the frame restatement equals Richardson central
    differences of the oracle's run along random directions, with the density bound
    active on boundary faces."""
    cons, dx, kw = boxed_waves(case)
    ny, nx = cons.shape[1:]
    lim = O.LIM_LMP
    cfg = _box_cfg(nx, ny, lim, kw, dx)
    lam = 1.05 * O.max_speed(cfg, O.new_state(cons))
    a = O.kinetic_speed(lam, 0.5)
    _, dbg = O.step(cfg, O.run(cfg, cons, dx, nsteps=3, lam_fixed=lam)["state"], a, debug=True)
    assert (dbg["theta_x"] < 1.0).sum() + (dbg["theta_y"] < 1.0).sum() > 60
    fr = TR.ghost_frame(cfg, a)
    nsteps = 6
    rng = np.random.default_rng(8)
    w = rng.uniform(0.5, 1.5, size=(4, ny, nx))
    u0 = torch.tensor(cons, requires_grad=True)
    (torch.tensor(w) * TR.rollout_frame(u0, nsteps, a, lim, fr)[:4]).sum().backward()
    g = u0.grad.numpy()
    for k in range(3):
        d = rng.standard_normal((4, ny, nx)) * np.abs(cons) * 1e-2
        h = 1e-5

        def L(x):
            return float((w * O.run(cfg, cons + x * d, dx, nsteps=nsteps, lam_fixed=lam)["state"][:4]).sum())

        fd = (4.0 * (L(h) - L(-h)) / (2 * h) - (L(2 * h) - L(-2 * h)) / (4 * h)) / 3.0
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (k, fd, ad)


@pytest.mark.parametrize("case", ["zg-mirror", "sponge"])
def test_frame_dynamic_rollout_matches_oracle(case):
    """The dynamic-speed rollout inside the frame follows the oracle's run with a^n =
    4 lambda(s^n) (Sec. 4 preamble)."""
    cons, dx, kw = boxed_waves(case)
    ny, nx = cons.shape[1:]
    cfg = _box_cfg(nx, ny, O.LIM_RLMP, kw, dx)
    fr = TR.ghost_frame(cfg, 1.0, sponge=kw["sponge"])
    got = TR.rollout_dynamic_frame(torch.tensor(cons), 8, O.LIM_RLMP, fr).numpy()
    ref = O.run(cfg, cons, dx, nsteps=8)["state"]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_frame_dynamic_rollout_with_prescribed_states_matches_oracle():
    """With prescribed states the frame's constants follow a^n (their Maxwellians), and
    lambda^n covers the states' speed: the dynamic rollout follows the oracle's run."""
    cons, dx, kw = boxed_waves("dirichlet-split")
    ny, nx = cons.shape[1:]
    for fast in (False, True):
        kw2 = dict(kw)
        if fast:   # a prescribed state faster than every cell: a^n = 4 lambda_bc
            st = W._conserved_state(1.0, 2.5, 0.0, 1.0, 1.4)
            kw2["field"] = O.Field(st, st, ())
        cfg = _box_cfg(nx, ny, O.LIM_LMP, kw2, dx)
        fr = TR.ghost_frame(cfg, 1.0, const_in_a=True)
        st = kw2["field"].inside
        r, m1, m2, E = st
        v2 = (m1 * m1 + m2 * m2) / (r * r)
        lam_bc = float(np.sqrt(v2) + np.sqrt(1.4 * 0.4 * (E - 0.5 * r * v2) / r))
        got = TR.rollout_dynamic_frame(torch.tensor(cons), 8, O.LIM_LMP, fr, lam_bc=lam_bc).numpy()
        ref = O.run(cfg, cons, dx, nsteps=8)["state"]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), fast
