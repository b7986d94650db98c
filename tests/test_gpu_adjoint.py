"""Adjoint of the rollout (vlbm_rollout / vlbm_adjoint) against central finite
differences of the forward map (needs a GB300).

The loss is L = 1/2 sum w (u^N - u_target)^2 over the conserved planes, so
dL/du^N = w (u^N - u_target). The kinetic speed is fixed (a state made with
lambda > 0, a = 4 lambda), so the forward map is the one the adjoint transposes.
Finite differences (smooth data only): central differences at h and 2h with
h = 1e-4 max(1, |u|), combined by one Richardson step, the loss difference
formed cell by cell; compared with the adjoint at a relative tolerance taken
against max(|g_i|, 1e-2 rms(g)) so that near-zero entries are judged on the
gradient's scale. Measured: plain central differences reach their smallest
error near h = 1e-5 (truncation below, FP64 round-off of the forward runs
above), and at h = 1e-6 the round-off alone is ~2e-5 of the smaller entries;
the Richardson pair at 1e-4 is ~1e-7.
Where the limiter is active, theta switches branch (min, max, clamps) on faces
within any finite h of a kink, so there the adjoint is compared over the whole
field with autograd through a plain PyTorch restatement of the step
(tests/torch_reference.py) that takes the same branches.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W
from tests import torch_reference as TR

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_15001_gb300 import vlbm as V  # noqa: E402

DEV = torch.device("cuda:0")


def _lam0(p):
    cfg = O.Config(p.nx, p.ny, p.bc, 0, p.gamma, 0.5, 1e-16)
    return O.max_speed(cfg, O.new_state(p.conserved()))


def _solver(p, limiter, prec, lam, kernel=V.KERNEL_AUTO, eps=1e-16):
    return V.VLBM(p.nx, p.ny, p.dx, bc=(0, 0, 0, 0), gamma=p.gamma, lam=lam, limiter=limiter,
                  precision=prec, eps=eps, kernel=kernel, device=DEV)


def _final(s, u0, nsteps):
    s.set_conserved(u0[0].contiguous(), u0[1:3].contiguous(), u0[3].contiguous())
    s.step(nsteps)
    rho, mom, E = s.moments()
    return torch.cat([rho[None], mom, E[None]])


def _setup(p, t_final, seed=5):
    rng = np.random.default_rng(seed)
    w = torch.tensor(rng.uniform(0.5, 1.5, size=(4, p.ny, p.nx)), dtype=torch.float64, device=DEV)
    tgt = W.isentropic_vortex(p.nx, t=t_final).conserved() if p.name.startswith("vortex") else \
        p.conserved() * 0.97
    return w, torch.tensor(tgt, dtype=torch.float64, device=DEV)


def _loss_diff(up, dn, w, tgt):
    """L(up) - L(dn) as 1/2 sum w (up - dn)(up + dn - 2 tgt): the difference is formed
    cell by cell before the sum, so the sum's round-off is relative to the difference
    (summing the two losses first loses ~1e-13 L to cancellation, which / 2h is the
    size of a small gradient entry)."""
    up, dn = up.double(), dn.double()
    return 0.5 * float((w * (up - dn) * (up + dn - 2.0 * tgt)).sum())


def _adjoint(s, u0, nsteps, every, w, tgt):
    """(u^N, dL/du_0) through VLBMRollout."""
    rho = u0[0].clone().requires_grad_(True)
    mom = u0[1:3].clone().requires_grad_(True)
    E = u0[3].clone().requires_grad_(True)
    rN, mN, EN = V.VLBMRollout.apply(rho, mom, E, s, nsteps, every)
    uN = torch.cat([rN[None], mN, EN[None]])
    L = 0.5 * (w.to(uN.dtype) * (uN - tgt.to(uN.dtype)) ** 2).sum()
    L.backward()
    g = torch.cat([rho.grad[None], mom.grad, E.grad[None]]).double()
    return uN.detach(), g


def _fd_check(s, u0, nsteps, w, tgt, g, cells, h_rel=1e-4, tol=1e-5):
    """Central differences with one Richardson step: D(h), D(2h) at h = h_rel max(1, |u|),
    (4 D(h) - D(2h)) / 3, so that the h^2 truncation term cancels and h can stay
    where the forward runs' round-off is negligible."""
    scale = 1e-2 * float(torch.sqrt((g * g).mean()))
    worst = 0.0

    def D(c, j, i, h):
        up = u0.clone()
        up[c, j, i] += h
        dn = u0.clone()
        dn[c, j, i] -= h
        return _loss_diff(_final(s, up, nsteps), _final(s, dn, nsteps), w, tgt) / (2 * h)

    for (j, i) in cells:
        for c in range(4):
            h = h_rel * max(1.0, abs(float(u0[c, j, i])))
            fd = (4.0 * D(c, j, i, h) - D(c, j, i, 2.0 * h)) / 3.0
            ad = float(g[c, j, i])
            err = abs(fd - ad) / max(abs(ad), scale)
            worst = max(worst, err)
            assert err <= tol, (j, i, c, fd, ad, err)
    return worst


def _cells(p, n, seed):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(p.ny)), int(rng.integers(p.nx))) for _ in range(n)]


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("limiter", [V.LIM_FIRST_ORDER, V.LIM_NONE, V.LIM_PP])
def test_adjoint_fd_fp64_vortex(limiter, kernel):
    p = W.vortex_with_bumps(48)
    lam = 1.05 * _lam0(p)
    nsteps, every = 60, 16            # a ragged last segment of 12 steps
    tN = nsteps * p.dx / (4.0 * lam)
    w, tgt = _setup(p, tN)
    s = _solver(p, limiter, V.FP64, lam, kernel)
    u0 = torch.tensor(p.conserved(), dtype=torch.float64, device=DEV)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert torch.equal(uN, _final(s, u0, nsteps))       # rollout = plain stepping, bit for bit
    _fd_check(s, u0, nsteps, w, tgt, g, _cells(p, 12, 7))
    s.close()


def _expansion(nx=40, ny=36, p0=1e-2):
    """Periodic strong expansion: v1 = +-2 tanh profiles pulling the gas apart around
    x = 1/2 (and colliding at x = 0), rho modulated in x and y, p = 1e-2. With a
    fixed speed of 1.6 lambda_0 the PP limiter's internal-energy bound is active
    on 250-700 faces in every one of the first 20 steps (theta down to ~0.1).
    The fields carry a seeded 1e-3 relative perturbation: a mirror-symmetric state
    puts dF^rho exactly at 0 on the symmetry planes, a kink of theta where two
    implementations that round differently take different one-sided derivatives."""
    X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)   # unit periods
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * X)
    v1 = 2.0 * np.tanh((X - 0.5) / 0.05) * np.where(np.abs(X - 0.5) < 0.25, 1.0, -1.0)
    v2 = 0.3 * np.sin(2 * np.pi * Y)
    cons = np.stack(W.primitive_to_conserved(rho, v1, v2, np.full((ny, nx), p0)))
    cons = cons * (1.0 + 1e-3 * np.random.default_rng(11).uniform(-1.0, 1.0, cons.shape))
    return cons, 1.0 / nx


def _autograd_gradient(cons, nsteps, a, limiter, w, tgt, eps):
    u0 = torch.tensor(cons, dtype=torch.float64, requires_grad=True)
    sN = TR.rollout(u0, nsteps, a, limiter, eps=eps)
    L = 0.5 * (w.cpu() * (sN[:4] - tgt.cpu()) ** 2).sum()
    L.backward()
    return sN.detach().numpy(), u0.grad.numpy()


def _bumps(n):
    p = W.vortex_with_bumps(n)
    return p.conserved(), p.dx


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("case", ["bumps-first", "bumps-none", "bumps-pp", "expansion-pp"])
def test_adjoint_matches_autograd(case, kernel):
    """The whole gradient field against autograd of the PyTorch restatement, FP64:
    smooth data with every limiter, and the strong expansion where theta < 1 on
    hundreds of faces in every step."""
    name, lim = case.split("-")
    limiter = {"first": V.LIM_FIRST_ORDER, "none": V.LIM_NONE, "pp": V.LIM_PP}[lim]
    if name == "bumps":
        cons, dx = _bumps(32)
        nsteps, every, eps = 30, 7, 1e-16
    else:
        cons, dx = _expansion()
        nsteps, every, eps = 20, 8, 1e-13
    ny, nx = cons.shape[1:]
    cfg = O.Config(nx, ny, (0, 0, 0, 0), limiter, 1.4, 0.5, eps)
    # the expansion speeds the gas up (lambda 2.19 -> 2.64): a fixed speed of
    # 1.6 lambda_0 keeps the CFL bound, and so admissibility, along the whole run
    lam = (1.6 if name == "expansion" else 1.05) * O.max_speed(cfg, O.new_state(cons))
    a = O.kinetic_speed(lam, 0.5)
    if name == "expansion":
        for k in (1, 10, 19):   # the limiter is active along the run
            st = O.run(cfg, cons, dx, nsteps=k, lam_fixed=lam)["state"]
            _, dbg = O.step(cfg, st, a, debug=True)
            th = np.concatenate([dbg["theta_x"].ravel(), dbg["theta_y"].ravel()])
            assert (th < 1.0).sum() > 100
    p = W.Problem(name, nx, ny, dx, 0.0, 0.0, cons[0], cons[1], cons[2], cons[3])
    w, tgt = _setup(p, 0.0)
    s = _solver(p, limiter, V.FP64, lam, kernel, eps=eps)
    u0 = torch.tensor(cons, dtype=torch.float64, device=DEV)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert s.monitors()["status"] == 0
    s.close()
    ref = O.run(cfg, cons, dx, nsteps=nsteps, lam_fixed=lam)["state"]
    assert np.array_equal(uN.cpu().numpy(), ref[:4])          # the forward map is the oracle's
    sN, g_ref = _autograd_gradient(cons, nsteps, a, limiter, w, tgt, eps)
    assert np.abs(sN - ref).max() <= 1e-12 * np.abs(ref).max()
    err = np.abs(g.cpu().numpy() - g_ref)
    assert err.max() <= 1e-10 * np.abs(g_ref).max(), (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_adjoint_zero_steps_and_linearity():
    p = W.vortex_with_bumps(32)
    lam = 1.05 * _lam0(p)
    s = _solver(p, V.LIM_PP, V.FP64, lam)
    u0 = torch.tensor(p.conserved(), dtype=torch.float64, device=DEV)
    scratch = s.adjoint_scratch(0, 4)
    gN = torch.randn((4, p.ny, p.nx), dtype=torch.float64, device=DEV, generator=torch.Generator(DEV).manual_seed(1))
    g0 = s.adjoint(gN, 0, 4, scratch, u0=u0)
    assert torch.equal(g0, gN)            # N = 0: u^0 = u_0, the identity
    nsteps, every = 9, 4
    scratch = s.adjoint_scratch(nsteps, every)
    g1 = s.adjoint(gN, nsteps, every, scratch, u0=u0)
    g2 = s.adjoint(2.0 * gN, nsteps, every, scratch)        # reuses the checkpoints
    g3 = s.adjoint(gN, nsteps, 1, s.adjoint_scratch(nsteps, 1), u0=u0)
    assert torch.equal(g2, 2.0 * g1)      # the transpose is linear in the cotangent
    assert torch.equal(g3, g1)            # independent of the checkpoint interval
    s.close()


def test_adjoint_dynamic_a_matches_fixed_on_uniform_flow():
    """A uniform state keeps lambda constant, so the recorded dynamic a^n equals the
    fixed speed 4 lambda(u_0) and both adjoints must agree (to round-off)."""
    nx, ny = 40, 24
    rho = np.full((ny, nx), 0.8)
    v1, v2, pr = np.full((ny, nx), 0.3), np.full((ny, nx), -0.2), np.full((ny, nx), 0.9)
    cons = W.primitive_to_conserved(rho, v1, v2, pr)
    u0 = torch.tensor(np.stack(cons), dtype=torch.float64, device=DEV)
    gN = torch.randn((4, ny, nx), dtype=torch.float64, device=DEV, generator=torch.Generator(DEV).manual_seed(3))
    dyn = V.VLBM(nx, ny, 0.1, limiter=V.LIM_PP, precision=V.FP64, device=DEV)
    dyn.set_conserved(u0[0].contiguous(), u0[1:3].contiguous(), u0[3].contiguous())
    lam = dyn.monitors()["lambda"]
    fix = V.VLBM(nx, ny, 0.1, lam=lam, limiter=V.LIM_PP, precision=V.FP64, device=DEV)
    ga = dyn.adjoint(gN, 12, 5, dyn.adjoint_scratch(12, 5), u0=u0)
    gb = fix.adjoint(gN, 12, 5, fix.adjoint_scratch(12, 5), u0=u0)
    # the uniform state may drift by an ulp per step, and a^n with it
    assert abs(dyn.monitors()["a"] / fix.monitors()["a"] - 1.0) < 1e-13
    assert torch.allclose(ga, gb, rtol=1e-12, atol=1e-12 * float(gb.abs().max()))
    dyn.close()
    fix.close()


def test_adjoint_against_oracle_fd():
    """GPU FP64 adjoint against central differences of the oracle (64^2, 100 steps)."""
    p = W.vortex_with_bumps(64)
    lam = 1.05 * _lam0(p)
    nsteps, every = 100, 25
    a = O.kinetic_speed(lam, 0.5)
    w, tgt = _setup(p, nsteps * p.dx / a)
    s = _solver(p, V.LIM_PP, V.FP64, lam)
    u0 = torch.tensor(p.conserved(), dtype=torch.float64, device=DEV)
    _, g = _adjoint(s, u0, nsteps, every, w, tgt)
    s.close()
    cfg = O.Config(p.nx, p.ny, (0, 0, 0, 0), O.LIM_PP, p.gamma, 0.5, 1e-16)
    wn, tn, c0 = w.cpu().numpy(), tgt.cpu().numpy(), p.conserved()

    def uN(c):
        return O.run(cfg, c, p.dx, nsteps=nsteps, lam_fixed=lam)["state"][:4]

    gn = g.cpu().numpy()
    scale = 1e-2 * float(np.sqrt((gn * gn).mean()))

    def D(c, j, i, h):
        up, dn = c0.copy(), c0.copy()
        up[c, j, i] += h
        dn[c, j, i] -= h
        a_, b_ = uN(up), uN(dn)
        return 0.5 * float((wn * (a_ - b_) * (a_ + b_ - 2.0 * tn)).sum()) / (2 * h)

    for (j, i) in _cells(p, 20, 2):
        for c in range(4):
            h = 1e-4 * max(1.0, abs(c0[c, j, i]))
            fd = (4.0 * D(c, j, i, h) - D(c, j, i, 2.0 * h)) / 3.0
            err = abs(fd - gn[c, j, i]) / max(abs(gn[c, j, i]), scale)
            assert err <= 1e-5, (j, i, c, fd, gn[c, j, i])


def test_adjoint_full_size_vortex_with_bumps():
    """512^2 vortex with 8 bumps, 500 steps, checkpoints every 50, loss against the
    unperturbed vortex advanced by the same scheme: the FP32 adjoint sweep against the
    FP64 one from the same dL/du^N (<= 1e-3 of max |g|; end to end, with the FP32
    forward's own loss, <= 5e-3), and the FP64 adjoint against differences of the
    FP64 GPU forward map on 20 cells (seed 2) x 4."""
    p = W.vortex_with_bumps(512)
    lam = 1.05 * _lam0(p)
    nsteps, every = 500, 50
    # L = dx^2 / 2 sum |u^N - u_target|^2, u_target = the unperturbed vortex advanced by
    # the same scheme (FP64)
    s64 = _solver(p, V.LIM_PP, V.FP64, lam)
    base = torch.tensor(W.isentropic_vortex(512).conserved(), dtype=torch.float64, device=DEV)
    tgt = _final(s64, base, nsteps)
    w = torch.full_like(tgt, p.dx * p.dx)
    u64 = torch.tensor(p.conserved(), dtype=torch.float64, device=DEV)
    _, g64 = _adjoint(s64, u64, nsteps, every, w, tgt)
    uN64 = _final(s64, u64, nsteps)
    seed = (w * (uN64 - tgt)).contiguous()               # dL/du^N of the FP64 run
    # FP32 sweep (FP32 rollout, recomputation and adjoint kernels) from the same dL/du^N
    s32 = _solver(p, V.LIM_PP, V.FP32, lam)
    scr = s32.adjoint_scratch(nsteps, every)
    u32 = u64.float()
    g32 = s32.adjoint(seed.float(), nsteps, every, scr, u0=u32).double()
    rel = float((g32 - g64).abs().max() / g64.abs().max())
    assert rel <= 1e-3, rel
    # end to end in FP32 (its own loss): the FP32 forward's rounding, ~1e-5 of u after
    # 500 steps, enters u^N - u_target, a difference of ~1e-2 of u
    tgt32 = _final(s32, base.float(), nsteps).double()
    _, g32e = _adjoint(s32, u32, nsteps, every, w, tgt32)
    rel_e2e = float((g32e - g64).abs().max() / g64.abs().max())
    assert rel_e2e <= 5e-3, rel_e2e
    s32.close()
    s64.close()
    # the finite differences step with the one-thread-per-cell kernel (2.4x faster than
    # the row-marching one on a 512^2 FP64 grid; both are bit-identical to the oracle)
    fd_solver = _solver(p, V.LIM_PP, V.FP64, lam, V.KERNEL_SIMPLE)
    _fd_check(fd_solver, u64, nsteps, w, tgt, g64, _cells(p, 20, 2))
    fd_solver.close()


def test_adjoint_rejects_unsupported():
    p = W.vortex_with_bumps(32)
    u0 = torch.tensor(p.conserved(), dtype=torch.float64, device=DEV)
    s = V.VLBM(p.nx, p.ny, p.dx, lam=1.0, limiter=V.LIM_PP, precision=V.FP64, device=DEV)
    s.set_conserved(u0[0].contiguous(), u0[1:3].contiguous(), u0[3].contiguous())
    with pytest.raises(V.VLBMError) as e:        # no rollout precedes it
        s.adjoint(u0, 4, 2, s.adjoint_scratch(4, 2))
    assert e.value.code == V.E_INVAL
    s.step(1)
    with pytest.raises(V.VLBMError):             # rollout must start at n = 0
        s.rollout(4, 2, s.adjoint_scratch(4, 2))
    s.close()


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("limiter", [V.LIM_NONE, V.LIM_PP])
def test_adjoint_dynamic_speed_matches_autograd(limiter, kernel):
    """ADJOINT_DIFF_A: the dynamic a^n = 4 lambda(s^n) differentiated through the max
    (its argmax cell), against autograd of the PyTorch restatement (FP64), and
    different from the gradient that holds a^n."""
    cons, dx = _bumps(32)
    nsteps, every = 24, 7
    p = W.Problem("bumps", 32, 32, dx, 0.0, 0.0, cons[0], cons[1], cons[2], cons[3])
    w, tgt = _setup(p, 0.0)
    s = _solver(p, limiter, V.FP64, 0.0, kernel)
    u0 = torch.tensor(cons, dtype=torch.float64, device=DEV)
    _, g_hold = _adjoint(s, u0, nsteps, every, w, tgt)
    s.set_adjoint_mode(V.ADJOINT_DIFF_A)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert s.monitors()["status"] == 0
    s.close()
    x = torch.tensor(cons, dtype=torch.float64, requires_grad=True)
    sN = TR.rollout_dynamic(x, nsteps, limiter)
    assert np.abs(sN[:4].detach().numpy() - uN.cpu().numpy()).max() <= 1e-12 * np.abs(cons).max()
    (0.5 * (w.cpu() * (sN[:4] - tgt.cpu()) ** 2).sum()).backward()
    g_ref = x.grad.numpy()
    err = np.abs(g.cpu().numpy() - g_ref)
    assert err.max() <= 1e-9 * np.abs(g_ref).max(), (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert np.abs(g_hold.cpu().numpy() - g_ref).max() > 1e-6 * np.abs(g_ref).max()


def test_adjoint_dynamic_speed_fp32_close_to_fp64():
    cons, dx = _bumps(32)
    p = W.Problem("bumps", 32, 32, dx, 0.0, 0.0, cons[0], cons[1], cons[2], cons[3])
    w, tgt = _setup(p, 0.0)
    gs = {}
    for prec, dt in ((V.FP64, torch.float64), (V.FP32, torch.float32)):
        s = _solver(p, V.LIM_PP, prec, 0.0, V.KERNEL_FUSED)
        s.set_adjoint_mode(V.ADJOINT_DIFF_A)
        u0 = torch.tensor(cons, dtype=dt, device=DEV)
        _, gs[prec] = _adjoint(s, u0, 20, 6, w, tgt)
        s.close()
    ref = gs[V.FP64].cpu().numpy()
    assert np.abs(gs[V.FP32].cpu().numpy() - ref).max() <= 5e-3 * np.abs(ref).max()


def test_adjoint_mode_is_checked():
    cons, dx = _bumps(16)
    p = W.Problem("bumps", 16, 16, dx, 0.0, 0.0, cons[0], cons[1], cons[2], cons[3])
    s = _solver(p, V.LIM_PP, V.FP64, 0.0)
    with pytest.raises(V.VLBMError):
        s.set_adjoint_mode(7)
    s.close()


def _boxed(case):
    """Smooth data in a box (Gaussian density and pressure bumps riding a uniform
    flow), with the sides of `case`: zero-gradient and mirror walls; zero-gradient
    sides with a sponge layer (periodic in y); prescribed states on two sides and a
    south side that switches from mirror to zero gradient."""
    nx, ny = 40, 32
    dx = 1.0 / nx
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    bump = np.exp(-((X - 0.45) ** 2 + (Y - 0.5) ** 2) / 0.02)
    base = (1.0, 0.3, 0.15, 1.0)
    cons = np.stack(W.primitive_to_conserved(1.0 + 0.2 * bump, base[1], base[2], 1.0 + 0.1 * bump))
    p = W.Problem(case, nx, ny, dx, 0.0, 0.0, cons[0], cons[1], cons[2], cons[3])
    sponge = 0
    if case == "zg-mirror":
        p.bc = (1, 1, 2, 2)
    elif case == "sponge":
        p.bc, sponge = (1, 1, 0, 0), 3
    else:
        p.bc, p.bc_hi, p.split = (3, 1, 2, 3), (3, 1, 1, 3), (0, 0, 15, 0)
        st = W._conserved_state(*base, 1.4)
        p.bfield = W.BoundaryField(st, st, ())
    return p, sponge


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("limiter", [V.LIM_FIRST_ORDER, V.LIM_NONE, V.LIM_PP])
@pytest.mark.parametrize("case", ["zg-mirror", "sponge", "dirichlet-split"])
def test_adjoint_fd_with_boundaries(case, limiter, kernel):
    """Grids with a boundary: the adjoint gathers over the first ghost layer too and
    folds the ghost cotangents back (transpose of the ghost fill); FP64 gradient
    against Richardson central differences at cells on every side and corner."""
    p, sponge = _boxed(case)
    cfg_bf = getattr(p, "bfield", None)
    boundary = V.make_boundary(p.bc, getattr(p, "bc_hi", None), getattr(p, "split", (0, 0, 0, 0)), p.x0, p.y0,
                               cfg_bf) if cfg_bf is not None or getattr(p, "bc_hi", None) else None
    lam = 1.1 * O.max_speed(O.Config(p.nx, p.ny, (1, 1, 1, 1), 0, 1.4, 0.5, 1e-16), O.new_state(p.conserved()))
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, lam=lam, limiter=limiter, precision=V.FP64, kernel=kernel,
               device=DEV, sponge=sponge, boundary=boundary)
    nsteps, every = 24, 7
    w, tgt = _setup(p, 0.0)
    u0 = torch.tensor(p.conserved(), dtype=torch.float64, device=DEV)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert torch.equal(uN, _final(s, u0, nsteps))
    ny, nx = p.ny, p.nx
    cells = [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1), (0, 17), (ny - 1, 9), (5, 0), (20, nx - 1),
             (1, 14), (16, 1), (14, 16), (1, 1)]
    _fd_check(s, u0, nsteps, w, tgt, g, cells)
    s.close()


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("case", ["pp", "lmp", "pp-fast-field", "lmp-fast-field"])
def test_adjoint_dynamic_speed_with_prescribed_states(case, kernel):
    """ADJOINT_DIFF_A with prescribed boundary states (two sides, and a south side that
    switches from mirror to zero gradient): a prescribed ghost's populations are its
    Maxwellians at a^n, so the fold adds their dL/da^n; when the prescribed state is
    faster than every cell (fast-field) lambda^n does not depend on the state. Against
    autograd of the restatement whose ghost constants follow a^n."""
    from tests.test_torch_reference import _box_cfg, boxed_waves
    limiter = V.LIM_LMP if case.startswith("lmp") else V.LIM_PP
    cons, dx, kw = boxed_waves("dirichlet-split")
    cons = cons * (1.0 + 1e-3 * np.random.default_rng(13).uniform(-1.0, 1.0, cons.shape))
    ny, nx = cons.shape[1:]
    if case.endswith("fast-field"):
        st = W._conserved_state(1.0, 2.5, 0.0, 1.0, 1.4)
        kw["field"] = O.Field(st, st, ())
    r, m1, m2, E = kw["field"].inside
    v2 = (m1 * m1 + m2 * m2) / (r * r)
    lam_bc = float(np.sqrt(v2) + np.sqrt(1.4 * 0.4 * (E - 0.5 * r * v2) / r))
    boundary = V.make_boundary(kw["bc"], kw["bc_hi"], kw["split"], 0.0, 0.0, kw["field"])
    s = V.VLBM(nx, ny, dx, bc=kw["bc"], limiter=limiter, precision=V.FP64, kernel=kernel, device=DEV,
               boundary=boundary)
    s.set_adjoint_mode(V.ADJOINT_DIFF_A)
    nsteps, every = 12, 5
    rng = np.random.default_rng(7)
    w = torch.tensor(rng.uniform(0.5, 1.5, size=(4, ny, nx)), dtype=torch.float64, device=DEV)
    tgt = torch.tensor(cons * 0.97, dtype=torch.float64, device=DEV)
    u0 = torch.tensor(cons, dtype=torch.float64, device=DEV)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert s.monitors()["status"] == 0
    s.close()
    fr = TR.ghost_frame(_box_cfg(nx, ny, limiter, kw, dx), 1.0, const_in_a=True)
    x = torch.tensor(cons, dtype=torch.float64, requires_grad=True)
    sN = TR.rollout_dynamic_frame(x, nsteps, limiter, fr, lam_bc=lam_bc)
    assert np.abs(sN[:4].detach().numpy() - uN.cpu().numpy()).max() <= 1e-12 * np.abs(cons).max()
    (0.5 * (w.cpu() * (sN[:4] - tgt.cpu()) ** 2).sum()).backward()
    g_ref = x.grad.numpy()
    err = np.abs(g.cpu().numpy() - g_ref)
    assert err.max() <= 1e-9 * np.abs(g_ref).max(), (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("limiter", [V.LIM_LMP, V.LIM_RLMP])
def test_adjoint_lmp_matches_autograd(limiter, kernel):
    """LMP / RLMP (periodic, a held): the three-pass adjoint (faces, bounds, gather)
    against autograd of the PyTorch restatement, FP64, on smooth waves where the
    density bound is active on 240-310 faces per step."""
    from tests.test_torch_reference import _waves
    cons, dx = _waves(32)
    n = cons.shape[1]
    cfg = O.Config(n, n, (0, 0, 0, 0), limiter, 1.4, 0.5, 1e-16)
    lam = 1.05 * O.max_speed(cfg, O.new_state(cons))
    a = O.kinetic_speed(lam, 0.5)
    st = O.run(cfg, cons, dx, nsteps=4, lam_fixed=lam)["state"]
    _, dbg = O.step(cfg, st, a, debug=True)
    assert (dbg["theta_x"] < 1.0).sum() + (dbg["theta_y"] < 1.0).sum() > 200
    p = W.Problem("waves", n, n, dx, 0.0, 0.0, cons[0], cons[1], cons[2], cons[3])
    w, tgt = _setup(p, 0.0)
    nsteps, every = 16, 5
    s = _solver(p, limiter, V.FP64, lam, kernel)
    u0 = torch.tensor(cons, dtype=torch.float64, device=DEV)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert s.monitors()["status"] == 0
    s.close()
    ref = O.run(cfg, cons, dx, nsteps=nsteps, lam_fixed=lam)["state"]
    assert np.array_equal(uN.cpu().numpy(), ref[:4])
    sN, g_ref = _autograd_gradient(cons, nsteps, a, limiter, w, tgt, 1e-16)
    err = np.abs(g.cpu().numpy() - g_ref)
    assert err.max() <= 1e-9 * np.abs(g_ref).max(), (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("limiter", [V.LIM_LMP, V.LIM_RLMP])
@pytest.mark.parametrize("case", ["zg-mirror", "sponge", "dirichlet-split"])
def test_adjoint_lmp_with_boundaries(case, limiter, kernel):
    """LMP / RLMP on grids with a boundary (a held): the bounds of the first ghost
    layer enter the boundary faces and reach rho* of faces in the second, so the
    three passes run over a two-layer frame and the fold undoes two ghost layers.
    FP64 gradient against autograd through the restatement inside the oracle's
    ghost frame, on smooth waves in a box."""
    from tests.test_torch_reference import _box_cfg, boxed_waves
    cons, dx, kw = boxed_waves(case)
    ny, nx = cons.shape[1:]
    cfg = _box_cfg(nx, ny, limiter, kw, dx)
    lam = 1.05 * O.max_speed(cfg, O.new_state(cons))
    a = O.kinetic_speed(lam, 0.5)
    boundary = V.make_boundary(kw["bc"], kw["bc_hi"], kw["split"], 0.0, 0.0, kw["field"]) if "field" in kw else None
    s = V.VLBM(nx, ny, dx, bc=kw["bc"], lam=lam, limiter=limiter, precision=V.FP64, kernel=kernel, device=DEV,
               sponge=kw["sponge"], boundary=boundary)
    nsteps, every = 16, 5
    rng = np.random.default_rng(5)
    w = torch.tensor(rng.uniform(0.5, 1.5, size=(4, ny, nx)), dtype=torch.float64, device=DEV)
    tgt = torch.tensor(cons * 0.97, dtype=torch.float64, device=DEV)
    u0 = torch.tensor(cons, dtype=torch.float64, device=DEV)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert s.monitors()["status"] == 0
    s.close()
    ref = O.run(cfg, cons, dx, nsteps=nsteps, lam_fixed=lam)["state"]
    assert np.array_equal(uN.cpu().numpy(), ref[:4])
    fr = TR.ghost_frame(cfg, a, sponge=kw["sponge"])
    x = torch.tensor(cons, dtype=torch.float64, requires_grad=True)
    sN = TR.rollout_frame(x, nsteps, a, limiter, fr)
    (0.5 * (w.cpu() * (sN[:4] - tgt.cpu()) ** 2).sum()).backward()
    g_ref = x.grad.numpy()
    err = np.abs(g.cpu().numpy() - g_ref)
    assert err.max() <= 1e-9 * np.abs(g_ref).max(), (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
@pytest.mark.parametrize("case", ["periodic-lmp", "periodic-rlmp", "zg-mirror-lmp", "sponge-rlmp"])
def test_adjoint_lmp_dynamic_speed(case, kernel):
    """ADJOINT_DIFF_A with LMP / RLMP: d theta / da of every face (kappa, u*, dF and the
    bound that won, through rho* of its face) from pass 1, handed to the argmax cell
    of lambda^n; against autograd of the restatement with a^n = 4 lambda(s^n)."""
    from tests.test_torch_reference import _box_cfg, _waves, boxed_waves
    name, lim = case.rsplit("-", 1)
    limiter = V.LIM_LMP if lim == "lmp" else V.LIM_RLMP
    if name == "periodic":
        cons, dx = _waves(32)
        kw = {"bc": (0, 0, 0, 0), "sponge": 0}
    else:
        cons, dx, kw = boxed_waves(name)
    # the waves' cell speeds come in near-equal pairs (maxima of smooth fields): a seeded
    # 1e-3 relative perturbation makes the max of lambda^n unique at every step, where
    # the gradient of the max is defined (at a tie any split between the cells is a
    # subgradient, and the library and autograd pick differently)
    cons = cons * (1.0 + 1e-3 * np.random.default_rng(12).uniform(-1.0, 1.0, cons.shape))
    ny, nx = cons.shape[1:]
    s = V.VLBM(nx, ny, dx, bc=kw["bc"], limiter=limiter, precision=V.FP64, kernel=kernel, device=DEV,
               sponge=kw["sponge"])
    s.set_adjoint_mode(V.ADJOINT_DIFF_A)
    nsteps, every = 16, 5
    rng = np.random.default_rng(6)
    w = torch.tensor(rng.uniform(0.5, 1.5, size=(4, ny, nx)), dtype=torch.float64, device=DEV)
    tgt = torch.tensor(cons * 0.97, dtype=torch.float64, device=DEV)
    u0 = torch.tensor(cons, dtype=torch.float64, device=DEV)
    uN, g = _adjoint(s, u0, nsteps, every, w, tgt)
    assert s.monitors()["status"] == 0
    s.close()
    x = torch.tensor(cons, dtype=torch.float64, requires_grad=True)
    fr = None if name == "periodic" else TR.ghost_frame(_box_cfg(nx, ny, limiter, kw, dx), 1.0, sponge=kw["sponge"])
    def speed_gap_and_a(u):   # (relative gap between the two largest cell speeds, 4 lambda)
        r, m1, m2, E = u[0], u[1], u[2], u[3]
        v2 = (m1 * m1 + m2 * m2) / (r * r)
        top = torch.topk((torch.sqrt(v2) + torch.sqrt(1.4 * 0.4 * (E - 0.5 * r * v2) / r)).flatten(), 2).values
        return float((top[0] - top[1]) / top[0]), 4.0 * float(top[0])

    with torch.no_grad():   # the largest cell speed leads the next by a clear margin at every step
        gap, a = speed_gap_and_a(x)
        st = TR.init_populations(x, a, 0.5, 1.4)
        for m in range(nsteps):
            assert gap > 1e-9, (m, gap)
            st = TR.step(st, a, limiter) if fr is None else TR.step_frame(st, a, limiter, fr)
            gap, a = speed_gap_and_a(st[0:4])
    sN = TR.rollout_dynamic(x, nsteps, limiter) if fr is None else TR.rollout_dynamic_frame(x, nsteps, limiter, fr)
    assert np.abs(sN[:4].detach().numpy() - uN.cpu().numpy()).max() <= 1e-12 * np.abs(cons).max()
    (0.5 * (w.cpu() * (sN[:4] - tgt.cpu()) ** 2).sum()).backward()
    g_ref = x.grad.numpy()
    err = np.abs(g.cpu().numpy() - g_ref)
    assert err.max() <= 1e-9 * np.abs(g_ref).max(), (err.max(), np.unravel_index(err.argmax(), err.shape))
