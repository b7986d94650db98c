"""The PyTorch binding orders its calls against torch's current stream.

A solver given its own stream reads inputs that the caller produced on the current
stream and writes outputs that the caller reads there. Delays on either stream
(torch.cuda._sleep) make a missing wait visible: without the ordering, the solver
would read inputs not yet written, or the caller would read outputs not yet written.
Results must equal the same run on the default stream bit for bit.

The autograd function: two rollouts on one solver before either backward; the first
backward must still get its own gradient (it recomputes its rollout from u_0).
"""
import numpy as np
import pytest

from paper_2411_15001_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_15001_gb300 import vlbm as V  # noqa: E402

DEV = torch.device("cuda:0")
SLEEP = 20_000_000          # GPU cycles, ~10 ms


def _planes(s):
    r, m, e = s.moments()
    return torch.cat([r[None], m, e[None]]).cpu().numpy()


@pytest.mark.parametrize("prec", [V.FP32, V.FP64])
def test_side_stream_solver_equals_default_stream(prec):
    p = W.quadrant_riemann(300, 200, seed=8)
    dt = torch.float64 if prec == V.FP64 else torch.float32
    c = torch.tensor(p.conserved(), dtype=dt, device=DEV)
    ref = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, limiter=V.LIM_LMP, precision=prec, device=DEV)
    ref.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    ref.step(70)
    want = _planes(ref)
    ref.close()

    side = torch.cuda.Stream(DEV)
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, limiter=V.LIM_LMP, precision=prec, device=DEV, stream=side)
    torch.cuda.synchronize(DEV)
    torch.cuda._sleep(SLEEP)                       # the inputs are produced late on the current stream
    rho, mom, E = c[0].clone(), c[1:3].clone(), c[3].clone()
    s.set_conserved(rho, mom, E)
    del rho, mom, E                                # freed while the solver may still read them
    s.step(70)
    with torch.cuda.stream(side):
        torch.cuda._sleep(SLEEP)                   # the outputs are written late on the solver's stream
    r, m, e = s.moments()
    got = torch.cat([r[None], m, e[None]]).cpu().numpy()    # read on the current stream right away
    assert np.array_equal(got, want)
    s.close()


def test_two_rollouts_before_their_backwards():
    p = W.isentropic_vortex(40)
    c = torch.tensor(p.conserved(), dtype=torch.float64, device=DEV)
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, lam=3.0, limiter=V.LIM_PP, precision=V.FP64, device=DEV)
    R = V.VLBMRollout

    def grad_of(scale):
        rho = (c[0] * scale).requires_grad_()
        mom, E = c[1:3].clone(), c[3].clone()
        out = R.apply(rho, mom, E, s, 30, 10)
        return rho, out

    # reference: one forward, its backward
    rho_a, out_a = grad_of(1.0)
    (out_a[0] ** 2).sum().backward()
    want = rho_a.grad.clone()
    # two forwards, then the first backward (the solver's latest rollout is the second)
    rho_1, out_1 = grad_of(1.0)
    rho_2, out_2 = grad_of(1.001)
    (out_1[0] ** 2).sum().backward()
    assert torch.equal(rho_1.grad, want)
    (out_2[0] ** 2).sum().backward()
    assert torch.isfinite(rho_2.grad).all() and not torch.equal(rho_2.grad, want)
    s.close()


@pytest.mark.parametrize("prec", [V.FP32, V.FP64])
def test_adjoint_on_side_stream_equals_default_stream(prec):
    """The reverse sweep runs its recomputation on a second stream of the library's;
    on a solver with its own stream, delayed inputs and outputs, the gradient over
    several segments equals the default-stream one bit for bit."""
    p = W.vortex_with_bumps(96)
    dt = torch.float64 if prec == V.FP64 else torch.float32
    c = torch.tensor(p.conserved(), dtype=dt, device=DEV)
    nsteps, every = 40, 7
    gN = torch.tensor(np.random.default_rng(11).standard_normal((4, p.ny, p.nx)), dtype=dt, device=DEV)

    def solver(stream=None):
        return V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, gamma=p.gamma, lam=4.0, limiter=V.LIM_PP, precision=prec,
                      device=DEV, stream=stream)

    ref = solver()
    want = ref.adjoint(gN, nsteps, every, ref.adjoint_scratch(nsteps, every), u0=c).cpu().numpy()
    ref.close()

    side = torch.cuda.Stream(DEV)
    s = solver(side)
    scratch = s.adjoint_scratch(nsteps, every)
    torch.cuda.synchronize(DEV)
    torch.cuda._sleep(SLEEP)                       # inputs produced late on the current stream
    u0, g_in = c.clone(), gN.clone()
    g = s.adjoint(g_in, nsteps, every, scratch, u0=u0)
    del u0, g_in
    with torch.cuda.stream(side):
        torch.cuda._sleep(SLEEP)
    got = g.cpu().numpy()
    assert np.isfinite(want).all() and np.array_equal(got, want)
    s.close()
