"""Failure detection of the step kernels, through the C-ABI, without faulting the GPU.

- The kinetic-speed monitor is the Euclidean |v| + c of Sec. 4 (preamble).
- A state that leaves G: the unlimited scheme on the Lax-Liu configuration 3, which
  Sec. 4.7 reports to crash; the device records VLBM_E_POSITIVITY at the step where
  the oracle's run first leaves G, with the same count of cells outside G.
- A non-finite value, planted on the host in a checkpoint and loaded: the next step
  reports VLBM_E_NONFINITE, the state stops advancing (the error is sticky) and a new
  vlbm_set_conserved clears it.
- A bounded device wait that runs out: the row-marching kernel's wait probe
  (vlbm_test_wait_probe) makes every CTA wait on a barrier nothing completes; each
  gives up after the armed limit, issues no load, and the call reports
  VLBM_E_TIMEOUT; the context stays usable and the next run is bit-exact.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_15001_gb300 import vlbm as V  # noqa: E402

DEV = "cuda:0"


def _solver(p, limiter, precision, kernel=V.KERNEL_AUTO, **kw):
    dt = torch.float64 if precision == V.FP64 else torch.float32
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, gamma=p.gamma, limiter=limiter, precision=precision,
               kernel=kernel, device=DEV, **kw)
    c = torch.tensor(p.conserved(), dtype=dt, device=DEV)
    s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    return s


@pytest.mark.parametrize("prec, rel", [(V.FP64, 1e-14), (V.FP32, 5e-6)])
def test_speed_monitor_is_euclidean(prec, rel):
    # (rho, v1, v2, p) = (1, 3, 4, 1), gamma = 1.4: lambda = |v| + c = 5 + sqrt(1.4); the
    # max-norm speed of Prop. convex_preservation_O1 would give 4 + sqrt(1.4). In FP32
    # the monitor is an upper bound of the exact speed of the float state (with the
    # float gamma and gamma - 1 the kernels use), at most a few 1e-6 above it.
    nx = ny = 16
    dt = torch.float64 if prec == V.FP64 else torch.float32
    rho = torch.ones((ny, nx), dtype=dt, device=DEV)
    mom = torch.empty((2, ny, nx), dtype=dt, device=DEV)
    mom[0], mom[1] = 3.0, 4.0
    E = torch.full((ny, nx), 1.0 / 0.4 + 12.5, dtype=dt, device=DEV)
    for kernel in (V.KERNEL_SIMPLE, V.KERNEL_FUSED):
        s = V.VLBM(nx, ny, 0.1, bc=(0, 0, 0, 0), gamma=1.4, limiter=V.LIM_PP, precision=prec, kernel=kernel,
                   device=DEV)
        s.set_conserved(rho, mom, E)
        lam = 5.0 + math.sqrt(1.4)
        if prec == V.FP32:   # p = (gamma - 1)(E - |m|^2 / 2 rho) = 2.5 (gamma - 1), float constants
            lam = 5.0 + math.sqrt(float(np.float32(1.4)) * float(np.float32(1.4 - 1.0)) * 2.5)
        m = s.monitors()
        assert m["lambda"] == pytest.approx(lam, rel=rel) and m["a"] == pytest.approx(4 * lam, rel=rel)
        if prec == V.FP32:
            assert m["lambda"] >= lam, (m["lambda"], lam)
        s.step(3)                                          # a uniform flow stays uniform
        m = s.monitors()
        assert m["status"] == V.OK and m["lambda"] == pytest.approx(lam, rel=rel), m
        if prec == V.FP32:
            assert m["lambda"] >= lam, (m["lambda"], lam)
        s.close()


def _oracle_first_bad_step(p, limiter, t_end):
    """(first step whose output has a cell outside G, cells outside G after it)."""
    first = []

    def check(k, st):
        u = st[:4]
        bad = ~((u[0] > 0) & (2.0 * u[0] * u[3] - (u[1] * u[1] + u[2] * u[2]) > 0))
        if bad.any() and not first:
            first.append((k, int(bad.sum())))

    with pytest.raises(FloatingPointError):        # Sec. 4.7: the unlimited scheme crashes
        O.run(O.Config(p.nx, p.ny, p.bc, limiter, p.gamma), p.conserved(), p.dx, t_end=t_end, callback=check)
    return first[0]


@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
def test_unlimited_scheme_leaves_G_where_the_oracle_does(kernel):
    p = W.lax_liu_config3(48)
    k_bad, n_bad = _oracle_first_bad_step(p, O.LIM_SECOND, 0.8)
    s = _solver(p, V.LIM_NONE, V.FP64, kernel)
    s.step(k_bad - 1)
    m = s.monitors()
    assert m["status"] == V.OK and m["first_bad_step"] == -1 and m["bad_cells"] == 0
    s.step(1)
    m = s.monitors()
    assert m["status"] == V.E_POSITIVITY, m
    assert m["first_bad_step"] == k_bad and m["bad_cells"] == n_bad and m["n"] == k_bad, (m, k_bad, n_bad)
    # carried on to the final time, the run stays flagged (sticky) and ends non-finite or at t
    rc = V.vlbm_step_to(s._s, 0.8, 10 ** 5)
    m = s.monitors()
    assert rc == V.E_POSITIVITY and m["status"] == V.E_POSITIVITY and m["first_bad_step"] == k_bad, (rc, m)
    assert V.vlbm_sync(s._s) == V.E_POSITIVITY
    s.close()


@pytest.mark.parametrize("prec", [V.FP64, V.FP32])
@pytest.mark.parametrize("kernel", [V.KERNEL_SIMPLE, V.KERNEL_FUSED])
def test_non_finite_value_is_reported_and_sticky(prec, kernel):
    p = W.quadrant_riemann(64, 48, seed=4)
    s = _solver(p, V.LIM_LMP, prec, kernel)
    s.step(5)
    ck = s.save()
    host = ck.cpu()
    dt = np.float64 if prec == V.FP64 else np.float32
    planes = host[64:].numpy().view(dt).reshape(20, p.ny, p.nx)
    planes[4, 20, 30] = np.nan                      # population u_1 of cell (30, 20)
    s.load(host.to(DEV))
    s.step(1)
    assert V.vlbm_sync(s._s) == V.E_NONFINITE
    m = s.monitors()
    assert m["status"] == V.E_NONFINITE and m["nonfinite_cells"] >= 1 and m["first_bad_step"] == 6, m
    assert m["n"] == 6 and m["done"] == 1
    s.step(4)                                        # nothing runs on a failed state
    m2 = s.monitors()
    assert m2["n"] == 6 and m2["status"] == V.E_NONFINITE
    # a new initial state clears the error
    c = torch.tensor(p.conserved(), dtype=torch.float64 if prec == V.FP64 else torch.float32, device=DEV)
    s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    s.step(3)
    m3 = s.monitors()
    assert m3["status"] == V.OK and m3["n"] == 3 and m3["first_bad_step"] == -1
    s.close()


@pytest.mark.parametrize("prec", [V.FP32, V.FP64])
def test_bounded_wait_runs_out_and_is_reported(prec):
    p = W.quadrant_riemann(256, 192, seed=5)
    ref = _solver(p, V.LIM_PP, prec, V.KERNEL_FUSED)
    ref.step(7)
    want = ref.state_planes().cpu().numpy()
    ref.close()

    s = _solver(p, V.LIM_PP, prec, V.KERNEL_FUSED)
    s.step(2)
    assert V.vlbm_test_wait_probe(s._s, 2_000_000) == V.OK     # 2 ms per CTA
    s.step(3)
    assert V.vlbm_sync(s._s) == V.E_TIMEOUT
    m = s.monitors()
    assert m["status"] == V.E_TIMEOUT and m["n"] == 2, m          # no step completed
    s.step(64)                                                    # (single launches while armed)
    m = s.monitors()
    assert m["status"] == V.E_TIMEOUT and m["n"] == 2, m
    # the context is intact: a new initial state disarms the probe, and the run that
    # follows is the reference run bit for bit (the work counter was left reset)
    c = torch.tensor(p.conserved(), dtype=torch.float64 if prec == V.FP64 else torch.float32, device=DEV)
    s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    s.step(7)
    m = s.monitors()
    assert m["status"] == V.OK and m["n"] == 7
    got = s.state_planes().cpu().numpy()
    assert np.array_equal(got, want)
    s.close()
