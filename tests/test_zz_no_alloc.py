"""The workspace-free step, vlbm_step_noalloc, against the regular path and the oracle.

Some callers cannot allocate device memory (a plugin whose host owns the device
memory pool, a real-time loop that may not synchronise on cudaMalloc); they
step their own 20-plane state with vlbm_step_noalloc, whose only scratch is a
fixed array inside the library. Both paths evaluate the same per-cell step, so two
calls in a row must give the regular workspace path's state bit for bit, in both
precisions; in FP64 one call on a state the oracle produced must also give the
oracle's next state bit for bit (the FP64 path reproduces the oracle's operation
order). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2411_15001_gb300 import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_15001_gb300 import vlbm as V  # noqa: E402


@pytest.mark.parametrize("prec", [V.FP64, V.FP32])
@pytest.mark.parametrize("lim,problem", [(V.LIM_LMP, "quadrant"), (V.LIM_PP, "vortex")])
def test_noalloc_matches_workspace_path(prec, lim, problem):
    if problem == "quadrant":
        p = W.quadrant_riemann(77, 53, seed=5, bc=(1, 2, 2, 1))
    else:
        p = W.isentropic_vortex(64)
    dt = torch.float64 if prec == V.FP64 else torch.float32
    dev = torch.device("cuda:0")
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, limiter=lim, precision=prec, kernel=V.KERNEL_SIMPLE,
               device=dev)
    c = torch.tensor(p.conserved(), dtype=dt, device=dev)
    s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    s.step(3)                                   # populations off equilibrium
    state = s.state_planes().clone()            # 20 compact planes on the device
    grid = V.vlbm_grid(p.nx, p.ny, p.dx, (ctypes.c_int32 * 4)(*p.bc))
    opts = V.vlbm_opts(0.5, 1e-16, 0, 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    bufs = [state, torch.empty_like(state)]
    for call in range(2):
        a = s.monitors()["a"]
        rc, res = V.vlbm_step_noalloc(grid, p.gamma, a, lim, prec, opts, bufs[call % 2].data_ptr(),
                                      bufs[(call + 1) % 2].data_ptr(), stream)
        assert rc == V.OK, V.vlbm_strerror(rc)
        s.step(1)
        ref = s.state_planes().cpu().numpy()
        got = bufs[(call + 1) % 2].cpu().numpy()
        assert np.array_equal(got, ref), float(np.abs(got.astype(np.float64) - ref).max())
        mon = s.monitors()
        assert res.a_next == pytest.approx(mon["a"], rel=1e-12 if prec == V.FP64 else 1e-6)
        assert res.bad_cells == 0 and res.nonfinite_cells == 0
        np.testing.assert_allclose(list(res.sum), mon["sum"], rtol=1e-12, atol=1e-9)
    s.close()


@pytest.mark.parametrize("lim,oracle_lim", [(V.LIM_LMP, O.LIM_LMP), (V.LIM_PP, O.LIM_PP)])
def test_noalloc_fp64_equals_oracle(lim, oracle_lim):
    p = W.quadrant_riemann(45, 38, seed=6, bc=(1, 2, 2, 1))
    cfg = O.Config(p.nx, p.ny, p.bc, oracle_lim, p.gamma)
    r = O.run(cfg, p.conserved(), p.dx, nsteps=4)           # populations off equilibrium
    a = O.kinetic_speed(O.max_speed(cfg, r["state"]), 0.5)
    want = O.step(cfg, r["state"], a)
    dev = torch.device("cuda:0")
    d_in = torch.tensor(r["state"], dtype=torch.float64, device=dev).contiguous()
    d_out = torch.empty_like(d_in)
    grid = V.vlbm_grid(p.nx, p.ny, p.dx, (ctypes.c_int32 * 4)(*p.bc))
    rc, res = V.vlbm_step_noalloc(grid, p.gamma, a, lim, V.FP64, None, d_in.data_ptr(), d_out.data_ptr(),
                                  torch.cuda.current_stream(dev).cuda_stream)
    assert rc == V.OK, V.vlbm_strerror(rc)
    assert np.array_equal(d_out.cpu().numpy(), want)
    assert res.lambda_ == O.max_speed(cfg, want)


def test_noalloc_rejects_oversized_grid():
    grid = V.vlbm_grid(4096, 4096, 1.0, (ctypes.c_int32 * 4)(0, 0, 0, 0))
    rc, _ = V.vlbm_step_noalloc(grid, 1.4, 1.0, V.LIM_PP, V.FP32, None, 256, 512, None)
    assert rc == V.E_INVAL
