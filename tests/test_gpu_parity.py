"""CUDA path against the FP64 oracle through the C-ABI (needs a GB300).

Tolerances: FP64 path 1e-12 relative (max over each of the 20 planes; the FP64
kernels evaluate every formula in the oracle's operation order with IEEE
rounding, so most cases are bit-identical and are checked as such); FP32 path
relative L1 of the conserved fields <= 1e-5 on smooth data and <= 1e-3 on
discontinuous data; zero cells outside G at every step.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W
from tests.gpu_helpers import gpu_run, l1_rel, oracle_run, plane_rel_err
from tests.helpers import rel_norms, table1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_15001_gb300 import vlbm as V  # noqa: E402

BCS = [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (0, 0, 2, 1), (2, 1, 0, 0)]


KERNELS = [V.KERNEL_SIMPLE, V.KERNEL_FUSED]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("lim", [V.LIM_FIRST_ORDER, V.LIM_PP, V.LIM_LMP, V.LIM_RLMP])
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(37, 29), (70, 45), (251, 19)])
def test_fp64_parity_random_quadrants(kernel, lim, bc, shape):
    """Ragged sizes: one partial strip, and three strips of the fused kernel."""
    nx, ny = shape
    p = W.quadrant_riemann(nx, ny, seed=7, bc=bc)
    got, mon = gpu_run(p, lim, V.FP64, nsteps=12, kernel=kernel)
    ref = oracle_run(p, lim, nsteps=12)
    assert mon["status"] == 0 and mon["n"] == 12
    assert mon["t"] == ref["t"]
    assert plane_rel_err(got, ref["state"]) <= 1e-12
    assert np.array_equal(got, ref["state"])


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("lim", [V.LIM_PP, V.LIM_LMP])
@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (0, 0, 1, 1), (1, 2, 2, 1)])
def test_fp64_parity_sponge(kernel, lim, bc):
    """Sponge layer of Sec. 4.2 (theta = 0 within 5 cells of a zero-gradient side),
    on a grid of two strips with a ragged tail."""
    p = W.quadrant_riemann(130, 37, seed=8, bc=bc)
    got, mon = gpu_run(p, lim, V.FP64, nsteps=15, kernel=kernel, sponge=5)
    ref = oracle_run(p, lim, nsteps=15, sponge=5)
    assert mon["status"] == 0
    assert np.array_equal(got, ref["state"])


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_parity_unlimited_smooth(kernel):
    p = W.isentropic_vortex(40)
    got, mon = gpu_run(p, V.LIM_NONE, V.FP64, nsteps=30, kernel=kernel)
    ref = oracle_run(p, V.LIM_NONE, nsteps=30)
    assert plane_rel_err(got, ref["state"]) <= 1e-12


@pytest.mark.parametrize("kernel", KERNELS)
def test_vortex_128_fp64_pp_200_steps(kernel):
    """128^2 periodic isentropic vortex, FP64, PP, dynamic a, 200 steps."""
    p = W.isentropic_vortex(128)
    got, mon = gpu_run(p, V.LIM_PP, V.FP64, nsteps=200, kernel=kernel)
    ref = oracle_run(p, V.LIM_PP, nsteps=200)
    assert mon["status"] == 0 and mon["bad_cells"] == 0 and mon["first_bad_step"] == -1
    assert abs(mon["t"] - ref["t"]) <= 1e-12 * ref["t"]
    assert plane_rel_err(got, ref["state"]) <= 1e-12


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_blast_parity(kernel):
    """Near-vacuum blast (reflective walls, PP, eps = 1e-13) in FP64 against the oracle."""
    p = W.blast(64)
    got, mon = gpu_run(p, V.LIM_PP, V.FP64, nsteps=80, eps=1e-13, kernel=kernel)
    ref = oracle_run(p, V.LIM_PP, nsteps=80, eps=1e-13)
    assert mon["status"] == 0 and mon["first_bad_step"] == -1
    assert plane_rel_err(got, ref["state"]) <= 1e-12


@pytest.mark.parametrize("lim", ["PP", "LMP", "RLMP"])
def test_table1_on_gpu_fp64(lim):
    """Table 1 by the FP64 CUDA path (fused kernel), at every printed mesh.

    PP and RLMP (L1, L2) agree to the 6 printed digits at every mesh; LMP to 6 digits
    up to dx = 1/160. At dx = 1/320 and 1/640 the LMP bound of Sec. 3.3.1 jumps at
    faces where dF^rho is at round-off level near the extrema of the wave, so any two
    FP64 implementations that round differently differ in the 5th digit there (the
    oracle gives 5.86559e-5 at 1/320 where the paper prints 5.86654e-5); those
    entries are held to 1%."""
    code = {"PP": V.LIM_PP, "LMP": V.LIM_LMP, "RLMP": V.LIM_RLMP}[lim]
    for N in (20, 40, 80, 160, 320, 640):
        p = W.entropy_wave(N)
        got, mon = gpu_run(p, code, V.FP64, nsteps=int(round(10.7 * N)), lam=10.7 / 4,
                           kernel=V.KERNEL_FUSED)
        assert abs(mon["t"] - 1.0) < 1e-11
        err = rel_norms(got[0], W.entropy_wave(N).rho)
        ref = table1()[(lim, N)]
        rel = 1e-2 if (lim == "LMP" and N >= 320) else 1.5e-5
        for k in range(3 if lim != "RLMP" else 2):
            assert float("%.5e" % err[k]) == pytest.approx(ref[k], rel=rel), (N, k, err, ref)


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_smooth_vortex(kernel):
    p = W.isentropic_vortex(128)
    got, mon = gpu_run(p, V.LIM_PP, V.FP32, nsteps=200, kernel=kernel)
    ref = oracle_run(p, V.LIM_PP, nsteps=200)
    assert mon["status"] == 0 and mon["first_bad_step"] == -1
    assert l1_rel(got[:4], ref["state"][:4]) <= 1e-5


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("lim", [V.LIM_PP, V.LIM_LMP, V.LIM_RLMP])
def test_fp32_discontinuous_quadrants(kernel, lim):
    p = W.quadrant_riemann(200, 160, seed=0)
    got, mon = gpu_run(p, lim, V.FP32, t_end=0.05, kernel=kernel)
    ref = oracle_run(p, lim, t_end=0.05)
    assert mon["status"] == 0 and mon["first_bad_step"] == -1 and mon["n"] == ref["n"]
    assert l1_rel(got[:4], ref["state"][:4]) <= 1e-3


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_near_vacuum_blast(kernel):
    """Sedov-type blast, p = 1e-6 ambient, reflective walls, PP with eps = 1e-13.

    The near-vacuum core of this blast amplifies round-off exponentially (see
    test_blast_amplifies_round_off), so the FP32 path is held to the discontinuous
    tolerance over the first 40 steps and to the invariants (admissibility, mass and
    energy conserved by the walls) over 150."""
    p = W.blast(96)
    got, mon = gpu_run(p, V.LIM_PP, V.FP32, nsteps=40, eps=1e-13, kernel=kernel)
    ref = oracle_run(p, V.LIM_PP, nsteps=40, eps=1e-13)
    assert mon["status"] == 0 and mon["first_bad_step"] == -1
    assert l1_rel(got[:4], ref["state"][:4]) <= 1e-3
    got, mon = gpu_run(p, V.LIM_PP, V.FP32, nsteps=150, eps=1e-13, kernel=kernel)
    assert mon["status"] == 0 and mon["first_bad_step"] == -1 and mon["bad_cells"] == 0
    c0 = p.conserved().astype(np.float32).astype(np.float64).reshape(4, -1).sum(axis=1)
    assert abs(mon["sum"][0] - c0[0]) <= 1e-5 * c0[0]
    assert abs(mon["sum"][3] - c0[3]) <= 1e-5 * c0[3]


def test_blast_amplifies_round_off():
    """FP64 only: a relative perturbation of 1e-12 of the initial energy grows by many
    orders of magnitude over 150 steps of the near-vacuum blast, so no two
    implementations that round differently can agree there to FP32 round-off."""
    p = W.blast(96)
    a, _ = gpu_run(p, V.LIM_PP, V.FP64, nsteps=150, eps=1e-13)
    q = W.blast(96)
    q.E = q.E * (1.0 + 1e-12 * np.cos(np.arange(q.E.size).reshape(q.E.shape)))
    b, _ = gpu_run(q, V.LIM_PP, V.FP64, nsteps=150, eps=1e-13)
    growth = l1_rel(b[:4], a[:4]) / 1e-12
    assert growth > 1e4, growth


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,tol", [(V.FP64, 1e-13), (V.FP32, 1e-6)])
def test_conservation_monitor_periodic(prec, tol, kernel):
    p = W.quadrant_riemann(300, 80, seed=4, bc=(0, 0, 0, 0))
    got, mon = gpu_run(p, V.LIM_LMP, prec, nsteps=100, kernel=kernel)
    s0 = p.conserved().reshape(4, -1)
    if prec == V.FP32:
        s0 = s0.astype(np.float32).astype(np.float64)
    ref = s0.sum(axis=1)
    scale = np.abs(s0).sum(axis=1)
    assert np.all(np.abs(np.array(mon["sum"]) - ref) <= tol * scale)
    # the monitor sums are the FP64 sums of the stored state (FP32: Kahan-compensated
    # float partial sums, far below the state's own round-off)
    np.testing.assert_allclose(mon["sum"], got[:4].reshape(4, -1).sum(axis=1),
                               rtol=1e-12 if prec == V.FP64 else 1e-9, atol=1e-9)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec", [V.FP64, V.FP32])
def test_save_load_resume_is_bitwise(prec, kernel):
    p = W.quadrant_riemann(64, 48, seed=2)
    full, _, s = gpu_run(p, V.LIM_LMP, prec, nsteps=0, return_solver=True, kernel=kernel)
    s.step(7)
    ck = s.save()
    s.step(9)
    a = s.state_planes().cpu().numpy().copy()
    s.step(5)
    s.load(ck)
    s.step(9)
    b = s.state_planes().cpu().numpy()
    assert np.array_equal(a, b)
    assert s.time()[1] == 16
    s.close()


def test_step_to_lands_on_final_time():
    """The last step is shortened to land on t_end. t_end is put half-way through a
    step: when the remainder is tiny, a = dx / (t_end - t) is huge and amplifies the
    last bit of t, so only n and t are comparable then."""
    p = W.quadrant_riemann(64, 64, seed=3)
    r20 = oracle_run(p, V.LIM_LMP, nsteps=20)
    t_end = r20["t"] + 0.5 * p.dx / r20["a"][-1]
    got, mon = gpu_run(p, V.LIM_LMP, V.FP64, t_end=t_end)
    ref = oracle_run(p, V.LIM_LMP, t_end=t_end)
    assert mon["done"] == 1 and mon["n"] == ref["n"]
    assert mon["t"] == ref["t"] and abs(mon["t"] - t_end) <= 1e-15
    assert plane_rel_err(got, ref["state"]) <= 1e-12
    # a tiny remainder: the same number of steps and the same final time
    t_end2 = r20["t"] + 1e-9 * p.dx / r20["a"][-1]
    got2, mon2 = gpu_run(p, V.LIM_LMP, V.FP64, t_end=t_end2)
    ref2 = oracle_run(p, V.LIM_LMP, t_end=t_end2)
    assert mon2["n"] == ref2["n"] and abs(mon2["t"] - t_end2) <= 1e-15


def test_inadmissible_initial_state_is_rejected():
    p = W.quadrant_riemann(32, 32, seed=1)
    p.E[5, 5] = 0.0   # zero internal energy
    with pytest.raises(V.VLBMError) as e:
        gpu_run(p, V.LIM_PP, V.FP64, nsteps=1)
    assert e.value.code == V.E_INVAL


@pytest.mark.parametrize("lim,tol", [(V.LIM_PP, 1e-5), (V.LIM_LMP, 1e-3)])
def test_fused_equals_simple_fp32(lim, tol):
    """The two FP32 kernels evaluate the same formulas in a different order. With PP
    they agree to FP32 round-off; LMP takes different branches at ties (dF^rho at
    round-off level), so it is held to the discontinuous tolerance."""
    p = W.quadrant_riemann(300, 130, seed=9)
    a, _ = gpu_run(p, lim, V.FP32, nsteps=50, kernel=V.KERNEL_SIMPLE)
    b, _ = gpu_run(p, lim, V.FP32, nsteps=50, kernel=V.KERNEL_FUSED)
    assert l1_rel(b[:4], a[:4]) <= tol


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec", [V.FP64, V.FP32])
def test_graph_replay_equals_single_launches(kernel, prec):
    """vlbm_step replays whole groups of 64 steps from a CUDA graph; with kernel
    timing on it launches every step alone. Both give the same state bit for bit."""
    import torch

    p = W.quadrant_riemann(70, 45, seed=3, bc=(2, 1, 0, 0))
    out = []
    for timed in (False, True):
        s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, limiter=V.LIM_LMP, precision=prec, kernel=kernel,
                   device="cuda:0")
        dt = torch.float64 if prec == V.FP64 else torch.float32
        c = torch.tensor(p.conserved(), dtype=dt, device="cuda:0")
        s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
        s.profile(timed)
        s.step(200)          # 3 graph replays + 8 single launches when not timed
        s.step(64)
        out.append((s.state_planes().cpu().numpy(), s.monitors()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1]["n"] == out[1][1]["n"] == 264 and out[0][1]["t"] == out[1][1]["t"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec,rtol", [(V.FP64, 1e-13), (V.FP32, 1e-5)])
def test_monitor_min_density_and_internal_energy(kernel, prec, rtol):
    """min rho and min (E - |m|^2 / (2 rho)) of the current state against the oracle's."""
    p = W.quadrant_riemann(70, 45, seed=5, bc=(1, 1, 2, 2))
    got, mon = gpu_run(p, V.LIM_PP, prec, nsteps=25, kernel=kernel)
    ref = oracle_run(p, V.LIM_PP, nsteps=25)["state"]
    rhoe = ref[3] - 0.5 * (ref[1] ** 2 + ref[2] ** 2) / ref[0]
    assert abs(mon["min_rho"] - ref[0].min()) <= rtol * ref[0].min()
    assert abs(mon["min_internal_energy"] - rhoe.min()) <= 10 * rtol * rhoe.min()


def test_async_monitors_match_synchronous_ones():
    """vlbm_monitors_async / vlbm_monitors_decode: each step's record, copied while the
    next step is already enqueued, equals what vlbm_monitors reports after that step."""
    p = W.quadrant_riemann(96, 64, seed=3)
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, limiter=V.LIM_PP, precision=V.FP32, device="cuda:0")
    c = torch.tensor(p.conserved(), dtype=torch.float32, device="cuda:0")
    s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    bufs = [s.monitor_buffer() for _ in range(3)]
    evs = [torch.cuda.Event() for _ in range(3)]
    for k in range(3):
        s.step(1)
        s.monitors_async(bufs[k])
        evs[k].record(s.stream)
    sync = s.monitors()   # after the third step
    seen = []
    for k in range(3):
        evs[k].synchronize()
        seen.append(s.decode_monitors(bufs[k]))
    assert [m["n"] for m in seen] == [1, 2, 3]
    assert seen[2] == sync
    assert seen[0]["t"] < seen[1]["t"] < seen[2]["t"]
    s.close()
