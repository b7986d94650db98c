"""Batched solver (vlbm_batch_*) against single-grid solves and the oracle (needs a GB300).

The batch runs the same row-marching kernel over the work items of all grids, so
every grid must evolve exactly as it does alone: bit for bit in both precisions.
"""
import numpy as np
import pytest

from paper_2411_15001_gb300 import workloads as W
from tests.gpu_helpers import gpu_run, oracle_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_15001_gb300 import vlbm as V  # noqa: E402

DEV = torch.device("cuda:0")


def _problems():
    return [W.quadrant_riemann(70, 45, seed=11),
            W.quadrant_riemann(130, 64, seed=12, bc=(2, 1, 0, 0)),
            W.quadrant_riemann(64, 200, seed=13, bc=(0, 0, 2, 2)),
            W.quadrant_riemann(37, 29, seed=14),
            W.quadrant_riemann(251, 19, seed=15, bc=(1, 2, 2, 1))]


def _batch(probs, lim, prec):
    dt = torch.float64 if prec == V.FP64 else torch.float32
    b = V.VLBMBatch([(p.nx, p.ny, p.dx, p.bc) for p in probs], limiter=lim, precision=prec, device=DEV)
    for i, p in enumerate(probs):
        c = torch.tensor(p.conserved(), dtype=dt, device=DEV)
        b.set_conserved(i, c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    return b


@pytest.mark.parametrize("prec", [V.FP64, V.FP32])
@pytest.mark.parametrize("lim", [V.LIM_PP, V.LIM_LMP])
def test_batch_equals_single_grids(prec, lim):
    probs = _problems()
    b = _batch(probs, lim, prec)
    b.step(70)   # one graph replay of 64 steps plus single launches
    for i, p in enumerate(probs):
        got = b.state_planes(i).cpu().numpy()
        ref, mon = gpu_run(p, lim, prec, nsteps=70, kernel=V.KERNEL_FUSED)
        assert np.array_equal(got, ref.astype(got.dtype)), i
        bm = b.monitors(i)
        assert bm["n"] == 70 and bm["t"] == mon["t"] and bm["status"] == 0
    b.close()


def test_batch_fp64_matches_oracle():
    probs = _problems()[:3]
    b = _batch(probs, V.LIM_LMP, V.FP64)
    b.step(9)
    for i, p in enumerate(probs):
        ref = oracle_run(p, V.LIM_LMP, nsteps=9)
        assert np.array_equal(b.state_planes(i).cpu().numpy(), ref["state"])
    b.close()


def test_autotune_keeps_results_exact():
    """Tuning steps are real steps and the decomposition does not change arithmetic."""
    probs = _problems()
    b = _batch(probs, V.LIM_PP, V.FP32)
    best = b.autotune(trial_steps=2)
    n = b.monitors(0)["n"]
    assert n > 0 and best["ms_per_step"] > 0 and best["items"] > 0
    for chunk, cps, order in ((16, 1, V.ORDER_LPT), (64, 3, V.ORDER_INDEX), (128, 3, V.ORDER_GUIDED),
                              (16, 2, V.ORDER_GUIDED), (256, 3, V.ORDER_GUIDED), (4, 3, V.ORDER_LPT),
                              (1024, 2, V.ORDER_INDEX)):
        b.set_tuning(chunk, cps, order)
        assert b.tuning()["order"] == order
        b.step(3)
        n += 3
    for i, p in enumerate(probs):
        ref, _ = gpu_run(p, V.LIM_PP, V.FP32, nsteps=n, kernel=V.KERNEL_FUSED)
        assert np.array_equal(b.state_planes(i).cpu().numpy(), ref.astype(np.float32)), i
    b.close()
