"""Helpers for the GPU tests: run one problem through the C-ABI and through the oracle."""
import numpy as np

from oracle import oracle as O

LIM_NAMES = {0: "first", 1: "none", 2: "PP", 3: "LMP", 4: "RLMP"}


def gpu_run(p, limiter, precision, nsteps=None, t_end=None, lam=0.0, eps=1e-16, kernel=0,
            return_solver=False, sponge=0):
    import torch

    from paper_2411_15001_gb300 import vlbm as V

    dt = torch.float64 if precision == V.FP64 else torch.float32
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, gamma=p.gamma, lam=lam, limiter=limiter,
               precision=precision, eps=eps, kernel=kernel, device="cuda:0", sponge=sponge)
    c = torch.tensor(p.conserved(), dtype=dt, device="cuda:0")
    s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    if nsteps is not None:
        s.step(nsteps)
    if t_end is not None:
        s.step_to(t_end, 10 ** 7)
    planes = s.state_planes().double().cpu().numpy()
    mon = s.monitors()
    if return_solver:
        return planes, mon, s
    s.close()
    return planes, mon


def oracle_cfg(p, limiter, eps=1e-16, sponge=0):
    """The oracle's configuration of a workload, boundary field and split sides included."""
    bf = getattr(p, "bfield", None)
    field = O.Field(bf.inside, bf.outside, bf.planes) if bf is not None else None
    return O.Config(p.nx, p.ny, p.bc, limiter, p.gamma, 0.5, eps, sponge,
                    bc_hi=getattr(p, "bc_hi", None), split=getattr(p, "split", (0, 0, 0, 0)),
                    x0=p.x0, y0=p.y0, dx=p.dx, field=field)


def oracle_run(p, limiter, nsteps=None, t_end=None, lam=0.0, eps=1e-16, sponge=0):
    cfg = oracle_cfg(p, limiter, eps, sponge)
    return O.run(cfg, p.conserved(), p.dx, nsteps=nsteps, t_end=t_end,
                 lam_fixed=lam if lam > 0 else None)


def plane_rel_err(got, ref):
    """max over planes of max|got - ref| / max|ref| (planes with max|ref| = 0 use 1)."""
    d = np.abs(got - ref).reshape(ref.shape[0], -1).max(axis=1)
    s = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return float((d / np.where(s > 0, s, 1.0)).max())


def l1_rel(got, ref):
    return float(np.abs(got - ref).sum() / np.abs(ref).sum())
