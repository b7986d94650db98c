"""The FP32 theta of the step kernels, face by face, on the GPU (Sec. 3.2-3.4).

The FP32 kernels settle theta = min(1, theta_rho, theta_p) of each face in up to
three stages -- a float endpoint screen, a float interval of the spectral radius,
a double-precision interval -- and every stage must return a theta that never
exceeds the exact theta_p of the stored float face state (so the decomposition
states stay in G: the positivity of Sec. 3.4) and sits close below it. Here
vlbm_test_theta_faces runs the kernels' own function on about a million
adversarial faces plus the faces of a near-vacuum blast computed by the oracle,
and each result is checked exactly (tests/theta_faces.py: endpoints of the segment
u* +- (theta + eps) / kappa dF in the closure of G, in exact rational arithmetic
where double precision cannot decide), and against the oracle's theta_p where its
plain double evaluation is accurate.
"""
import numpy as np
import pytest

import theta_faces as TF
from oracle import oracle as O
from paper_2411_15001_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# how far below theta_p each stage may sit (relative): the screen returns min(1,
# theta_rho) itself; the float interval is tight to 2^-14 (+ 16 u for the
# reciprocals); the double-precision stage is held to the bound it documents
# (tests/theta_faces.py: fp64_stage_model -- tight to a few float roundings unless
# gamma_0, gamma_1 or c cancel, where its error bound grows with the cancellation)
# within the float roundings of its last steps
TOL = {0: 0.0, 1: 0.0, 2: 6.5e-5, 3: 4e-6}


def gpu_theta(F, a, eps, alpha=0.5):
    import torch

    from paper_2411_15001_gb300 import vlbm as V

    d = torch.from_numpy(np.ascontiguousarray(F, dtype=np.float32)).to("cuda:0")
    th = torch.empty(len(F), dtype=torch.float32, device="cuda:0")
    st = torch.empty(len(F), dtype=torch.int32, device="cuda:0")
    stream = torch.cuda.current_stream("cuda:0")
    rc = V.vlbm_test_theta_faces(len(F), a, alpha, eps, d.data_ptr(), th.data_ptr(), st.data_ptr(),
                                 stream.cuda_stream)
    assert rc == V.OK, V.vlbm_last_error_detail()
    stream.synchronize()
    return th.cpu().numpy(), st.cpu().numpy()


def blast_faces(n=256, steps=240, eps=1e-13):
    """Face states of the oracle's near-vacuum blast (PP) after `steps` steps: u* and
    dF of every x- and y-face, rounded to float as the FP32 kernels hold them, and
    the kinetic speed of the next step."""
    p = W.blast(n)
    cfg = O.Config(n, n, p.bc, O.LIM_PP, p.gamma, 0.5, eps)
    r = O.run(cfg, p.conserved(), p.dx, nsteps=steps)
    a = O.kinetic_speed(O.max_speed(cfg, r["state"]), 0.5)
    _, dbg = O.step(cfg, r["state"], a, debug=True)
    us = np.concatenate([dbg["ustar_x"].reshape(-1, 4), dbg["ustar_y"].reshape(-1, 4)])
    df = np.concatenate([dbg["dflux_x"].reshape(-1, 4), dbg["dflux_y"].reshape(-1, 4)])
    keep = np.any(df != 0.0, axis=1)          # the quiet gas outside the ring has dF = 0
    F = np.empty((int(keep.sum()), 9), dtype=np.float32)
    F[:, 0:4] = us[keep]
    F[:, 4:8] = df[keep]
    F[:, 8] = 1.0
    return F, a


def _check(F, a, eps, label):
    kappa = a / 4.0
    th, st = gpu_theta(F, a, eps)
    res = TF.check_certificate(F, th, st, kappa, eps, TOL, model=TF.fp64_stage_model(F, kappa, eps))
    hist = {k: int((st == k).sum()) for k in range(4)}
    print(f"{label}: {len(F)} faces, stages none/screen/interval/fp64 = "
          f"{hist[0]}/{hist[1]}/{hist[2]}/{hist[3]}, min theta {th.min():.3g}")
    for what, idx in res.items():
        assert idx.size == 0, (label, what, idx.size, F[idx[:3]], th[idx[:3]], st[idx[:3]])
    s3 = np.nonzero((st == 3) & (th < np.minimum(1.0, F[:, 8])))[0]
    if s3.size:   # how far below theta_p the double-precision stage sat (for the record)
        tp = np.array([O.theta_p(kappa, eps, F[i, :4].astype(np.float64), F[i, 4:8].astype(np.float64))
                       for i in s3[:2000]])
        ok = tp > 1e-6
        gap = (1.0 - th[s3[:2000]][ok] / tp[ok]) if ok.any() else np.zeros(1)
        print(f"   stage 3 below theta_p (oracle, first 2000): median {np.median(gap):.2e}, max {gap.max():.2e}")
    # the oracle's theta_p where its plain double evaluation is accurate
    good = np.nonzero(TF.gamma0_ratio(F[:, :4]) > 1e-7)[0]
    f = F[good].astype(np.float64)
    tp = np.array([O.theta_p(kappa, eps, f[i, :4], f[i, 4:8]) for i in range(len(f))])
    ref = np.maximum(np.minimum(np.minimum(1.0, f[:, 8]), tp), 0.0)
    g = th[good].astype(np.float64)
    tol = np.array([TOL[int(k)] for k in st[good]])
    low = np.where(st[good] == 3, np.minimum(ref, TF.fp64_stage_model(F[good], kappa, eps)), ref)
    over = np.nonzero(g > ref * (1.0 + 1e-9))[0]
    under = np.nonzero(g < low * (1.0 - tol) - 3.0 * eps)[0]
    assert over.size == 0, (label, "above the oracle", F[good][over[:3]], g[over[:3]], ref[over[:3]])
    assert under.size == 0, (label, "below the oracle", F[good][under[:3]], g[under[:3]], ref[under[:3]])
    return hist


def test_theta_p_certificate_face_by_face():
    rng = np.random.default_rng(2024)
    a, eps = 8.0, 1e-13           # kappa = 2
    sets = [
        ("random", TF.random_faces(rng, 400_000, 2.0)),
        ("near vacuum", TF.random_faces(rng, 200_000, 2.0, near_vacuum=True)),
        ("cancelling gamma_0", TF.cancelling_faces(rng, 200_000, 2.0)),
        ("large jumps", TF.large_jump_faces(rng, 100_000, 2.0)),
        ("boundary of G", TF.boundary_faces(rng, 20_000, 2.0, pool=4_000_000)),
    ]
    total = {k: 0 for k in range(4)}
    for label, F in sets:
        for k, v in _check(F, a, eps, label).items():
            total[k] += v
    F, ab = blast_faces()
    for k, v in _check(F, ab, 1e-13, "blast 256^2 (oracle), step 240").items():
        total[k] += v
    print("all faces:", total)
    assert sum(total.values()) >= 1_000_000
    assert all(total[k] > 100 for k in range(4)), total     # every stage exercised
