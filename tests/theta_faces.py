"""Faces for the FP32 theta_p certificate and an exact check of it (no GPU here).

theta_p of Sec. 3.4 (eq. GQL) is max(0, kappa / varrho - eps), varrho the spectral
radius of the face. theta <= theta_p holds exactly when the segment u* + s dF,
|s| <= (theta + eps) / kappa, lies in the closure of G (the density root r1 and the
internal-energy quadratic r2 are the two ends of that segment's admissible part),
and G is convex with u* inside it, so it suffices that both endpoints
u* +- (theta + eps) / kappa dF have rho >= 0 and 2 rho E - |m|^2 >= 0. That test
needs no square root: it is decided here in double precision where an error bound
proves its sign, else in exact rational arithmetic (fractions.Fraction). The same
test at a slightly larger theta tells whether a computed theta is also close to
theta_p from below.

Inputs are float32 face records (u*[4], dF[4], theta_rho), as the kernels store them.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

U64 = 2.0 ** -53


def _fr(x):
    return Fraction(float(x))


def endpoints_in_closed_G(us, df, s):
    """For faces (n, 4) us, df and half-lengths s (n,) as float64: True where both
    u* +- s dF have rho >= 0 and 2 rho E - |m|^2 >= 0, decided exactly. s must be
    exactly representable (float64); us, df exact float64 values."""
    us = np.asarray(us, dtype=np.float64)
    df = np.asarray(df, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    n = us.shape[0]
    out = np.ones(n, dtype=bool)
    undecided = np.zeros(n, dtype=bool)
    for sign in (1.0, -1.0):
        sd = sign * s[:, None] * df                       # products rounded
        end = us + sd
        mag = np.abs(us) + np.abs(sd)
        err = 4.0 * U64 * mag                             # |end - exact| bound per component
        r, a, b, e = end.T
        er, ea, eb, ee = err.T
        q = 2.0 * r * e - (a * a + b * b)
        # bound of |q - exact q|: propagation of the component errors and the rounding of q
        qerr = (2.0 * (np.abs(r) * ee + np.abs(e) * er + er * ee) + 2.0 * (np.abs(a) * ea + np.abs(b) * eb)
                + ea * ea + eb * eb) + 8.0 * U64 * (2.0 * np.abs(r * e) + a * a + b * b)
        sure_in = (r - er >= 0.0) & (q - qerr >= 0.0)
        sure_out = (r + er < 0.0) | (q + qerr < 0.0)     # rho < 0, or q < 0 whatever the sign of rho
        out &= ~sure_out
        undecided |= ~(sure_in | sure_out)
    for i in np.nonzero(undecided & out)[0]:
        out[i] = _exact_in_closed_G(us[i], df[i], s[i])
    return out


def _exact_in_closed_G(us, df, s):
    S = _fr(s)
    for sign in (1, -1):
        r, a, b, e = (_fr(us[k]) + sign * S * _fr(df[k]) for k in range(4))
        if r < 0 or 2 * r * e - a * a - b * b < 0:
            return False
    return True


def half_length(theta, eps, kappa, up=True):
    """(theta + eps) / kappa as float64, rounded up (up=True) or down by a margin
    that covers the rounding of the two operations."""
    s = (np.asarray(theta, dtype=np.float64) + eps) / kappa
    return s * (1.0 + 4 * U64) if up else s * (1.0 - 4 * U64)


def check_certificate(faces, theta, stage, kappa, eps, tol, model=None):
    """Per-face checks of a theta computed for float32 `faces` (n, 9):
    - 0 <= theta <= min(1, theta_rho) (theta = 0 where min(1, theta_rho) <= 0);
    - soundness: theta > 0 => theta <= theta_p exactly (endpoints in the closure of G);
    - tightness: theta = min(1, theta_rho), or theta_p < theta / (1 - tol[stage]) + 3 eps
      (endpoints at that larger theta leave G); for faces of stage 3, when `model` (the
      bound that stage documents, per face) is given: theta >= model (1 - tol[3]) - eps.
    Returns a dict of index arrays of the faces that fail each check."""
    f = np.asarray(faces, dtype=np.float32).astype(np.float64)
    th = np.asarray(theta, dtype=np.float32).astype(np.float64)
    stage = np.asarray(stage)
    us, df, tr = f[:, 0:4], f[:, 4:8], f[:, 8]
    t = np.minimum(1.0, tr)
    bad_range = np.nonzero(~((th >= 0.0) & (th <= np.maximum(t, 0.0))))[0]
    pos = np.nonzero(th > 0.0)[0]
    ok = endpoints_in_closed_G(us[pos], df[pos], half_length(th[pos], eps, kappa, up=True))
    bad_sound = pos[~ok]
    below = np.nonzero(th < t)[0]
    if model is not None:
        s3 = below[stage[below] == 3]
        bad_model = s3[th[s3] < np.minimum(model[s3], t[s3]) * (1.0 - tol[3]) - eps]
        below = below[stage[below] != 3]
    else:
        bad_model = np.zeros(0, dtype=np.int64)
    tl = np.asarray([tol[int(k)] for k in stage[below]]) if below.size else np.zeros(0)
    th_hi = th[below] / (1.0 - tl) + 3.0 * eps
    still_in = endpoints_in_closed_G(us[below], df[below], half_length(th_hi, eps, kappa, up=False))
    bad_tight = np.concatenate([below[still_in & (th_hi < t[below])], bad_model])
    return {"range": bad_range, "sound": bad_sound, "tight": bad_tight}


def _sum_dd(*terms):
    """Sum of exact double terms, accurate to ~2^-104 of their magnitudes (TwoSum cascade)."""
    s, c = terms[0], np.zeros_like(terms[0])
    for t in terms[1:]:
        s, e = _two_sum(s, t)
        c = c + e
    return s + c


def fp64_stage_model(faces, kappa, eps):
    """The lower bound of theta_p that the FP32 kernels' double-precision stage documents
    (Sec. 3.4, eq. GQL), per face: gamma_0 = m1^2 + m2^2 - 2 rho E, gamma_1 / 2 and the
    quadratic's coefficient c, each a chain of fused multiply-adds whose rounding error is
    at most e = 2^-52 times the sum of the chain's partial results. The stage widens its
    computed value by e; its computed value may itself sit e from the exact one, so in
    terms of the exact values: D = -2 gamma_0 >= D_lo = -2 (gamma_0 + 2 e0), |gamma_1| <= G_hi
    = 2 (|gamma_1 / 2| + 2 e1), c <= c_hi = c + 2 ec; Delta <= G_hi^2 + 2 max(D c);
    theta >= kappa min(rho / |drho|, D_lo / (G_hi + sqrt(Delta_hi))) - 2 eps. Evaluated here
    with the chains summed accurately; 0 where D_lo <= 0."""
    f = np.asarray(faces, dtype=np.float32).astype(np.float64)
    rs, m1, m2, E, dr, dm1, dm2, dE = f[:, :8].T
    g0i = _sum_dd(m2 * m2, -2.0 * rs * E)
    g0 = _sum_dd(m1 * m1, m2 * m2, -2.0 * rs * E)
    e0 = (np.abs(g0i) + np.abs(g0)) * 2.0 ** -52
    D_lo, D_hi = -2.0 * (g0 + 2.0 * e0), -2.0 * (g0 - 2.0 * e0)
    h1 = _sum_dd(dm1 * m1, dm2 * m2)
    h2 = _sum_dd(dE * rs, -(dm1 * m1), -(dm2 * m2))
    h3 = _sum_dd(dr * E, dE * rs, -(dm1 * m1), -(dm2 * m2))
    G_hi = 2.0 * (np.abs(h3) + 2.0 * (np.abs(h1) + np.abs(h2) + np.abs(h3)) * 2.0 ** -52)
    ci = _sum_dd(dm2 * dm2, -2.0 * dr * dE)
    cq = _sum_dd(dm1 * dm1, dm2 * dm2, -2.0 * dr * dE)
    c_hi = cq + 2.0 * (np.abs(ci) + np.abs(cq)) * 2.0 ** -52
    Dc_hi = np.where(c_hi >= 0.0, D_hi * c_hi, D_lo * c_hi)
    N_hi = G_hi + np.sqrt(np.maximum(G_hi * G_hi + 2.0 * Dc_hi, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(np.abs(dr) > 0, rs / np.abs(dr), np.inf)
        inv = np.where(N_hi > 0, np.minimum(inv, D_lo / N_hi), inv)
    th = kappa * inv - 2.0 * eps
    th = np.where(np.isinf(inv), 1.0, th)
    return np.where((D_lo > 0.0) & (rs > 0.0), np.maximum(th, 0.0), 0.0)


# ---------------------------------------------------------------- face generators

def _records(us, df, theta_rho):
    out = np.empty((us.shape[0], 9), dtype=np.float32)
    out[:, 0:4] = us
    out[:, 4:8] = df
    out[:, 8] = theta_rho
    return out


def _theta_rho(rng, n):
    """1 (PP in FP32: theta_p carries the density bound) for most faces, a value in
    (0, 1) or a non-positive one (LMP-like) for the rest."""
    tr = np.ones(n)
    k = rng.random(n)
    tr[k < 0.25] = rng.random(int((k < 0.25).sum()))
    tr[k < 0.03] = -rng.random(int((k < 0.03).sum()))
    tr[k < 0.01] = 0.0
    return tr


def random_faces(rng, n, kappa=1.0, near_vacuum=False):
    """Admissible u* (density 1e-6..1e2, speeds up to 5, internal energy a fraction
    1e-3..1 of E, or 1e-12..1e-4 near the vacuum) and dF of every size from 1e-3 to
    1e3 times kappa u*, with independent signs (mixed-sign components)."""
    rho = 10.0 ** rng.uniform(-6, 2, n)
    speed = rng.uniform(0.1 if near_vacuum else 0.0, 5.0, n)
    ang = rng.uniform(0, 2 * np.pi, n)
    v1, v2 = speed * np.cos(ang), speed * np.sin(ang)
    ratio = 10.0 ** (rng.uniform(-12, -4, n) if near_vacuum else rng.uniform(-3, 0, n))
    ke = 0.5 * rho * (v1 * v1 + v2 * v2)
    E = np.where(ke > 0, ke / (1.0 - ratio), rho)
    us = np.stack([rho, rho * v1, rho * v2, E], axis=1).astype(np.float32)
    scale = kappa * 10.0 ** rng.uniform(-3, 3, n)
    comp = rng.uniform(-1, 1, (n, 4)) * np.abs(us.astype(np.float64)).max(axis=1, keepdims=True)
    comp[:, 0] = rng.uniform(-1, 1, n) * us[:, 0]
    comp[:, 3] = rng.uniform(-1, 1, n) * us[:, 3]
    zero = rng.random((n, 4)) < 0.05                      # some components exactly 0
    comp[zero] = 0.0
    df = (scale[:, None] * comp).astype(np.float32)
    return _records(us, df, _theta_rho(rng, n))


def cancelling_faces(rng, n, kappa=1.0):
    """u* whose gamma_0 = m1^2 + m2^2 - 2 rho* E* nearly cancels in float: E* is the
    float nearest to |m|^2 / (2 rho*) (1 + ratio), ratio down to 1e-9, with one
    velocity component much smaller than the other (the products then differ in
    exponent and their sum does not fit a double). Faces whose rounded E* falls
    outside G are kept: theta must then be 0."""
    rho = (10.0 ** rng.uniform(-3, 1, n)).astype(np.float32)
    big = rng.uniform(0.5, 5.0, n) * np.where(rng.random(n) < 0.5, -1, 1)
    small = big * 10.0 ** rng.uniform(-6, -1, n) * np.where(rng.random(n) < 0.5, -1, 1)
    swap = rng.random(n) < 0.5
    v1, v2 = np.where(swap, small, big), np.where(swap, big, small)
    m1 = (rho * v1).astype(np.float32)
    m2 = (rho * v2).astype(np.float32)
    r64 = rho.astype(np.float64)
    ke = (m1.astype(np.float64) ** 2 + m2.astype(np.float64) ** 2) / (2 * r64)
    E = (ke * (1.0 + 10.0 ** rng.uniform(-9, -5, n))).astype(np.float32)
    us = np.stack([rho, m1, m2, E], axis=1)
    scale = kappa * 10.0 ** rng.uniform(-9, 0, n)
    comp = rng.uniform(-1, 1, (n, 4)) * np.abs(us.astype(np.float64))
    df = (scale[:, None] * comp).astype(np.float32)
    return _records(us, df, _theta_rho(rng, n))


def large_jump_faces(rng, n, kappa=1.0):
    """|dF| far above kappa rho* (1e3..1e8 times): theta_p close to 0."""
    f = random_faces(rng, n, kappa)
    f[:, 4:8] *= (10.0 ** rng.uniform(3, 8, n)).astype(np.float32)[:, None]
    return f


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def gamma0_ratio(us):
    """-gamma_0 / (2 rho* E*) of float32 u*, gamma_0 = m1^2 + m2^2 - 2 rho* E* summed
    without error (every product of two floats is exact in double; two TwoSums)."""
    u = np.asarray(us, dtype=np.float32).astype(np.float64)
    t1, t2, t3 = u[:, 1] * u[:, 1], u[:, 2] * u[:, 2], -2.0 * u[:, 0] * u[:, 3]
    s1, e1 = _two_sum(t1, t2)
    s2, e2 = _two_sum(s1, t3)
    g0 = s2 + (e1 + e2)
    return -g0 / (2.0 * u[:, 0] * u[:, 3])


def boundary_faces(rng, n, kappa=1.0, pool=4_000_000):
    """u* inside G but as close to its boundary as float data allows: E* is the
    smallest float above |m|^2 / (2 rho*), and of a large pool the n states with the
    smallest -gamma_0 / (2 rho* E*) are kept (down to ~1e-14, where gamma_0 has
    cancelled to a few units of the last of its 48 product bits). dF is scaled so
    that theta_p stays of order one."""
    rho = (10.0 ** rng.uniform(-2, 1, pool)).astype(np.float32)
    v1 = rng.uniform(-5, 5, pool)
    v2 = v1 * 10.0 ** rng.uniform(-8, 0, pool) * np.where(rng.random(pool) < 0.5, -1, 1)
    m1 = (rho * v1).astype(np.float32)
    m2 = (rho * v2).astype(np.float32)
    r64 = rho.astype(np.float64)
    ke = (m1.astype(np.float64) ** 2 + m2.astype(np.float64) ** 2) / (2 * r64)
    E = ke.astype(np.float32)
    us = np.stack([rho, m1, m2, E], axis=1)
    ratio = gamma0_ratio(us)
    E = np.where(ratio > 0, E, np.nextafter(E, np.float32(np.inf)))
    us[:, 3] = E
    ratio = gamma0_ratio(us)
    keep = np.argsort(np.where(ratio > 0, ratio, np.inf))[:n]
    us = us[keep]
    ratio = ratio[keep]
    scale = kappa * ratio * 10.0 ** rng.uniform(-1, 2, n)
    comp = rng.uniform(-1, 1, (n, 4)) * np.abs(us.astype(np.float64))
    df = (scale[:, None] * comp).astype(np.float32)
    return _records(us, df, _theta_rho(rng, n))
