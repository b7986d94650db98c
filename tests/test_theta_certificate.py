"""The FP32 internal-energy bound (Sec. 3.4, eq. GQL) without a GPU.

1. The exact endpoint check of tests/theta_faces.py, pinned to the oracle's
   closed-form theta_p on well-conditioned faces: it accepts theta_p (1 - 1e-6),
   rejects theta_p (1 + 1e-5) and flags theta_p (1 - 1e-3) as too far below.
2. The float endpoint screen of the FP32 kernels, emulated operation by operation
   (correctly rounded float adds and multiplies, fused multiply-adds rounded once)
   on adversarial faces: whenever it passes for a target t = min(1, theta_rho), both
   endpoints u* +- T dF lie in G exactly and T >= (t + eps) / kappa exactly, so
   theta_p >= t -- the screen's proof, checked face by face.
"""
from fractions import Fraction

import numpy as np
import pytest

import theta_faces as TF
from oracle import oracle as O

F32 = np.float32
U = F32(5.9604645e-08)


def _faces(kind, rng, n, kappa):
    if kind == "random":
        return TF.random_faces(rng, n, kappa)
    if kind == "near_vacuum":
        return TF.random_faces(rng, n, kappa, near_vacuum=True)
    if kind == "cancelling":
        return TF.cancelling_faces(rng, n, kappa)
    if kind == "large_jump":
        return TF.large_jump_faces(rng, n, kappa)
    return TF.boundary_faces(rng, n, kappa, pool=400_000)


@pytest.mark.parametrize("kind", ["random", "near_vacuum", "cancelling", "large_jump"])
def test_exact_check_agrees_with_the_oracle(kind):
    rng = np.random.default_rng(11)
    kappa, eps = 2.0, 1e-13
    F = _faces(kind, rng, 3000, kappa)
    # the closed form in plain double is itself accurate to 1e-6 only where gamma_0 does
    # not cancel by more than 1e-7 of its terms (the kernels form it from exact sums)
    F = F[TF.gamma0_ratio(F[:, :4]) > 1e-7]
    f = F.astype(np.float64)
    tp = np.array([O.theta_p(kappa, eps, f[i, :4], f[i, 4:8]) for i in range(len(F))])
    t = np.minimum(1.0, f[:, 8])
    ref = np.maximum(np.minimum(t, tp), 0.0)
    active = np.nonzero((tp < t) & (tp > 1e-6))[0]
    assert active.size > 300
    tol = {k: 6.5e-5 for k in range(4)}
    st = np.full(len(F), 2)
    ok = TF.check_certificate(F, (ref * (1 - 1e-6)).astype(F32), st, kappa, eps, tol)
    assert ok["sound"].size == 0 and ok["tight"].size == 0 and ok["range"].size == 0
    hi = TF.check_certificate(F, (ref * (1 + 1e-5)).astype(F32), st, kappa, eps, tol)
    assert np.array_equal(np.intersect1d(hi["sound"], active), active)
    lo = TF.check_certificate(F, (ref * (1 - 1e-3)).astype(F32), st, kappa, eps, tol)
    assert np.array_equal(np.intersect1d(lo["tight"], active), active)


# ---------------------------------------------------------------- float emulation

def _round_f32(s, e):
    """float32 nearest to the exact value s + e (s a double, |e| <= ulp(s) / 2),
    ties to even: a second rounding of s alone could differ at a float midpoint."""
    r = s.astype(F32)
    r64 = r.astype(np.float64)
    lo = np.where(r64 > s, np.nextafter(r, F32(-np.inf)), r)
    hi = np.nextafter(lo, F32(np.inf))
    mid = (lo.astype(np.float64) + hi.astype(np.float64)) / 2.0   # exact
    d = (s - mid) + e
    even = (lo.view(np.int32) & 1) == 0
    return np.where(d > 0, hi, np.where(d < 0, lo, np.where(even, lo, hi)))


def fma32(a, b, c):
    """Fused multiply-add of float32 arrays, rounded once: a b is exact in double,
    the sum's rounding error is kept by TwoSum and decides the float rounding."""
    p = a.astype(np.float64) * b.astype(np.float64)
    c = c.astype(np.float64)
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    return _round_f32(s, e)


def mul32(a, b):
    return (a.astype(np.float64) * b.astype(np.float64)).astype(F32)   # exact product, one rounding


def screen_T(th, eps, kappa):
    """The kernels' T for target th: the per-step constant T1 (an upper bound of (1 + 2 eps)
    / kappa (1 + 64 u)) at th >= 1, else ((th + 2 eps) / kappa) (1 + 64 u) in float."""
    T1 = (1.0 + 2.0 * eps) / kappa * (1.0 + 64.0 * 2.0 ** -24)
    T1f = F32(T1)
    if float(T1f) < T1:
        T1f = np.nextafter(T1f, F32(np.inf))
    em, ik = F32(2.0 * eps), F32(1.0 / kappa)
    T = ((th + em) * ik) * F32(1.0 + 64.0 * 2.0 ** -24)
    return np.where(th >= F32(1.0), T1f, T)


def screen(us, df, T):
    """The FP32 endpoint screen, operation by operation: True where both endpoints
    u* +- T dF are proved inside G."""
    tiny, huge, c2 = F32(2.0 ** -100), F32(2.0 ** 100), F32(2.0 - 2.0 ** -19)
    ok = np.ones(us.shape[0], dtype=bool)
    for sgn in (1, -1):
        t = (T * F32(sgn)).astype(F32)
        r = fma32(t, df[:, 0], us[:, 0])
        a = fma32(t, df[:, 1], us[:, 1])
        b = fma32(t, df[:, 2], us[:, 2])
        e = fma32(t, df[:, 3], us[:, 3])
        p = mul32(r, e)
        x = fma32(-b, b, fma32(np.full_like(p, c2), p, -mul32(a, a)))
        ok &= (r >= tiny) & (e >= tiny) & (p >= tiny) & (p <= huge) & (x > 0)
    return ok


def _strictly_in_G(us, df, T):
    S = Fraction(float(T))
    for sign in (1, -1):
        r, a, b, e = (Fraction(float(us[k])) + sign * S * Fraction(float(df[k])) for k in range(4))
        if not (r > 0 and 2 * r * e - a * a - b * b > 0):
            return False
    return True


@pytest.mark.parametrize("kind", ["random", "near_vacuum", "cancelling", "large_jump", "boundary"])
def test_float_screen_passes_only_proved_faces(kind):
    rng = np.random.default_rng(23)
    kappa, eps = 2.0, 1e-13
    F = _faces(kind, rng, 4000, kappa)
    us, df, tr = F[:, 0:4], F[:, 4:8], F[:, 8]
    th = np.minimum(F32(1.0), tr)
    pos = th > 0
    T = screen_T(th, eps, kappa)
    passed = np.nonzero(screen(us, df, T) & pos)[0]
    failed = np.nonzero(~screen(us, df, T) & pos)[0]
    # near the vacuum and for large jumps theta_p is mostly below t: few faces pass
    assert passed.size >= {"random": 500, "cancelling": 200}.get(kind, 0)
    # T >= (t + eps) / kappa exactly
    for i in passed:
        assert Fraction(float(T[i])) >= (Fraction(float(th[i])) + Fraction(eps)) / Fraction(kappa)
    # both endpoints in G: double with an error bound, exact where that cannot decide
    s = T[passed].astype(np.float64)
    inside = TF.endpoints_in_closed_G(us[passed].astype(np.float64), df[passed].astype(np.float64), s)
    assert inside.all(), passed[~inside][:10]
    for i in passed[:: max(1, passed.size // 200)]:       # strict membership, exactly, on a sample
        assert _strictly_in_G(us[i], df[i], T[i])
    # the screen is not vacuous: on the faces it leaves, theta_p is often below t
    if failed.size and kind != "boundary":
        f = F[failed].astype(np.float64)
        tp = np.array([O.theta_p(kappa, eps, f[i, :4], f[i, 4:8]) for i in range(len(f))])
        assert (tp < th[failed]).mean() > 0.5


@pytest.mark.parametrize("kind", ["random", "near_vacuum", "cancelling", "large_jump", "boundary"])
def test_double_stage_bound_is_sound_and_tight_where_conditioned(kind):
    """The bound the double-precision stage documents (theta_faces.fp64_stage_model) never
    exceeds theta_p (exact endpoint check), and on faces where gamma_0 cancels by at most
    1e-7 of its terms it is within the documented error, 2^-52 over that ratio (a few
    1e-9), of the oracle's theta_p."""
    rng = np.random.default_rng(31)
    kappa, eps = 2.0, 1e-13
    F = _faces(kind, rng, 3000, kappa)
    model = TF.fp64_stage_model(F, kappa, eps)
    t = np.minimum(1.0, F[:, 8].astype(np.float64))
    th = np.maximum(np.minimum(model, t), 0.0)
    pos = np.nonzero(th > 0)[0]
    ok = TF.endpoints_in_closed_G(F[pos, :4].astype(np.float64), F[pos, 4:8].astype(np.float64),
                                  TF.half_length(th[pos] * (1 - 1e-12), eps, kappa))
    assert ok.all(), pos[~ok][:5]
    ratio = TF.gamma0_ratio(F[:, :4])
    good = np.nonzero(ratio > 1e-7)[0]
    f = F[good].astype(np.float64)
    tp = np.array([O.theta_p(kappa, eps, f[i, :4], f[i, 4:8]) for i in range(len(f))])
    ref = np.maximum(np.minimum(t[good], tp), 0.0)
    rel = 1e-12 + 8 * 2.0 ** -52 / ratio[good]
    assert np.all(th[good] >= ref * (1 - rel) - 2 * eps), np.max((ref - th[good]) / np.maximum(ref, 1e-300))
