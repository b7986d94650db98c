"""Exact density of the near-vacuum isentropic wave of Sec. 4.4 (gamma = 3), by
characteristics: a test reference for the oracle's 1D validation runs
(workloads.near_vacuum_wave defines the initial data)."""
import numpy as np


def near_vacuum_wave_exact(x, t: float, amp: float = 0.9999995):
    """Exact density of the wave above for t before the first shock (t < ~0.18): with
    gamma = 3 the Riemann invariants w = v +- sqrt(3) rho are constant along
    dx/dt = w, so w(x, t) = w0(x - w t), solved by Newton's method."""
    s3 = np.sqrt(3.0)
    x = np.asarray(x, dtype=np.float64)

    def solve(sign):
        w0 = lambda y: sign * s3 * (1.0 + amp * np.sin(np.pi * y))
        dw0 = lambda y: sign * s3 * amp * np.pi * np.cos(np.pi * y)
        w = w0(x)
        for _ in range(100):
            r = w - w0(x - w * t)
            w = w - r / (1.0 + t * dw0(x - w * t))
        return w

    return (solve(1.0) - solve(-1.0)) / (2.0 * s3)
