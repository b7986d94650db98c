"""Writes quadrant1024_lmp_jitter.txt: how far float-level noise alone moves the
1024^2 LMP quadrant problem at t = 0.25 (workloads.quadrant_riemann(1024, seed=0),
zero-gradient sides, dynamic a^n, last step shortened to land on t).

Runs the FP64 oracle twice: clean, and with every value of the state multiplied by
(1 + d), d uniform in [-2^-24, 2^-24] (float's unit roundoff, seeded), after every
step. The L1 distance of the two final densities, relative to the clean one, is the
spread that any float-precision run of this configuration can be held to: LMP's
theta^rho jumps where dF^rho changes sign (Sec. 3.3.1), so rounding-level changes
grow. Calls only the oracle.

    python tests/golden/make_quadrant_jitter.py [n]        (n = 1024; ~5 min on 8 cores)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2411_15001_gb300 import workloads as W  # noqa: E402


def main(n=1024, t_end=0.25, seed=7):
    p = W.quadrant_riemann(n, seed=0)
    cfg = O.Config(n, n, p.bc, O.LIM_LMP, p.gamma)
    O.set_threads(os.cpu_count() or 1)
    clean = O.run(cfg, p.conserved(), p.dx, t_end=t_end)
    rng = np.random.default_rng(seed)

    def jitter(k, state):
        state *= 1.0 + rng.uniform(-2.0 ** -24, 2.0 ** -24, state.shape)

    noisy = O.run(cfg, p.conserved(), p.dx, t_end=t_end, callback=jitter)
    r0, r1 = clean["state"][0], noisy["state"][0]
    spread = float(np.abs(r1 - r0).sum() / np.abs(r0).sum())
    out = os.path.join(HERE, f"quadrant{n}_lmp_jitter.txt")
    with open(out, "w") as f:
        f.write(f"# written by: python tests/golden/make_quadrant_jitter.py {n}\n")
        f.write("# L1(rho) of the jittered FP64 oracle run relative to the clean one at t = 0.25;\n")
        f.write("# steps of the clean and the jittered runs\n")
        f.write(f"spread {spread:.6e}\n")
        f.write(f"steps_clean {clean['n']}\n")
        f.write(f"steps_jittered {noisy['n']}\n")
    print(open(out).read())


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1024)
