"""Write tests/golden/oracle_cells8_nb21.txt from the oracle alone.

The file is a regression fixture of the oracle: 8 cells x 21 bins of the
64-cell workload (random-phase forcing 0.5 p0 at 100 kHz, s = 0.3), 200 flow
steps of 1e-8 s, adaptive stepping at tol 1e-4.  It records the final R and
Rdot of every (bin, cell), the per-call attempt total and the 7 moments.
Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2511_21031_gb300 import workloads  # noqa: E402

N_STEPS = 200


def run():
    wl = workloads.config_small().subset(np.arange(8))
    P = oracle.Params(**wl.fluid)
    R0, w = oracle.bins(wl.n_bins, wl.R0ref, wl.s, wl.span_K)
    R = np.repeat(R0[:, None], wl.n_cells, axis=1).copy()
    V = np.zeros_like(R)
    h = np.zeros(R.shape, dtype=np.float32)
    nb = np.full(wl.n_cells, oracle.equilibrium_nb(wl.alpha0, R0, w))
    attempts = 0
    for n in range(N_STEPS):
        fl, na = oracle.step(P, R0, wl.pressure_step(n), wl.dt, R, V, h)
        assert not fl.any()
        attempts += int(na.sum())
    mom = oracle.moments(P, R0, w, nb, R, V)
    return R, V, attempts, mom


if __name__ == "__main__":
    R, V, attempts, mom = run()
    path = os.path.join(HERE, "oracle_cells8_nb21.txt")
    with open(path, "w") as f:
        f.write("# oracle regression fixture, written by tests/golden/make_golden.py\n")
        f.write(f"attempts {attempts}\n")
        for name, arr in (("R", R), ("Rdot", V), ("moments", mom)):
            f.write(f"{name} " + " ".join(repr(float(x)) for x in arr.ravel()) + "\n")
    print("wrote", path, "attempts", attempts)
