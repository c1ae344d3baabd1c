"""Mixed precision (FP32 right-hand sides, FP64 state, error estimate, controller
bookkeeping, collapse fallback and compensated alpha sum) against the FP64
oracle.  Target: alpha within 1e-5 relative; the errors of R and <R^2 Rdot>
are stated beside it."""
import numpy as np
import pytest

import oracle
from paper_2511_21031_gb300 import pab, workloads
from tests.gpu_helpers import moment_errors, rel_err_R, rel_err_V, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

ALPHA_TOL = 1e-5


def _errors(g, o, fluid):
    em = moment_errors(g["moments"], o["moments"], o["R"], o["V"], o["w"])
    return dict(R=rel_err_R(g["R"], o["R"]), Rdot=rel_err_V(g["V"], o["V"], fluid),
                alpha=em[1], R2Rdot=em[3], S_alpha=em[4], pbw=em[5], rdot2=em[6])


def test_mixed_small_workload_full_1000_steps():
    wl = workloads.config_small()
    g = run_gpu(wl, wl.n_steps, precision="mixed", record=False)
    o = run_oracle(wl, wl.n_steps)
    e = _errors(g, o, wl.fluid)
    print("mixed vs FP64 oracle, 64 cells x 21 bins x 1000 steps:", e)
    assert e["alpha"] <= ALPHA_TOL
    assert e["R"] <= 1e-5 and e["R2Rdot"] <= 1e-4
    assert g["status"]["flags"] == 0 and g["status"]["n_fp64"] == 0


def test_mixed_full_size_grid256_sampled_cells():
    """256^3 cells x Nb 31 in mixed precision, 10 flow steps on the whole grid,
    256 seeded cells compared with the FP64 oracle run on those cells."""
    wl = workloads.config_grid256_mixed()
    n = 10
    ps = [wl.pressure_step(k) for k in range(n)]
    g = run_gpu(wl, n, pressures=ps, precision="mixed", record=False)
    cells = np.sort(np.random.default_rng(8).choice(wl.n_cells, 256, replace=False))
    o = run_oracle(wl.subset(cells), n, pressures=[p[cells] for p in ps])
    gs = dict(R=g["R"][:, cells], V=g["V"][:, cells], moments=g["moments"][:, cells])
    e = _errors(gs, o, wl.fluid)
    print("mixed vs FP64 oracle, 256^3 x 31, 10 steps, 256 sampled cells:", e)
    assert e["alpha"] <= ALPHA_TOL
    assert np.all(np.isfinite(g["moments"]))


def test_mixed_collapse_uses_fp64_fallback_and_stays_close():
    """Ohl-like 21.4 kHz forcing at 1.2 p0: bins grow several-fold and collapse, so
    the FP64 trial must fire near collapse; the result stays close to the oracle."""
    base = workloads.config_collapse(edge=8)
    cells = np.arange(0, base.n_cells, 8)          # 64 cells spread along the wave
    wl = base.subset(cells)
    n = 11000                                      # 55 us: growth and first collapse
    g = run_gpu(wl, n, precision="mixed", record=False)
    o = run_oracle(wl, n)
    e = _errors(g, o, wl.fluid)
    st = g["status"]
    print("collapse stress, mixed vs FP64 oracle:", e, "FP64 trials:", st["n_fp64"],
          "of", st["n_attempts"])
    assert st["n_fp64"] > 0
    r = o["R"] / o["R0"][:, None]
    assert r.min() < 0.3 and np.abs(o["V"]).max() > 75.0   # a collapse was reached
    assert e["alpha"] <= ALPHA_TOL
    # the other outputs, a few times above their errors on this build (alpha 3.8e-7,
    # R 3.1e-5, Rdot 2.9e-3, <R^2 Rdot> and S_alpha 7.7e-6, <R^3 p_bw>/<R^3> 2.3e-5,
    # <R^3 Rdot^2>/<R^3> 1.2e-5): a weaker FP64 fallback fails here
    assert e["R"] <= 1e-4 and e["Rdot"] <= 1e-2
    assert e["R2Rdot"] <= 5e-5 and e["S_alpha"] <= 5e-5
    assert e["pbw"] <= 1e-4 and e["rdot2"] <= 1e-4


def test_compensated_alpha_sum_keeps_bins_below_half_an_ulp():
    """Mixed mode sums <R^3> (and so alpha) with a compensated FP64 sum.  State:
    one dominant bin and 62 bins each worth 0.3 ulp of it, which a plain FP64
    sum drops (the oracle's plain sum loses ~18 ulp here); the compensated sum
    stays within the rounding of its terms (<= 3 ulp for <R^3>, 6 ulp for alpha)."""
    import torch
    C, B = 32, 63
    R0, w = oracle.bins(B, 10e-6, 0.7, 5.0)
    big = w[0] * (1e-4) ** 3
    ulp = np.spacing(big)
    R = np.empty((B, C))
    R[0] = 1e-4
    for b in range(1, B):
        R[b] = np.cbrt(0.3 * ulp / w[b])
    V = np.zeros((B, C))
    sol = pab.Solver(C, B, precision="mixed", s_lognormal=0.7)
    sol.set_state(torch.as_tensor(R, device="cuda"), torch.as_tensor(V, device="cuda"))
    m = sol.moments().cpu().numpy()
    P = oracle.Params()
    plain, ald = oracle.moments(P, R0, w, np.full(C, sol.nb_default), R, V, with_long_double=True)
    m3_ld = ald / (4.0 / 3.0 * np.pi * sol.nb_default)
    u = float(np.spacing(m3_ld[0].astype(np.float64)))
    assert float(np.max(np.abs(plain[2] - m3_ld))) >= 10 * u        # plain summation fails here
    assert float(np.max(np.abs(m[2] - m3_ld))) <= 3 * u              # compensated does not
    assert float(np.max(np.abs(m[1] - ald) / ald)) <= 6 * 2.2e-16
    sol.close()
