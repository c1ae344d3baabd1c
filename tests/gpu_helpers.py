"""Shared drivers for the GPU parity tests: run a workload through the C ABI and
through the oracle on identical host-generated inputs, and compare."""
import math

import numpy as np

import oracle

V_FLOOR_SCALE = 1e-3  # Rdot errors are judged against max(|Rdot|, 1e-3 sqrt(p0/rho))


def oracle_params(wl, **over):
    kw = dict(wl.fluid)
    kw.update(over)
    return oracle.Params(**kw)


def run_oracle(wl, n_steps, pressures=None, n_fixed=0, params=None, R0w=None, state=None,
               nb=None, record=False):
    P = params or oracle_params(wl)
    R0, w = R0w if R0w is not None else oracle.bins(wl.n_bins, wl.R0ref, wl.s, wl.span_K)
    if state is None:
        R = np.repeat(R0[:, None], wl.n_cells, axis=1).copy()
        V = np.zeros_like(R)
        h = np.zeros(R.shape, dtype=np.float32)
    else:
        R, V, h = (np.array(a, copy=True) for a in state)
    att_total = np.zeros(R.shape, dtype=np.int64)
    last_att = None
    flags_or = 0
    for n in range(n_steps):
        p = pressures[n] if pressures is not None else wl.pressure_step(n)
        fl, na = oracle.step(P, R0, p, wl.dt, R, V, h, n_fixed=n_fixed)
        flags_or |= int(np.bitwise_or.reduce(fl.ravel()))
        att_total += na
        last_att = na
    if nb is None:
        nb = np.full(wl.n_cells, oracle.equilibrium_nb(wl.alpha0, R0, w))
    mom = oracle.moments(P, R0, w, nb, R, V)
    return dict(R=R, V=V, h=h, moments=mom, R0=R0, w=w, attempts=att_total, last_attempts=last_att,
                flags=flags_or, nb=nb)


def run_gpu(wl, n_steps, pressures=None, precision="fp64", n_fixed=0, block_warps=0, record=True,
            solver=None, **cfg):
    import torch

    from paper_2511_21031_gb300 import pab
    own = solver is None
    if own:
        kw = dict(s_lognormal=wl.s, R0ref=wl.R0ref, span_K=wl.span_K, alpha0=wl.alpha0,
                  record_attempts=1 if record else 0)
        kw.update({k: v for k, v in wl.fluid.items()})
        kw.update(cfg)
        solver = pab.Solver(wl.n_cells, wl.n_bins, precision=precision, fixed_substeps=n_fixed, **kw)
        if block_warps:
            solver.set_block_warps(block_warps)
    mom = torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64, device="cuda")
    att_total = torch.zeros((wl.n_bins, wl.n_cells), dtype=torch.int64, device="cuda") if record else None
    for n in range(n_steps):
        p = pressures[n] if pressures is not None else wl.pressure_step(n)
        pt = torch.as_tensor(np.ascontiguousarray(p), dtype=torch.float64, device="cuda")
        solver.step(pt, wl.dt, moments=mom)
        if record:
            att_total += solver.attempts().to(torch.int64)
    st = solver.status()
    R, V, h = solver.get_state()
    torch.cuda.synchronize()
    out = dict(R=R.cpu().numpy(), V=V.cpu().numpy(), h=h.cpu().numpy(), moments=mom.cpu().numpy(),
               status=st, solver=solver, R0=np.array(solver.R0), w=np.array(solver.w),
               attempts=att_total.cpu().numpy() if record else None)
    if own:
        out["solver"] = solver
    return out


def rel_err_R(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def rel_err_V(a, b, fluid):
    floor = V_FLOOR_SCALE * math.sqrt(fluid["p0"] / fluid["rho"])
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def moment_errors(g, o, R, V, w):
    """Per-row relative error of the 7 moments.  Signed rows (<R^2 Rdot> and the
    alpha source) are judged against the sum of absolute terms sum w R^2 |Rdot|
    plus the Rdot floor, the condition scale of that sum."""
    w = np.asarray(w)[:, None]
    m3 = o[2]
    abs_m2v = np.sum(w * R * R * np.abs(V), axis=0) + np.sum(w * R * R, axis=0) * 1e-2
    errs = {}
    for k in (0, 1, 2, 5):
        errs[k] = float(np.max(np.abs(g[k] - o[k]) / np.maximum(np.abs(o[k]), 1e-300)))
    errs[6] = float(np.max(np.abs(g[6] - o[6]) / np.maximum(np.abs(o[6]), 1e-4)))
    errs[3] = float(np.max(np.abs(g[3] - o[3]) / abs_m2v))
    errs[4] = float(np.max(np.abs(g[4] - o[4]) / (3 * o[1] * abs_m2v / m3)))
    return errs
