"""GPU FP64 path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated by the method's targets): fixed-step mode relative 1e-9,
adaptive mode relative 1e-6 on R, Rdot (Rdot against max(|Rdot|, 0.01 m/s))
and on every moment (signed moments against their sum of absolute terms).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_21031_gb300 import pab, workloads
from tests.gpu_helpers import moment_errors, rel_err_R, rel_err_V, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL_FIXED = 1e-9
TOL_ADAPT = 1e-6


def _check(g, o, fluid, tol, attempts=True):
    eR = rel_err_R(g["R"], o["R"])
    eV = rel_err_V(g["V"], o["V"], fluid)
    em = moment_errors(g["moments"], o["moments"], o["R"], o["V"], o["w"])
    assert eR <= tol, eR
    assert eV <= tol, eV
    for k, e in em.items():
        assert e <= tol, (pab.MOMENT_NAMES[k], e)
    if attempts and g["attempts"] is not None:
        differ = float(np.mean(g["attempts"] != o["attempts"]))
        assert differ <= 1e-3, differ
    return eR, eV, em


def test_bin_table_matches_oracle():
    for B, s in ((1, 0.3), (3, 0.2), (21, 0.3), (31, 0.5), (51, 0.7), (63, 0.7)):
        sol = pab.Solver(4, B, s_lognormal=s)
        R0, w = oracle.bins(B, 10e-6, s, 5.0)
        np.testing.assert_allclose(sol.R0, R0, rtol=1e-14)
        np.testing.assert_allclose(sol.w, w, rtol=1e-13)
        assert sol.nb_default == pytest.approx(oracle.equilibrium_nb(4e-5, R0, w), rel=1e-13)
        sol.close()


def test_initial_state_and_equilibrium_moments():
    import torch
    sol = pab.Solver(100, 31, s_lognormal=0.5, Rdot0_ref=0.015)
    R, V, h = sol.get_state()
    R0 = torch.tensor(sol.R0, dtype=torch.float64, device="cuda")[:, None]
    assert torch.equal(R, R0.expand(-1, 100))
    torch.testing.assert_close(V, (0.015 / 10e-6) * R0.expand(-1, 100), rtol=1e-15, atol=0)
    assert torch.all(h == 0)
    sol.close()
    sol = pab.Solver(100, 31, s_lognormal=0.5)
    m = sol.moments().cpu().numpy()
    np.testing.assert_allclose(m[1], 4e-5, rtol=1e-13)
    np.testing.assert_allclose(m[5], 101325.0, rtol=1e-13)
    assert np.all(m[3] == 0) and np.all(m[4] == 0) and np.all(m[6] == 0)
    sol.close()


@pytest.mark.parametrize("n_fixed", [1, 3])
def test_fixed_mode_parity_small(n_fixed):
    wl = workloads.config_small()
    g = run_gpu(wl, 300, n_fixed=n_fixed)
    o = run_oracle(wl, 300, n_fixed=n_fixed)
    _check(g, o, wl.fluid, TOL_FIXED, attempts=False)


def test_adaptive_parity_64_cells_full_1000_steps():
    """64 cells x Nb 21, 0.5 p0 at 100 kHz, 1000 steps of 1e-8 s (the small workload in full)."""
    wl = workloads.config_small()
    g = run_gpu(wl, wl.n_steps)
    o = run_oracle(wl, wl.n_steps)
    assert g["status"]["flags"] == 0 and o["flags"] == 0
    eR, eV, em = _check(g, o, wl.fluid, TOL_ADAPT)
    assert g["status"]["n_attempts"] == int(o["attempts"].sum()) or \
        abs(g["status"]["n_attempts"] / o["attempts"].sum() - 1) < 1e-4
    np.testing.assert_array_equal(g["h"] > 0, o["h"] > 0)


@pytest.mark.parametrize("C,B,s", [(1, 21, 0.3), (33, 31, 0.5), (1000, 31, 0.5), (257, 51, 0.7),
                                   (70, 63, 0.6), (45, 1, 0.0), (40, 3, 0.2)])
def test_adaptive_parity_ragged_tiles_and_bin_counts(C, B, s):
    """Several 32-cell tiles with a ragged tail; Nb from 1 to the maximum 63;
    1.2 p0 forcing (tension), 150 steps of 5e-9 s."""
    base = workloads.config_grid128(edge=8)
    cells = np.arange(C) % base.n_cells
    wl = base.subset(cells)
    wl.n_bins = B
    wl.s = s if B > 1 else 0.3
    g = run_gpu(wl, 150)
    o = run_oracle(wl, 150)
    _check(g, o, wl.fluid, TOL_ADAPT)


@pytest.mark.parametrize("bw", [1, 2, 4, 16])
def test_launch_shape_does_not_change_the_state(bw):
    wl = workloads.config_small()
    ref = run_gpu(wl, 100, block_warps=8)
    g = run_gpu(wl, 100, block_warps=bw)
    np.testing.assert_array_equal(g["R"], ref["R"])
    np.testing.assert_array_equal(g["V"], ref["V"])
    np.testing.assert_array_equal(g["h"], ref["h"])
    np.testing.assert_allclose(g["moments"], ref["moments"], rtol=1e-14, atol=0)


def test_full_size_grid128_sampled_cells():
    """128^3 cells x Nb 31 (the timed workload) in the launch shape the bench
    uses: 12 flow steps on the whole grid, then 384 seeded cells compared with
    the oracle run on exactly those cells (cells are independent)."""
    wl = workloads.config_grid128()
    n = 12
    ps = [wl.pressure_step(k) for k in range(n)]
    g = run_gpu(wl, n, pressures=ps, record=False)
    cells = np.sort(np.random.default_rng(7).choice(wl.n_cells, 384, replace=False))
    sub = wl.subset(cells)
    o = run_oracle(sub, n, pressures=[p[cells] for p in ps])
    gs = dict(R=g["R"][:, cells], V=g["V"][:, cells], moments=g["moments"][:, cells], attempts=None)
    _check(gs, o, wl.fluid, TOL_ADAPT, attempts=False)
    assert g["status"]["flags"] == 0
    # every cell of the grid moved and stayed physical
    assert np.all(np.isfinite(g["moments"])) and np.all(g["moments"][1] > 0)


def test_adaptive_parity_through_growth_and_collapse():
    """The collapse-stress forcing (1.2 p0 plane wave at 21.4 kHz, 5e-9 s steps) on 64 cells
    spread along the wave x 31 bins, through the first growth and collapse (11000 steps):
    the regime of the paper's Ohl-type validation case (Sec. 5), with sub-step cascades and
    rejections near collapse and the gas term far from equilibrium.  FP64
    kernel against the oracle at the adaptive tolerance on R, Rdot and every moment, with at
    most 0.1 % of bins taking a different number of trials."""
    base = workloads.config_collapse(edge=8)
    cells = np.arange(0, base.n_cells, 8)
    wl = base.subset(cells)
    n = 11000
    g = run_gpu(wl, n)
    o = run_oracle(wl, n)
    x = o["R"] / o["R0"][:, None]
    per_bin = o["attempts"] / n
    print(f"collapse FP64 parity: R/R0 in [{x.min():.3f}, {x.max():.3f}], max |Rdot| "
          f"{np.abs(o['V']).max():.1f} m/s, trials per bin-step mean {per_bin.mean():.3f} max "
          f"{per_bin.max():.3f}, GPU trials {g['status']['n_attempts']} oracle {int(o['attempts'].sum())}")
    assert g["status"]["flags"] == 0 and o["flags"] == 0
    assert x.min() < 0.3 and np.abs(o["V"]).max() > 75.0      # bins are collapsing at the end
    eR, eV, em = _check(g, o, wl.fluid, TOL_ADAPT)
    print("errors: R", eR, "Rdot", eV, {pab.MOMENT_NAMES[k]: e for k, e in em.items()})


def test_rayleigh_collapse_and_incompressible_limit_on_gpu():
    """Empty cavity, inviscid, c = inf: GPU equals the oracle (which is pinned to
    the Rayleigh collapse time)."""
    over = dict(mu=0.0, sigma=0.0, c=math.inf, gas_mode=1)
    wl = workloads.config_small().subset(np.arange(3))
    wl.n_bins = 1
    wl.fluid = dict(wl.fluid, mu=0.0, sigma=0.0, c=math.inf)
    tc = 0.914681 * 10e-6 * math.sqrt(1000.0 / 101325.0)
    wl.dt = tc / 400
    ps = [np.full(3, 101325.0)] * 380
    P = oracle.Params(**dict(wl.fluid, gas_mode=1))
    g = run_gpu(wl, 380, pressures=ps, gas_mode=1)
    o = run_oracle(wl, 380, pressures=ps, params=P)
    assert g["R"][0, 0] / 10e-6 < 0.45   # R/R0 ~ 0.39 at 0.95 t_c
    _check(g, o, wl.fluid, TOL_ADAPT)
    del over


def test_nonfinite_pressure_and_step_limit_are_flagged():
    import torch
    sol = pab.Solver(64, 21, record_attempts=1)
    p = torch.full((64,), 101325.0, dtype=torch.float64, device="cuda")
    p[5] = float("nan")
    sol.step(p, 1e-8)
    st = sol.status()
    assert st["status"] == pab.PAB_ENONFINITE and st["flags"] & pab.FLAG_NONFINITE
    assert st["n_flagged"] == 21
    R, V, _ = sol.get_state()
    assert torch.all(R[:, 5] == torch.tensor(sol.R0, device="cuda", dtype=torch.float64))
    sol.close()
    sol = pab.Solver(64, 21, max_attempts=1, tol=1e-14)
    p = torch.full((64,), 3 * 101325.0, dtype=torch.float64, device="cuda")
    sol.step(p, 1e-6)
    st = sol.status()
    assert st["status"] == pab.PAB_ESTEP_LIMIT and st["flags"] & pab.FLAG_STEP_LIMIT
    assert st["n_attempts"] == 64 * 21
    # status is reset by reading it
    st2 = sol.status()
    assert st2["flags"] == 0 and st2["n_attempts"] == 0
    sol.close()


def test_invalid_step_arguments():
    import torch
    sol = pab.Solver(8, 3, s_lognormal=0.2)
    p = torch.full((8,), 101325.0, dtype=torch.float64, device="cuda")
    for dt in (0.0, -1e-8, float("nan"), float("inf")):
        with pytest.raises(pab.PabError) as ei:
            sol.step(p, dt)
        assert ei.value.status == pab.PAB_EINVAL
    with pytest.raises(pab.PabError):
        pab.pab_bubble_step(sol.handle, 0, 0, 1e-8, 0)
    with pytest.raises(ValueError):
        sol.step(p.float(), 1e-8)
    with pytest.raises(pab.PabError) as ei:
        pab.Solver(8, 3, s_lognormal=0.2).attempts()
    assert ei.value.status == pab.PAB_ESTATE
    sol.close()
    sol.close()  # double close is safe


def test_checkpoint_resume_is_bit_identical():
    import torch
    wl = workloads.config_small()
    a = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    ps = [torch.as_tensor(wl.pressure_step(k), device="cuda") for k in range(40)]
    for k in range(20):
        a.step(ps[k], wl.dt)
    ck = a.get_state()
    for k in range(20, 40):
        a.step(ps[k], wl.dt)
    ra = a.get_state()
    b = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    b.set_state(*ck)
    for k in range(20, 40):
        b.step(ps[k], wl.dt)
    rb = b.get_state()
    for x, y in zip(ra, rb):
        assert torch.equal(x, y)
    a.close()
    b.close()


def test_moments_only_kernel_and_host_entry_match_fused_step():
    import torch
    wl = workloads.config_small()
    a = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    b = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    nb = torch.linspace(1e9, 5e9, wl.n_cells, dtype=torch.float64, device="cuda")
    mom = torch.empty((7, wl.n_cells), dtype=torch.float64, device="cuda")
    mh = torch.empty((7, wl.n_cells), dtype=torch.float64).pin_memory()
    for k in range(30):
        p = wl.pressure_step(k)
        a.step(torch.as_tensor(p, device="cuda"), wl.dt, moments=mom, nb=nb)
        b.step_host(torch.as_tensor(p).pin_memory(), wl.dt, moments_host=mh, nb_host=nb.cpu())
    m2 = a.moments(nb=nb)
    torch.cuda.synchronize()
    # the step ends with the reduce-only kernel's pass over the new state: the same bits
    assert torch.equal(m2, mom)
    assert torch.equal(mom.cpu(), mh)
    a.close()
    b.close()


def test_external_nb_field_scales_alpha_linearly():
    """alpha and its source are linear in n_b; the other moments do not depend on it."""
    import torch
    wl = workloads.config_small()
    a = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    p = torch.as_tensor(wl.pressure_step(0), device="cuda")
    nb = torch.full((wl.n_cells,), 2.0 * a.nb_default, dtype=torch.float64, device="cuda")
    m1 = torch.empty((7, wl.n_cells), dtype=torch.float64, device="cuda")
    a.step(p, wl.dt, moments=m1)
    m2 = a.moments(nb=nb)
    for k in (0, 1, 4):
        torch.testing.assert_close(m2[k], 2 * m1[k], rtol=1e-15, atol=0)
    for k in (2, 3, 6):
        assert torch.equal(m2[k], m1[k])
    # p_bw: the step's closing pass and the reduce-only kernel are the same arithmetic
    assert torch.equal(m2[5], m1[5])
    a.close()


def _planted_proposals(wl):
    """Carried step proposals [B][C] that the controller must fall back from (NaN, zeros,
    negative, infinite, beyond 2^104, huge but exactly convertible, above dt) next to valid
    ones (subnormal, a third of dt, dt itself); returns (h, the mask of the valid ones)."""
    dt = np.float32(wl.dt)
    special = np.array([np.nan, 0.0, -0.0, -1e-9, np.inf, 3e38, 1e31, 2.0 * dt,
                        1e-40, dt / np.float32(3.0), dt], dtype=np.float32)
    valid = np.array([False] * 8 + [True] * 3)
    idx = np.arange(wl.n_bins * wl.n_cells).reshape(wl.n_bins, wl.n_cells) % special.size
    return special[idx], valid[idx]


def test_invalid_carried_step_size_falls_back_to_dt():
    """The first trial of a flow step is min(h, dt) for a positive finite carried h and dt
    otherwise: the FP64 path against the oracle from the same planted proposals, and the
    mixed path bit for bit against the same run with every invalid proposal set to 0."""
    import torch
    wl = workloads.config_small()
    R0, _ = oracle.bins(wl.n_bins, wl.R0ref, wl.s, wl.span_K)
    R = np.repeat(R0[:, None], wl.n_cells, axis=1)
    V = np.zeros_like(R)
    h, valid = _planted_proposals(wl)
    steps = 5
    o = run_oracle(wl, steps, state=(R, V, h))
    s = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s, R0ref=wl.R0ref, span_K=wl.span_K,
                   alpha0=wl.alpha0, record_attempts=1, **wl.fluid)
    s.set_state(torch.as_tensor(R, device="cuda"), torch.as_tensor(V, device="cuda"),
                torch.as_tensor(h, device="cuda"))
    g = run_gpu(wl, steps, solver=s)
    _check(g, o, wl.fluid, TOL_ADAPT)
    assert g["status"]["flags"] == 0
    s.close()

    outs = []
    for hh in (h, np.where(valid, h, np.float32(0.0))):
        m = pab.Solver(wl.n_cells, wl.n_bins, precision="mixed", s_lognormal=wl.s, R0ref=wl.R0ref,
                       span_K=wl.span_K, alpha0=wl.alpha0, **wl.fluid)
        m.set_state(torch.as_tensor(R, device="cuda"), torch.as_tensor(V, device="cuda"),
                    torch.as_tensor(hh, device="cuda"))
        for n in range(steps):
            m.step(torch.as_tensor(wl.pressure_step(n), device="cuda"), wl.dt)
        outs.append([x.cpu() for x in m.get_state()])
        m.close()
    for x, y in zip(*outs):
        assert torch.equal(x, y)


def test_calls_on_other_streams_give_the_create_streams_bits():
    """Every call is ordered on the stream it is given, not on the one the handle was created
    on: steps issued on a side stream and then on the legacy default stream (the caller ordering
    the two) give the bits of the same steps on the create stream."""
    import torch
    wl = workloads.config_small()
    ps = [torch.as_tensor(wl.pressure_step(k), device="cuda") for k in range(30)]
    s_create, s_side = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    a = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s, stream=s_create)
    b = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s, stream=s_create)
    ma = torch.empty((7, wl.n_cells), dtype=torch.float64, device="cuda")
    mb = torch.empty_like(ma)
    torch.cuda.synchronize()
    for k in range(30):
        a.step(ps[k], wl.dt, moments=ma, stream=s_create)
    for k in range(15):
        b.step(ps[k], wl.dt, moments=mb, stream=s_side)
    legacy = torch.cuda.default_stream()
    legacy.wait_stream(s_side)
    for k in range(15, 30):
        b.step(ps[k], wl.dt, moments=mb, stream=legacy)
    ra = a.get_state(stream=s_create)
    rb = b.get_state(stream=legacy)
    torch.cuda.synchronize()
    for x, y in zip(ra, rb):
        assert torch.equal(x, y)
    assert torch.equal(ma, mb)
    assert a.status(stream=s_create)["n_attempts"] == b.status(stream=legacy)["n_attempts"]
    a.close()
    b.close()


def test_mixed_parked_items_and_lot_overflow_give_the_same_bits_in_every_launch_shape():
    """Every bin starts near collapse (R = 0.18 R0, below the FP64 threshold of 0.2 R0), so every
    item parks in its CTA's lot (32 per warp) until the lot is full and the rest take their FP64
    trials where they are (5000 cells: 157 tiles, no split by bins); the state and moments are the
    same bits for CTAs of 1, 4 and 16 warps, and match the oracle at the adaptive tolerance."""
    import torch
    wl = workloads.config_small().subset(np.arange(5000) % 64)
    wl.n_bins = 31
    wl.s = 0.5
    R0, _ = oracle.bins(wl.n_bins, wl.R0ref, wl.s, wl.span_K)
    R = np.repeat(0.18 * R0[:, None], wl.n_cells, axis=1)
    V = np.zeros_like(R)
    h = np.zeros(R.shape, dtype=np.float32)
    steps = 3
    outs = []
    for bw in (1, 4, 16):
        s = pab.Solver(wl.n_cells, wl.n_bins, precision="mixed", s_lognormal=wl.s, R0ref=wl.R0ref,
                       span_K=wl.span_K, alpha0=wl.alpha0, **wl.fluid)
        s.set_block_warps(bw)
        s.set_state(torch.as_tensor(R, device="cuda"), torch.as_tensor(V, device="cuda"),
                    torch.as_tensor(h, device="cuda"))
        g = run_gpu(wl, steps, solver=s, record=False)
        assert g["status"]["n_fp64"] > 0 and g["status"]["flags"] == 0
        outs.append(g)
        s.close()
    for g in outs[1:]:
        for k in ("R", "V", "h", "moments"):
            np.testing.assert_array_equal(g[k], outs[0][k])
    o = run_oracle(wl, steps, state=(R, V, h))
    assert rel_err_R(outs[0]["R"], o["R"]) <= TOL_ADAPT
    assert rel_err_V(outs[0]["V"], o["V"], wl.fluid) <= TOL_ADAPT


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [1, 70, 96, 4700])
def test_small_grid_split_by_bins_gives_the_bits_of_a_large_grid(precision, m):
    """A grid of fewer tiles than SMs is split by bins over more CTAs, and the last CTA of each
    tile sums the terms the others stored (one bin per CTA at 1-96 cells, two bin ranges at 147
    tiles, a ragged last tile at 70 and 4700 cells; the tiles' counters reset by every one of the
    30 calls); the same cells inside a large grid (one CTA per 128 cells, moments from the closing
    pass) give the same state and moments, bit for bit."""
    big = workloads.config_grid128(edge=32)               # 32768 cells: 256 CTAs
    small = big.subset(np.arange(m))                       # fewer tiles than SMs: split by bins
    n = 30
    ps = [big.pressure_step(k) for k in range(n)]
    gb = run_gpu(big, n, pressures=ps, precision=precision, record=False)
    gs = run_gpu(small, n, pressures=[p[:m] for p in ps], precision=precision, record=False)
    np.testing.assert_array_equal(gs["R"], gb["R"][:, :m])
    np.testing.assert_array_equal(gs["V"], gb["V"][:, :m])
    np.testing.assert_array_equal(gs["h"], gb["h"][:, :m])
    np.testing.assert_array_equal(gs["moments"], gb["moments"][:, :m])
