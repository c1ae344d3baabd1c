"""Carrier-facing forms on the GPU against the oracle: conservative bubble
variables (Listing 2, Eq. e:ndf), mixture pressure (Eq. e:pressure),
stiffened-gas liquid pressure (Eq. eos_liquid) and the Strang half step."""
import numpy as np
import pytest

import oracle
from paper_2511_21031_gb300 import pab, workloads

pytestmark = pytest.mark.gpu


def _evolved_solver(n_steps=40, C=300, B=31, s=0.5):
    import torch
    base = workloads.config_grid128(edge=8)
    wl = base.subset(np.arange(C) % base.n_cells)
    wl.n_bins, wl.s = B, s
    sol = pab.Solver(C, B, s_lognormal=s)
    for n in range(n_steps):
        sol.step(torch.as_tensor(wl.pressure_step(n), device="cuda"), wl.dt)
    return sol, wl


def test_conservative_variables_match_oracle_and_round_trip():
    import torch
    sol, wl = _evolved_solver()
    nb = torch.linspace(1e9, 4e9, sol.n_cells, dtype=torch.float64, device="cuda")
    R, V, h = sol.get_state()
    qR, qV = sol.get_conservative(nb=nb)
    oqR, oqV = oracle.cons_from_prim(nb.cpu().numpy(), R.cpu().numpy(), V.cpu().numpy())
    np.testing.assert_array_equal(qR.cpu().numpy(), oqR)
    np.testing.assert_array_equal(qV.cpu().numpy(), oqV)
    alpha = sol.moments(nb=nb)[1].clone()
    other = pab.Solver(sol.n_cells, sol.n_bins, s_lognormal=wl.s)
    nb_back = other.set_conservative(alpha, qR, qV)
    R2, V2, _ = other.get_state()
    oR, oV, onb = oracle.prim_from_cons(np.array(sol.w), alpha.cpu().numpy(), oqR, oqV)
    np.testing.assert_allclose(nb_back.cpu().numpy(), onb, rtol=1e-14)
    np.testing.assert_allclose(nb_back.cpu().numpy(), nb.cpu().numpy(), rtol=1e-13)
    np.testing.assert_allclose(R2.cpu().numpy(), oR, rtol=1e-14)
    np.testing.assert_allclose(R2.cpu().numpy(), R.cpu().numpy(), rtol=1e-13)
    np.testing.assert_allclose(V2.cpu().numpy(), V.cpu().numpy(), rtol=1e-13, atol=1e-18)
    sol.close()
    other.close()


def test_nonpositive_alpha_gives_nan_nb_and_a_flag_on_the_next_step():
    import torch
    sol = pab.Solver(40, 21)
    qR, qV = sol.get_conservative()
    alpha = torch.full((40,), 4e-5, dtype=torch.float64, device="cuda")
    alpha[3] = 0.0
    nb = sol.set_conservative(alpha, qR, qV)
    assert torch.isnan(nb[3]) and torch.all(torch.isfinite(torch.cat([nb[:3], nb[4:]])))
    sol.step(torch.full((40,), 101325.0, dtype=torch.float64, device="cuda"), 1e-8)
    st = sol.status()
    assert st["flags"] & pab.FLAG_NONFINITE and st["n_flagged"] == 21
    sol.close()


def test_mixture_pressure_and_stiffened_gas_match_oracle():
    import torch
    sol, wl = _evolved_solver()
    m = sol.moments()
    g = np.random.default_rng(50)
    rho = torch.as_tensor(g.uniform(950, 1050, size=sol.n_cells), device="cuda")
    e = torch.as_tensor(g.uniform(3.6e5, 3.7e5, size=sol.n_cells), device="cuda")
    p_l = pab.pab_stiffened_gas(rho, e, 6.12, 3.43e8)
    np.testing.assert_allclose(p_l.cpu().numpy(),
                               oracle.stiffened_gas(rho.cpu().numpy(), e.cpu().numpy(), 6.12, 3.43e8),
                               rtol=1e-15, atol=1e-6)
    p_l = torch.as_tensor(g.uniform(5e4, 2e5, size=sol.n_cells), device="cuda")
    for rl in (None, rho):
        p = sol.mixture_pressure(m, p_l, rho_l=rl)
        op = oracle.mixture_pressure(m.cpu().numpy(), p_l.cpu().numpy(),
                                     rl.cpu().numpy() if rl is not None else None, 1000.0)
        np.testing.assert_allclose(p.cpu().numpy(), op, rtol=1e-15)
    sol.close()


def test_strang_half_is_a_bubble_step_of_half_the_flow_step():
    import torch
    wl = workloads.config_small()
    a = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    b = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    ma = torch.empty((7, wl.n_cells), dtype=torch.float64, device="cuda")
    mb = torch.empty_like(ma)
    for n in range(10):
        p_start = torch.as_tensor(wl.pressure_at(n * 2 * wl.dt), device="cuda")
        p_end = torch.as_tensor(wl.pressure_at((n + 1) * 2 * wl.dt), device="cuda")
        a.strang_half(p_start, 2 * wl.dt)
        # (the carrier would advance here)
        a.strang_half(p_end, 2 * wl.dt, moments=ma)
        b.step(p_start, wl.dt)
        b.step(p_end, wl.dt, moments=mb)
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    assert torch.equal(ma, mb)
    with pytest.raises(pab.PabError):
        a.strang_half(p_start, 0.0)
    a.close()
    b.close()
