"""Volume-averaged (EL) model on the GPU against the oracle: Lagrangian bubbles
advanced by the Keller-Miksis stepper under their cell's pressure, and the
truncated Gaussian smearing of Eq. (kernel3D) into alpha and its growth rate."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_21031_gb300 import pab, workloads
from paper_2511_21031_gb300.el import BubbleCloud

pytestmark = pytest.mark.gpu


def _cloud(edge=20, alpha0=2e-3, s=0.4, seed=70):
    return workloads.bubble_cloud(edge=edge, dx=60e-6, alpha0=alpha0, R0ref=10e-6, s=s, seed=seed)


def test_smear_matches_oracle_including_wide_kernels_and_edges():
    import torch
    wl = _cloud()
    g = np.random.default_rng(71)
    R = wl.R0 * g.uniform(0.5, 9.0, size=wl.n_bubbles)          # some R > dx: h = R
    V = g.normal(size=wl.n_bubbles)
    cl = BubbleCloud(wl.pos, wl.R0, wl.edge, wl.edge, wl.edge, wl.dx)
    cl.set_state(torch.as_tensor(R, device="cuda"), torch.as_tensor(V, device="cuda"))
    a = torch.empty(wl.edge ** 3, dtype=torch.float64, device="cuda")
    ad = torch.empty_like(a)
    cl.smear(a, ad)
    oa, oad = oracle.el_smear(wl.pos, R, V, wl.edge, wl.edge, wl.edge, wl.dx)
    assert R.max() > wl.dx and wl.n_bubbles > 50
    np.testing.assert_allclose(a.cpu().numpy(), oa, rtol=1e-12, atol=1e-14 * oa.max())
    np.testing.assert_allclose(ad.cpu().numpy(), oad, rtol=1e-12, atol=1e-14 * np.abs(oad).max())
    cl.close()


def test_bubble_with_nan_radius_adds_nothing_to_the_smear():
    import torch
    wl = _cloud(seed=73)
    g = np.random.default_rng(73)
    R = wl.R0 * g.uniform(0.5, 3.0, size=wl.n_bubbles)
    V = g.normal(size=wl.n_bubbles)
    k = wl.n_bubbles // 2
    Rn = R.copy()
    Rn[k] = np.nan
    cl = BubbleCloud(wl.pos, wl.R0, wl.edge, wl.edge, wl.edge, wl.dx)
    cl.set_state(torch.as_tensor(Rn, device="cuda"), torch.as_tensor(V, device="cuda"))
    a = torch.empty(wl.edge ** 3, dtype=torch.float64, device="cuda")
    ad = torch.empty_like(a)
    cl.smear(a, ad)
    keep = np.arange(wl.n_bubbles) != k
    oa, oad = oracle.el_smear(wl.pos[:, keep], R[keep], V[keep], wl.edge, wl.edge, wl.edge, wl.dx)
    a, ad = a.cpu().numpy(), ad.cpu().numpy()
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(ad))
    np.testing.assert_allclose(a, oa, rtol=1e-12, atol=1e-14 * oa.max())
    np.testing.assert_allclose(ad, oad, rtol=1e-12, atol=1e-14 * np.abs(oad).max())
    cl.close()


def test_advance_and_smear_match_oracle_over_steps():
    import torch
    wl = _cloud(edge=16, alpha0=3e-3, seed=72)
    P = oracle.Params(**wl.fluid)
    cl = BubbleCloud(wl.pos, wl.R0, wl.edge, wl.edge, wl.edge, wl.dx)
    cell = (np.floor(wl.pos[2] / wl.dx) * wl.edge + np.floor(wl.pos[1] / wl.dx)) * wl.edge \
        + np.floor(wl.pos[0] / wl.dx)
    R = wl.R0.copy()
    V = np.zeros(wl.n_bubbles)
    h = np.zeros(wl.n_bubbles, dtype=np.float32)
    a = torch.empty(wl.edge ** 3, dtype=torch.float64, device="cuda")
    for n in range(60):
        p = wl.pressure_step(n)
        cl.step(torch.as_tensor(p, device="cuda"), wl.dt, alpha=a)
        oracle.el_advance(P, wl.R0, cell.astype(np.int64), p, wl.dt, R, V, h)
    Rg, Vg, hg = cl.get_state()
    st = cl.status()
    assert st["flags"] == 0 and st["n_attempts"] >= 60 * wl.n_bubbles
    np.testing.assert_allclose(Rg.cpu().numpy(), R, rtol=1e-6)
    vf = 1e-3 * math.sqrt(P.p0 / P.rho)
    assert np.max(np.abs(Vg.cpu().numpy() - V) / np.maximum(np.abs(V), vf)) <= 1e-6
    oa = oracle.el_smear(wl.pos, R, V, wl.edge, wl.edge, wl.edge, wl.dx, with_rate=False)
    np.testing.assert_allclose(a.cpu().numpy(), oa, rtol=1e-5, atol=1e-9 * oa.max())
    cl.close()


def test_bubble_outside_the_grid_is_flagged_and_left_alone():
    import torch
    pos = np.array([[1e-4, 5e-3], [1e-4, 1e-4], [1e-4, 1e-4]])      # second is outside x
    cl = BubbleCloud(pos, np.array([10e-6, 10e-6]), 8, 8, 8, 50e-6)
    p = torch.full((512,), 2 * 101325.0, dtype=torch.float64, device="cuda")
    cl.step(p, 1e-8)
    st = cl.status()
    assert st["status"] == pab.PAB_ENONFINITE and st["n_flagged"] == 1
    R, _, _ = cl.get_state()
    assert float(R[1]) == 10e-6 and float(R[0]) < 10e-6
    cl.close()
