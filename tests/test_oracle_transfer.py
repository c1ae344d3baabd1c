"""Pins of the oracle's non-polytropic contents (Sec. 2: Ando's pressure
equation, the vapour flux of Eq. massVaporRate, constant-coefficient wall
gradients). Each pin follows from physics the oracle does not spell out that
way: the equilibrium fixed point, the exact polytropic law without transfer,
the first law of thermodynamics at constant volume (heat term), the enthalpy
carried by condensing or evaporating vapour (coupling of the two equations),
diffusive equilibrium of the vapour, and third-order convergence of the
four-component trial."""
import math

import numpy as np
import pytest

import oracle

scipy_integrate = pytest.importorskip("scipy.integrate")

R0 = 10e-6


def _params(**kw):
    d = dict(pv=2338.0)
    d.update(kw)
    return oracle.Params(**d)


def test_equilibrium_is_a_fixed_point():
    P, T = _params(), oracle.Transfer()
    R0s = np.array([5e-6, 10e-6, 20e-6])
    C = 3
    y = np.array([oracle.transfer_init(P, T, r) for r in R0s])  # [B][4]
    R = np.repeat(y[:, 0:1], C, 1).copy()
    V = np.repeat(y[:, 1:2], C, 1).copy()
    pb = np.repeat(y[:, 2:3], C, 1).copy()
    mv = np.repeat(y[:, 3:4], C, 1).copy()
    h = np.zeros((3, C), np.float32)
    R_in, pb_in, mv_in = R.copy(), pb.copy(), mv.copy()
    for _ in range(20):
        fl, _ = oracle.transfer_step(P, T, R0s, np.full(C, P.p0), 1e-8, R, V, pb, mv, h)
        assert not fl.any()
    np.testing.assert_allclose(R, R_in, rtol=1e-14)
    np.testing.assert_allclose(pb, pb_in, rtol=1e-14)
    np.testing.assert_allclose(mv, mv_in, rtol=1e-14)
    np.testing.assert_allclose(V, 0.0, atol=1e-12)
    # the equilibrium gas mass is the ideal-gas law at R0 for the gas partial pressure
    mg = oracle.transfer_gas_mass(P, T, R0)
    V0 = 4 / 3 * math.pi * R0 ** 3
    assert mg * T.R_g * T.T_w == pytest.approx((P.p0 + 2 * P.sigma / R0 - P.pv) * V0, rel=1e-14)


def test_without_transfer_the_contents_are_polytropic():
    """beta_T = beta_c = 0: dp_b/dt = -3 gamma Rdot p_b/R, so p_b R^(3 gamma) is invariant, and
    with p_v = 0 the radius follows the polytropic model (gas_mode 0) to integration error."""
    T = oracle.Transfer(beta_T=0.0, beta_c=0.0)
    for pv in (2338.0, 0.0):
        P = _params(pv=pv)
        y = oracle.transfer_init(P, T, R0)
        R, V, pb, mv = (np.full((1, 1), v) for v in y)
        h = np.zeros((1, 1), np.float32)
        inv0 = pb[0, 0] * R[0, 0] ** (3 * P.gamma)
        p = np.array([1.4 * P.p0])
        for _ in range(40):
            oracle.transfer_step(P, T, [R0], p, 5e-9, R, V, pb, mv, h, n_fixed=20)
            assert pb[0, 0] * R[0, 0] ** (3 * P.gamma) == pytest.approx(inv0, rel=1e-9)
            assert mv[0, 0] == y[3]
    # same trajectory as the polytropic oracle (p_v = 0: all of p_b is gas)
    P = _params(pv=0.0)
    y = oracle.transfer_init(P, T, R0)
    R, V, pb, mv = (np.full((1, 1), v) for v in y)
    Rp, Vp = np.full((1, 1), R0), np.zeros((1, 1))
    h = np.zeros((1, 1), np.float32)
    hp = np.zeros((1, 1), np.float32)
    p = np.array([1.4 * P.p0])
    for _ in range(60):
        oracle.transfer_step(P, T, [R0], p, 5e-9, R, V, pb, mv, h, n_fixed=40)
        oracle.step(P, [R0], p, 5e-9, Rp, Vp, hp, n_fixed=40)
    assert abs(R[0, 0] / R0 - 1) > 0.01  # the bubble moved
    assert R[0, 0] == pytest.approx(Rp[0, 0], rel=1e-9)
    assert V[0, 0] == pytest.approx(Vp[0, 0], rel=1e-7, abs=1e-9)


def test_heat_term_is_the_first_law_at_constant_volume():
    """Rdot = 0, beta_c = 0, no vapour: the contents exchange only heat Q = 4 pi R^2 k dT/dr
    through the wall, with dT/dr = beta_T (T_w - T)/R. At constant volume dU = Q dt with
    U = p V/(gamma - 1) and p V = m_g R_g T, so p relaxes exponentially to the isothermal
    pressure m_g R_g T_w / V with time constant m_g R_g / ((gamma - 1) 4 pi R k beta_T)."""
    P, T = _params(pv=0.0), oracle.Transfer(beta_c=0.0, beta_T=7.0)
    mg = oracle.transfer_gas_mass(P, T, R0)
    R = 1.3 * R0  # held fixed, expanded: the gas is colder than the wall
    V = 4 / 3 * math.pi * R ** 3
    p_iso = mg * T.R_g * T.T_w / V
    p_start = 0.7 * p_iso
    tau = mg * T.R_g / ((P.gamma - 1) * 4 * math.pi * R * T.k_bw * T.beta_T)

    def f(t, u):
        return [oracle.transfer_rates(P, T, mg, [R, 0.0, u[0], 0.0])[0]]

    t_end = 3 * tau
    sol = scipy_integrate.solve_ivp(f, (0, t_end), [p_start], rtol=1e-11, atol=1e-6,
                                    t_eval=np.linspace(0, t_end, 7))
    want = p_iso + (p_start - p_iso) * np.exp(-sol.t / tau)
    np.testing.assert_allclose(sol.y[0], want, rtol=1e-8)
    assert sol.y[0, -1] > p_start  # heat flowed in


def test_vapour_enthalpy_and_diffusive_equilibrium():
    """Rdot = 0, beta_T = 0: vapour entering at the wall temperature brings its enthalpy, so at
    constant volume dp_b = gamma R_v T_w dm_v / V and p_b - gamma R_v T_w m_v / V is invariant.
    The flux stops when the mean vapour fraction equals the saturated wall value."""
    P, T = _params(pv=2338.0), oracle.Transfer(beta_T=0.0, beta_c=4.0)
    mg = oracle.transfer_gas_mass(P, T, R0)
    R = R0
    V = 4 / 3 * math.pi * R ** 3
    y0 = oracle.transfer_init(P, T, R0)
    u0 = [y0[2], 0.2 * y0[3]]  # vapour-starved bubble: evaporation into it

    def f(t, u):
        return list(oracle.transfer_rates(P, T, mg, [R, 0.0, u[0], u[1]]))

    t_end = 1e-5  # the flux relaxes within about a microsecond at this size
    sol = scipy_integrate.solve_ivp(f, (0, t_end), u0, method="LSODA", rtol=1e-11,
                                    atol=[1e-6, 1e-30], t_eval=np.linspace(0, t_end, 9))
    k = P.gamma * T.R_v * T.T_w / V
    inv = sol.y[0] - k * sol.y[1]
    np.testing.assert_allclose(inv, inv[0], rtol=1e-9)
    assert sol.y[1, 1] > sol.y[1, 0] and np.all(np.diff(sol.y[1]) >= -1e-12 * sol.y[1, 0])  # evaporation
    pb, mv = sol.y[0, -1], sol.y[1, -1]
    chi_mean = mv / (mv + mg)
    chi_wall = (P.pv / T.R_v) / (P.pv / T.R_v + (pb - P.pv) / T.R_g)
    assert chi_mean == pytest.approx(chi_wall, rel=1e-6)


def test_four_component_trial_is_third_order():
    """Fixed sub-steps n, 2n, 4n over the same flow step: errors against a fine reference fall
    by 2^3 per halving for every component."""
    P, T = _params(), oracle.Transfer()
    y0 = oracle.transfer_init(P, T, R0)
    p = np.array([1.8 * P.p0])
    dt = 2e-7

    def run(n):
        R, V, pb, mv = (np.full((1, 1), v) for v in y0)
        h = np.zeros((1, 1), np.float32)
        oracle.transfer_step(P, T, [R0], p, dt, R, V, pb, mv, h, n_fixed=n)
        return np.array([R[0, 0], V[0, 0], pb[0, 0], mv[0, 0]])

    ref = run(2048)
    e = [np.abs(run(n) - ref) for n in (16, 32, 64)]
    for c in range(4):
        r1, r2 = e[0][c] / e[1][c], e[1][c] / e[2][c]
        assert 6.0 < r1 < 10.5 and 6.0 < r2 < 10.5, (c, r1, r2)


def test_transfer_moments_use_the_state_pressure():
    """With p_b set to the polytropic value, the moments equal those of the polytropic model."""
    P = _params(pv=0.0)
    R0s, w = oracle.bins(5, R0ref=R0, s=0.3)
    rng = np.random.default_rng(3)
    C = 4
    R = (R0s[:, None] * rng.uniform(0.8, 1.2, size=(5, C))).copy()
    V = rng.normal(scale=0.5, size=(5, C))
    pg0 = P.p0 + 2 * P.sigma / R0s
    pb = (pg0[:, None] * (R0s[:, None] / R) ** (3 * P.gamma)).copy()
    nb = np.full(C, 1e12)
    a = oracle.transfer_moments(P, w, nb, R, V, pb)
    b = oracle.moments(P, R0s, w, nb, R, V)
    np.testing.assert_allclose(a, b, rtol=1e-13)
