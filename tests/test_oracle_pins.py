"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a textbook special case, an invariant of the paper's equations or a
brute-force evaluation, chosen so that a dropped term, a wrong sign or index
or a transposed coefficient in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special  # noqa: F401

import oracle
from paper_2511_21031_gb300 import workloads

WATER = oracle.Params()


# ----------------------------------------------------------------------------
# a1. Lognormal bins + Simpson quadrature (Sec. 2.2)
# ----------------------------------------------------------------------------
def _truncated_lognormal_moment(k, R0ref, s, K):
    """E[R0^k] of the lognormal cut to |ln(R0/R0ref)| <= K s (closed form)."""
    mu = math.log(R0ref)
    full = math.exp(k * mu + 0.5 * k * k * s * s)
    num = special.ndtr(K - k * s) - special.ndtr(-K - k * s)
    den = special.ndtr(K) - special.ndtr(-K)
    return full * num / den


@pytest.mark.parametrize("B,s", [(21, 0.3), (31, 0.5), (51, 0.7), (11, 0.3)])
def test_bins_integrate_lognormal_moments(B, s):
    R0, w = oracle.bins(B, 10e-6, s, 5.0)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.all(w > 0)
    assert np.all(np.diff(R0) > 0)
    assert R0[B // 2] == pytest.approx(10e-6, rel=1e-15)
    for k in (1, 2, 3):
        exact = _truncated_lognormal_moment(k, 10e-6, s, 5.0)
        approx = float(np.dot(w, R0 ** k))
        # Simpson on [-5s, 5s] with B nodes: error O(dphi^4) of the integrand scale
        dphi = 10 * s / (B - 1)
        bound = 2.0 * (k * s + 5.0) ** 4 * dphi ** 4 / 180.0 * 10
        assert abs(approx / exact - 1.0) < max(bound, 1e-12)


def test_bins_simpson_fourth_order():
    """Halving dphi divides the quadrature error by ~16 (composite Simpson)."""
    errs = []
    for B in (11, 21, 41, 81):
        R0, w = oracle.bins(B, 10e-6, 0.5, 5.0)
        exact = _truncated_lognormal_moment(3, 10e-6, 0.5, 5.0)
        errs.append(abs(float(np.dot(w, R0 ** 3)) / exact - 1.0))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert 12.0 < ratios[1] < 20.0 and 12.0 < ratios[2] < 20.0, ratios


def test_bins_truncation_to_full_lognormal():
    """As the span K grows, the moments approach exp(k mu + k^2 s^2/2)."""
    for k in (1, 2, 3):
        prev = None
        for K in (3.0, 4.0, 5.0, 6.0):
            R0, w = oracle.bins(201, 10e-6, 0.3, K)
            full = math.exp(k * math.log(10e-6) + 0.5 * k * k * 0.09)
            e = abs(float(np.dot(w, R0 ** k)) / full - 1.0)
            if prev is not None:
                assert e < prev
            prev = e
        assert prev < 1e-4


def test_bins_monodisperse_and_invalid():
    R0, w = oracle.bins(1, 7e-6, 0.0, 5.0)
    assert R0[0] == 7e-6 and w[0] == 1.0
    for B in (2, 4, 20):
        with pytest.raises(ValueError):
            oracle.bins(B, 10e-6, 0.3, 5.0)
    with pytest.raises(ValueError):
        oracle.bins(21, 10e-6, 0.0, 5.0)


# ----------------------------------------------------------------------------
# a3. Keller-Miksis right-hand side, Eq. (keller_miksis)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("R0", [2.2e-6, 10e-6, 44e-6])
def test_rhs_equilibrium_fixed_point(R0):
    Rd, Rdd, pbw = oracle.rhs(WATER, R0, WATER.p0, R0, 0.0)
    assert Rd == 0.0
    assert abs(Rdd) < 1e-6          # m/s^2; one rounding of p0 + 2 sigma/R0 at most
    assert pbw == pytest.approx(WATER.p0, rel=1e-15)


def test_rhs_rayleigh_plesset_limit():
    """c -> infinity: R Rddot + 3/2 Rdot^2 = (p_bw - p_inf)/rho (textbook RP)."""
    P = oracle.Params(c=math.inf)
    g = np.random.default_rng(0)
    for _ in range(50):
        R0 = g.uniform(2e-6, 50e-6)
        R = R0 * g.uniform(0.3, 3.0)
        V = g.uniform(-20, 20)
        pinf = g.uniform(-0.5, 3.0) * P.p0
        _, Rdd, pbw = oracle.rhs(P, R0, pinf, R, V)
        pg0 = P.p0 + 2 * P.sigma / R0
        pbw_def = pg0 * (R0 / R) ** (3 * P.gamma) - 4 * P.mu * V / R - 2 * P.sigma / R
        assert pbw == pytest.approx(pbw_def, rel=1e-12)
        lhs = R * Rdd + 1.5 * V * V
        rhs = (pbw - pinf) / P.rho
        assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-9 * abs(pinf) / P.rho)


def _pbw_paper(P, R0, R, V):
    """Wall pressure as Eq. (keller_miksis) defines it, polytropic gas."""
    pg0 = P.p0 + 2 * P.sigma / R0 - P.pv
    pb = P.pv + pg0 * (R0 / R) ** (3 * P.gamma)
    return pb - 4 * P.mu * V / R - 2 * P.sigma / R


@pytest.mark.parametrize("mu,c", [(1e-3, 1500.0), (6e-3, 1500.0), (0.05, 300.0)])
def test_rhs_satisfies_keller_miksis_with_time_derivative_of_pbw(mu, c):
    """Plug Rddot into the KM equation with d/dt p_bw taken by finite differences
    along the motion (so the Rddot hidden in d/dt p_bw is included)."""
    P = oracle.Params(mu=mu, c=c, pv=1000.0)
    g = np.random.default_rng(1)
    for _ in range(40):
        R0 = g.uniform(2e-6, 50e-6)
        R = R0 * g.uniform(0.4, 2.5)
        V = g.uniform(-30, 30)
        pinf = g.uniform(-0.3, 2.5) * P.p0
        _, Rdd, pbw = oracle.rhs(P, R0, pinf, R, V)
        eps = 1e-6 * R / max(abs(V), 1.0)

        def pbw_at(tau):
            return _pbw_paper(P, R0, R + V * tau + 0.5 * Rdd * tau * tau, V + Rdd * tau)

        dpbw = (pbw_at(eps) - pbw_at(-eps)) / (2 * eps)
        lhs = R * (1 - V / c) * Rdd + 1.5 * V * V * (1 - V / (3 * c))
        rhs = (pbw - pinf) / P.rho * (1 + V / c) + R * dpbw / (P.rho * c)
        scale = abs(R * Rdd) + 1.5 * V * V + abs(pbw - pinf) / P.rho + abs(R * dpbw / (P.rho * c))
        assert abs(lhs - rhs) <= 1e-6 * scale


# ----------------------------------------------------------------------------
# a4. SSP-RK3 with embedded SSP-RK2, error norm and controller (Sec. 3)
# ----------------------------------------------------------------------------
def test_trial_is_third_and_second_order_taylor_polynomials():
    """On y' = A y the SSP-RK3 result is (I + hA + (hA)^2/2 + (hA)^3/6) y and the
    embedded Heun result is (I + hA + (hA)^2/2) y."""
    g = np.random.default_rng(2)
    for _ in range(20):
        A = g.normal(size=(2, 2))
        y = g.normal(size=2)
        h = g.uniform(0.01, 0.5)
        M = h * A
        I = np.eye(2)
        y3_exact = (I + M + M @ M / 2 + M @ M @ M / 6) @ y
        z_exact = (I + M + M @ M / 2) @ y
        y3, z = oracle.linear_trial(A, y, h)
        np.testing.assert_allclose(y3, y3_exact, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(z, z_exact, rtol=1e-13, atol=1e-14)


def test_error_norm_and_step_factor_reading():
    vf = 0.01
    assert oracle.error_norm([2.0, 1.0], [2.0, 1.0], vf) == 0.0
    assert oracle.error_norm([2.0, 1.0], [2.002, 1.0], vf) == pytest.approx(1e-3)
    assert oracle.error_norm([2.0, 0.0], [2.0, 1e-5], vf) == pytest.approx(1e-3)   # floor
    assert oracle.error_norm([2.0, -4.0], [2.0, -4.004], vf) == pytest.approx(1e-3)
    tol = 1e-4
    assert oracle.step_factor(0.0, tol) == 5.0
    assert oracle.step_factor(tol, tol) == pytest.approx(0.9)
    assert oracle.step_factor(8 * tol, tol) == pytest.approx(0.45)
    assert oracle.step_factor(1e6 * tol, tol) == 0.2
    assert oracle.step_factor(1e-12 * tol, tol) == 5.0
    assert oracle.step_factor(float("nan"), tol) == 0.2


def test_adaptive_driver_tracks_exact_linear_solution_and_lands_on_dt():
    """Decaying linear system: every call ends exactly at the flow-step end and
    the global error stays at the tolerance scale."""
    A = np.array([[-2.0e5, 1.0e-6], [3.0e9, -5.0e5]])
    lam, vec = np.linalg.eig(A)
    y0 = np.array([1e-5, 0.3])
    y = y0.copy()
    h = np.zeros(1, dtype=np.float32)
    dt = 2e-6
    total_attempts = 0
    for n in range(1, 11):
        fl, na = oracle.linear_advance(A, y, h, dt, 1e-6, 1e-3)
        assert fl == 0
        total_attempts += na
        coef = np.linalg.solve(vec, y0)
        exact = (vec @ (coef * np.exp(lam * n * dt))).real
        assert abs(y[0] / exact[0] - 1) < 1e-4
    assert total_attempts > 10  # the controller had to sub-step
    assert 0 < h[0] <= dt * 5


def test_adaptive_driver_step_limit_flag_keeps_last_accepted_state():
    A = np.array([[-1.0e9, 0.0], [0.0, -1.0e9]])
    y = np.array([1.0, 1.0])
    h = np.array([1e-6], dtype=np.float32)
    fl, na = oracle.linear_advance(A, y, h, 1e-6, 1e-12, 1e-3, max_attempts=5)
    assert fl == oracle.FLAG_STEP_LIMIT and na == 5
    assert np.all(np.isfinite(y))


def _taylor3(x):
    return 1.0 + x + x * x / 2.0 + x ** 3 / 6.0


def test_controller_carries_unclipped_proposal_when_last_trial_was_clipped():
    """Sec. 3 leaves the controller open; the reading keeps the unclipped proposal when the
    last trial was shortened to land on dt and the error would let the step grow (fac >= 1),
    and otherwise carries h_try * fac.  On y' = 0 the error is exactly zero, so fac = 5."""
    zero = np.zeros((2, 2))
    # One trial of exactly dt: not clipped, so the carried proposal is dt * 5.
    y = np.array([1.0, 0.0])
    h = np.zeros(1, dtype=np.float32)
    assert oracle.linear_advance(zero, y, h, 1.0, 1e-4, 1e-3) == (0, 1)
    assert h[0] == 5.0
    # Carried 3/8: the first trial grows the proposal to 15/8; the second is clipped to the
    # 5/8 left and fac = 5 >= 1, so 15/8 is carried (h_try * fac would give 25/8).
    y = np.array([1.0, 0.0])
    h = np.array([0.375], dtype=np.float32)
    assert oracle.linear_advance(zero, y, h, 1.0, 1e-4, 1e-3) == (0, 2)
    assert h[0] == 1.875
    # y' = -y from a carried 1/4 at tol 0.18: trial 1 (x = -1/4) grows h to 1/4 * fac1 > 3/4,
    # so trial 2 is clipped to 3/4; its error lies between 0.729 tol and tol, so it is
    # accepted with fac < 1 and the carried proposal is 3/4 * fac2, not the unclipped h.
    A = np.array([[-1.0, 0.0], [0.0, 0.0]])
    tol = 0.18
    err = [abs(x ** 3 / 6.0) / abs(_taylor3(x)) for x in (-0.25, -0.75)]
    fac = [0.9 * (tol / e) ** (1.0 / 3.0) for e in err]
    assert 0.25 * fac[0] > 0.75 and 0.729 * tol < err[1] <= tol and fac[1] < 1.0
    y = np.array([1.0, 0.0])
    h = np.array([0.25], dtype=np.float32)
    assert oracle.linear_advance(A, y, h, 1.0, tol, 1e-3) == (0, 2)
    assert h[0] == pytest.approx(0.75 * fac[1], rel=1e-7)
    assert y[0] == pytest.approx(_taylor3(-0.25) * _taylor3(-0.75), rel=1e-14)


def test_controller_retries_at_one_fifth_after_a_non_positive_stage():
    """A trial whose stage radius goes non-positive is rejected and retried at 0.2 h_try,
    whatever its error norm allows.  On R' = -R with dt = 1.5 and tol = 100 the Euler stage
    1 - h goes negative for h > 1 while the error (9 at h = 1.5) would allow fac = 2; the
    sequence by hand: reject 1.5 -> accept 0.3 (fac 5) -> reject the clipped 1.2 -> accept
    0.24 (fac 5) -> accept the clipped 0.96 (fac 5 >= 1, so the unclipped 1.2 is carried)."""
    A = np.array([[-1.0, 0.0], [0.0, 0.0]])
    assert 0.9 * (100.0 / 9.0) ** (1.0 / 3.0) > 0.2      # the error alone would not force 0.2
    y = np.array([1.0, 0.0])
    h = np.zeros(1, dtype=np.float32)
    assert oracle.linear_advance(A, y, h, 1.5, 100.0, 1e-3, max_attempts=50) == (0, 5)
    assert y[0] == pytest.approx(_taylor3(-0.3) * _taylor3(-0.24) * _taylor3(-0.96), rel=1e-14)
    assert h[0] == pytest.approx(1.2, rel=1e-7)


# ----------------------------------------------------------------------------
# Whole-path pins: fixed point, linear frequency, Rayleigh collapse, order
# ----------------------------------------------------------------------------
def _single(R0s, R=None, V=None):
    R0s = np.asarray(R0s, dtype=np.float64)
    B = len(R0s)
    Rs = np.array(R0s if R is None else R, dtype=np.float64).reshape(B, 1)
    Vs = np.zeros((B, 1)) if V is None else np.array(V, dtype=np.float64).reshape(B, 1)
    hs = np.zeros((B, 1), dtype=np.float32)
    return Rs, Vs, hs


def test_fixed_point_over_1000_steps_every_bin():
    R0, w = oracle.bins(21, 10e-6, 0.3, 5.0)
    C = 3
    R = np.repeat(R0[:, None], C, axis=1).copy()
    V = np.zeros_like(R)
    h = np.zeros(R.shape, dtype=np.float32)
    p = np.full(C, WATER.p0)
    dt = 1e-8
    for _ in range(1000):
        fl, na = oracle.step(WATER, R0, p, dt, R, V, h)
        assert not fl.any()
    assert np.max(np.abs(R / R0[:, None] - 1)) <= 1e-12
    assert np.max(np.abs(V) / (R0[:, None] / dt)) <= 1e-12


def _linear_km(P, R0):
    pg0 = P.p0 + 2 * P.sigma / R0 - P.pv
    w0sq = (3 * P.gamma * pg0 - 2 * P.sigma / R0) / (P.rho * R0 * R0)
    M = R0 + 4 * P.mu / (P.rho * P.c)
    damp = 4 * P.mu / (P.rho * R0) + R0 * R0 * w0sq / P.c
    beta = damp / (2 * M)
    Om2 = R0 * w0sq / M
    return math.sqrt(w0sq), math.sqrt(Om2 - beta * beta), beta


@pytest.mark.parametrize("R0", [5e-6, 10e-6, 20e-6])
def test_linear_natural_frequency_and_damping(R0):
    """Small oscillation about R0 at p0 follows the linearised KM equation
    (R0 + 4mu/(rho c)) x'' + (4mu/(rho R0) + R0^2 w0^2/c) x' + R0 w0^2 x = 0."""
    w0, wd, beta = _linear_km(WATER, R0)
    if R0 == 10e-6:
        assert w0 / (2 * math.pi) == pytest.approx(345.64e3, rel=1e-4)
    T = 2 * math.pi / wd
    nsamp = 400
    dt = T / nsamp
    R, V, h = _single([R0], R=[R0 * (1 + 1e-5)])
    p = np.array([WATER.p0])
    ts, xs, vs = [0.0], [1e-5], [0.0]
    for n in range(1, 10 * nsamp + 1):
        oracle.step(WATER, [R0], p, dt, R, V, h, n_fixed=16)
        ts.append(n * dt)
        xs.append(R[0, 0] / R0 - 1)
        vs.append(V[0, 0] / R0)
    ts, xs, vs = map(np.array, (ts, xs, vs))
    cross_t, cross_v = [], []
    for i in range(len(xs) - 1):
        if xs[i] == 0 or xs[i] * xs[i + 1] < 0:
            # cubic Hermite root between samples
            t0, t1 = ts[i], ts[i + 1]
            hh = t1 - t0

            def herm(tau):
                s = (tau - t0) / hh
                h00 = 2 * s**3 - 3 * s**2 + 1
                h10 = s**3 - 2 * s**2 + s
                h01 = -2 * s**3 + 3 * s**2
                h11 = s**3 - s**2
                return h00 * xs[i] + h10 * hh * vs[i] + h01 * xs[i + 1] + h11 * hh * vs[i + 1]

            from scipy.optimize import brentq
            tc = brentq(herm, t0, t1, xtol=1e-22)
            cross_t.append(tc)
            cross_v.append(abs(np.interp(tc, ts, vs)))
    cross_t = np.array(cross_t)
    half = np.polyfit(np.arange(len(cross_t)), cross_t, 1)[0]
    wd_meas = math.pi / half
    assert wd_meas == pytest.approx(wd, rel=3e-6)
    # the viscous Rddot kept inside d/dt p_bw shifts wd by ~1.3e-4 relative at 10 um
    beta_meas = -np.polyfit(cross_t, np.log(cross_v), 1)[0]
    assert beta_meas == pytest.approx(beta, rel=2e-3)


@pytest.mark.parametrize("tol,bound", [(1e-4, 3e-5), (1e-6, 1e-6), (1e-8, 2e-8)])
def test_rayleigh_collapse_time(tol, bound):
    """Empty cavity, inviscid, incompressible, no surface tension:
    t(R) = R0 sqrt(3 rho/(2 dp)) int_{R/R0}^1 x^{3/2} (1-x^3)^{-1/2} dx,
    collapse time 0.914681 R0 sqrt(rho/dp)."""
    P = oracle.Params(mu=0.0, sigma=0.0, c=math.inf, gas_mode=1, tol=tol)
    R0 = 10e-6
    dp = P.p0
    tc = math.sqrt(1.5) * special.beta(5 / 6, 0.5) / 3 * R0 * math.sqrt(P.rho / dp)
    assert tc / (R0 * math.sqrt(P.rho / dp)) == pytest.approx(0.915, abs=5e-4)
    nflow = 400
    dt = tc / nflow
    R, V, h = _single([R0])
    p = np.array([P.p0])
    worst = 0.0
    for n in range(1, nflow):
        fl, _ = oracle.step(P, [R0], p, dt, R, V, h)
        assert fl[0, 0] == 0
        x = R[0, 0] / R0
        if n * dt > 0.99 * tc:
            break
        # int_x^1 u^{3/2} (1-u^3)^{-1/2} du = B(5/6, 1/2)/3 * (1 - I_{x^3}(5/6, 1/2))
        integ = special.beta(5 / 6, 0.5) / 3 * special.betaincc(5 / 6, 0.5, x ** 3)
        t_exact = R0 * math.sqrt(1.5 * P.rho / dp) * integ
        worst = max(worst, abs(n * dt - t_exact) / tc)
    assert x < 0.25
    assert worst < bound, worst


def test_rayleigh_integral_closed_form_matches_quadrature():
    x = 0.6
    q, _ = integrate.quad(lambda u: u ** 1.5 / math.sqrt(1 - u ** 3), x, 1.0, limit=200)
    assert special.beta(5 / 6, 0.5) / 3 * special.betaincc(5 / 6, 0.5, x ** 3) == pytest.approx(q, rel=1e-8)


def _forced_run(n_fixed, nsteps=100, dt=1e-8, tol=1e-4):
    P = oracle.Params(tol=tol)
    R0 = np.array([4e-6, 10e-6, 25e-6])
    R, V, h = _single(R0)
    for n in range(nsteps):
        p = np.array([P.p0 * (1 + 0.9 * math.sin(2 * math.pi * 3e5 * (n + 0.5) * dt))])
        oracle.step(P, R0, p, dt, R.reshape(3, 1), V.reshape(3, 1), h.reshape(3, 1),
                    n_fixed=n_fixed)
    return R.ravel().copy(), V.ravel().copy()


def test_fixed_substep_refinement_is_third_order():
    Rref, Vref = _forced_run(512)
    errs = [np.max(np.abs(_forced_run(n)[0] - Rref) / Rref) for n in (1, 2, 4, 8)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    for r in ratios[1:]:
        assert 6.5 < r < 9.5, (errs, ratios)


def test_adaptive_converges_to_fine_fixed_solution():
    Rref, Vref = _forced_run(512)
    e4 = np.max(np.abs(_forced_run(0, tol=1e-4)[0] - Rref) / Rref)
    e8 = np.max(np.abs(_forced_run(0, tol=1e-8)[0] - Rref) / Rref)
    e10 = np.max(np.abs(_forced_run(0, tol=1e-10)[0] - Rref) / Rref)
    assert e8 < e4 and e10 < e8
    assert e10 < 1e-9


# ----------------------------------------------------------------------------
# a6. Moments (Eqs. e:ndf, e:alpha, e:pressure)
# ----------------------------------------------------------------------------
def test_moments_at_equilibrium():
    R0, w = oracle.bins(31, 10e-6, 0.5, 5.0)
    C = 5
    nb = np.array([oracle.equilibrium_nb(a, R0, w) for a in (1e-7, 1e-5, 4e-5, 1e-3, 1e-2)])
    R = np.repeat(R0[:, None], C, axis=1)
    V = np.zeros_like(R)
    out = oracle.moments(WATER, R0, w, nb, R, V)
    np.testing.assert_allclose(out[0], nb, rtol=0)
    np.testing.assert_allclose(out[1], [1e-7, 1e-5, 4e-5, 1e-3, 1e-2], rtol=1e-14)
    np.testing.assert_allclose(out[2], _truncated_lognormal_moment(3, 10e-6, 0.5, 5.0), rtol=1e-4)
    assert np.all(out[3] == 0) and np.all(out[4] == 0) and np.all(out[6] == 0)
    np.testing.assert_allclose(out[5], WATER.p0, rtol=1e-14)


def test_alpha_source_is_time_derivative_of_alpha():
    """With n_b constant, d alpha/dt from Eq. (e:ndf) equals 3 alpha <R^2 Rdot>/<R^3>."""
    P = oracle.Params()
    R0, w = oracle.bins(21, 10e-6, 0.3, 5.0)
    C = 4
    nb = np.full(C, oracle.equilibrium_nb(4e-5, R0, w))
    R = np.repeat(R0[:, None], C, axis=1).copy()
    V = np.zeros_like(R)
    h = np.zeros(R.shape, dtype=np.float32)
    th = np.linspace(0, 2, C)
    dt = 2e-10
    alphas, sources = [], []
    for n in range(400):
        p = P.p0 * (1 + 0.8 * np.sin(2 * math.pi * 2e5 * n * dt + th))
        oracle.step(P, R0, p, dt, R, V, h, n_fixed=4)
        out = oracle.moments(P, R0, w, nb, R, V)
        alphas.append(out[1].copy())
        sources.append(out[4].copy())
    alphas = np.array(alphas)
    sources = np.array(sources)
    dadt = (alphas[2:] - alphas[:-2]) / (2 * dt)
    scale = np.max(np.abs(sources))
    assert scale > 0
    assert np.max(np.abs(dadt - sources[1:-1])) < 2e-3 * scale


def test_moments_single_bin_reduce_to_wall_pressure_and_rdot_squared():
    """B = 1, c -> infinity: <R^3 p_bw>/<R^3> = p_inf + rho (R Rddot + 3/2 Rdot^2) and
    <R^3 Rdot^2>/<R^3> = Rdot^2 for any p_inf (Rayleigh-Plesset balance)."""
    P = oracle.Params(c=math.inf)
    g = np.random.default_rng(3)
    for _ in range(20):
        R0 = g.uniform(3e-6, 30e-6)
        R = R0 * g.uniform(0.5, 2.0)
        V = g.uniform(-10, 10)
        pinf = g.uniform(0.2, 2.0) * P.p0
        out = oracle.moments(P, [R0], [1.0], [1e12], np.array([[R]]), np.array([[V]]))
        _, Rdd, _ = oracle.rhs(P, R0, pinf, R, V)
        assert out[5, 0] == pytest.approx(pinf + P.rho * (R * Rdd + 1.5 * V * V), rel=1e-9)
        assert out[6, 0] == pytest.approx(V * V, rel=1e-14)
        assert out[2, 0] == pytest.approx(R ** 3, rel=1e-14)
        assert out[1, 0] == pytest.approx(4 / 3 * math.pi * 1e12 * R ** 3, rel=1e-14)


def test_moments_brute_force_tiny():
    """Two cells, three bins: each moment equals the weighted sum written out term by term."""
    P = oracle.Params()
    R0 = np.array([5e-6, 10e-6, 20e-6])
    w = np.array([0.2, 0.5, 0.3])
    R = np.array([[5.5e-6, 4e-6], [9e-6, 12e-6], [21e-6, 18e-6]])
    V = np.array([[1.0, -2.0], [0.5, 3.0], [-0.25, 0.0]])
    nb = np.array([1e10, 2e10])
    out = oracle.moments(P, R0, w, nb, R, V)
    for c in range(2):
        terms = [(w[i], R[i, c], V[i, c], oracle.rhs(P, R0[i], 0.0, R[i, c], V[i, c])[2])
                 for i in range(3)]
        m3 = sum(wi * r ** 3 for wi, r, v, pb in terms)
        m2v = sum(wi * r ** 2 * v for wi, r, v, pb in terms)
        m3p = sum(wi * r ** 3 * pb for wi, r, v, pb in terms)
        m3v2 = sum(wi * r ** 3 * v * v for wi, r, v, pb in terms)
        alpha = 4 / 3 * math.pi * nb[c] * m3
        expect = [nb[c], alpha, m3, m2v, 3 * alpha * m2v / m3, m3p / m3, m3v2 / m3]
        np.testing.assert_allclose(out[:, c], expect, rtol=1e-13)


# ----------------------------------------------------------------------------
# a7. Status
# ----------------------------------------------------------------------------
def test_nonfinite_pressure_flags_and_leaves_state():
    R0, w = oracle.bins(3, 10e-6, 0.3, 5.0)
    R = np.repeat(R0[:, None], 2, axis=1).copy()
    V = np.zeros_like(R)
    h = np.zeros(R.shape, dtype=np.float32)
    fl, na = oracle.step(WATER, R0, np.array([np.nan, WATER.p0]), 1e-8, R, V, h)
    assert np.all(fl[:, 0] == oracle.FLAG_NONFINITE) and np.all(fl[:, 1] == 0)
    np.testing.assert_array_equal(R[:, 0], R0)
    assert np.all(na[:, 0] == 0)


def test_workload_generators_are_seeded():
    a = workloads.config_small()
    b = workloads.config_small()
    np.testing.assert_array_equal(a.pressure_step(7), b.pressure_step(7))
    assert a.pressure_step(0).shape == (64,)
    g = workloads.config_grid128(edge=8)
    assert g.theta.shape == (512,)


def test_oracle_matches_its_golden_regression_fixture():
    """Guards the pinned oracle against unnoticed drift (fixture written by
    tests/golden/make_golden.py, which calls only the oracle)."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    stored = {}
    for line in open(os.path.join(here, "oracle_cells8_nb21.txt")):
        if line.startswith("#"):
            continue
        key, *vals = line.split()
        stored[key] = np.array([float(v) for v in vals])
    R, V, attempts, mom = mg.run()
    assert attempts == int(stored["attempts"][0])
    np.testing.assert_allclose(R.ravel(), stored["R"], rtol=1e-13)
    np.testing.assert_allclose(V.ravel(), stored["Rdot"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(mom.ravel(), stored["moments"], rtol=1e-9, atol=1e-20)


# ----------------------------------------------------------------------------
# Carrier-facing forms: conservative variables, mixture pressure, stiffened gas
# ----------------------------------------------------------------------------
def test_conservative_round_trip_recovers_nb_from_alpha():
    """n_b from alpha (Eq. e:ndf) inverts the product n_b R: alpha computed by the
    moments (independent code) and q = n_b R give back n_b, R and Rdot."""
    g = np.random.default_rng(40)
    R0, w = oracle.bins(21, 10e-6, 0.3, 5.0)
    C = 50
    R = R0[:, None] * g.uniform(0.3, 3.0, size=(21, C))
    V = g.normal(size=(21, C))
    nb = g.uniform(1e8, 1e12, size=C)
    alpha = oracle.moments(WATER, R0, w, nb, R, V)[1]
    qR, qV = oracle.cons_from_prim(nb, R, V)
    np.testing.assert_allclose(qR, nb * R, rtol=1e-15)
    R2, V2, nb2 = oracle.prim_from_cons(w, alpha, qR, qV)
    np.testing.assert_allclose(nb2, nb, rtol=1e-14)
    np.testing.assert_allclose(R2, R, rtol=1e-14)
    np.testing.assert_allclose(V2, V, rtol=1e-14, atol=1e-30)


def test_mixture_pressure_limits_and_equilibrium():
    R0, w = oracle.bins(31, 10e-6, 0.5, 5.0)
    C = 4
    alphas = np.array([0.0, 1e-5, 1e-2, 1.0])
    nb = np.array([oracle.equilibrium_nb(max(a, 1e-30), R0, w) for a in alphas])
    R = np.repeat(R0[:, None], C, axis=1)
    V = np.zeros_like(R)
    m = oracle.moments(WATER, R0, w, nb, R, V)
    p_l = np.full(C, 2.5e5)
    p = oracle.mixture_pressure(m, p_l)
    # at rest the bubbles contribute p_bw = p0: p = (1 - alpha) p_l + alpha p0
    np.testing.assert_allclose(p, (1 - m[1]) * p_l + m[1] * WATER.p0, rtol=1e-14)
    assert p[0] == pytest.approx(2.5e5, rel=1e-15)
    np.testing.assert_allclose(oracle.mixture_pressure(m, np.full(C, WATER.p0)), WATER.p0, rtol=1e-14)


def test_mixture_pressure_is_linear_in_the_moments():
    g = np.random.default_rng(41)
    C = 30
    m = g.uniform(0.1, 1.0, size=(7, C))
    m[1] = g.uniform(0, 0.05, size=C)
    m[5] = g.uniform(5e4, 2e5, size=C)
    m[6] = g.uniform(0, 100, size=C)
    p_l = g.uniform(5e4, 3e5, size=C)
    rho = g.uniform(900, 1100, size=C)
    p = oracle.mixture_pressure(m, p_l, rho)
    a = m[1]
    expect = p_l - a * p_l + a * m[5] - a * rho * m[6]
    np.testing.assert_allclose(p, expect, rtol=1e-12)


def test_stiffened_gas_inverts_its_energy():
    """e_l = (p_l + gamma_l pi_inf) / ((gamma_l - 1) rho_l) gives back p_l."""
    g = np.random.default_rng(42)
    gam, pinf = 6.12, 3.43e8
    p_l = g.uniform(-5e4, 5e6, size=100)
    rho = g.uniform(950, 1050, size=100)
    e = (p_l + gam * pinf) / ((gam - 1.0) * rho)
    np.testing.assert_allclose(oracle.stiffened_gas(rho, e, gam, pinf), p_l, rtol=0, atol=1e-6 * gam * pinf * 1e-3)


# ----------------------------------------------------------------------------
# Volume-averaged (EL) model: Gaussian smearing, Eq. (kernel3D)
# ----------------------------------------------------------------------------
def test_el_smear_single_bubble_closed_forms():
    """One bubble at a cell centre with R < dx (h = dx): the centre value is
    V/(h^3 (2 pi)^{3/2}); values at equal distance agree; cells at d >= 3h get
    nothing; the grid sum equals V/(2 pi)^{3/2} times the lattice sum of
    exp(-|m|^2/2) over integer vectors with |m| < 3."""
    dx = 75e-6
    n = 9
    pos = np.array([[4.5 * dx], [4.5 * dx], [4.5 * dx]])
    R = np.array([10e-6])
    V = 4 / 3 * math.pi * R[0] ** 3
    a, ad = oracle.el_smear(pos, R, np.array([2.0]), n, n, n, dx)
    a = a.reshape(n, n, n)
    norm = (2 * math.pi) ** 1.5
    assert a[4, 4, 4] == pytest.approx(V / (dx ** 3 * norm), rel=1e-14)
    assert a[4, 4, 5] == pytest.approx(a[4, 5, 4], rel=1e-14) == pytest.approx(a[3, 4, 4], rel=1e-14)
    assert a[4, 4, 5] / a[4, 4, 4] == pytest.approx(math.exp(-0.5), rel=1e-13)
    assert a[4, 4, 7] == 0.0 and a[4, 4, 1] == 0.0            # d = 3h exactly: outside
    assert a[4, 6, 6] > 0                                       # d = 2.83 h: inside
    lattice = sum(math.exp(-(i * i + j * j + k * k) / 2.0)
                  for i in range(-3, 4) for j in range(-3, 4) for k in range(-3, 4)
                  if i * i + j * j + k * k < 9)
    assert a.sum() * dx ** 3 == pytest.approx(V * lattice / norm, rel=1e-13)
    # the growth rate uses 4 pi R^2 Rdot in place of V
    np.testing.assert_allclose(ad.reshape(n, n, n), a * (4 * math.pi * R[0] ** 2 * 2.0) / V, rtol=1e-13)


def test_el_smear_width_follows_radius_and_superposes():
    """h = max(dx, R): a bubble larger than the cell spreads over 3 R; two bubbles add."""
    dx = 50e-6
    n = 16
    big = np.array([[8 * dx], [8 * dx], [8 * dx]])
    a = oracle.el_smear(big, np.array([80e-6]), np.array([0.0]), n, n, n, dx, with_rate=False)
    a = a.reshape(n, n, n)
    h = 80e-6
    d = math.sqrt(3) * 0.5 * dx                                 # nearest cell centres
    assert a[8, 8, 8] == pytest.approx(4 / 3 * math.pi * h ** 3 * math.exp(-d * d / (2 * h * h))
                                       / (h ** 3 * (2 * math.pi) ** 1.5), rel=1e-13)
    assert a[8, 8, 8 + 4] > 0                                   # 3.5 dx < 3 h = 4.8 dx
    g = np.random.default_rng(43)
    pos = g.uniform(0, n * dx, size=(3, 5))
    Rs = g.uniform(5e-6, 60e-6, size=5)
    Vd = g.normal(size=5)
    tot = oracle.el_smear(pos, Rs, Vd, n, n, n, dx)[0]
    parts = sum(oracle.el_smear(pos[:, i:i + 1], Rs[i:i + 1], Vd[i:i + 1], n, n, n, dx)[0] for i in range(5))
    np.testing.assert_allclose(tot, parts, rtol=1e-13, atol=1e-30)


def test_el_advance_matches_ee_bins_with_the_same_pressure():
    """A Lagrangian bubble follows the same Keller-Miksis stepper as an EE bin
    of the same R0 under the same pressure."""
    P = oracle.Params()
    g = np.random.default_rng(44)
    N = 6
    R0 = g.uniform(3e-6, 30e-6, size=N)
    p_cell = np.array([P.p0 * 1.3, P.p0 * 0.6])
    cell = np.array([0, 1, 0, 1, 0, 1])
    R = R0.copy()
    V = np.zeros(N)
    h = np.zeros(N, dtype=np.float32)
    for _ in range(50):
        fl, na = oracle.el_advance(P, R0, cell, p_cell, 1e-8, R, V, h)
        assert not fl.any()
    for n in range(N):
        Rb = np.array([[R0[n]]])
        Vb = np.zeros((1, 1))
        hb = np.zeros((1, 1), dtype=np.float32)
        for _ in range(50):
            oracle.step(P, [R0[n]], [p_cell[cell[n]]], 1e-8, Rb, Vb, hb)
        assert R[n] == Rb[0, 0] and V[n] == Vb[0, 0]
