"""The synthetic inputs match their stated recipe (sizes, ranges and distributions), on the CPU.

Every GPU parity test, smoke check and bench line draws its inputs from these generators, and
the oracle sees the same arrays; this checks the recipe itself: the water constants, the
forcing p_c(t) = p0 + a p0 sin(2 pi f t + theta_c) sampled at mid-step, the plane wave's phase
along x over one wavelength with its 5 % jitter, the batched instances' ranges, and the request
stream's Poisson arrivals and clipped lognormal edges."""
import math

import numpy as np
import pytest

from paper_2511_21031_gb300 import workloads


def test_water_and_paper_defaults():
    assert workloads.WATER == dict(rho=1000.0, c=1500.0, mu=1e-3, sigma=0.072, p0=101325.0, gamma=1.4,
                                   pv=0.0)
    w = workloads.config_small()
    assert (w.R0ref, w.span_K, w.alpha0) == (10e-6, 5.0, 4e-5)


@pytest.mark.parametrize("make,cells,nb,s,dt,steps,amp,freq", [
    (lambda: workloads.config_small(), 64, 21, 0.3, 1e-8, 1000, 0.5, 1e5),
    (lambda: workloads.config_grid128(edge=16), 16 ** 3, 31, 0.5, 5e-9, 500, 1.2, 1e5),
    (lambda: workloads.config_grid256_mixed(edge=16), 16 ** 3, 31, 0.5, 1e-8, 1000, 0.5, 1e5),
    (lambda: workloads.config_collapse(edge=16), 16 ** 3, 31, 0.5, 5e-9, 10000, 1.2, 21.4e3),
])
def test_configs_and_their_forcing(make, cells, nb, s, dt, steps, amp, freq):
    w = make()
    assert (w.n_cells, w.n_bins, w.s, w.dt, w.n_steps, w.amp, w.freq) == (cells, nb, s, dt, steps, amp, freq)
    p0 = w.fluid["p0"]
    for n in (0, 3, steps - 1):
        t = (n + 0.5) * dt
        expect = p0 * (1.0 + amp * np.sin(2.0 * math.pi * freq * t + w.theta))
        # absolute, on the scale of p0: with a > 1 the pressure passes through zero
        np.testing.assert_allclose(w.pressure_step(n), expect, rtol=0.0, atol=1e-14 * p0)
    p = w.pressure_step(1)
    assert p.min() >= p0 * (1.0 - amp) - 1e-6 and p.max() <= p0 * (1.0 + amp) + 1e-6


def test_random_phase_is_uniform_on_the_circle():
    th = workloads.random_phase(200_000, seed=9)
    assert th.min() >= 0.0 and th.max() < 2.0 * math.pi
    hist, _ = np.histogram(th, bins=20, range=(0.0, 2.0 * math.pi))
    assert np.all(np.abs(hist / 10_000 - 1.0) < 0.05)


def test_plane_wave_phase_runs_one_wavelength_along_x_with_jitter():
    nx, ny, nz, f, c = 32, 4, 3, 1e5, 1500.0
    th = workloads.plane_wave_phase(nx, ny, nz, f, c, seed=3).reshape(nz, ny, nx)
    k = 2.0 * math.pi * f / c
    dx = (c / f) / nx
    base = -k * (np.arange(nx) + 0.5) * dx
    jit = th - base[None, None, :]
    assert np.all(np.abs(jit) <= 0.05 * 2.0 * math.pi)
    assert np.std(jit) > 0.05 * 2.0 * math.pi / 3.0        # the jitter is there, uniform-sized
    assert base[0] - base[-1] == pytest.approx(2.0 * math.pi * (nx - 1) / nx)


def test_batched_instances_span_their_ranges():
    insts = workloads.batched_instances(n=512)
    edges = np.array([round(w.n_cells ** (1 / 3)) for w in insts])
    assert np.all(edges ** 3 == [w.n_cells for w in insts])
    assert edges.min() >= 16 and edges.max() <= 96 and edges.min() < 24 and edges.max() > 88
    assert {w.n_bins for w in insts} == {11, 21, 31, 51}
    amps = np.array([w.amp for w in insts])
    ss = np.array([w.s for w in insts])
    assert amps.min() >= 0.3 and amps.max() <= 1.5 and ss.min() >= 0.2 and ss.max() <= 0.7
    assert all(w.precision == "mixed" and w.dt == 1e-8 and w.freq == 1e5 for w in insts)
    bins = sum(w.n_cells * w.n_bins for w in insts)
    assert 3e9 < bins < 6e9                                    # the benchmark's few-1e9 bin-states
    assert len({w.seed for w in insts}) == len(insts)


def test_sliced_instances_cover_the_workload_in_order():
    wl = workloads.config_grid128(edge=16)
    insts = workloads.sliced_instances(wl, 8)
    assert len(insts) == 8 and all(w.n_cells == 512 for w in insts)
    assert np.array_equal(np.concatenate([w.theta for w in insts]), wl.theta)
    assert all(w.precision == "mixed" and (w.n_bins, w.s, w.dt, w.amp, w.freq)
               == (wl.n_bins, wl.s, wl.dt, wl.amp, wl.freq) for w in insts)
    with pytest.raises(ValueError):
        workloads.sliced_instances(wl, 7)


def test_request_stream_is_poisson_with_clipped_lognormal_edges():
    reqs = workloads.request_stream(n=4000, rate=200.0)
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0.0)
    assert gaps.mean() == pytest.approx(1.0 / 200.0, rel=0.05)
    assert gaps.std() == pytest.approx(1.0 / 200.0, rel=0.08)   # exponential: sd = mean
    edges = np.array([round(r.work.n_cells ** (1 / 3)) for r in reqs])
    assert edges.min() >= 32 and edges.max() <= 192
    inner = edges[(edges > 32) & (edges < 192)]
    assert np.median(edges) == pytest.approx(78.4, abs=3)
    assert np.std(np.log(inner)) == pytest.approx(math.log(6.0) / 4.0, rel=0.15)
    assert {r.work.n_bins for r in reqs} == {21, 31}
    assert all(r.work.s == 0.3 and r.work.amp == 0.5 and r.work.n_steps == 200 for r in reqs)
