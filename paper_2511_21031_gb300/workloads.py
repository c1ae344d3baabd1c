"""Seeded synthetic inputs for the bubble source update.

This module holds no arithmetic of the method: it draws the per-cell forcing
parameters and evaluates the synthetic carrier pressure field that stands in for
the flow solver, and it describes the workload sizes.  The same generators feed
the CUDA library and the oracle, so both see identical inputs.

Water throughout (rho = 1000, c = 1500, mu = 1e-3, sigma = 0.072, p0 = 101325,
gamma = 1.4, p_v = 0), bins centred at R0ref = 10 um with span +-5 s, initial
void fraction 4e-5 (the bubble-screen case of Sec. 5.1), equilibrium start.

Forcing: p_c(t) = p0 + a p0 sin(2 pi f t + theta_c) sampled at the mid-point of
each flow step (the carrier is frozen during the bubble half of the Strang
split, Sec. 3).  Per-cell phases theta_c:
  - "random phase": theta_c ~ U[0, 2 pi);
  - "plane wave": theta_c = -k x_c + d_c with k = 2 pi f / c, x_c the cell
    centre along x over one wavelength, d_c ~ U(-0.05 * 2 pi, 0.05 * 2 pi).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

WATER = dict(rho=1000.0, c=1500.0, mu=1e-3, sigma=0.072, p0=101325.0, gamma=1.4, pv=0.0)


@dataclasses.dataclass
class Workload:
    name: str
    n_cells: int
    n_bins: int
    s: float
    dt: float
    n_steps: int
    amp: float           # forcing amplitude in units of p0
    freq: float          # forcing frequency [Hz]
    theta_spec: tuple    # ("random", seed) | ("plane", nx, ny, nz, seed) | ("given", array)
    R0ref: float = 10e-6
    span_K: float = 5.0
    alpha0: float = 4e-5
    seed: int = 0
    precision: str = "fp64"
    fluid: dict = dataclasses.field(default_factory=lambda: dict(WATER))

    @property
    def bins_total(self) -> int:
        return self.n_cells * self.n_bins

    @property
    def theta(self) -> np.ndarray:
        """Per-cell forcing phase [n_cells] (drawn on first use)."""
        th = self.__dict__.get("_theta")
        if th is None:
            kind = self.theta_spec[0]
            if kind == "random":
                th = random_phase(self.n_cells, self.theta_spec[1])
            elif kind == "plane":
                _, nx, ny, nz, sd = self.theta_spec
                th = plane_wave_phase(nx, ny, nz, self.freq, self.fluid["c"], sd)
            else:
                th = np.ascontiguousarray(self.theta_spec[1], dtype=np.float64)
            if th.shape != (self.n_cells,):
                raise ValueError("phase array does not match n_cells")
            self.__dict__["_theta"] = th
        return th

    def pressure_at(self, t: float, xp=np, device=None):
        """Carrier pressure [n_cells] at time t (xp = numpy or torch)."""
        p0 = self.fluid["p0"]
        w = 2.0 * math.pi * self.freq
        if xp is np:
            return p0 + self.amp * p0 * np.sin(w * t + self.theta)
        th = self.theta_device(xp, device)
        return p0 + self.amp * p0 * xp.sin(th + w * t)

    def theta_device(self, torch, device):
        key = (str(device),)
        cache = self.__dict__.setdefault("_theta_cache", {})
        if key not in cache:
            cache[key] = torch.as_tensor(self.theta, dtype=torch.float64, device=device)
        return cache[key]

    def pressure_step(self, n: int, xp=np, device=None):
        """Pressure for flow step n, sampled at t_n + dt/2."""
        return self.pressure_at((n + 0.5) * self.dt, xp=xp, device=device)

    def subset(self, cells: np.ndarray, name: Optional[str] = None) -> "Workload":
        """The same workload restricted to the given cell indices."""
        th = np.ascontiguousarray(self.theta[np.asarray(cells)])
        return dataclasses.replace(self, name=name or f"{self.name}[sample {len(cells)}]",
                                   n_cells=int(len(cells)), theta_spec=("given", th))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_phase(n_cells: int, seed: int) -> np.ndarray:
    return _rng(seed).uniform(0.0, 2.0 * math.pi, size=n_cells)


def plane_wave_phase(nx: int, ny: int, nz: int, freq: float, c: float, seed: int,
                     jitter: float = 0.05) -> np.ndarray:
    """theta for a plane wave along x over one wavelength, x fastest in memory."""
    k = 2.0 * math.pi * freq / c
    lam = c / freq
    dx = lam / nx
    x = (np.arange(nx) + 0.5) * dx
    base = np.broadcast_to(-k * x, (nz, ny, nx)).reshape(-1)
    d = _rng(seed).uniform(-jitter * 2.0 * math.pi, jitter * 2.0 * math.pi, size=nx * ny * nz)
    return np.ascontiguousarray(base + d)


def config_small(seed: int = 1) -> Workload:
    """64 cells x Nb = 21 (s = 0.3), 0.5 p0 at 100 kHz with random phases, 1000 x 1e-8 s."""
    return Workload("cells64_nb21_fp64", 64, 21, 0.3, 1e-8, 1000, 0.5, 1e5,
                    ("random", seed), seed=seed)


def config_grid128(seed: int = 2, edge: int = 128) -> Workload:
    """edge^3 cells x Nb = 31 (s = 0.5), 1.2 p0 plane wave at 100 kHz + 5 % phase jitter, 500 x 5e-9 s."""
    return Workload(f"grid{edge}^3_nb31_fp64", edge ** 3, 31, 0.5, 5e-9, 500, 1.2, 1e5,
                    ("plane", edge, edge, edge, seed), seed=seed)


def config_grid256_mixed(seed: int = 3, edge: int = 256) -> Workload:
    """edge^3 cells x Nb = 31 (s = 0.5), config-small forcing, 1000 x 1e-8 s, mixed precision."""
    n = edge ** 3
    return Workload(f"grid{edge}^3_nb31_mixed", n, 31, 0.5, 1e-8, 1000, 0.5, 1e5,
                    ("random", seed), seed=seed, precision="mixed")


def config_collapse(seed: int = 5, edge: int = 64, n_steps: int = 10000) -> Workload:
    """Collapse-stress variant: 1.2 p0 at 21.4 kHz plane wave, 5e-9 s steps."""
    return Workload(f"grid{edge}^3_nb31_collapse", edge ** 3, 31, 0.5, 5e-9, n_steps, 1.2, 21.4e3,
                    ("plane", edge, edge, edge, seed), seed=seed)


def batched_instances(n: int = 512, seed: int = 4, edge_lo: int = 16, edge_hi: int = 96,
                      nb_choices=(11, 21, 31, 51), n_steps: int = 200) -> List[Workload]:
    """Independent instances of uneven size, Nb, amplitude and distribution width."""
    g = _rng(seed)
    out = []
    for i in range(n):
        L = int(g.integers(edge_lo, edge_hi + 1))
        nb = int(g.choice(nb_choices))
        amp = float(g.uniform(0.3, 1.5))
        s = float(g.uniform(0.2, 0.7))
        sd = seed * 100003 + i
        out.append(Workload(f"inst{i}_L{L}_nb{nb}", L ** 3, nb, s, 1e-8, n_steps, amp, 1e5,
                            ("random", sd), seed=sd, precision="mixed"))
    return out


def sliced_instances(wl: Workload, n: int, precision: str = "mixed") -> List[Workload]:
    """The workload's cells cut into n contiguous, equal instances (the same forcing, bins and
    steps): a batch of them does exactly the single instance's work."""
    if n <= 0 or wl.n_cells % n:
        raise ValueError("n must divide the workload's cell count")
    m = wl.n_cells // n
    return [dataclasses.replace(wl.subset(np.arange(i * m, (i + 1) * m), name=f"{wl.name}[slice {i}]"),
                                precision=precision) for i in range(n)]


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float   # seconds from stream start
    work: Workload


def request_stream(n: int = 2000, rate: float = 200.0, seed: int = 6, n_steps: int = 200,
                   edge_lo: int = 32, edge_hi: int = 192, edge_median: float = 78.4) -> List[Request]:
    """Poisson arrivals; edge L lognormal (median 78.4, log-sd ln6/4) clipped; Nb in {21, 31}."""
    g = _rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(g.exponential(1.0 / rate))
        L = int(round(math.exp(g.normal(math.log(edge_median), math.log(6.0) / 4.0))))
        L = min(max(L, edge_lo), edge_hi)
        nb = int(g.choice((21, 31)))
        sd = seed * 100003 + i
        out.append(Request(i, t, Workload(f"req{i}_L{L}_nb{nb}", L ** 3, nb, 0.3, 1e-8, n_steps, 0.5,
                                          1e5, ("random", sd), seed=sd, precision="mixed")))
    return out


@dataclasses.dataclass
class BubbleCloud:
    """Volume-averaged (EL) workload: fixed bubbles on a grid, forced cell by cell."""
    name: str
    edge: int
    dx: float
    pos: np.ndarray      # [3][N]
    R0: np.ndarray       # [N]
    theta: np.ndarray    # per-cell forcing phase [edge^3]
    amp: float = 0.5
    freq: float = 1e5
    dt: float = 1e-8
    n_steps: int = 100
    fluid: dict = dataclasses.field(default_factory=lambda: dict(WATER))

    @property
    def n_bubbles(self) -> int:
        return int(self.R0.shape[0])

    def pressure_step(self, n: int, xp=np, device=None):
        p0 = self.fluid["p0"]
        w = 2.0 * math.pi * self.freq
        t = (n + 0.5) * self.dt
        if xp is np:
            return p0 + self.amp * p0 * np.sin(w * t + self.theta)
        th = self.__dict__.setdefault("_th_dev", xp.as_tensor(self.theta, device=device))
        return p0 + self.amp * p0 * xp.sin(th + w * t)


def bubble_cloud(edge: int = 128, dx: float = 75e-6, alpha0: float = 1e-3, R0ref: float = 10e-6,
                 s: float = 0.0, seed: int = 7, n_steps: int = 100) -> BubbleCloud:
    """Bubbles placed uniformly in an edge^3 grid of cells dx (the cost test of Sec. 5.2:
    75 um cells, R0 = 10 um); their number gives void fraction alpha0; s > 0 draws
    lognormal radii (median R0ref), s = 0 is monodisperse."""
    g = _rng(seed)
    L = edge * dx
    n = int(round(alpha0 * L ** 3 / (4.0 / 3.0 * math.pi * R0ref ** 3)))
    pos = g.uniform(0.0, L, size=(3, n))
    R0 = R0ref * np.exp(s * g.normal(size=n)) if s > 0 else np.full(n, R0ref)
    th = g.uniform(0.0, 2.0 * math.pi, size=edge ** 3)
    return BubbleCloud(f"el_cloud{edge}^3_a{alpha0:g}", edge, dx, np.ascontiguousarray(pos), R0, th,
                       n_steps=n_steps)
