"""FP64 CPU oracle of the ensemble-averaged bubble-dynamics source update.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()``, and the
CPU-baseline leg and the ``--impl reference`` arm of ``bench.py`` may import this package; the product path
(``paper_2511_21031_gb300``) never does, and this package never imports it.

This module only marshals numpy arrays into the plain C oracle
(``pab_oracle.c``), which holds all of the arithmetic; see that file for the
paper passages each function follows.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pab_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

FLAG_STEP_LIMIT = 1
FLAG_NONFINITE = 2
FLAG_SUPERSONIC = 4
FLAG_NONPOS = 8


CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
          "-D_GNU_SOURCE"]


def compile_to(src: str, out: str) -> str:
    """Compile an oracle source file to a shared library (FP64, no FMA contraction, no fast-math)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle in place when missing or older than its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_to(_SRC, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("c", ctypes.c_double), ("mu", ctypes.c_double),
                ("sigma", ctypes.c_double), ("p0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("pv", ctypes.c_double), ("gas_mode", ctypes.c_int32),
                ("max_attempts", ctypes.c_int32), ("tol", ctypes.c_double),
                ("v_floor", ctypes.c_double)]


@dataclasses.dataclass
class Params:
    """Liquid, gas and stepper constants (SI units). Defaults: water, Sec. 5."""
    rho: float = 1000.0
    c: float = 1500.0
    mu: float = 1e-3
    sigma: float = 0.072
    p0: float = 101325.0
    gamma: float = 1.4
    pv: float = 0.0
    gas_mode: int = 0
    max_attempts: int = 100000
    tol: float = 1e-4
    v_floor: float = -1.0  # < 0: 1e-3 * sqrt(p0 / rho)

    def as_c(self) -> _Params:
        vf = self.v_floor if self.v_floor >= 0 else 1e-3 * math.sqrt(self.p0 / self.rho)
        return _Params(self.rho, self.c, self.mu, self.sigma, self.p0, self.gamma, self.pv,
                       int(self.gas_mode), int(self.max_attempts), self.tol, vf)


class _Transfer(ctypes.Structure):
    _fields_ = [("R_g", ctypes.c_double), ("R_v", ctypes.c_double), ("T_w", ctypes.c_double),
                ("k_bw", ctypes.c_double), ("D", ctypes.c_double), ("beta_T", ctypes.c_double),
                ("beta_c", ctypes.c_double)]


@dataclasses.dataclass
class Transfer:
    """Gas/vapour contents with constant wall transfer coefficients (SI units).
    Defaults: air and water vapour at 20 C; beta_T and beta_c are inputs."""
    R_g: float = 287.05
    R_v: float = 461.5
    T_w: float = 293.15
    k_bw: float = 0.0257
    D: float = 2.42e-5
    beta_T: float = 5.0
    beta_c: float = 5.0

    def as_c(self) -> _Transfer:
        return _Transfer(self.R_g, self.R_v, self.T_w, self.k_bw, self.D, self.beta_T, self.beta_c)


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_ldp = ctypes.POINTER(ctypes.c_longdouble)


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            # PAB_ORACLE_LIB: a compiled copy of this oracle with one planted mistake,
            # used only by tests/test_oracle_mutations.py to show the pins catch it
            alt = os.environ.get("PAB_ORACLE_LIB")
            lib = ctypes.CDLL(alt if alt else build())
            P = ctypes.POINTER(_Params)
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = ctypes.c_int
            lib.orc_bins.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _dp, _dp]
            lib.orc_bins.restype = ctypes.c_int
            lib.orc_rhs.argtypes = [P, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            lib.orc_rhs.restype = None
            lib.orc_step.argtypes = [P, ctypes.c_int64, ctypes.c_int32, _dp, _dp, ctypes.c_double,
                                     ctypes.c_int32, _dp, _dp, _fp, _u32p, _i32p]
            lib.orc_step.restype = None
            lib.orc_moments.argtypes = [P, ctypes.c_int64, ctypes.c_int32, _dp, _dp, _dp, _dp,
                                        _dp, _dp, _ldp]
            lib.orc_moments.restype = None
            lib.orc_error_norm.argtypes = [_dp, _dp, ctypes.c_double]
            lib.orc_error_norm.restype = ctypes.c_double
            lib.orc_step_factor.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_step_factor.restype = ctypes.c_double
            lib.orc_linear_trial.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp]
            lib.orc_linear_trial.restype = None
            lib.orc_linear_advance.argtypes = [_dp, _dp, _fp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int32, _i32p]
            lib.orc_linear_advance.restype = ctypes.c_uint32
            lib.orc_cons_from_prim.argtypes = [ctypes.c_int64, ctypes.c_int32, _dp, _dp, _dp, _dp, _dp]
            lib.orc_cons_from_prim.restype = None
            lib.orc_prim_from_cons.argtypes = [ctypes.c_int64, ctypes.c_int32, _dp, _dp, _dp, _dp,
                                               _dp, _dp, _dp]
            lib.orc_prim_from_cons.restype = None
            lib.orc_mixture_pressure.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, _dp]
            lib.orc_mixture_pressure.restype = None
            lib.orc_stiffened_gas.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double,
                                              ctypes.c_double, _dp]
            lib.orc_stiffened_gas.restype = None
            _i64p = ctypes.POINTER(ctypes.c_int64)
            lib.orc_el_advance.argtypes = [P, ctypes.c_int64, _dp, _i64p, _dp, ctypes.c_double, _dp, _dp,
                                           _fp, _u32p, _i32p]
            lib.orc_el_advance.restype = None
            lib.orc_el_smear.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_double, _dp, _dp]
            lib.orc_el_smear.restype = None
            T = ctypes.POINTER(_Transfer)
            lib.orc_transfer_gas_mass.argtypes = [P, T, ctypes.c_double]
            lib.orc_transfer_gas_mass.restype = ctypes.c_double
            lib.orc_transfer_init.argtypes = [P, T, ctypes.c_double, _dp]
            lib.orc_transfer_init.restype = None
            lib.orc_transfer_rates.argtypes = [P, T, ctypes.c_double, _dp, _dp, _dp]
            lib.orc_transfer_rates.restype = None
            lib.orc_transfer_rhs.argtypes = [P, T, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            lib.orc_transfer_rhs.restype = None
            lib.orc_transfer_step.argtypes = [P, T, ctypes.c_int64, ctypes.c_int32, _dp, _dp,
                                              ctypes.c_double, ctypes.c_int32, _dp, _dp, _dp, _dp,
                                              _fp, _u32p, _i32p]
            lib.orc_transfer_step.restype = None
            lib.orc_transfer_moments.argtypes = [P, ctypes.c_int64, ctypes.c_int32, _dp, _dp, _dp,
                                                 _dp, _dp, _dp]
            lib.orc_transfer_moments.restype = None
            _LIB = lib
    return _LIB


def _ptr(a, typ):
    return a.ctypes.data_as(typ)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    """Threads the oracle's OpenMP loops run with."""
    return int(_lib().orc_max_threads())


def bins(n_bins: int, R0ref: float = 10e-6, s: float = 0.3, K: float = 5.0):
    """Lognormal bin table (R0_i, w_i) with Simpson weights normalised to one."""
    R0 = np.zeros(n_bins)
    w = np.zeros(n_bins)
    rc = _lib().orc_bins(int(n_bins), R0ref, s, K, _ptr(R0, _dp), _ptr(w, _dp))
    if rc != 0:
        raise ValueError(f"invalid bin request: n_bins={n_bins} s={s} K={K}")
    return R0, w


def rhs(params: Params, R0: float, p_inf: float, R: float, Rdot: float):
    """Keller-Miksis right-hand side: returns (Rdot, Rddot, p_bw)."""
    y = np.array([R, Rdot], dtype=np.float64)
    f = np.zeros(2)
    pbw = np.zeros(1)
    cp = params.as_c()
    _lib().orc_rhs(ctypes.byref(cp), R0, p_inf, _ptr(y, _dp), _ptr(f, _dp), _ptr(pbw, _dp))
    return float(f[0]), float(f[1]), float(pbw[0])


def step(params: Params, R0, p_inf, dt, R, Rdot, h, n_fixed: int = 0):
    """Advance [B][C] state in place over one flow step; returns (flags, attempts)."""
    R0 = _f64(R0)
    p_inf = _f64(p_inf)
    B = R0.shape[0]
    C = p_inf.shape[0]
    for a, dt_ in ((R, np.float64), (Rdot, np.float64), (h, np.float32)):
        if a.dtype != dt_ or not a.flags.c_contiguous or a.size != B * C:
            raise ValueError("state arrays must be contiguous [B][C] (R, Rdot f64; h f32)")
    flags = np.zeros((B, C), dtype=np.uint32)
    attempts = np.zeros((B, C), dtype=np.int32)
    cp = params.as_c()
    _lib().orc_step(ctypes.byref(cp), C, B, _ptr(R0, _dp), _ptr(p_inf, _dp), float(dt),
                    int(n_fixed), _ptr(R, _dp), _ptr(Rdot, _dp), _ptr(h, _fp),
                    _ptr(flags, _u32p), _ptr(attempts, _i32p))
    return flags, attempts


def moments(params: Params, R0, w, n_b, R, Rdot, with_long_double: bool = False):
    """[7][C] moments (n_b, alpha, <R^3>, <R^2 Rdot>, S_alpha, <R^3 p_bw>/<R^3>, <R^3 Rdot^2>/<R^3>)."""
    R0 = _f64(R0)
    w = _f64(w)
    n_b = _f64(n_b)
    R = _f64(R)
    Rdot = _f64(Rdot)
    B = R0.shape[0]
    C = n_b.shape[0]
    out = np.zeros((7, C))
    ald = np.zeros(C, dtype=np.longdouble) if with_long_double else None
    cp = params.as_c()
    _lib().orc_moments(ctypes.byref(cp), C, B, _ptr(R0, _dp), _ptr(w, _dp), _ptr(n_b, _dp),
                       _ptr(R, _dp), _ptr(Rdot, _dp), _ptr(out, _dp),
                       _ptr(ald, _ldp) if ald is not None else None)
    if with_long_double:
        return out, ald
    return out


def error_norm(y3, z, v_floor):
    y3 = _f64(y3)
    z = _f64(z)
    return float(_lib().orc_error_norm(_ptr(y3, _dp), _ptr(z, _dp), v_floor))


def step_factor(err, tol):
    return float(_lib().orc_step_factor(err, tol))


def linear_trial(A, y, h):
    A = _f64(A).reshape(4)
    y = _f64(y)
    y3 = np.zeros(2)
    z = np.zeros(2)
    _lib().orc_linear_trial(_ptr(A, _dp), _ptr(y, _dp), h, _ptr(y3, _dp), _ptr(z, _dp))
    return y3, z


def linear_advance(A, y, h, dt, tol, v_floor, max_attempts=100000):
    """Adaptive driver on y' = A y; y (2,) f64 and h (1,) f32 updated in place."""
    A = _f64(A).reshape(4)
    na = np.zeros(1, dtype=np.int32)
    fl = _lib().orc_linear_advance(_ptr(A, _dp), _ptr(y, _dp), _ptr(h, _fp), dt, tol, v_floor,
                                   int(max_attempts), _ptr(na, _i32p))
    return int(fl), int(na[0])


def equilibrium_nb(alpha0: float, R0, w) -> float:
    """n_b from the initial void fraction at the equilibrium state (Eq. e:ndf)."""
    return alpha0 / (4.0 / 3.0 * math.pi * float(np.dot(_f64(w), _f64(R0) ** 3)))


def cons_from_prim(n_b, R, Rdot):
    """Conservative bubble variables qR = n_b R, qV = n_b Rdot ([B][C])."""
    n_b = _f64(n_b)
    R = _f64(R)
    Rdot = _f64(Rdot)
    B, C = R.shape
    qR = np.zeros_like(R)
    qV = np.zeros_like(R)
    _lib().orc_cons_from_prim(C, B, _ptr(n_b, _dp), _ptr(R, _dp), _ptr(Rdot, _dp), _ptr(qR, _dp),
                              _ptr(qV, _dp))
    return qR, qV


def prim_from_cons(w, alpha, qR, qV):
    """Primitive R, Rdot and n_b from alpha and the conservative variables (Eq. e:ndf)."""
    w = _f64(w)
    alpha = _f64(alpha)
    qR = _f64(qR)
    qV = _f64(qV)
    B, C = qR.shape
    R = np.zeros_like(qR)
    V = np.zeros_like(qR)
    nb = np.zeros(C)
    _lib().orc_prim_from_cons(C, B, _ptr(w, _dp), _ptr(alpha, _dp), _ptr(qR, _dp), _ptr(qV, _dp),
                              _ptr(R, _dp), _ptr(V, _dp), _ptr(nb, _dp))
    return R, V, nb


def mixture_pressure(moments, p_l, rho_l=None, rho_default=1000.0):
    """Mixture pressure of Eq. (e:pressure) from the [7][C] moments and p_l [C]."""
    moments = _f64(moments)
    p_l = _f64(p_l)
    C = p_l.shape[0]
    out = np.zeros(C)
    rl = _f64(rho_l) if rho_l is not None else None
    _lib().orc_mixture_pressure(C, _ptr(moments, _dp), _ptr(p_l, _dp),
                                _ptr(rl, _dp) if rl is not None else None, float(rho_default),
                                _ptr(out, _dp))
    return out


def stiffened_gas(rho_l, e_l, gamma_l, pi_inf):
    """Liquid pressure of the stiffened-gas EOS, Eq. (eos_liquid)."""
    rho_l = _f64(rho_l)
    e_l = _f64(e_l)
    out = np.zeros_like(rho_l)
    _lib().orc_stiffened_gas(rho_l.size, _ptr(rho_l, _dp), _ptr(e_l, _dp), float(gamma_l),
                             float(pi_inf), _ptr(out, _dp))
    return out


def el_advance(params: Params, R0, cell, p_cell, dt, R, Rdot, h):
    """Advance N Lagrangian bubbles in place (each under its cell's pressure); returns (flags, attempts)."""
    R0 = _f64(R0)
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    p_cell = _f64(p_cell)
    N = R0.shape[0]
    for a, dt_ in ((R, np.float64), (Rdot, np.float64), (h, np.float32)):
        if a.dtype != dt_ or not a.flags.c_contiguous or a.size != N:
            raise ValueError("bubble state arrays must be contiguous [N] (R, Rdot f64; h f32)")
    flags = np.zeros(N, dtype=np.uint32)
    att = np.zeros(N, dtype=np.int32)
    cp = params.as_c()
    _lib().orc_el_advance(ctypes.byref(cp), N, _ptr(R0, _dp), cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          _ptr(p_cell, _dp), float(dt), _ptr(R, _dp), _ptr(Rdot, _dp), _ptr(h, _fp),
                          _ptr(flags, _u32p), _ptr(att, _i32p))
    return flags, att


def el_smear(pos, R, Rdot, nx, ny, nz, dx, with_rate=True):
    """Void fraction (and its bubble-growth rate) of Eq. (kernel3D) at the cell centres."""
    pos = _f64(pos)
    R = _f64(R)
    Rdot = _f64(Rdot)
    N = R.shape[0]
    alpha = np.zeros(nx * ny * nz)
    adot = np.zeros(nx * ny * nz) if with_rate else None
    _lib().orc_el_smear(N, _ptr(pos[0], _dp), _ptr(pos[1], _dp), _ptr(pos[2], _dp), _ptr(R, _dp),
                        _ptr(Rdot, _dp), int(nx), int(ny), int(nz), float(dx), _ptr(alpha, _dp),
                        _ptr(adot, _dp) if adot is not None else None)
    return (alpha, adot) if with_rate else alpha


# ---------------------------------------------------------------------------
# Non-polytropic contents: state (R, Rdot, p_b, m_v) per bin.
# ---------------------------------------------------------------------------
def transfer_gas_mass(params: Params, tr: Transfer, R0: float) -> float:
    """Non-condensable gas mass of a bubble in equilibrium at R0."""
    cp, ct = params.as_c(), tr.as_c()
    return float(_lib().orc_transfer_gas_mass(ctypes.byref(cp), ctypes.byref(ct), float(R0)))


def transfer_init(params: Params, tr: Transfer, R0: float):
    """Equilibrium state (R, Rdot, p_b, m_v) of bin R0."""
    y = np.zeros(4)
    cp, ct = params.as_c(), tr.as_c()
    _lib().orc_transfer_init(ctypes.byref(cp), ctypes.byref(ct), float(R0), _ptr(y, _dp))
    return y


def transfer_rates(params: Params, tr: Transfer, m_g: float, y):
    """(dp_b/dt, dm_v/dt) at state y = (R, Rdot, p_b, m_v)."""
    y = _f64(y)
    a = np.zeros(1)
    b = np.zeros(1)
    cp, ct = params.as_c(), tr.as_c()
    _lib().orc_transfer_rates(ctypes.byref(cp), ctypes.byref(ct), float(m_g), _ptr(y, _dp),
                              _ptr(a, _dp), _ptr(b, _dp))
    return float(a[0]), float(b[0])


def transfer_rhs(params: Params, tr: Transfer, m_g: float, p_inf: float, y):
    """Right-hand side (f[4], p_bw) of the four-component system at y."""
    y = _f64(y)
    f = np.zeros(4)
    pbw = np.zeros(1)
    cp, ct = params.as_c(), tr.as_c()
    _lib().orc_transfer_rhs(ctypes.byref(cp), ctypes.byref(ct), float(m_g), float(p_inf),
                            _ptr(y, _dp), _ptr(f, _dp), _ptr(pbw, _dp))
    return f, float(pbw[0])


def transfer_step(params: Params, tr: Transfer, R0, p_inf, dt, R, Rdot, pb, mv, h, n_fixed: int = 0):
    """Advance [B][C] state (R, Rdot, p_b, m_v f64; h f32) in place; returns (flags, attempts)."""
    R0 = _f64(R0)
    p_inf = _f64(p_inf)
    B = R0.shape[0]
    C = p_inf.shape[0]
    for a, dt_ in ((R, np.float64), (Rdot, np.float64), (pb, np.float64), (mv, np.float64),
                   (h, np.float32)):
        if a.dtype != dt_ or not a.flags.c_contiguous or a.size != B * C:
            raise ValueError("state arrays must be contiguous [B][C]")
    flags = np.zeros((B, C), dtype=np.uint32)
    attempts = np.zeros((B, C), dtype=np.int32)
    cp, ct = params.as_c(), tr.as_c()
    _lib().orc_transfer_step(ctypes.byref(cp), ctypes.byref(ct), C, B, _ptr(R0, _dp), _ptr(p_inf, _dp),
                             float(dt), int(n_fixed), _ptr(R, _dp), _ptr(Rdot, _dp), _ptr(pb, _dp),
                             _ptr(mv, _dp), _ptr(h, _fp), _ptr(flags, _u32p), _ptr(attempts, _i32p))
    return flags, attempts


def transfer_moments(params: Params, w, n_b, R, Rdot, pb):
    """[7][C] moments with p_bw from the state p_b (rows as moments())."""
    w = _f64(w)
    n_b = _f64(n_b)
    R, Rdot, pb = _f64(R), _f64(Rdot), _f64(pb)
    B = w.shape[0]
    C = n_b.shape[0]
    out = np.zeros((7, C))
    cp = params.as_c()
    _lib().orc_transfer_moments(ctypes.byref(cp), C, B, _ptr(w, _dp), _ptr(n_b, _dp), _ptr(R, _dp),
                                _ptr(Rdot, _dp), _ptr(pb, _dp), _ptr(out, _dp))
    return out
