"""Thin ctypes binding of libpab (include/pab.h).

The module-level functions carry the C names and only marshal arguments
(integers for device pointers and streams).  ``Solver`` wraps one handle for
torch tensors: it checks dtype, device and contiguity and passes
``data_ptr()`` and the current CUDA stream.  Every step of the path runs in
the library's kernels; if the library is missing this module raises.
"""
from __future__ import annotations

import collections
import ctypes
import os
from typing import Optional

from . import _build

PAB_OK, PAB_EINVAL, PAB_ENOMEM, PAB_ECUDA, PAB_ESTEP_LIMIT, PAB_ENONFINITE, PAB_ESTATE = range(7)
PAB_FP64, PAB_MIXED = 0, 1
PAB_ADAPTIVE, PAB_FIXED = 0, 1
PAB_GAS_POLYTROPIC, PAB_GAS_EMPTY, PAB_GAS_TRANSFER = 0, 1, 2
FLAG_STEP_LIMIT, FLAG_NONFINITE, FLAG_SUPERSONIC, FLAG_NONPOS = 1, 2, 4, 8
MAX_BINS = 63
MAX_CELLS = 1 << 35
N_MOMENTS = 7
MOMENT_NAMES = ("n_b", "alpha", "R3", "R2Rdot", "S_alpha", "R3pbw_over_R3", "R3Rdot2_over_R3")

EXPORTS = ("pab_config_default", "pab_create", "pab_bubble_step", "pab_moments",
           "pab_bubble_step_host", "pab_bubble_step_host_async", "pab_host_wait", "pab_status_flags", "pab_get_state", "pab_set_state",
           "pab_get_attempts", "pab_get_bins", "pab_bin_table", "pab_set_block_warps", "pab_destroy",
           "pab_last_error", "pab_status_string", "pab_peak_fma", "pab_bubble_step_noalloc",
           "pab_strang_half", "pab_get_conservative", "pab_set_conservative", "pab_mixture_pressure",
           "pab_stiffened_gas", "pab_math_check", "pab_bits_check", "pab_gas32_check", "pab_gas_table",
           "pab_get_contents", "pab_set_contents", "pab_check_report", "pab_accept_check",
           "pab_exp_check", "pab_intmul_check")
NOALLOC_SCRATCH_BYTES = 256


class PabError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class pab_config(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_bins", ctypes.c_int32), ("gas_mode", ctypes.c_int32),
                ("rho", ctypes.c_double), ("c", ctypes.c_double), ("mu", ctypes.c_double),
                ("sigma", ctypes.c_double), ("p0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("pv", ctypes.c_double), ("R0ref", ctypes.c_double), ("s_lognormal", ctypes.c_double),
                ("span_K", ctypes.c_double), ("R0_host", ctypes.POINTER(ctypes.c_double)),
                ("w_host", ctypes.POINTER(ctypes.c_double)), ("precision", ctypes.c_int32),
                ("stepper", ctypes.c_int32), ("n_fixed_sub", ctypes.c_int32),
                ("max_attempts", ctypes.c_int32), ("tol", ctypes.c_double), ("v_floor", ctypes.c_double),
                ("alpha0", ctypes.c_double), ("Rdot0_ref", ctypes.c_double),
                ("record_attempts", ctypes.c_int32), ("block_warps", ctypes.c_int32),
                ("R_g", ctypes.c_double), ("R_v", ctypes.c_double), ("T_w", ctypes.c_double),
                ("k_bw", ctypes.c_double), ("D_vg", ctypes.c_double), ("beta_T", ctypes.c_double),
                ("beta_c", ctypes.c_double)]


_LIB = None


def checked() -> bool:
    """True when PAB_CHECKED=1 selects the checked build (libpab_checked.so: every kernel's
    global-memory index tested against its buffer; pab_check_report reads the findings)."""
    return os.environ.get("PAB_CHECKED", "") == "1"


def library_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpab.so (building it first if allowed); raises if it is unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    chk = checked()
    path = library_path()
    if not os.path.exists(path) or not _build.up_to_date(chk):
        if not build_if_missing:
            raise RuntimeError(f"{os.path.basename(path)} missing or stale at {path}; run __graft_entry__.build()")
        _build.build(checked=chk)
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    cfgp = ctypes.POINTER(pab_config)
    sig = {
        "pab_config_default": (None, [cfgp]),
        "pab_create": (i32, [cfgp, vp, ctypes.POINTER(vp)]),
        "pab_bubble_step": (i32, [vp, vp, vp, dbl, vp, vp]),
        "pab_moments": (i32, [vp, vp, vp, vp]),
        "pab_bubble_step_host": (i32, [vp, vp, vp, dbl, vp, vp]),
        "pab_status_flags": (i32, [vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64), ctypes.POINTER(i64), vp]),
        "pab_get_state": (i32, [vp, vp, vp, vp, vp]),
        "pab_get_contents": (i32, [vp, vp, vp, vp]),
        "pab_bubble_step_host_async": (i32, [vp, vp, vp, dbl, vp, vp]),
        "pab_host_wait": (i32, [vp]),
        "pab_set_contents": (i32, [vp, vp, vp, vp]),
        "pab_set_state": (i32, [vp, vp, vp, vp, vp]),
        "pab_get_attempts": (i32, [vp, vp, vp]),
        "pab_get_bins": (i32, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "pab_bin_table": (i32, [ctypes.POINTER(pab_config), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                ctypes.POINTER(dbl)]),
        "pab_gas_table": (i32, [dbl, vp, i64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(dbl)]),
        "pab_set_block_warps": (i32, [vp, i32]),
        "pab_destroy": (None, [vp]),
        "pab_last_error": (ctypes.c_char_p, [vp]),
        "pab_status_string": (ctypes.c_char_p, [i32]),
        "pab_peak_fma": (i32, [i32, i32, i32, i32, vp, ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(dbl), vp]),
        "pab_bubble_step_noalloc": (i32, [cfgp, vp, vp, dbl, vp, vp, vp, vp, vp, vp]),
        "pab_strang_half": (i32, [vp, vp, vp, dbl, vp, vp]),
        "pab_get_conservative": (i32, [vp, vp, vp, vp, vp]),
        "pab_set_conservative": (i32, [vp, vp, vp, vp, vp, vp]),
        "pab_mixture_pressure": (i32, [vp, vp, vp, vp, vp, vp]),
        "pab_stiffened_gas": (i32, [i64, vp, vp, dbl, dbl, vp, vp]),
        "pab_math_check": (i32, [i64, vp, vp, dbl, vp, vp, vp, vp]),
        "pab_bits_check": (i32, [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "pab_gas32_check": (i32, [i64, vp, ctypes.c_float, vp, vp, vp]),
        "pab_accept_check": (i32, [i64, vp, vp, dbl, dbl, vp, vp]),
        "pab_exp_check": (i32, [i64, vp, vp, vp, vp]),
        "pab_intmul_check": (i32, [i64, vp, vp, vp, vp, vp, vp]),
        "pab_check_report": (i32, [ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


# --------------------------------------------------------------------------
# C names, argument marshalling only
# --------------------------------------------------------------------------
def status_string(s: int) -> str:
    try:
        return load().pab_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


def pab_config_default(**overrides) -> pab_config:
    cfg = pab_config()
    load().pab_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(f"pab_config has no field {k}")
        setattr(cfg, k, v)
    return cfg


def _check(h, st, what):
    if st != PAB_OK:
        msg = load().pab_last_error(h).decode() if h else ""
        raise PabError(st, f"{what}: {msg}")


def pab_create(cfg: pab_config, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    st = load().pab_create(ctypes.byref(cfg), ctypes.c_void_p(stream), ctypes.byref(out))
    if st != PAB_OK:
        raise PabError(st, "pab_create rejected the configuration (details on stderr)")
    return out.value


def pab_bubble_step(h: int, p_inf_ptr: int, nb_ptr: int, dt: float, moments_ptr: int, stream: int = 0):
    _check(h, load().pab_bubble_step(h, p_inf_ptr or None, nb_ptr or None, float(dt),
                                     moments_ptr or None, stream or None), "pab_bubble_step")


def pab_moments(h: int, nb_ptr: int, moments_ptr: int, stream: int = 0):
    _check(h, load().pab_moments(h, nb_ptr or None, moments_ptr or None, stream or None), "pab_moments")


def pab_bubble_step_host(h: int, p_inf_host: int, nb_host: int, dt: float, moments_host: int,
                         stream: int = 0):
    _check(h, load().pab_bubble_step_host(h, p_inf_host or None, nb_host or None, float(dt),
                                          moments_host or None, stream or None), "pab_bubble_step_host")


def pab_status_flags(h: int, stream: int = 0, raise_on_error: bool = False):
    fl = ctypes.c_uint32()
    nf, na, n64 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = load().pab_status_flags(h, ctypes.byref(fl), ctypes.byref(nf), ctypes.byref(na),
                                 ctypes.byref(n64), stream or None)
    if st in (PAB_EINVAL, PAB_ECUDA) or (raise_on_error and st != PAB_OK):
        _check(h, st, "pab_status_flags")
    return dict(status=st, flags=fl.value, n_flagged=nf.value, n_attempts=na.value, n_fp64=n64.value)


def pab_get_state(h, R_ptr, Rdot_ptr, h_ptr, stream=0):
    _check(h, load().pab_get_state(h, R_ptr or None, Rdot_ptr or None, h_ptr or None, stream or None),
           "pab_get_state")


def pab_set_state(h, R_ptr, Rdot_ptr, h_ptr, stream=0):
    _check(h, load().pab_set_state(h, R_ptr or None, Rdot_ptr or None, h_ptr or None, stream or None),
           "pab_set_state")


def pab_get_attempts(h, att_ptr, stream=0):
    _check(h, load().pab_get_attempts(h, att_ptr or None, stream or None), "pab_get_attempts")


def pab_bin_table(**cfg):
    """(R0, w, n_b default) that pab_create builds for the config (host only, no device)."""
    c = pab_config_default(**cfg)
    R0 = (ctypes.c_double * c.n_bins)()
    w = (ctypes.c_double * c.n_bins)()
    nb = ctypes.c_double()
    st = load().pab_bin_table(ctypes.byref(c), R0, w, ctypes.byref(nb))
    if st != PAB_OK:
        raise PabError(st, "pab_bin_table rejected the configuration (details on stderr)")
    return list(R0), list(w), nb.value


def pab_gas_table(gamma: float):
    """(nodes [2J+1][stride] float64 array, dmax) of the host-built gas-term table (no device)."""
    import numpy as np
    lib = load()
    n, stride, dmax = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    st = lib.pab_gas_table(float(gamma), None, 0, ctypes.byref(n), ctypes.byref(stride), ctypes.byref(dmax))
    if st != PAB_OK:
        raise PabError(st, "pab_gas_table")
    tab = np.empty((n.value, stride.value), dtype=np.float64)
    st = lib.pab_gas_table(float(gamma), tab.ctypes.data, tab.size, ctypes.byref(n), ctypes.byref(stride),
                           ctypes.byref(dmax))
    if st != PAB_OK:
        raise PabError(st, "pab_gas_table")
    return tab, dmax.value


def pab_get_bins(h, n_bins: int):
    R0 = (ctypes.c_double * n_bins)()
    w = (ctypes.c_double * n_bins)()
    nb = ctypes.c_double()
    _check(h, load().pab_get_bins(h, R0, w, ctypes.byref(nb)), "pab_get_bins")
    return list(R0), list(w), nb.value


def pab_set_block_warps(h, w):
    _check(h, load().pab_set_block_warps(h, int(w)), "pab_set_block_warps")


def pab_peak_fma(precision: int, blocks: int, threads: int, iters: int, sink_ptr: int, stream: int = 0):
    """Returns (kernel ms, FMA count) of the FMA-throughput microbenchmark."""
    ms = ctypes.c_float()
    n = ctypes.c_double()
    st = load().pab_peak_fma(int(precision), int(blocks), int(threads), int(iters), sink_ptr,
                             ctypes.byref(ms), ctypes.byref(n), stream or None)
    if st != PAB_OK:
        raise PabError(st, "pab_peak_fma")
    return ms.value, n.value


def pab_bubble_step_noalloc(cfg: pab_config, p_inf_ptr: int, nb_ptr: int, dt: float, R_ptr: int,
                            Rdot_ptr: int, h_ptr: int, moments_ptr: int, status_ptr: int, stream: int = 0):
    """Allocation-free step on caller-owned state (no handle); see include/pab.h."""
    st = load().pab_bubble_step_noalloc(ctypes.byref(cfg), p_inf_ptr or None, nb_ptr or None, float(dt),
                                        R_ptr or None, Rdot_ptr or None, h_ptr or None,
                                        moments_ptr or None, status_ptr or None, stream or None)
    if st != PAB_OK:
        raise PabError(st, "pab_bubble_step_noalloc (details on stderr)")


def pab_stiffened_gas(rho_l, e_l, gamma_l: float, pi_inf: float, out=None, stream=None):
    """Stiffened-gas liquid pressure (torch float64 CUDA tensors of equal length)."""
    import torch
    if out is None:
        out = torch.empty_like(rho_l)
    for t in (rho_l, e_l, out):
        if t.dtype != torch.float64 or not t.is_contiguous() or not t.is_cuda or t.numel() != rho_l.numel():
            raise ValueError("rho_l, e_l and out must be contiguous float64 CUDA tensors of equal size")
    st = load().pab_stiffened_gas(rho_l.numel(), rho_l.data_ptr(), e_l.data_ptr(), float(gamma_l),
                                  float(pi_inf), out.data_ptr(), _stream_handle(stream) or None)
    if st != PAB_OK:
        raise PabError(st, "pab_stiffened_gas")
    return out


def pab_bits_check(f, x, y, stream=None):
    """Library helpers against the hardware: dict of f2d, f2d_hw, rcp, div, seed, cmp."""
    import torch
    out = {k: torch.empty_like(x) for k in ("f2d", "f2d_hw", "rcp", "div", "seed")}
    out["cmp"] = torch.empty(x.shape, dtype=torch.int16, device=x.device)  # uint16 bit masks
    st = load().pab_bits_check(x.numel(), f.data_ptr(), x.data_ptr(), y.data_ptr(),
                               out["f2d"].data_ptr(), out["f2d_hw"].data_ptr(),
                               out["rcp"].data_ptr(), out["div"].data_ptr(), out["seed"].data_ptr(),
                               out["cmp"].data_ptr(), _stream_handle(stream) or None)
    if st != PAB_OK:
        raise PabError(st, "pab_bits_check")
    return out


def pab_math_check(R, Rb, a: float, stream=None):
    """(base-series value, table value, exp/log value) of the library's gas-term helpers."""
    import torch
    g = torch.empty_like(R)
    gt = torch.empty_like(R)
    e = torch.empty_like(R)
    st = load().pab_math_check(R.numel(), R.data_ptr(), Rb.data_ptr(), float(a), g.data_ptr(),
                               gt.data_ptr(), e.data_ptr(), _stream_handle(stream) or None)
    if st != PAB_OK:
        raise PabError(st, "pab_math_check")
    return g, gt, e


def pab_gas32_check(u, a: float, stream=None):
    """(library value, CUDA expm1f/log1pf value) of the FP32 gas term (1 + u)^(-a) - 1."""
    import torch
    out = torch.empty_like(u)
    lib = torch.empty_like(u)
    st = load().pab_gas32_check(u.numel(), u.data_ptr(), float(a), out.data_ptr(), lib.data_ptr(),
                                _stream_handle(stream) or None)
    if st != PAB_OK:
        raise PabError(st, "pab_gas32_check")
    return out, lib


def pab_exp_check(x, stream=None):
    """(the smear's table-driven e^x, the CUDA library's exp) of x (float64, on the device)."""
    import torch
    mine = torch.empty_like(x)
    lib = torch.empty_like(x)
    st = load().pab_exp_check(x.numel(), x.data_ptr(), mine.data_ptr(), lib.data_ptr(),
                              _stream_handle(stream) or None)
    if st != PAB_OK:
        raise PabError(st, "pab_exp_check")
    return mine, lib


def pab_intmul_check(x, y, stream=None):
    """(x y, x^3, 1/x) formed on the integer pipe as the kernels form them, for x, y float64 on
    the device."""
    import torch
    prod = torch.empty_like(x)
    cube = torch.empty_like(x)
    rcp = torch.empty_like(x)
    st = load().pab_intmul_check(x.numel(), x.data_ptr(), y.data_ptr(), prod.data_ptr(),
                                 cube.data_ptr(), rcp.data_ptr(), _stream_handle(stream) or None)
    if st != PAB_OK:
        raise PabError(st, "pab_intmul_check")
    return prod, cube, rcp


def pab_accept_check(trial, k, tol: float, v_floor: float, stream=None):
    """[n, 4] uint8: the FP64 trial's bracketed accept decision and the exact FP64 test on
    trial [n, 4] float64 (R3, Rdot3, e_R, e_Rdot), then the mixed trial's bracketed component
    test and its exact form on k [n, 4] float32 (k1, k2, k3, T)."""
    import torch
    n = trial.shape[0]
    if tuple(trial.shape) != (n, 4) or tuple(k.shape) != (n, 4) or trial.dtype != torch.float64 \
            or k.dtype != torch.float32 or not trial.is_contiguous() or not k.is_contiguous():
        raise ValueError("trial must be [n, 4] float64 and k [n, 4] float32, contiguous")
    out = torch.empty((n, 4), dtype=torch.uint8, device=trial.device)
    st = load().pab_accept_check(n, trial.data_ptr(), k.data_ptr(), float(tol), float(v_floor),
                                 out.data_ptr(), _stream_handle(stream) or None)
    if st != PAB_OK:
        raise PabError(st, "pab_accept_check")
    return out


CHECK_UNITS = {1: "step kernels", 2: "batch", 3: "carrier coupling", 4: "Euler-Lagrange", 5: "transfer contents"}


def pab_check_report():
    """The checked build's first out-of-bounds index since the last call (count 0: none), or
    None from a library built without the checks.  Waits for the device."""
    n, u, ln, i, b = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    st = load().pab_check_report(ctypes.byref(n), ctypes.byref(u), ctypes.byref(ln), ctypes.byref(i),
                                 ctypes.byref(b))
    if st == PAB_ESTATE:
        return None
    if st != PAB_OK:
        raise PabError(st, "pab_check_report")
    return dict(count=n.value, unit=CHECK_UNITS.get(u.value, ""), line=ln.value, index=i.value, bound=b.value)


def pab_destroy(h):
    if h:
        load().pab_destroy(h)


# --------------------------------------------------------------------------
# torch convenience wrapper around one handle
# --------------------------------------------------------------------------
def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Solver:
    """One resident ensemble: n_cells x n_bins bubble state on the current GPU."""

    def __init__(self, n_cells: int, n_bins: int = 21, *, precision: str = "fp64",
                 fixed_substeps: int = 0, stream=None, **cfg_overrides):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Solver needs a CUDA device; there is no CPU fallback")
        self.device = torch.device("cuda", torch.cuda.current_device())
        prec = {"fp64": PAB_FP64, "mixed": PAB_MIXED}[precision]
        kw = dict(n_cells=int(n_cells), n_bins=int(n_bins), precision=prec)
        if fixed_substeps:
            kw.update(stepper=PAB_FIXED, n_fixed_sub=int(fixed_substeps))
        kw.update(cfg_overrides)
        self._keep = []
        for key in ("R0_host", "w_host"):
            if key in kw and kw[key] is not None and not isinstance(kw[key], ctypes.POINTER(ctypes.c_double)):
                arr = (ctypes.c_double * len(kw[key]))(*[float(x) for x in kw[key]])
                self._keep.append(arr)
                kw[key] = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        self.cfg = pab_config_default(**kw)
        self._in_flight = collections.deque(maxlen=2)  # host tensors of pipelined calls
        self.n_cells = int(n_cells)
        self.n_bins = int(n_bins)
        self.precision = precision
        self.handle = pab_create(self.cfg, _stream_handle(stream))
        self.R0, self.w, self.nb_default = pab_get_bins(self.handle, self.n_bins)

    # ---- checks -----------------------------------------------------------
    def _dev(self, t, shape, dtype, name):
        import torch
        if t is None:
            return 0
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype \
                or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)} "
                             f"on {self.device}")
        return t.data_ptr()

    # ---- entry points -----------------------------------------------------
    def step(self, p_inf, dt: float, moments=None, nb=None, stream=None):
        import torch
        pab_bubble_step(self.handle, self._dev(p_inf, (self.n_cells,), torch.float64, "p_inf"),
                        self._dev(nb, (self.n_cells,), torch.float64, "nb"), dt,
                        self._dev(moments, (N_MOMENTS, self.n_cells), torch.float64, "moments"),
                        _stream_handle(stream))
        return moments

    def moments(self, out=None, nb=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((N_MOMENTS, self.n_cells), dtype=torch.float64, device=self.device)
        pab_moments(self.handle, self._dev(nb, (self.n_cells,), torch.float64, "nb"),
                    self._dev(out, (N_MOMENTS, self.n_cells), torch.float64, "moments"),
                    _stream_handle(stream))
        return out

    def step_host(self, p_inf_host, dt: float, moments_host=None, nb_host=None, stream=None):
        """End-to-end form with host (CPU, ideally pinned) float64 tensors."""
        import torch

        def hp(t, shape, name):
            if t is None:
                return 0
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous() \
                    or tuple(t.shape) != tuple(shape):
                raise ValueError(f"{name} must be a contiguous float64 CPU tensor of shape {shape}")
            return t.data_ptr()
        pab_bubble_step_host(self.handle, hp(p_inf_host, (self.n_cells,), "p_inf_host"),
                             hp(nb_host, (self.n_cells,), "nb_host"), dt,
                             hp(moments_host, (N_MOMENTS, self.n_cells), "moments_host"),
                             _stream_handle(stream))
        return moments_host

    def step_host_async(self, p_inf_host, dt: float, moments_host=None, nb_host=None, stream=None):
        """Pipelined end-to-end form: returns at once; moments_host is ready (and the host
        tensors free) after host_wait() or after the second call after this one.  The solver
        holds the host tensors of the calls that may still be in flight, so temporaries passed
        here stay alive until their copies have run."""
        import torch
        if p_inf_host is None:
            raise ValueError("p_inf_host is required")
        for t, shape, name in ((p_inf_host, (self.n_cells,), "p_inf_host"), (nb_host, (self.n_cells,), "nb_host"),
                               (moments_host, (N_MOMENTS, self.n_cells), "moments_host")):
            if t is not None and (t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous()
                                  or tuple(t.shape) != shape):
                raise ValueError(f"{name} must be a contiguous float64 CPU tensor of shape {shape}")
        st = load().pab_bubble_step_host_async(
            self.handle, p_inf_host.data_ptr(), nb_host.data_ptr() if nb_host is not None else None, float(dt),
            moments_host.data_ptr() if moments_host is not None else None, _stream_handle(stream) or None)
        _check(self.handle, st, "pab_bubble_step_host_async")
        # a call returns only once the call two before it has finished, so the last two
        # calls' tensors are all that can still be in flight
        self._in_flight.append((p_inf_host, nb_host, moments_host))
        return moments_host

    def host_wait(self):
        _check(self.handle, load().pab_host_wait(self.handle), "pab_host_wait")
        self._in_flight.clear()

    def status(self, stream=None, raise_on_error=False):
        return pab_status_flags(self.handle, _stream_handle(stream), raise_on_error)

    def get_state(self, stream=None):
        import torch
        shp = (self.n_bins, self.n_cells)
        R = torch.empty(shp, dtype=torch.float64, device=self.device)
        V = torch.empty_like(R)
        h = torch.empty(shp, dtype=torch.float32, device=self.device)
        pab_get_state(self.handle, R.data_ptr(), V.data_ptr(), h.data_ptr(), _stream_handle(stream))
        return R, V, h

    def set_state(self, R, V, h=None, stream=None):
        import torch
        shp = (self.n_bins, self.n_cells)
        pab_set_state(self.handle, self._dev(R, shp, torch.float64, "R"),
                      self._dev(V, shp, torch.float64, "Rdot"),
                      self._dev(h, shp, torch.float32, "h"), _stream_handle(stream))

    def get_contents(self, stream=None):
        """(p_b, m_v) [Nb][C] of a PAB_GAS_TRANSFER handle."""
        import torch
        shp = (self.n_bins, self.n_cells)
        pb = torch.empty(shp, dtype=torch.float64, device=self.device)
        mv = torch.empty_like(pb)
        _check(self.handle, load().pab_get_contents(self.handle, pb.data_ptr(), mv.data_ptr(),
                                                    _stream_handle(stream) or None), "pab_get_contents")
        return pb, mv

    def set_contents(self, pb=None, mv=None, stream=None):
        import torch
        shp = (self.n_bins, self.n_cells)
        _check(self.handle, load().pab_set_contents(self.handle, self._dev(pb, shp, torch.float64, "pb") or None,
                                                    self._dev(mv, shp, torch.float64, "mv") or None,
                                                    _stream_handle(stream) or None), "pab_set_contents")

    def attempts(self, stream=None):
        import torch
        a = torch.empty((self.n_bins, self.n_cells), dtype=torch.int32, device=self.device)
        pab_get_attempts(self.handle, a.data_ptr(), _stream_handle(stream))
        return a

    def set_block_warps(self, w: int):
        pab_set_block_warps(self.handle, w)

    # ---- carrier-facing forms (pab_closure.h) -----------------------------
    def strang_half(self, p_inf, dt_flow: float, moments=None, nb=None, stream=None):
        import torch
        _check(self.handle, load().pab_strang_half(
            self.handle, self._dev(p_inf, (self.n_cells,), torch.float64, "p_inf") or None,
            self._dev(nb, (self.n_cells,), torch.float64, "nb") or None, float(dt_flow),
            self._dev(moments, (N_MOMENTS, self.n_cells), torch.float64, "moments") or None,
            _stream_handle(stream) or None), "pab_strang_half")
        return moments

    def get_conservative(self, nb=None, stream=None):
        import torch
        shp = (self.n_bins, self.n_cells)
        qR = torch.empty(shp, dtype=torch.float64, device=self.device)
        qV = torch.empty_like(qR)
        _check(self.handle, load().pab_get_conservative(
            self.handle, self._dev(nb, (self.n_cells,), torch.float64, "nb") or None, qR.data_ptr(),
            qV.data_ptr(), _stream_handle(stream) or None), "pab_get_conservative")
        return qR, qV

    def set_conservative(self, alpha, qR, qV, stream=None):
        import torch
        shp = (self.n_bins, self.n_cells)
        nb = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        _check(self.handle, load().pab_set_conservative(
            self.handle, self._dev(alpha, (self.n_cells,), torch.float64, "alpha"),
            self._dev(qR, shp, torch.float64, "qR"), self._dev(qV, shp, torch.float64, "qV"),
            nb.data_ptr(), _stream_handle(stream) or None), "pab_set_conservative")
        return nb

    def mixture_pressure(self, moments, p_l, rho_l=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        _check(self.handle, load().pab_mixture_pressure(
            self.handle, self._dev(moments, (N_MOMENTS, self.n_cells), torch.float64, "moments"),
            self._dev(p_l, (self.n_cells,), torch.float64, "p_l"),
            self._dev(rho_l, (self.n_cells,), torch.float64, "rho_l") or None,
            self._dev(out, (self.n_cells,), torch.float64, "p"), _stream_handle(stream) or None),
            "pab_mixture_pressure")
        return out

    def close(self):
        if getattr(self, "handle", None):
            pab_destroy(self.handle)  # waits for the pipelined calls' copies
            self.handle = None
        if hasattr(self, "_in_flight"):
            self._in_flight.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
