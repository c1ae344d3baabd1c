"""ctypes binding of the volume-averaged (Euler-Lagrange) model (include/pab_el.h)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import pab
from .pab import PabError, pab_config, pab_config_default

EXPORTS = ("pab_el_create", "pab_el_step", "pab_el_smear", "pab_el_status", "pab_el_get_state",
           "pab_el_set_state", "pab_el_destroy", "pab_el_last_error")
_BOUND = False


def load():
    global _BOUND
    lib = pab.load()
    if _BOUND:
        return lib
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "pab_el_create": (i32, [ctypes.POINTER(pab_config), i64, vp, vp, i32, i32, i32, dbl, vp,
                                ctypes.POINTER(vp)]),
        "pab_el_step": (i32, [vp, vp, dbl, vp, vp, vp]),
        "pab_el_smear": (i32, [vp, vp, vp, vp]),
        "pab_el_status": (i32, [vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(i64),
                                ctypes.POINTER(i64), vp]),
        "pab_el_get_state": (i32, [vp, vp, vp, vp, vp]),
        "pab_el_set_state": (i32, [vp, vp, vp, vp, vp]),
        "pab_el_destroy": (None, [vp]),
        "pab_el_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _BOUND = True
    return lib


def _stream(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class BubbleCloud:
    """N fixed Lagrangian bubbles on an nx x ny x nz grid of cell size dx."""

    def __init__(self, pos, R0, nx: int, ny: int, nz: int, dx: float, stream=None, **liquid):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("BubbleCloud needs a CUDA device; there is no CPU fallback")
        self.device = torch.device("cuda", torch.cuda.current_device())
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        R0 = np.ascontiguousarray(R0, dtype=np.float64)
        if pos.ndim != 2 or pos.shape[0] != 3 or pos.shape[1] != R0.shape[0]:
            raise ValueError("pos must be [3][N] and R0 [N]")
        self.N = int(R0.shape[0])
        self.shape = (int(nz), int(ny), int(nx))
        self.dx = float(dx)
        cfg = pab_config_default(**liquid)
        out = ctypes.c_void_p()
        st = load().pab_el_create(ctypes.byref(cfg), self.N, pos.ctypes.data if self.N else None,
                                  R0.ctypes.data if self.N else None, int(nx), int(ny), int(nz), float(dx),
                                  _stream(stream) or None, ctypes.byref(out))
        if st != pab.PAB_OK:
            raise PabError(st, "pab_el_create (details on stderr)")
        self.handle = out.value

    def _check(self, st, what):
        if st != pab.PAB_OK:
            raise PabError(st, f"{what}: {load().pab_el_last_error(self.handle).decode()}")

    @property
    def n_cells(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def _field(self, t, name):
        import torch
        if t is None:
            return None
        if t.device != self.device or t.dtype != torch.float64 or not t.is_contiguous() \
                or t.numel() != self.n_cells:
            raise ValueError(f"{name} must be a contiguous float64 tensor of {self.n_cells} cells")
        return t.data_ptr()

    def step(self, p_cell, dt: float, alpha=None, alpha_dot=None, stream=None):
        self._check(load().pab_el_step(self.handle, self._field(p_cell, "p_cell"), float(dt),
                                       self._field(alpha, "alpha"), self._field(alpha_dot, "alpha_dot"),
                                       _stream(stream) or None), "pab_el_step")

    def smear(self, alpha, alpha_dot=None, stream=None):
        self._check(load().pab_el_smear(self.handle, self._field(alpha, "alpha"),
                                        self._field(alpha_dot, "alpha_dot"), _stream(stream) or None),
                    "pab_el_smear")

    def status(self, stream=None):
        fl = ctypes.c_uint32()
        nf, na = ctypes.c_int64(), ctypes.c_int64()
        st = load().pab_el_status(self.handle, ctypes.byref(fl), ctypes.byref(nf), ctypes.byref(na),
                                  _stream(stream) or None)
        if st in (pab.PAB_EINVAL, pab.PAB_ECUDA):
            self._check(st, "pab_el_status")
        return dict(status=st, flags=fl.value, n_flagged=nf.value, n_attempts=na.value)

    def get_state(self, stream=None):
        import torch
        R = torch.empty(self.N, dtype=torch.float64, device=self.device)
        V = torch.empty_like(R)
        h = torch.empty(self.N, dtype=torch.float32, device=self.device)
        self._check(load().pab_el_get_state(self.handle, R.data_ptr(), V.data_ptr(), h.data_ptr(),
                                            _stream(stream) or None), "pab_el_get_state")
        return R, V, h

    def _bubbles(self, t, dtype, name):
        if t is None:
            return None
        if t.device != self.device or t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != (self.N,):
            raise ValueError(f"{name} must be a contiguous {dtype} tensor of {self.N} bubbles on {self.device}")
        return t.data_ptr()

    def set_state(self, R, V, h=None, stream=None):
        import torch
        if R is None or V is None:
            raise ValueError("R and Rdot are required")
        self._check(load().pab_el_set_state(self.handle, self._bubbles(R, torch.float64, "R"),
                                            self._bubbles(V, torch.float64, "Rdot"),
                                            self._bubbles(h, torch.float32, "h"),
                                            _stream(stream) or None), "pab_el_set_state")

    def close(self):
        if getattr(self, "handle", None):
            load().pab_el_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
