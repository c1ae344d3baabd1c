"""ctypes binding of the batched form (include/pab_batch.h).

``Batch`` owns one pab_batch_t: an arena of slots on the current GPU, each
holding one independent bubble ensemble.  Methods take torch tensors and pass
``data_ptr()`` and the current stream; the library does all the work.
"""
from __future__ import annotations

import ctypes

from . import pab
from .pab import PabError, pab_config, pab_config_default


class pab_batch_config(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("capacity_bins", ctypes.c_int64), ("block_warps", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("bins_per_grab", ctypes.c_int32),
                ("max_bins", ctypes.c_int32)]


EXPORTS = ("pab_batch_config_default", "pab_batch_create", "pab_batch_admit", "pab_batch_bind",
           "pab_batch_release", "pab_batch_step", "pab_batch_step_graph", "pab_batch_status",
           "pab_batch_get_state", "pab_batch_set_state", "pab_batch_usage", "pab_batch_set_launch",
           "pab_batch_destroy", "pab_batch_last_error")

_BOUND = False


def load():
    global _BOUND
    lib = pab.load()
    if _BOUND:
        return lib
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    bcp = ctypes.POINTER(pab_batch_config)
    sig = {
        "pab_batch_config_default": (None, [bcp]),
        "pab_batch_create": (i32, [bcp, vp, ctypes.POINTER(vp)]),
        "pab_batch_admit": (i32, [vp, ctypes.POINTER(pab_config), vp, ctypes.POINTER(i32)]),
        "pab_batch_bind": (i32, [vp, i32, vp, vp, vp, dbl]),
        "pab_batch_release": (i32, [vp, i32, vp]),
        "pab_batch_step": (i32, [vp, vp]),
        "pab_batch_step_graph": (i32, [vp, vp]),
        "pab_batch_status": (i32, [vp, i32, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64), ctypes.POINTER(i64), vp]),
        "pab_batch_get_state": (i32, [vp, i32, vp, vp, vp, vp]),
        "pab_batch_set_state": (i32, [vp, i32, vp, vp, vp, vp]),
        "pab_batch_usage": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "pab_batch_set_launch": (i32, [vp, i32, i32, i32]),
        "pab_batch_destroy": (None, [vp]),
        "pab_batch_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _BOUND = True
    return lib


def pab_batch_config_default(**overrides) -> pab_batch_config:
    c = pab_batch_config()
    load().pab_batch_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise AttributeError(f"pab_batch_config has no field {k}")
        setattr(c, k, v)
    return c


def _stream(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Batch:
    """An arena of resident bubble ensembles stepped together by one persistent kernel."""

    def __init__(self, max_slots: int = 512, precision: str = "mixed", capacity_bins: int = 0,
                 max_bins: int = 0, stream=None, **launch):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device; there is no CPU fallback")
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.precision = precision
        cfg = pab_batch_config_default(
            max_slots=int(max_slots), capacity_bins=int(capacity_bins), max_bins=int(max_bins),
            precision={"fp64": pab.PAB_FP64, "mixed": pab.PAB_MIXED}[precision], **launch)
        out = ctypes.c_void_p()
        st = load().pab_batch_create(ctypes.byref(cfg), _stream(stream) or None, ctypes.byref(out))
        if st != pab.PAB_OK:
            raise PabError(st, "pab_batch_create (details on stderr)")
        self.handle = out.value
        self.slots = {}  # slot -> (n_cells, n_bins)
        self._bound = {}  # slot -> the tensors whose pointers the library holds for its steps

    def _check(self, st, what):
        if st != pab.PAB_OK:
            raise PabError(st, f"{what}: {load().pab_batch_last_error(self.handle).decode()}")

    def admit(self, n_cells: int, n_bins: int, stream=None, **cfg) -> int:
        c = pab_config_default(n_cells=int(n_cells), n_bins=int(n_bins), **cfg)
        slot = ctypes.c_int32(-1)
        self._check(load().pab_batch_admit(self.handle, ctypes.byref(c), _stream(stream) or None,
                                           ctypes.byref(slot)), "pab_batch_admit")
        self.slots[slot.value] = (int(n_cells), int(n_bins))
        return slot.value

    def try_admit(self, n_cells: int, n_bins: int, stream=None, **cfg):
        """Admit or return None when the arena or the slots are full (PAB_ENOMEM)."""
        try:
            return self.admit(n_cells, n_bins, stream=stream, **cfg)
        except PabError as e:
            if e.status == pab.PAB_ENOMEM:
                return None
            raise

    def _ptr(self, t, shape, dtype, name):
        if t is None:
            return None
        if t.device != self.device or t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != shape:
            raise ValueError(f"{name} must be a contiguous {dtype} tensor {shape} on {self.device}")
        return t.data_ptr()

    def bind(self, slot: int, p_inf, dt: float, moments=None, nb=None):
        """Bind the slot's inputs and outputs for the following steps.  The library keeps the
        pointers, so the batch holds the tensors until the slot is bound again or released."""
        import torch
        C, _ = self.slots[slot]
        f64 = torch.float64
        self._check(load().pab_batch_bind(self.handle, int(slot), self._ptr(p_inf, (C,), f64, "p_inf"),
                                          self._ptr(nb, (C,), f64, "nb"),
                                          self._ptr(moments, (pab.N_MOMENTS, C), f64, "moments"),
                                          float(dt)), "pab_batch_bind")
        self._bound[slot] = (p_inf, nb, moments)

    def release(self, slot: int, stream=None):
        self._check(load().pab_batch_release(self.handle, int(slot), _stream(stream) or None),
                    "pab_batch_release")
        self.slots.pop(slot, None)
        self._bound.pop(slot, None)

    def step(self, graph: bool = False, stream=None):
        fn = load().pab_batch_step_graph if graph else load().pab_batch_step
        self._check(fn(self.handle, _stream(stream) or None), "pab_batch_step")

    def status(self, slot: int, stream=None, raise_on_error: bool = False):
        fl = ctypes.c_uint32()
        nf, na, n64 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        st = load().pab_batch_status(self.handle, int(slot), ctypes.byref(fl), ctypes.byref(nf),
                                     ctypes.byref(na), ctypes.byref(n64), _stream(stream) or None)
        if st in (pab.PAB_EINVAL, pab.PAB_ECUDA) or (raise_on_error and st != pab.PAB_OK):
            self._check(st, "pab_batch_status")
        return dict(status=st, flags=fl.value, n_flagged=nf.value, n_attempts=na.value, n_fp64=n64.value)

    def get_state(self, slot: int, stream=None):
        import torch
        C, B = self.slots[slot]
        R = torch.empty((B, C), dtype=torch.float64, device=self.device)
        V = torch.empty_like(R)
        h = torch.empty((B, C), dtype=torch.float32, device=self.device)
        self._check(load().pab_batch_get_state(self.handle, int(slot), R.data_ptr(), V.data_ptr(),
                                               h.data_ptr(), _stream(stream) or None), "pab_batch_get_state")
        return R, V, h

    def set_state(self, slot: int, R, V, h=None, stream=None):
        import torch
        C, B = self.slots[slot]
        if R is None or V is None:
            raise ValueError("R and Rdot are required")
        self._check(load().pab_batch_set_state(self.handle, int(slot), self._ptr(R, (B, C), torch.float64, "R"),
                                               self._ptr(V, (B, C), torch.float64, "Rdot"),
                                               self._ptr(h, (B, C), torch.float32, "h"),
                                               _stream(stream) or None), "pab_batch_set_state")

    def usage(self):
        a = ctypes.c_int32()
        used, cap = ctypes.c_int64(), ctypes.c_int64()
        self._check(load().pab_batch_usage(self.handle, ctypes.byref(a), ctypes.byref(used),
                                           ctypes.byref(cap)), "pab_batch_usage")
        return dict(active_slots=a.value, bins_used=used.value, capacity_bins=cap.value)

    def set_launch(self, block_warps: int, ctas_per_sm: int, bins_per_grab: int):
        self._check(load().pab_batch_set_launch(self.handle, int(block_warps), int(ctas_per_sm),
                                                int(bins_per_grab)), "pab_batch_set_launch")
        self.launch = (int(block_warps), int(ctas_per_sm), int(bins_per_grab))

    def close(self):
        if getattr(self, "handle", None):
            load().pab_batch_destroy(self.handle)
            self.handle = None
        if hasattr(self, "_bound"):
            self._bound.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
