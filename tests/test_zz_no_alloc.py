"""The allocation-free step (pab_bubble_step_noalloc) against the handle path.

Some callers may not allocate device memory: a flow solver that hands the
library pointers into its own fixed pools, or a plugin whose memory belongs to
a host framework's allocator.  For them the library offers a step that takes
the whole state from the caller and keeps its only scratch (a status block) in
a static device array.  This test allocates the buffers itself (as such a
caller's owner would), runs two steps in a row through both entry points on the
same inputs, and requires the same state, moments and status within the
adaptive parity tolerance.  It sits in its own file, collected last, and works
alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2511_21031_gb300 import pab, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-6  # the adaptive-mode parity tolerance of the other GPU tests


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_step_matches_handle_step_on_two_calls(precision):
    import torch
    wl = workloads.config_grid128(edge=8)
    C, B = wl.n_cells, wl.n_bins
    prec = pab.PAB_FP64 if precision == "fp64" else pab.PAB_MIXED
    ref = pab.Solver(C, B, precision=precision, s_lognormal=wl.s)
    R, V, h = ref.get_state()          # caller-owned copies of the initial state
    R0s = [x.clone() for x in (R, V, h)]
    counts = []
    cfg = pab.pab_config_default(n_cells=C, n_bins=B, s_lognormal=wl.s, precision=prec)
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    m_ref = torch.empty((7, C), dtype=torch.float64, device="cuda")
    m_na = torch.empty((7, C), dtype=torch.float64, device="cuda")
    status = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    for k in range(2):
        p = torch.as_tensor(wl.pressure_step(k), device="cuda")
        ref.step(p, wl.dt, moments=m_ref)
        pab.pab_bubble_step_noalloc(cfg, p.data_ptr(), 0, wl.dt, R.data_ptr(), V.data_ptr(),
                                    h.data_ptr(), m_na.data_ptr(), status.data_ptr(), sp)
        st = ref.status()
        torch.cuda.synchronize()
        Rr, Vr, hr = ref.get_state()
        torch.testing.assert_close(R, Rr, rtol=TOL, atol=0)
        vfloor = 1e-3 * (101325.0 / 1000.0) ** 0.5
        assert float(((V - Vr).abs() / Vr.abs().clamp_min(vfloor)).max()) <= TOL
        torch.testing.assert_close(h, hr, rtol=TOL, atol=0)
        torch.testing.assert_close(m_na, m_ref, rtol=TOL, atol=1e-12 * float(m_ref.abs().max()))
        s = status.cpu().numpy()
        assert s[0] == st["flags"] == 0
        assert s[1] == st["n_flagged"] and s[3] == st["n_fp64"]
        if precision == "fp64":
            assert s[2] == st["n_attempts"] > 0  # the scratch was cleared before this call
        else:
            # the mixed gas term here is the series, the handle's its node table: equal to
            # rounding, so an accept decision at the tolerance's edge may differ
            assert s[2] > 0 and abs(s[2] / st["n_attempts"] - 1.0) <= 1e-3
            counts.append(int(s[2]))
    if precision == "mixed":
        # the same inputs again from the same start: the same count, so each call cleared
        # the block instead of adding to the previous call's counts
        R2, V2, h2 = R0s
        m2 = torch.empty_like(m_na)
        for k in range(2):
            p = torch.as_tensor(wl.pressure_step(k), device="cuda")
            pab.pab_bubble_step_noalloc(cfg, p.data_ptr(), 0, wl.dt, R2.data_ptr(), V2.data_ptr(),
                                        h2.data_ptr(), m2.data_ptr(), status.data_ptr(), sp)
            torch.cuda.synchronize()
            assert int(status[2]) == counts[k]
        assert torch.equal(R2, R) and torch.equal(m2, m_na)
    ref.close()


def test_noalloc_fixed_mode_without_a_step_size_array():
    """PAB_FIXED needs no carried step size, so h may be NULL: the fixed-step parity
    tolerance (1e-9) against the handle path, over two calls."""
    import torch
    wl = workloads.config_grid128(edge=8)
    C, B = wl.n_cells, wl.n_bins
    ref = pab.Solver(C, B, s_lognormal=wl.s, fixed_substeps=3)
    R, V, _ = ref.get_state()
    cfg = pab.pab_config_default(n_cells=C, n_bins=B, s_lognormal=wl.s, stepper=pab.PAB_FIXED,
                                 n_fixed_sub=3)
    sp = int(torch.cuda.current_stream().cuda_stream)
    m_ref = torch.empty((7, C), dtype=torch.float64, device="cuda")
    m_na = torch.empty_like(m_ref)
    for k in range(2):
        p = torch.as_tensor(wl.pressure_step(k), device="cuda")
        ref.step(p, wl.dt, moments=m_ref)
        pab.pab_bubble_step_noalloc(cfg, p.data_ptr(), 0, wl.dt, R.data_ptr(), V.data_ptr(),
                                    0, m_na.data_ptr(), 0, sp)
        torch.cuda.synchronize()
        Rr, Vr, _ = ref.get_state()
        torch.testing.assert_close(R, Rr, rtol=1e-9, atol=0)
        vfloor = 1e-3 * (101325.0 / 1000.0) ** 0.5
        assert float(((V - Vr).abs() / Vr.abs().clamp_min(vfloor)).max()) <= 1e-9
        torch.testing.assert_close(m_na, m_ref, rtol=1e-9, atol=1e-15 * float(m_ref.abs().max()))
    ref.close()


def test_noalloc_refuses_bad_sizes_and_pointers():
    import torch
    lib = pab.load()
    p = torch.full((8,), 101325.0, dtype=torch.float64, device="cuda")
    R = torch.full((3, 8), 10e-6, dtype=torch.float64, device="cuda")
    V = torch.zeros_like(R)
    h = torch.zeros((3, 8), dtype=torch.float32, device="cuda")
    for bad in (dict(n_bins=64 + 1), dict(n_bins=4), dict(n_cells=0)):
        cfg = pab.pab_config_default(**{"n_cells": 8, "n_bins": 3, "s_lognormal": 0.2, **bad})
        st = lib.pab_bubble_step_noalloc(ctypes.byref(cfg), p.data_ptr(), None, 1e-8, R.data_ptr(),
                                         V.data_ptr(), h.data_ptr(), None, None, None)
        assert st == pab.PAB_EINVAL
    # explicit bins whose weights sum to zero: refused as pab_create refuses them
    R0x = (ctypes.c_double * 3)(5e-6, 10e-6, 20e-6)
    wx = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    cfg = pab.pab_config_default(n_cells=8, n_bins=3, s_lognormal=0.2)
    cfg.R0_host = ctypes.cast(R0x, ctypes.POINTER(ctypes.c_double))
    cfg.w_host = ctypes.cast(wx, ctypes.POINTER(ctypes.c_double))
    assert lib.pab_bubble_step_noalloc(ctypes.byref(cfg), p.data_ptr(), None, 1e-8, R.data_ptr(),
                                       V.data_ptr(), h.data_ptr(), None, None, None) == pab.PAB_EINVAL
    with pytest.raises(pab.PabError):
        pab.Solver(8, 3, R0_host=[5e-6, 10e-6, 20e-6], w_host=[0.0, 0.0, 0.0])
    cfg = pab.pab_config_default(n_cells=8, n_bins=3, s_lognormal=0.2)
    assert lib.pab_bubble_step_noalloc(ctypes.byref(cfg), p.data_ptr(), None, 1e-8, R.data_ptr(),
                                       V.data_ptr(), None, None, None, None) == pab.PAB_EINVAL
    assert lib.pab_bubble_step_noalloc(ctypes.byref(cfg), p.data_ptr(), None, -1.0, R.data_ptr(),
                                       V.data_ptr(), h.data_ptr(), None, None, None) == pab.PAB_EINVAL
    torch.cuda.synchronize()
    assert np.all(R.cpu().numpy() == 10e-6)
