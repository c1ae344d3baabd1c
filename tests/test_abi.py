"""Host-side checks of the C ABI: the library loads, exports every entry point
include/pab.h declares, the ctypes config matches the C layout, and invalid
calls are refused before any device work (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess
import tempfile

import pytest

from paper_2511_21031_gb300 import pab

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def _declared():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pab_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    lib = pab.load()
    declared = _declared()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    from paper_2511_21031_gb300 import batch, el
    batch.load()
    el.load()
    assert set(declared) == set(pab.EXPORTS) | set(batch.EXPORTS) | set(el.EXPORTS)


def test_config_layout_matches_c():
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "pab.h"
int main(void) {
  printf("%zu", sizeof(pab_config));
#define O(f) printf(" %s=%zu", #f, offsetof(pab_config, f));
  O(n_cells) O(n_bins) O(gas_mode) O(rho) O(c) O(mu) O(sigma) O(p0) O(gamma) O(pv) O(R0ref)
  O(s_lognormal) O(span_K) O(R0_host) O(w_host) O(precision) O(stepper) O(n_fixed_sub)
  O(max_attempts) O(tol) O(v_floor) O(alpha0) O(Rdot0_ref) O(record_attempts) O(block_warps)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(pab.pab_config)
    for item in out[1:]:
        k, v = item.split("=")
        assert getattr(pab.pab_config, k).offset == int(v), k


def test_batch_config_layout_matches_c():
    from paper_2511_21031_gb300 import batch
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "pab_batch.h"
int main(void) {
  printf("%zu", sizeof(pab_batch_config));
#define O(f) printf(" %s=%zu", #f, offsetof(pab_batch_config, f));
  O(max_slots) O(precision) O(capacity_bins) O(block_warps) O(ctas_per_sm) O(bins_per_grab) O(max_bins)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(batch.pab_batch_config)
    for item in out[1:]:
        k, v = item.split("=")
        assert getattr(batch.pab_batch_config, k).offset == int(v), k
    c = batch.pab_batch_config_default()
    assert c.max_slots == 512 and c.precision == pab.PAB_MIXED and c.max_bins == pab.MAX_BINS


def test_invalid_batch_configs_are_refused_without_device_work():
    from paper_2511_21031_gb300 import batch
    lib = batch.load()
    for bad in (dict(max_slots=0), dict(max_slots=5000), dict(precision=3), dict(block_warps=17),
                dict(ctas_per_sm=33), dict(bins_per_grab=9), dict(max_bins=64), dict(capacity_bins=-1),
                dict(capacity_bins=pab.MAX_CELLS * pab.MAX_BINS + 1)):
        c = batch.pab_batch_config_default(**bad)
        out = ctypes.c_void_p()
        assert lib.pab_batch_create(ctypes.byref(c), None, ctypes.byref(out)) == pab.PAB_EINVAL
        assert out.value is None
    assert lib.pab_batch_step(None, None) == pab.PAB_EINVAL
    assert lib.pab_batch_bind(None, 0, None, None, None, 1e-8) == pab.PAB_EINVAL
    lib.pab_batch_destroy(None)


def test_config_defaults_are_water_and_paper_tolerance():
    c = pab.pab_config_default()
    assert (c.rho, c.c, c.mu, c.sigma, c.p0, c.gamma, c.pv) == (1000.0, 1500.0, 1e-3, 0.072, 101325.0, 1.4, 0.0)
    assert c.tol == 1e-4 and c.n_bins == 21 and c.R0ref == 10e-6 and c.alpha0 == 4e-5


@pytest.mark.parametrize("bad", [dict(n_bins=20), dict(n_bins=2), dict(n_bins=65), dict(n_cells=0),
                                 dict(rho=-1.0), dict(tol=0.0), dict(stepper=1, n_fixed_sub=0),
                                 dict(precision=7), dict(gas_mode=3), dict(max_attempts=0),
                                 dict(n_bins=21, s_lognormal=0.0), dict(block_warps=17),
                                 dict(n_cells=pab.MAX_CELLS + 1), dict(n_cells=-(1 << 62))])
def test_invalid_configs_are_refused_without_device_work(bad):
    cfg = pab.pab_config_default(**{"n_cells": 8, **bad})
    out = ctypes.c_void_p()
    st = pab.load().pab_create(ctypes.byref(cfg), None, ctypes.byref(out))
    assert st == pab.PAB_EINVAL
    assert out.value is None


@pytest.mark.parametrize("n,nx,ny,nz,dx", [(-1, 4, 4, 4, 1e-3), (1, 0, 4, 4, 1e-3), (1, 4, 4, 4, 0.0),
                                          (1, 4, 4, 4, float("inf")),
                                          (1, 1 << 12, 1 << 12, (1 << 11) + 1, 1e-3),
                                          (pab.MAX_CELLS + 1, 4, 4, 4, 1e-3)])
def test_invalid_el_populations_are_refused_without_device_work(n, nx, ny, nz, dx):
    """Sizes the EL grid and its cell indices cannot hold (nx ny nz or N above the cell cap)
    are refused like the others, before any device call and before any position is read."""
    from paper_2511_21031_gb300 import el
    lib = el.load()
    cfg = pab.pab_config_default()
    out = ctypes.c_void_p()
    pos = (ctypes.c_double * 3)(1e-4, 1e-4, 1e-4)
    R0 = (ctypes.c_double * 1)(1e-5)
    st = lib.pab_el_create(ctypes.byref(cfg), n, ctypes.addressof(pos) if n >= 1 else None,
                           ctypes.addressof(R0) if n >= 1 else None, nx, ny, nz, dx, None,
                           ctypes.byref(out))
    assert st == pab.PAB_EINVAL
    assert out.value is None


def test_null_handle_calls_return_einval():
    lib = pab.load()
    assert lib.pab_bubble_step(None, None, None, 1e-8, None, None) == pab.PAB_EINVAL
    assert lib.pab_moments(None, None, None, None) == pab.PAB_EINVAL
    assert lib.pab_status_flags(None, None, None, None, None, None) == pab.PAB_EINVAL
    assert lib.pab_get_state(None, None, None, None, None) == pab.PAB_EINVAL
    assert lib.pab_set_state(None, None, None, None, None) == pab.PAB_EINVAL
    assert lib.pab_set_block_warps(None, 4) == pab.PAB_EINVAL
    lib.pab_destroy(None)
    assert lib.pab_last_error(None) == b"NULL handle"
    assert pab.status_string(pab.PAB_ESTEP_LIMIT) == "PAB_ESTEP_LIMIT"


def test_pipelined_host_calls_keep_their_host_tensors_alive(monkeypatch):
    """Solver.step_host_async returns before its copies run: the tensors of the last two calls
    (the ones the library may still be copying) stay referenced until host_wait, those of older
    calls are dropped, and a refused call holds nothing."""
    import collections
    import gc
    import types
    import weakref

    import torch
    status = {"rc": pab.PAB_OK}

    class FakeLib:
        def pab_bubble_step_host_async(self, h, p, nb, dt, m, s):
            return status["rc"]

        def pab_host_wait(self, h):
            return pab.PAB_OK

        def pab_last_error(self, h):
            return b"fake"

        def pab_status_string(self, s):
            return b"PAB_ECUDA"

    monkeypatch.setattr(pab, "load", lambda *a, **k: FakeLib())
    sol = object.__new__(pab.Solver)
    sol.handle, sol.n_cells, sol.n_bins = 1, 4, 1
    sol._in_flight = collections.deque(maxlen=2)
    stream = types.SimpleNamespace(cuda_stream=0)
    refs = []
    for k in range(3):
        p = torch.full((4,), float(k), dtype=torch.float64)
        m = torch.empty((7, 4), dtype=torch.float64)
        refs.append((weakref.ref(p), weakref.ref(m)))
        sol.step_host_async(p, 1e-8, moments_host=m, stream=stream)
        del p, m
    gc.collect()
    assert refs[0][0]() is None and refs[0][1]() is None
    assert all(r() is not None for pair in refs[1:] for r in pair)
    sol.host_wait()
    gc.collect()
    assert all(r() is None for pair in refs for r in pair)
    status["rc"] = pab.PAB_ECUDA
    p = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(pab.PabError):
        sol.step_host_async(p, 1e-8, stream=stream)
    assert len(sol._in_flight) == 0
    with pytest.raises(ValueError):
        sol.step_host_async(None, 1e-8, stream=stream)
    sol.handle = None


def test_batch_binding_holds_bound_tensors_and_checks_state_shapes(monkeypatch):
    """The library keeps a bound slot's pointers for every later step, so the Batch holds the
    tensors until the slot is re-bound or released; set_state refuses tensors of the wrong
    shape or type before the library sees them."""
    import gc
    import types
    import weakref

    import torch
    from paper_2511_21031_gb300 import batch

    class FakeLib:
        def pab_batch_bind(self, h, slot, p, nb, m, dt):
            return pab.PAB_OK

        def pab_batch_release(self, h, slot, s):
            return pab.PAB_OK

        def pab_batch_set_state(self, h, slot, R, V, hh, s):
            return pab.PAB_OK

    monkeypatch.setattr(batch, "load", lambda *a, **k: FakeLib())
    b = object.__new__(batch.Batch)
    b.handle, b.device = 1, torch.device("cpu")
    b.slots, b._bound = {0: (4, 3)}, {}
    stream = types.SimpleNamespace(cuda_stream=0)
    p = torch.zeros(4, dtype=torch.float64)
    m = torch.empty((7, 4), dtype=torch.float64)
    rp, rm = weakref.ref(p), weakref.ref(m)
    b.bind(0, p, 1e-8, moments=m)
    del p, m
    gc.collect()
    assert rp() is not None and rm() is not None
    b.bind(0, torch.ones(4, dtype=torch.float64), 1e-8)
    gc.collect()
    assert rp() is None and rm() is None
    q = b._bound[0][0]
    rq = weakref.ref(q)
    del q
    b.release(0, stream=stream)
    gc.collect()
    assert rq() is None and 0 not in b.slots
    b.slots[1] = (4, 3)
    R = torch.zeros((3, 4), dtype=torch.float64)
    b.set_state(1, R, R.clone(), torch.zeros((3, 4), dtype=torch.float32), stream=stream)
    for bad in (dict(R=torch.zeros((4, 3), dtype=torch.float64)), dict(R=torch.zeros((3, 4), dtype=torch.float32)),
                dict(h=torch.zeros((3, 4), dtype=torch.float64)), dict(R=None)):
        kw = dict(R=R, V=R.clone(), h=None)
        kw.update(bad)
        with pytest.raises(ValueError):
            b.set_state(1, kw["R"], kw["V"], kw["h"], stream=stream)
    with pytest.raises(ValueError):
        b.bind(1, torch.zeros(5, dtype=torch.float64), 1e-8)
    b.handle = None


def test_product_path_fails_loudly_without_its_library_or_a_device(monkeypatch, tmp_path):
    """No CPU fallback: a missing library is an error, not a silent substitute, and the solver,
    batch and bubble-cloud classes refuse to run without a CUDA device."""
    import torch
    from paper_2511_21031_gb300 import _build, batch, el
    monkeypatch.setattr(pab, "_LIB", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libpab.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pab.load(build_if_missing=False)
    monkeypatch.undo()
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pab.Solver(8)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        batch.Batch(max_slots=2, capacity_bins=100)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        el.BubbleCloud([[0.0], [0.0], [0.0]], [1e-5], 4, 4, 4, 1e-4)


@pytest.mark.parametrize("header", [os.path.basename(h) for h in HEADERS])
def test_header_compiles_standalone_as_c_and_cpp(header):
    """Each public header is a C ABI: it compiles on its own as C99, C11 and C++17 with all
    warnings as errors, and pulls in nothing but the standard integer types and pab.h."""
    with tempfile.TemporaryDirectory() as d:
        for std, ext, cc in (("c99", "c", "gcc"), ("c11", "c", "gcc"), ("c++17", "cpp", "g++")):
            src = os.path.join(d, "t." + ext)
            open(src, "w").write(f'#include "{header}"\nint main(void) {{ return 0; }}\n')
            r = subprocess.run([cc, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic",
                                "-I", os.path.join(ROOT, "include"), "-c", src, "-o", os.path.join(d, "t.o")],
                               capture_output=True, text=True)
            assert r.returncode == 0, (header, std, r.stderr[-800:])
    text = open(os.path.join(ROOT, "include", header)).read()
    includes = set(re.findall(r'#include\s+[<"]([^>"]+)[>"]', text))
    assert includes <= {"stdint.h", "stddef.h", "pab.h"}, includes


def test_bubble_cloud_set_state_checks_shapes(monkeypatch):
    """The volume-averaged binding refuses state tensors of the wrong length, type or device
    before the library sees them."""
    import torch
    from paper_2511_21031_gb300 import el
    calls = []

    class FakeLib:
        def pab_el_set_state(self, h, R, V, hh, s):
            calls.append((R, V, hh))
            return pab.PAB_OK

    monkeypatch.setattr(el, "load", lambda *a, **k: FakeLib())
    cl = object.__new__(el.BubbleCloud)
    cl.handle, cl.device, cl.N = 1, torch.device("cpu"), 3
    import types
    s = types.SimpleNamespace(cuda_stream=0)
    R = torch.ones(3, dtype=torch.float64)
    cl.set_state(R, R.clone(), torch.ones(3, dtype=torch.float32), stream=s)
    cl.set_state(R, R.clone(), stream=s)
    assert len(calls) == 2 and calls[1][2] is None
    for bad in (dict(R=torch.ones(4, dtype=torch.float64)), dict(R=torch.ones(3, dtype=torch.float32)),
                dict(h=torch.ones(3, dtype=torch.float64)), dict(V=None),
                dict(R=torch.ones((3, 1), dtype=torch.float64))):
        kw = dict(R=R, V=R.clone(), h=None)
        kw.update(bad)
        with pytest.raises(ValueError):
            cl.set_state(kw["R"], kw["V"], kw["h"], stream=s)
    assert len(calls) == 2
    cl.handle = None
