"""The checked build compiles on the CPU: every kernel source with -DPAB_CHECKED, linked into
libpab_checked.so, which exports the whole C ABI plus the bounds report.  (The GPU suite runs
under it with PAB_CHECKED=1; the report is read after every GPU test by tests/conftest.py.)"""
import ctypes
import os

import pytest

from paper_2511_21031_gb300 import _build, pab


@pytest.mark.slow
def test_checked_library_builds_and_exports_the_abi():
    lib = _build.build(checked=True)
    assert lib == _build.LIB_CHECKED and os.path.exists(lib)
    handle = ctypes.CDLL(lib)
    for name in pab.EXPORTS:
        getattr(handle, name)
    # the unchecked library carries the same entry points
    plain = ctypes.CDLL(_build.build())
    getattr(plain, "pab_check_report")
