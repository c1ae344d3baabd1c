"""Static checks of the repository's separation rules, on the CPU.

- The product package (the CUDA library and its Python binding) never imports or loads the
  oracle, so no product path can route through it.
- The oracle never imports the product package, and the two share no C source or header.
- Only the tests, the smoke check and the benchmark name the oracle among the top-level files.
- No committed file reads, runs or imports anything under the working folder `_work/`."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2511_21031_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _tracked():
    r = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    if r.returncode != 0:
        return None
    return [os.path.join(ROOT, p) for p in r.stdout.split()]


def test_product_package_never_uses_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|liboracle|pab_oracle", re.M)
    for f in _files(PKG, (".py", ".cu", ".cuh", ".h", ".c")):
        assert not pat.search(open(f).read()), f


def test_oracle_never_uses_the_product_package():
    for f in _files(ORACLE, (".py", ".c", ".h")):
        text = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2511_21031_gb300\b|libpab", text, re.M), f
        assert not re.search(r'#include\s+"(pab|\.\./)', text), f
    for f in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h")):
        assert "orc_" not in open(f).read(), f


def test_only_tests_smoke_and_bench_name_the_oracle_at_top_level():
    allowed = {"__graft_entry__.py", "bench.py"}
    for n in os.listdir(ROOT):
        if n.endswith(".py") and n not in allowed:
            assert not re.search(r"^\s*(import|from)\s+oracle\b", open(os.path.join(ROOT, n)).read(),
                                 re.M), n


def test_nothing_committed_uses_the_working_folder():
    files = _tracked()
    if files is None:
        return
    pat = re.compile(r"""["'/]_work/|_work\.|sys\.path.*_work""")
    for f in files:
        if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".sh", ".ini", ".cfg", ".toml")) and os.path.exists(f):
            if os.path.basename(f) == "test_layout.py":
                continue
            assert not pat.search(open(f, errors="replace").read()), f
