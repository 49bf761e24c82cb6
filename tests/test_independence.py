"""The oracle and the CUDA path share no code: neither imports the other, the seeded input
generators (synthetic/) import neither, and only the tests, the smoke entry point and the bench's
CPU-baseline legs import the oracle.  Checked by reading the sources."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SKIP = {".git", "_work", "gpurun_out", "baseline", "_build", "__pycache__", ".pytest_cache"}
IMPORTS_ORACLE = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)|importlib\.import_module\(\s*['\"]oracle", re.M)
IMPORTS_PACKAGE = re.compile(r"^\s*(import\s+paper_2105_04940_gb300\b|from\s+paper_2105_04940_gb300\b|from\s+\.\.)", re.M)


def _sources(*exts):
    for dirpath, dirnames, filenames in os.walk(ROOT):
        dirnames[:] = [d for d in dirnames if d not in SKIP]
        for f in filenames:
            if f.endswith(exts):
                path = os.path.join(dirpath, f)
                yield os.path.relpath(path, ROOT), open(path, encoding="utf-8", errors="replace").read()


def test_only_tests_smoke_and_bench_import_the_oracle():
    allowed = ("tests/", "oracle/")
    users = sorted(p for p, text in _sources(".py") if IMPORTS_ORACLE.search(text))
    assert users, "the oracle is imported somewhere"
    for p in users:
        assert p.startswith(allowed) or p in ("__graft_entry__.py", "bench.py"), p


def test_the_package_never_names_the_oracle():
    pkg = "paper_2105_04940_gb300" + os.sep
    for p, text in _sources(".py", ".cu", ".cuh", ".h", ".c", ".cpp"):
        if p.startswith(pkg) or p.startswith("include" + os.sep):
            assert not IMPORTS_ORACLE.search(text), p
            assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", text), p


def test_oracle_and_generators_never_import_the_package():
    for p, text in _sources(".py"):
        if p.startswith(("oracle" + os.sep, "synthetic" + os.sep)):
            assert not IMPORTS_PACKAGE.search(text), p
        if p.startswith("synthetic" + os.sep):
            assert not IMPORTS_ORACLE.search(text), p
