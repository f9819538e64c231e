"""The C-ABI library builds for sm_103a and exports every entry point that
include/psso.h declares (no GPU needed: nothing is called)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "psso.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psso_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2110_01470_gb300.build import build_library
    return build_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("psso_create", "psso_create_ex", "psso_run", "psso_best", "psso_destroy",
                     "psso_evaluate", "psso_get_state", "psso_get_log", "psso_save", "psso_load",
                     "psso_last_error", "psso_sync", "psso_stats", "psso_generation"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (psso_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    import ctypes
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n)
    import paper_2110_01470_gb300 as psso
    assert psso.load() is not None


def test_binding_names_match_header():
    import paper_2110_01470_gb300 as psso
    for n in _declared():
        assert callable(getattr(psso, n)), n


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2110_01470_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "psso_oracle" not in text and "liboracle" not in text, f
