"""The C-ABI library builds for sm_103a and exports every entry point that
include/psso.h declares (no GPU needed: nothing is called)."""
import ctypes
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


def test_binding_structs_match_header(tmp_path):
    """Every struct of the ABI has the same size and field offsets in the C
    header (compiled by gcc) and in the ctypes binding."""
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    import paper_2110_01470_gb300 as psso
    structs = {"psso_problem": psso.psso_problem, "psso_config": psso.psso_config,
               "psso_log_entry": psso.psso_log_entry, "psso_stats_t": psso.psso_stats_t,
               "psso_tune_report": psso.psso_tune_report, "psso_peaks": psso.psso_peaks}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "psso.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines))
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {tuple(l.split()[:2]): int(l.split()[2]) for l in got if l.strip()}
    for name, cls in structs.items():
        assert c[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert c[(name, field)] == getattr(cls, field).offset, (name, field)


def test_binding_config_fields():
    """The binding builds a psso_config from field names and rejects unknown ones."""
    import paper_2110_01470_gb300 as psso
    cfg = psso._config("f32", {"batch_blocks_per_sm": 3, "threads_per_block": 384, "log_stride": 1})
    assert (cfg.precision, cfg.batch_blocks_per_sm, cfg.threads_per_block, cfg.log_stride) == (1, 3, 384, 1)
    assert cfg.flow == 0 and cfg.stream is None
    with pytest.raises(TypeError):
        psso._config("f64", {"threads": 64})


def test_entry_points_fail_cleanly_without_gpu(libpath):
    """Without a GPU, the entry points return an error status (no crash, no
    CPU fallback); the NVTX ranges around them are inert."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU tests cover the entry points")
    import paper_2110_01470_gb300 as psso
    import workload
    psso.load(libpath)
    p = workload.problem("sphere", 16, 4, seed=1)
    with pytest.raises(psso.PssoError) as e:
        psso.psso_create_ex([p], "f64")
    assert e.value.status == psso.PSSO_ERR_CUDA
    with pytest.raises(psso.PssoError):
        psso.psso_run(None, 1)
    with pytest.raises(psso.PssoError):
        psso.psso_autotune([p], "f64", generations=1)


def test_check_entry_points_unsupported_in_default_build(libpath):
    """The index-check calls exist in every build; the default build answers
    PSSO_ERR_UNSUPPORTED without touching the device."""
    import paper_2110_01470_gb300 as psso
    psso.load(libpath)
    for call in (lambda: psso.psso_check_report(), lambda: psso.psso_check_selftest(5)):
        with pytest.raises(psso.PssoError) as e:
            call()
        assert e.value.status == psso.PSSO_ERR_UNSUPPORTED
        assert "checked build" in psso.psso_last_error()
