"""The index-checked build (-DPSSO_CHECKED): every kernel verifies each index
it computes into a buffer before the access and records the first failure.

The GPU suite runs again, in a child process, against the checked copy of the
library (PSSO_LIBRARY): every test must pass, and afterwards the library must
report no failed check.  The record-and-report path itself is proven by the
self-test entry point, a failed check with no memory access."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the timing-only files add nothing to index coverage
SKIP_FILES = ("test_gpu_checked.py", "test_gpu_microbench.py", "test_gpu_autotune.py")


@pytest.fixture(scope="module")
def checked_lib():
    if os.environ.get("PSSO_LIBRARY"):
        pytest.skip("already running against another library build")
    from paper_2110_01470_gb300.build import build_library
    return build_library(checked=True)


def _child_env(path, **extra):
    env = dict(os.environ, PSSO_LIBRARY=path, PYTHONPATH=ROOT)
    env.update(extra)
    return env


def test_selftest_records_and_clears(checked_lib):
    code = ("import paper_2110_01470_gb300 as p\n"
            "p.load()\n"
            "out = [p.psso_check_report()]\n"
            "p.psso_check_selftest(123456789)\n"
            "p.psso_check_selftest(-5)\n"
            "out.append(p.psso_check_report(clear=True))\n"
            "out.append(p.psso_check_report())\n"
            "p.psso_check_selftest(-5)\n"
            "out.append(p.psso_check_report(clear=True))\n"
            "print(out)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=_child_env(checked_lib),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    # first failure wins; clearing resets the record; negative indices survive
    assert r.stdout.strip() == str([(0, 0), (1, 123456789), (0, 0), (1, -5)])


def test_gpu_suite_under_index_checks(checked_lib, tmp_path):
    report = tmp_path / "report.json"
    files = sorted(f for f in os.listdir(os.path.join(ROOT, "tests"))
                   if f.startswith("test_") and f.endswith(".py") and f not in SKIP_FILES)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           *[os.path.join("tests", f) for f in files]]
    r = subprocess.run(cmd, cwd=ROOT, env=_child_env(checked_lib, PSSO_CHECK_REPORT=str(report)),
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert "passed" in r.stdout.splitlines()[-1]
    rep = json.loads(report.read_text())
    assert rep == {"site": 0, "index": 0}, rep
