import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library handle (GPU tests only)."""
    import paper_2110_01470_gb300 as psso
    psso.load()
    return psso


def pytest_sessionfinish(session, exitstatus):
    """With PSSO_CHECK_REPORT=<file> (a run against the index-checked library),
    writes the library's first failed index check, {"site": 0} if none."""
    out = os.environ.get("PSSO_CHECK_REPORT")
    if not out:
        return
    import json
    import paper_2110_01470_gb300 as psso
    site, index = psso.psso_check_report()
    with open(out, "w") as f:
        json.dump({"site": site, "index": index}, f)
