import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_sessionfinish(session, exitstatus):
    """Under TUCKER_CHECK_REPORT (set by the checked-build test for its child run): write the
    library's tucker_check_site() after all tests, from the process that ran the kernels."""
    out = os.environ.get("TUCKER_CHECK_REPORT")
    if not out:
        return
    from paper_2010_10638_gb300 import tucker
    with open(out, "w") as f:
        f.write(str(tucker.tucker_check_site()))


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


@pytest.fixture(params=["cluster", "persistent", "multi"])
def qrp_form(request, monkeypatch):
    """Runs a test with each form of the QRP: the cluster form (one grid barrier per
    reflector; the default wherever its shared-memory plan fits), the persistent
    cooperative form (two grid barriers per reflector), and the multi-kernel form (three
    launches per reflector; what runs when neither single-launch form fits)."""
    monkeypatch.setenv("TUCKER_QRP_FORM", request.param)
    return request.param
