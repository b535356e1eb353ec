import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


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
