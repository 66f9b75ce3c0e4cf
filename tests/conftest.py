import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(autouse=True)
def _checked_build_index_checks():
    """Under the index-checked build (UTRACK_CHECKED=1) every handle a test
    closed must have passed its kernels' index checks."""
    yield
    if os.environ.get("UTRACK_CHECKED", "") != "1" or "paper_2505_08222_gb300" not in sys.modules:
        return
    import gc

    ut = sys.modules["paper_2505_08222_gb300"]
    gc.collect()
    failures = list(ut.CHECK_FAILURES)
    ut.CHECK_FAILURES.clear()
    assert not failures, failures
