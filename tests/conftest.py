import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def lope():
    """The CUDA library, built in-tree if needed (no GPU required to build or load)."""
    from paper_1502_03504_gb300 import build

    build.build()
    import paper_1502_03504_gb300 as L

    L.load()
    return L


# Measured errors of the reduced-precision parity tests against the FP64
# oracle, next to the bound each test asserts: one entry per configuration.
# When LOPE_ERROR_REPORT names a file, the session writes them there as JSON.
_ERRORS = {}


@pytest.fixture(scope="session")
def error_report():
    return _ERRORS


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("LOPE_ERROR_REPORT")
    if path and _ERRORS:
        import json

        with open(path, "w") as fh:
            json.dump(_ERRORS, fh, indent=1, sort_keys=True)
