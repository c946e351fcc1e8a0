import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Measured errors of the parity checks that go through the `meas` fixture: (test, quantity,
# value, tolerance).  With KS_ERRLOG set, the session writes them there as JSON (the per-result
# error tables are built from that file).
_ERRORS = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("KS_ERRLOG")
    if path and _ERRORS:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(_ERRORS, f, indent=0)


@pytest.fixture
def meas(request):
    """meas(quantity, value, tol): records the measured error and asserts value <= tol."""
    def check(what, value, tol):
        value = float(value)
        _ERRORS.append({"test": request.node.nodeid, "what": what, "value": value, "tol": float(tol)})
        assert value <= tol, (what, value, tol)
    return check
