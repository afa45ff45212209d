import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionfinish(session, exitstatus):
    """Write the achieved parity errors (tests/parity.py) to $PTYLM_PARITY_LOG, if set."""
    path = os.environ.get("PTYLM_PARITY_LOG")
    if path:
        from tests import parity
        parity.write_log(path)
