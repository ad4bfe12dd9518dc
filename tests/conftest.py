import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def built_lib():
    """libevo.so, built in-tree first if missing or stale."""
    from paper_2207_05477_gb300 import build, evo
    build.build()
    return evo.lib()


def pytest_sessionfinish(session, exitstatus):
    """EVO_PARITY_REPORT=<path>: write every parity check's measured errors and bounds."""
    path = os.environ.get("EVO_PARITY_REPORT")
    if not path:
        return
    mod = sys.modules.get("tolerances")
    if mod is not None:
        mod.write_report(path)
