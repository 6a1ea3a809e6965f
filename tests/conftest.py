import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger CPU case")


@pytest.fixture(scope="session")
def olib():
    import oracle
    return oracle.load()


def pytest_terminal_summary(terminalreporter):
    # the precision report of the GPU parity tests: every comparison with the
    # FP64 oracle, largest errors per method and precision
    util = sys.modules.get("tests.gpu_util") or sys.modules.get("gpu_util")
    if util is None or not getattr(util, "PRECISION_LOG", None):
        return
    terminalreporter.section("precision vs the FP64 oracle")
    for line in util.precision_summary():
        terminalreporter.write_line(line)
