import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU statistics")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


# Counts that a parity test tolerates (rounding-level mismatches it has explained), printed at
# the end of the run so that drift shows even when every test passes.
_PARITY_NOTES = []


def parity_note(msg: str) -> None:
    _PARITY_NOTES.append(msg)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if _PARITY_NOTES:
        terminalreporter.section("parity notes")
        for m in _PARITY_NOTES:
            terminalreporter.write_line(m)
