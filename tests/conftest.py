import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running oracle physics check")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Errors of every GPU-vs-oracle comparison of the run: rho and u as the tests bound them, the
    plain field-relative L-infinity error of u beside the scaled one, and the momentum totals."""
    try:
        from tests import parity_util
    except Exception:
        return
    if not parity_util.RECORDS:
        return
    tr = terminalreporter
    tr.write_sep("-", "GPU vs FP64 oracle")
    tr.write_line(f"{'test':<86} {'rho':>9} {'u/scale':>9} {'u plain':>9} {'sum rho u':>9}")
    for name, er, eu, eup, em in parity_util.RECORDS:
        tr.write_line(f"{name[-86:]:<86} {er:9.2e} {eu:9.2e} {eup:9.2e} {em:9.2e}")
