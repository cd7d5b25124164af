import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build_oracle()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """Achieved errors of the GPU parity checks, one line each."""
    from tests import gpu_util
    rows = gpu_util.PARITY
    if not rows:
        return
    tr = terminalreporter
    tr.section("parity: achieved error vs the FP64 oracle (or closed form)")
    for wl, prec, q, err, tol in rows:
        tr.write_line("%-34s %-10s %-34s %.3e  (tol %.0e)" % (wl, prec, q, err, tol))
    path = os.environ.get("XX_PARITY_JSON")
    if path:
        import json
        with open(path, "w") as f:
            json.dump([dict(workload=w, precision=p, quantity=q, error=e, tol=t)
                       for w, p, q, e, t in rows], f, indent=1)
