import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    try:
        from tests.parity_util import VISIT_LOG
    except Exception:
        return
    if not VISIT_LOG:
        return
    tr = terminalreporter
    tr.write_sep("-", "visit lists that differ from the oracle's, each explained by the margin")
    lines = [f"{bad:6d} of {n:9d} rays ({100.0 * bad / max(n, 1):.3f}%)  {name}"
             for name, n, bad in VISIT_LOG]
    for ln in lines:
        tr.write_line(ln)
    path = os.environ.get("SALF_VISIT_LOG")
    if path:
        with open(path, "w") as f:
            f.write("\n".join(lines) + "\n")
