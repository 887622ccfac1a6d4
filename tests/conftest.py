import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_sessionfinish(session, exitstatus):
    """With CEMTAMP_DEBUG=1 the tests run on the bounds-checked library: the
    session fails if any of its index checks fired."""
    if os.environ.get("CEMTAMP_DEBUG") != "1":
        return
    P = sys.modules.get("paper_2512_11571_gb300")
    torch = sys.modules.get("torch")
    if P is None or P._lib is None or torch is None or not torch.cuda.is_available():
        return
    code = P.cem_debug_status()
    if code != 0:
        print(f"\nbounds check fired in the debug library: code {code}")
        session.exitstatus = 1


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle
