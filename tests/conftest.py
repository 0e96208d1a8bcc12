import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    from oracle import build
    build.build()
    return oracle


def jl_mpmath(l, x, dps=30):
    """Reference j_l(x) from mpmath's Bessel J of half-integer order."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    if x == 0:
        return 1.0 if l == 0 else 0.0
    v = mp.besselj(l + 0.5, x, maxterms=10 ** 7, maxprec=60000) * mp.sqrt(mp.pi / (2 * mp.mpf(x)))
    return float(v)
