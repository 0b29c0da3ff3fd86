import os
import sys

import pytest

# The oracle's OpenMP threads wait briefly, then sleep, at the end of each
# parallel loop (libgomp reads this when it loads, before any test imports the
# oracle). Its many small loops on small lattices otherwise spin at every barrier,
# and on a machine whose cores are shared a test can then run a hundred times
# slower than alone.
os.environ.setdefault("GOMP_SPINCOUNT", "10000")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
