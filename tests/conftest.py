import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))
for _p in (ROOT, TESTS):
    if _p not in sys.path:
        sys.path.insert(0, _p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def oracle_mod():
    # QLBM_ORACLE_DIR names a directory holding a (deliberately altered) copy
    # of the oracle package; the mutation tests run the pins against it.
    alt = os.environ.get("QLBM_ORACLE_DIR")
    if alt:
        sys.path.insert(0, alt)
    import oracle
    if alt:
        assert os.path.dirname(os.path.dirname(os.path.abspath(oracle.__file__))) == os.path.abspath(alt)
    oracle.build()
    return oracle
