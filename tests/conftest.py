import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); parity tests of the device path")
    config.addinivalue_line("markers", "slow: full-size cases (minutes of CPU)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build_lib()
    return oracle


@pytest.fixture(scope="session")
def matgen_mod():
    from paper_1907_06487_gb300 import matgen
    matgen.build_lib()
    return matgen
