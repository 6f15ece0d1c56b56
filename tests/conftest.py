import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def pytest_collection_modifyitems(config, items):
    # GPU tests fail loudly (not skip) when the GPU is missing: run them with -m gpu
    # only where a GPU exists.
    pass


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.lib()
