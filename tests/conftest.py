import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libspca.so")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped (not failed) on machines without a GPU only when the user
    # asked for them explicitly there; the default CPU run deselects them with -m "not gpu".
    pass


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O
