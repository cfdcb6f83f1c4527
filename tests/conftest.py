import os
import sys

import pytest

# The full-size tests hold most of the device at once (ResNet-50's tensor-core
# weight tiles, outputs and masks); growable segments keep freed blocks of
# one size usable for allocations of another.  Read when CUDA starts.
os.environ.setdefault("PYTORCH_ALLOC_CONF", "expandable_segments:True")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O
