import os
import sys

import pytest

# before anything initialises CUDA: hardware queues for the pipelined Parareal
# streams (see paper_2507_19246_gb300/mqs.py)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # a GPU test cannot run without a device: fail loudly rather than skip if
    # the user explicitly selected gpu tests on a machine without one is left
    # to the tests themselves (they require the library and a device).
    pass
