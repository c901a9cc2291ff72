import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")

# liboci honours its OCI_* test and profiling overrides only with this switch
# set; tests that pin a kernel or a shape set the override itself.
os.environ.setdefault("OCI_TEST_HOOKS", "1")
