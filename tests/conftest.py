import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs through the C-ABI library)")
    config.addinivalue_line("markers", "slow: longer CPU checks")


def pytest_collection_modifyitems(config, items):
    # run the no-allocation entry point's test file (if any) last
    items.sort(key=lambda it: os.path.basename(str(it.fspath)).startswith("test_zz"))
