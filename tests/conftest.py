import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


def pytest_sessionstart(session):
    # the host-side tests call libfth.so (fitter, transforms, validation) on the CPU:
    # build it once up front (nvcc cross-compiles without a GPU)
    from paper_1402_2095_gb300 import build
    build.build()
