"""Shared pytest setup: markers and import paths."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


import pytest


@pytest.fixture(scope="session")
def gpu_library():
    """Build and load libvplbm.so; GPU tests fail (not skip) without CUDA."""
    import torch
    import paper_1905_05110_gb300 as vp
    from paper_1905_05110_gb300 import build as vbuild
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    vbuild.build()
    lib = vp.load_library()
    torch.cuda.init()
    return lib
