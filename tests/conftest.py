import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")


@pytest.fixture(scope="session")
def lib():
    """The built C library (compiled in-tree on first use)."""
    from paper_2101_04847_gb300 import build, lbm

    build.build_library()
    return lbm.load_library()


@pytest.fixture(scope="session")
def gpu(lib):
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return lib
