import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def tc():
    """The library's Python binding, loaded on a GPU machine (fails loudly if absent)."""
    if not cuda_available():
        pytest.skip("no CUDA device")
    import paper_1602_02740_gb300 as lib
    from paper_1602_02740_gb300 import tc as _binding  # noqa: F401  (loads the submodule)
    return lib
