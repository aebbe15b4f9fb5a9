import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def gpu_lib():
    """The C-ABI library, built in-tree; skips when no GPU is present."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12430_gb300 import gwstream

    return gwstream.lib()


@pytest.fixture(scope="session")
def gpu_free_lib():
    """The C-ABI library for its host-only entry points (no GPU needed)."""
    from paper_2108_12430_gb300 import gwstream

    return gwstream.lib()
