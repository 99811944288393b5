import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def mp():
    """The built library's binding on a CUDA device (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_21694_gb300 import build
    build.build()
    from paper_2509_21694_gb300 import binding
    return binding
