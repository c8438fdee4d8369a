import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libte")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    """`slow` CPU tests (minutes of oracle work on the paper's full-size system)
    run only when TE_RUN_SLOW=1 is set."""
    if os.environ.get("TE_RUN_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow oracle pin: set TE_RUN_SLOW=1 to run")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def te():
    """The CUDA library binding; GPU tests fail loudly if it cannot load."""
    if not cuda_available():
        pytest.fail("gpu test selected but no CUDA device is visible")
    from paper_2205_15346_gb300 import te as _te
    return _te
