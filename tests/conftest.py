"""Shared test setup: the ``gpu`` marker, module paths and builders."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def cuda_lib():
    """Builds (if stale) and loads the CUDA library; skips without a GPU."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_07826_gb300 import build as B
    B.build()
    from paper_1706_07826_gb300 import spvar
    spvar.lib()
    return spvar
