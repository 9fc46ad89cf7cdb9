import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libaesgb.so")


@pytest.fixture(scope="session")
def orc():
    import oracle

    return oracle.oracle()


@pytest.fixture(scope="session")
def aes():
    """The CUDA library binding, built in-tree if needed.  Fails (does not skip) when the
    library cannot be built or loaded: there is no fallback."""
    import paper_1506_08503_gb300 as aes

    if not aes.LIB_PATH.exists():
        aes.build()
    aes.lib()
    return aes


@pytest.fixture(scope="session")
def cuda(aes):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a visible CUDA device")
    torch.cuda.init()
    return torch.device("cuda:0")


@pytest.fixture(scope="session")
def aes_lib_ready(aes, cuda):
    return aes
