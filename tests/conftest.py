import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def repo_root():
    return ROOT


def pytest_collection_modifyitems(session, config, items):
    # the all-steps parity tests need minutes of oracle work: start it in background processes
    # now, so that it runs while the other tests run
    if any("test_gpu_zlong" in it.nodeid for it in items):
        try:
            import torch

            if not torch.cuda.is_available():
                return
        except Exception:
            return
        import long_oracle

        long_oracle.start()
