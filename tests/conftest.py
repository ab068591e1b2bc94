import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


class HostBuffers:
    """Two host byte buffers shared by the full-size tests of a session, grown
    (never shrunk) to the largest request.  The inputs of every full-size test
    are generated into them: allocating and freeing tens of GB per test leaves
    the host reclaiming memory, which stalls host-device copies for a while
    afterwards."""

    def __init__(self):
        self.a = self.b = None

    def views(self, n, stride):
        import numpy as np
        need = n * stride
        if self.a is None or self.a.size < need:
            self.a = self.b = None
            self.a, self.b = np.empty(need, np.uint8), np.empty(need, np.uint8)
        return self.a[:need].reshape(n, stride), self.b[:need].reshape(n, stride)


@pytest.fixture(scope="session")
def host_buffers():
    return HostBuffers()
