import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def cov():
    """The CUDA binding, with libcov.so built for sm_103a."""
    from paper_2511_11514_b300 import build_lib
    build_lib.build()
    from paper_2511_11514_b300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="session")
def _session_ctx(cov):
    c = cov.Context(0)
    yield c
    c.close()


@pytest.fixture
def ctx(_session_ctx):
    """The shared context, with its device status cleared before each test."""
    _session_ctx.device_status()
    return _session_ctx


def dev32(a):
    import torch
    return torch.as_tensor(a, dtype=torch.float32).cuda().contiguous()


def dev64(a):
    import torch
    return torch.as_tensor(a, dtype=torch.float64).cuda().contiguous()


def host(t):
    return t.detach().cpu().double().numpy()


def rel_norm(a, b):
    import numpy as np
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))
