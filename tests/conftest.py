import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def bbox_diag(pos, n):
    """Bounding-box diagonal of the first n initial positions of each mechanism."""
    import numpy as np
    p = np.asarray(pos, dtype=np.float64)
    m = np.arange(p.shape[1])[None, :] < np.asarray(n)[:, None]
    hi = np.where(m[..., None], p, -np.inf).max(1)
    lo = np.where(m[..., None], p, np.inf).min(1)
    return np.sqrt(((hi - lo) ** 2).sum(-1))


@pytest.fixture(scope="session")
def oracle_lib():
    from oracle import oracle
    oracle.lib()
    return oracle
