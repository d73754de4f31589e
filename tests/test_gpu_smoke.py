"""__graft_entry__.smoke(): the small end-to-end check (plan build, both precisions, FULL
rows against the oracle) runs as a test too, so that a change that breaks it shows up
with the rest of the GPU suite."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_smoke():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import __graft_entry__ as entry
    entry.smoke()
