"""The allocation-free compaction entry point, called through the C ABI.

It serves callers that cannot allocate device memory (a host framework that owns the
memory pool, or code on a latency budget), so its scratch is a static device array
inside the library.  Its rows must equal those links_simulate writes in VALID_ONLY
mode, on two calls in a row (the second call finds the first call's leftovers in the
shared array).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2208_14567_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_14567_gb300 import links
    links.lib()
    return links


def test_static_compaction_matches_links_simulate(L):
    from paper_2208_14567_gb300.api import Simulator, to_device
    stream = torch.cuda.current_stream()
    for seed, B in ((21, 9000), (22, 5000)):  # two calls in a row, the second smaller
        batch = I.dyad_batch(B, 6, 10, seed=seed)
        with Simulator(B, batch.nmax, stream=stream) as s:
            s.build(to_device(batch))
            o = s.simulate(96, L.MIXED, L.OUT_VALID_ONLY, traj=False, path=False)
            s.sync()
            n_ref = int(o.n_out[0])
            ref = o.out_index[:n_ref].cpu().numpy()
            idx = torch.full((B,), -7, dtype=torch.int32, device="cuda")
            n = torch.full((1,), -7, dtype=torch.int32, device="cuda")
            L.links_compact_valid_static(o.valid, idx, n, stream)
            torch.cuda.synchronize()
            assert int(n[0]) == n_ref
            assert np.array_equal(idx[:n_ref].cpu().numpy(), ref)
            assert (idx[n_ref:].cpu().numpy() == -7).all()
            assert np.array_equal(ref, np.nonzero(o.valid.cpu().numpy())[0])


def test_static_compaction_rejects_oversized_batches(L):
    big = torch.zeros(4194304 + 1, dtype=torch.uint8, device="cuda")
    idx = torch.empty(16, dtype=torch.int32, device="cuda")
    n = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(L.LinksError) as e:
        L.links_compact_valid_static(big, idx, n)
    assert e.value.status == L.EINVAL and "4194304" in str(e.value)
