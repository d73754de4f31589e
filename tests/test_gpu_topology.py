"""The topology-specialised screen (links_topo_create / links_simulate_topology).

Its mechanisms get the generic screen's flags, lock steps and minimum discriminants
bit for bit (the same operations in the same order), the others go to the generic
screen, so every output of a simulation equals that of links_simulate (MIXED): the
generic path is itself checked against the FP64 oracle in test_gpu_sim.py.
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


def both(L, batch, T, out_mode, topo_of=0, lanes=0):
    from paper_2208_14567_gb300.api import Simulator, to_device
    with Simulator(batch.B, batch.nmax) as s:
        s.build(to_device(batch))
        a = s.simulate(T, L.MIXED, out_mode)
        s.sync()
        ra = {k: None if v is None else v.cpu().numpy() for k, v in a.__dict__.items()}
        topo = L.links_topo_create(s.ctx, int(batch.n_joints[topo_of]), batch.adj[topo_of], batch.jtype[topo_of],
                                   lanes)
        try:
            esc = torch.zeros(1, dtype=torch.int32, device="cuda")
            o = s.simulate_topology(topo, T, out_mode, n_escaped=esc)
            s.sync()
            rb = {k: None if v is None else v.cpu().numpy() for k, v in o.__dict__.items()}
            info = L.links_topo_info(topo)
        finally:
            L.links_topo_free(topo)
    return ra, rb, int(esc.item()), info


def check_same(ra, rb, out_mode, L):
    for k in ("valid", "lock_step", "min_disc"):
        assert np.array_equal(ra[k], rb[k], equal_nan=True), k
    if out_mode == L.OUT_VALID_ONLY:
        n = int(ra["n_out"][0])
        assert int(rb["n_out"][0]) == n
        assert np.array_equal(ra["out_index"][:n], rb["out_index"][:n])
        assert np.array_equal(ra["traj"][:n], rb["traj"][:n], equal_nan=True)
        assert np.array_equal(ra["path"][:n], rb["path"][:n], equal_nan=True)
    else:
        assert np.array_equal(ra["traj"], rb["traj"], equal_nan=True)
        assert np.array_equal(ra["path"], rb["path"], equal_nan=True)


@pytest.mark.parametrize("n,T,lanes", [(6, 200, 0), (8, 200, 8), (8, 200, 32), (10, 64, 16), (5, 37, 0)])
def test_one_topology_matches_generic(L, n, T, lanes):
    """All samples of one topology of the paper's generator: identical outputs, and the
    specialised kernel decides most of them itself."""
    batch = I.paper_batch(1, 20000, n, seed=n)
    for out_mode in (L.OUT_FULL, L.OUT_VALID_ONLY):
        ra, rb, esc, info = both(L, batch, T, out_mode, lanes=lanes)
        check_same(ra, rb, out_mode, L)
        assert esc == 0
    print(f"[topology n={n} T={T} lanes={lanes}] dyads {info['dyads']} valid {ra['valid'].mean():.3f} escaped {esc} "
          f"compile {info['compile_ms']:.0f} ms")


def test_other_topologies_escape(L):
    """A batch of eight topologies with the kernel of the first: the other seven's
    mechanisms escape to the generic screen and every output is still the same."""
    batch = I.paper_batch(8, 1500, 8, seed=21)
    ra, rb, esc, _ = both(L, batch, 200, L.OUT_FULL)
    check_same(ra, rb, L.OUT_FULL, L)
    assert esc == 7 * 1500


def test_dyad_workload_and_bad_topology(L):
    """Random dyad-built candidates (mostly other topologies) and planted ill-formed
    mechanisms; a topology that does not plan is refused."""
    batch = I.dyad_batch(5000, 6, 8, seed=5)
    ra, rb, esc, _ = both(L, batch, 200, L.OUT_FULL, topo_of=3)
    check_same(ra, rb, L.OUT_FULL, L)
    from paper_2208_14567_gb300.api import Simulator
    adj = np.zeros((6, 6), np.uint8)
    jt = np.array([0, 2, 1, 1, 1, 1], np.int8)
    with Simulator(4, 6) as s:
        with pytest.raises(L.LinksError):
            L.links_topo_create(s.ctx, 6, adj, jt)
        with pytest.raises(L.LinksError):
            L.links_topo_create(s.ctx, int(batch.n_joints[0]), batch.adj[0], batch.jtype[0], 12)


def test_topology_plan_mismatch_refused(L):
    """A topology with more joints than the plan's n_max is refused (its kernel would read
    past the plan's rows)."""
    from paper_2208_14567_gb300.api import Simulator, to_device
    small = I.paper_batch(1, 64, 6, seed=1)
    big = I.paper_batch(1, 4, 8, seed=2)
    with Simulator(small.B, small.nmax) as s:
        s.build(to_device(small))
        topo = L.links_topo_create(s.ctx, int(big.n_joints[0]), big.adj[0], big.jtype[0])
        try:
            with pytest.raises(L.LinksError):
                s.simulate_topology(topo, 50, L.OUT_FULL)
        finally:
            L.links_topo_free(topo)
