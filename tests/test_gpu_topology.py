"""The topology-specialised screen (links_topo_create / links_simulate_topology).

Its mechanisms get the generic screen's flags, lock steps and minimum discriminants
bit for bit (the same operations in the same order), the others go to the generic
screen, so every output of a simulation equals that of links_simulate (MIXED).  The
specialised path is also checked against the FP64 oracle directly.
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


@pytest.mark.parametrize("n,lanes", [(6, 0), (8, 16), (10, 32), (12, 0)])
def test_topology_screen_matches_oracle(L, n, lanes):
    """The topology-specialised path against the FP64 oracle directly: 4000 position
    samples of one paper topology, LINKS_MIXED FULL through links_simulate_topology --
    flags identical outside the oracle's margin (min |q| <= 1e-9), positions within
    1e-5 of the bounding-box diagonal at every step both sides simulated, NaN from the
    lock on, min_disc within 1e-4 + 1e-3 q."""
    from conftest import bbox_diag
    from oracle import oracle as O
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = I.paper_batch(1, 4000, n, seed=40 + n)
    T = 200
    ref = O.simulate(batch, T)
    with Simulator(batch.B, batch.nmax) as s:
        s.build(to_device(batch))
        topo = L.links_topo_create(s.ctx, int(batch.n_joints[0]), batch.adj[0], batch.jtype[0], lanes)
        try:
            esc = torch.zeros(1, dtype=torch.int32, device="cuda")
            o = s.simulate_topology(topo, T, L.OUT_FULL, n_escaped=esc)
            s.sync()
            g = {k: None if v is None else v.cpu().numpy() for k, v in o.__dict__.items()}
        finally:
            L.links_topo_free(topo)
    assert int(esc.item()) == 0
    margin = ~(ref.min_abs_q > 1e-9)
    mism = (g["valid"] != ref.valid) | (g["lock_step"] != ref.lock_step)
    assert not (mism & ~margin).any()
    Ld = bbox_diag(batch.pos, batch.n_joints)
    lr = np.where(ref.lock_step < 0, T, ref.lock_step)
    lg = np.where(g["lock_step"] < 0, T, g["lock_step"])
    stop = np.minimum(lr, lg)
    tm = np.arange(T)[None, :] < stop[:, None]
    err = np.abs(g["traj"][:, :n].astype(np.float64) - ref.traj[:, :n]).max(-1)  # [B, n, T]
    e = np.where(tm[:, None, :], err, 0.0).max((1, 2)) / Ld
    assert (e <= 1e-5).all(), e.max()
    after = np.arange(T)[None, :] >= lg[:, None]
    assert np.isnan(g["traj"][:, :n][np.broadcast_to(after[:, None, :], (batch.B, n, T))]).all()
    pe = np.where(tm, np.abs(g["path"].astype(np.float64) - ref.path).max(-1), 0.0).max(1) / Ld
    assert (pe <= 1e-5).all()
    ok = (ref.lock_step != 0) & (g["lock_step"] == ref.lock_step)
    dq = np.abs(g["min_disc"][ok] - ref.min_disc[ok])
    assert (dq <= 1e-4 + 1e-3 * ref.min_disc[ok]).all()
    print(f"[topology vs oracle n={n}] valid {g['valid'].mean():.3f} margin cases {int(margin.sum())} "
          f"max position error / L {e.max():.2e}")


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
