"""The seeded input generator: determinism and the structure the recipes promise."""
import numpy as np
import pytest

from paper_2208_14567_gb300 import inputs as I


def test_stream_is_counter_addressed():
    s = I.Stream(7, 3)
    a = s.u64(np.arange(100))
    b = s.u64(np.arange(50, 100))
    assert np.array_equal(a[50:], b)
    assert not np.array_equal(I.Stream(7, 4).u64(np.arange(10)), a[:10])
    u = s.uniform(np.arange(100000))
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_splitmix64_reference_value():
    # splitmix64 with state 0: first output of the published generator (Vigna).
    z = I._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_dyad_batch_structure():
    b = I.dyad_batch(4000, 6, 8, seed=0)
    assert b.adj.dtype == np.uint8 and b.jtype.dtype == np.int8 and b.pos.dtype == np.float32
    assert np.array_equal(b.adj, b.adj.transpose(0, 2, 1))
    assert not b.adj[:, np.arange(8), np.arange(8)].any()
    assert set(np.unique(b.n_joints)) == {6, 7, 8}
    nfix = (b.jtype == 0).sum(1)
    assert nfix.min() >= 2 and nfix.max() <= 3
    assert ((b.jtype == 2).sum(1) == 1).all()
    # every simple joint has exactly two links to lower-index joints (sequential dyad addition)
    for m in range(200):
        for k in range(3, b.n_joints[m]):
            if b.jtype[m, k] == 1:
                assert b.adj[m, k, :k].sum() == 2
                par = np.nonzero(b.adj[m, k, :k])[0]
                assert not (b.jtype[m, par] == 0).all()
    pad = np.arange(8)[None, :] >= b.n_joints[:, None]
    assert (b.jtype[pad] == -1).all() and (b.pos[pad] == 0).all()
    live = ~pad
    assert b.pos[live].min() >= 0.0 and b.pos[live].max() < 1.0


def test_dyad_batch_deterministic_and_seeded():
    a = I.dyad_batch(300, 6, 20, seed=3)
    b = I.dyad_batch(300, 6, 20, seed=3)
    c = I.dyad_batch(300, 6, 20, seed=4)
    for x, y in ((a.adj, b.adj), (a.pos, b.pos), (a.jtype, b.jtype), (a.n_joints, b.n_joints)):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.pos, c.pos)
    # prefix property: the first rows do not depend on the batch size
    d = I.dyad_batch(100, 6, 20, seed=3)
    assert np.array_equal(d.adj, a.adj[:100]) and np.array_equal(d.pos, a.pos[:100])


def test_permute_is_a_relabeling():
    a = I.dyad_batch(50, 6, 10, seed=1)
    p = I.dyad_batch(50, 6, 10, seed=1, permute=True)
    for m in range(50):
        n = a.n_joints[m]
        # same multiset of degrees and types, same number of links
        assert sorted(a.adj[m, :n, :n].sum(0)) == sorted(p.adj[m, :n, :n].sum(0))
        assert sorted(a.jtype[m, :n]) == sorted(p.jtype[m, :n])
        assert a.adj[m].sum() == p.adj[m].sum()


def test_fourbar_batch():
    f = I.fourbar_batch(16)
    assert f.pos.dtype == np.float64 and f.adj.shape == (16, 5, 5)
    assert list(f.jtype[0]) == [0, 2, 0, 1, 1]
    assert f.adj[0, 1, 3] and f.adj[0, 2, 3] and f.adj[0, 1, 4] and f.adj[0, 3, 4] and f.adj[0, 0, 1]


def test_perturb_and_requests():
    c = np.zeros((100, 200, 2), np.float32)
    q = I.perturb_curves(c, 0.02, seed=0)
    assert abs(q.std() - 0.02) < 0.001 and abs(q.mean()) < 0.001
    t, n = I.poisson_requests(20000, 2000.0, 65536, seed=0)
    assert abs(t[-1] / 20000 - 1 / 2000) < 5e-5
    assert n.min() >= 1 and n.max() <= 65536
    # log-uniform: the median is near sqrt(65537)
    assert 150 < np.median(n) < 350


@pytest.mark.parametrize("n", [6, 9, 14, 20])
def test_paper_topologies_meet_the_rules(n):
    """The paper's topology rules, checked from the oracle's solve path: every joint is an
    ancestor of the last-solved joint, which has no fixed neighbour; 1-DOF and
    dyad-solvable (oracle status OK)."""
    from oracle import oracle as O
    t = I.paper_topologies(24, n, seed=n)
    for b in range(t.B):
        P = O.plan(n, t.adj[b], t.jtype[b], np.zeros((n, 2)))
        assert P.status == 0
        assert P.coupler == n - 1
        parents = {P.k[d]: (P.i[d], P.j[d]) for d in range(P.n_dyads)}
        parents[P.motor] = (P.pivot,)
        seen, stack = set(), [P.coupler]
        while stack:
            a = stack.pop()
            if a not in seen:
                seen.add(a)
                stack.extend(parents.get(a, ()))
        assert seen == set(range(n))
        fixed = set(np.nonzero(t.jtype[b, :n] == I.FIXED)[0].tolist())
        assert not (set(np.nonzero(t.adj[b, n - 1, :n])[0].tolist()) & fixed)


def test_topology_rules_flags_breaking_topologies():
    """topology_rules against a direct check on random J-operator candidates: most of them
    break a rule, and the masks agree with the solve-path check."""
    from oracle import oracle as O
    d = I.dyad_batch(400, 7, 7, seed=3)
    irr, free = I.topology_rules(d)
    assert 0 < irr.mean() < 1 and 0 < free.mean() < 1
    for b in range(60):
        n = int(d.n_joints[b])
        P = O.plan(n, d.adj[b], d.jtype[b], d.pos[b].astype(np.float64))
        parents = {P.k[q]: (P.i[q], P.j[q]) for q in range(P.n_dyads)}
        parents[P.motor] = (P.pivot,)
        seen, stack = set(), [P.coupler]
        while stack:
            a = stack.pop()
            if a not in seen:
                seen.add(a)
                stack.extend(parents.get(a, ()))
        assert irr[b] == (seen == set(range(n)))
        assert free[b] == (not (d.adj[b, P.coupler, :n] & (d.jtype[b, :n] == I.FIXED)).any())


def test_paper_batch_standardised_positions():
    b = I.paper_batch(8, 16, 10, seed=5)
    assert b.B == 128 and b.nmax == 10
    assert np.all(b.pos[:, 0] == np.float32(0.5)) and np.all(b.pos[:, 1, 0] == np.float32(0.55))
    assert np.all(b.pos[:, 1, 1] == np.float32(0.5))
    assert (b.pos >= 0).all() and (b.pos <= 1).all()
    assert np.array_equal(b.adj[0], b.adj[15])  # topology-major: 16 samples per topology
    assert np.array_equal(b.pos, I.paper_batch(8, 16, 10, seed=5).pos)


def test_paper_batch_reproduces_the_papers_infeasibility_scale(oracle_lib):
    """The paper reports that at least 99% of random samples are wasted for mechanisms of
    more than 10 joints (Sec. "Scale of Infeasibilities").  With every joint drawn
    uniformly and then standardised by a similarity (ground joint at (0.5, 0.5), actuator
    arm 0.05 and horizontal), the oracle finds that scale: a few valid in a hundred at 6
    joints, under 2% at 12, and fewer at 15 than at 12."""
    rates = {}
    for n in (6, 12, 15):
        b = I.paper_batch(32, 128, n, seed=n)
        rates[n] = float(oracle_lib.simulate(b, 200, traj=False, path=False).valid.mean())
    assert rates[6] > 0.08 and rates[12] < 0.02 and rates[15] < rates[12]
    # the standardisation is a similarity of a uniform draw: the arm is exactly (0.05, 0)
    b = I.paper_batch(4, 64, 9, seed=1)
    arm = b.pos[:, 1].astype(np.float64) - b.pos[:, 0]
    assert np.allclose(arm, [0.05, 0.0], atol=1e-7)
    assert np.ptp(b.pos[:, 2:].reshape(-1, 2), axis=0).min() > 0.2  # the other joints spread over the box


def test_adjacency_masks_are_the_adjacency_bits():
    """MechBatch.masks(): bit c of row a is set exactly where adj[a, c] is nonzero, for
    n_max 8, 20 and 32 (the top bit), across chunk boundaries."""
    for lo, hi, nmax in ((6, 8, 8), (6, 20, 20), (3, 6, 32)):
        b = I.dyad_batch(700, lo, hi, seed=nmax, nmax=nmax)
        b.adj[3, 0, nmax - 1] = 7  # any nonzero byte is a link
        m = b.masks(chunk=256)
        want = ((b.adj != 0).astype(np.uint64) << np.arange(nmax, dtype=np.uint64)).sum(-1)
        assert m.dtype == np.uint32 and m.shape == (b.B, nmax)
        assert np.array_equal(m.astype(np.uint64), want)
