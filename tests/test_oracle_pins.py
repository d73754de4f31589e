"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: they use identities of the
construction (step 0, rigidity, closure), an independent trigonometric solution
of the four-bar, the Grashof-type full-rotation condition, brute force over both
circle-intersection branches, the mobility equation (Eq. 1) on the joint graph,
and library routines (scipy cdist, numpy sorting, SVD).
"""
import math

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from conftest import bbox_diag
from paper_2208_14567_gb300 import inputs as I

T = 200


# ----------------------------------------------------------------------------- plans

def mech(n, edges, types, pos=None, nmax=None):
    nmax = nmax or n
    adj = np.zeros((nmax, nmax), np.uint8)
    for a, b in edges:
        adj[a, b] = adj[b, a] = 1
    jt = np.full(nmax, -1, np.int8)
    jt[:n] = types
    if pos is None:
        pos = np.random.default_rng(n).random((nmax, 2))
    return adj, jt, np.asarray(pos, np.float64)


FOURBAR_E = [(0, 1), (1, 3), (2, 3), (1, 4), (3, 4)]


def test_plan_fourbar(oracle_lib):
    adj, jt, pos = mech(5, FOURBAR_E, [0, 2, 0, 1, 1])
    P = oracle_lib.plan(5, adj, jt, pos)
    assert P.status == 0 and P.motor == 1 and P.pivot == 0 and P.n_dyads == 2 and P.coupler == 4
    assert (P.k[0], P.i[0], P.j[0]) == (3, 1, 2)
    assert (P.k[1], P.i[1], P.j[1]) == (4, 1, 3)
    # lengths are the initial link lengths
    assert P.r1sq[0] == pytest.approx(((pos[3] - pos[1]) ** 2).sum(), rel=1e-15)
    assert P.r2sq[1] == pytest.approx(((pos[4] - pos[3]) ** 2).sum(), rel=1e-15)


def test_plan_solve_order_follows_lowest_ready_joint(oracle_lib):
    # joint 5 becomes solvable first (neighbours 1 and 2 known); joint 3 needs 5
    edges = [(0, 1), (3, 5), (3, 1), (4, 3), (4, 2), (5, 1), (5, 2)]
    adj, jt, pos = mech(6, edges, [0, 2, 0, 1, 1, 1])
    P = oracle_lib.plan(6, adj, jt, pos)
    assert P.status == 0
    assert [P.k[d] for d in range(3)] == [5, 3, 4]
    assert P.coupler == 4
    # joints 3 (on 1, 2) and 4 (on 0, 1) are ready together: the lower index goes first
    edges = [(0, 1), (1, 3), (2, 3), (0, 4), (1, 4), (3, 5), (4, 5)]
    adj, jt, pos = mech(6, edges, [0, 2, 0, 1, 1, 1])
    P = oracle_lib.plan(6, adj, jt, pos)
    assert P.status == 0 and [P.k[d] for d in range(3)] == [3, 4, 5]
    assert (P.i[1], P.j[1]) == (0, 1) and (P.i[2], P.j[2]) == (3, 4)


@pytest.mark.parametrize("edges,types,n,status", [
    (FOURBAR_E, [0, 1, 0, 1, 1], 5, 4),                       # no actuated joint
    (FOURBAR_E, [0, 2, 0, 2, 1], 5, 4),                       # two actuated joints
    ([(1, 3), (2, 3), (1, 4), (3, 4)], [0, 2, 0, 1, 1], 5, 5),  # crank not on a fixed joint
    ([(0, 1), (1, 3), (3, 4), (2, 4)], [0, 2, 0, 1, 1], 5, 6),  # two joints each with one known neighbour
    ([(0, 1), (1, 3), (2, 3), (0, 3)], [0, 2, 0, 1], 4, 7),   # three known neighbours
    ([(0, 1), (1, 2), (1, 3), (2, 3)], [0, 2, 0, 1], 4, 7),   # crank also linked to another ground joint
    (FOURBAR_E, [0, 2, 0, 3, 1], 5, 2),                       # bad type
])
def test_plan_statuses(oracle_lib, edges, types, n, status):
    adj, jt, pos = mech(n, edges, types)
    assert oracle_lib.plan(n, adj, jt, pos).status == status


def test_plan_bad_adjacency_and_size(oracle_lib):
    adj, jt, pos = mech(5, FOURBAR_E, [0, 2, 0, 1, 1])
    a2 = adj.copy()
    a2[3, 1] = 0
    assert oracle_lib.plan(5, a2, jt, pos).status == 3
    a3 = adj.copy()
    a3[2, 2] = 1
    assert oracle_lib.plan(5, a3, jt, pos).status == 3
    assert oracle_lib.plan(1, adj, jt, pos).status == 1
    assert oracle_lib.plan(6, adj, jt, pos).status == 1


def mobility(adj, jt, n):
    """Eq. 1 with j2 = 0 on the joint graph: bodies = ground + every link that is not
    ground-to-ground; j1 = sum over joints of (bodies meeting there - 1)."""
    fixed = jt[:n] == 0
    bars = [(a, b) for a in range(n) for b in range(a + 1, n) if adj[a, b] and not (fixed[a] and fixed[b])]
    bodies = 1 + len(bars)
    j1 = 0
    for a in range(n):
        meet = sum(1 for (x, y) in bars if a in (x, y)) + (1 if fixed[a] else 0)
        j1 += max(meet - 1, 0)
    return 3 * (bodies - 1) - 2 * j1


def test_generated_candidates_have_mobility_one_and_plan(oracle_lib):
    b = I.dyad_batch(300, 6, 12, seed=5, permute=True)
    for m in range(b.B):
        n = b.n_joints[m]
        assert mobility(b.adj[m], b.jtype[m], n) == 1
        assert oracle_lib.plan(n, b.adj[m], b.jtype[m], b.pos[m].astype(np.float64)).status == 0


def test_extra_link_breaks_mobility_and_plan(oracle_lib):
    b = I.dyad_batch(100, 7, 10, seed=6)
    rng = np.random.default_rng(0)
    seen = 0
    for m in range(b.B):
        n = b.n_joints[m]
        free = [(x, y) for x in range(n) for y in range(x + 1, n)
                if not b.adj[m, x, y] and not (b.jtype[m, x] == 0 and b.jtype[m, y] == 0)]
        x, y = free[rng.integers(len(free))]
        adj = b.adj[m].copy()
        adj[x, y] = adj[y, x] = 1
        assert mobility(adj, b.jtype[m], n) == 0
        st = oracle_lib.plan(n, adj, b.jtype[m], b.pos[m].astype(np.float64)).status
        assert st in (6, 7)
        seen += st == 7
    assert seen > 50


# ------------------------------------------------------------------------- simulation

@pytest.fixture(scope="module")
def fourbars(oracle_lib):
    f = I.fourbar_batch(2048, seed=0)
    return f, oracle_lib.simulate(f, T)


@pytest.fixture(scope="module")
def dyads(oracle_lib):
    b = I.dyad_batch(3000, 6, 14, seed=1, permute=True)
    return b, oracle_lib.simulate(b, T)


def test_step0_reproduces_initial_positions(fourbars, dyads):
    for batch, r in (fourbars, dyads):
        L = bbox_diag(batch.pos, batch.n_joints)
        ok = r.lock_step != 0
        assert ok.mean() > 0.99
        for m in np.nonzero(ok)[0]:
            n = batch.n_joints[m]
            err = np.abs(r.traj[m, :n, 0] - batch.pos[m, :n]).max()
            # FP64 rounding is amplified by 1/sin(gamma) = q^-1/2 per dyad (q >= min_disc)
            kappa = 1.0 / math.sqrt(min(1.0, max(r.min_disc[m], 1e-300)))
            assert err <= 1e-13 * L[m] * kappa


def test_rigidity_every_link_keeps_its_length(dyads, fourbars):
    for batch, r in (fourbars, dyads):
        for m in range(batch.B):
            n = batch.n_joints[m]
            stop = T if r.lock_step[m] < 0 else r.lock_step[m]
            if stop == 0:
                continue
            a, b = np.nonzero(np.triu(batch.adj[m, :n, :n]))
            tr = r.traj[m, :n, :stop]
            l0 = np.linalg.norm(batch.pos[m, a].astype(np.float64) - batch.pos[m, b], axis=-1)
            lt = np.linalg.norm(tr[a] - tr[b], axis=-1)
            assert np.abs(lt - l0[:, None]).max() <= 1e-9 * max(1.0, l0.max())


def test_nan_from_lock_and_flags(dyads):
    batch, r = dyads
    lk = r.lock_step
    assert set(np.unique(r.valid)) <= {0, 1}
    assert ((lk == -1) == (r.valid == 1)).all()
    for m in np.nonzero(lk >= 0)[0][:200]:
        n = batch.n_joints[m]
        assert np.isnan(r.traj[m, :n, lk[m]:]).all()
        assert not np.isnan(r.traj[m, :n, :lk[m]]).any()
    assert np.isnan(r.traj[:, 14:]).all() if batch.nmax > 14 else True
    # min_disc: q of the unlocked steps is a squared sine in (0, 1]
    md = r.min_disc[lk != 0]
    assert (md > 0).all() and (md <= 1 + 1e-12).all()


def test_closure_at_full_turn(oracle_lib, dyads):
    batch, r = dyads
    L = bbox_diag(batch.pos, batch.n_joints)
    for m in np.nonzero(r.valid)[0][:300]:
        P = oracle_lib.plan(batch.n_joints[m], batch.adj[m], batch.jtype[m], batch.pos[m].astype(np.float64))
        out, locked, *_ = oracle_lib.solve_at(P, batch.pos[m], 2 * math.pi)
        assert not locked
        n = batch.n_joints[m]
        assert np.abs(out[:n] - batch.pos[m, :n]).max() <= 1e-10 * L[m]


def fourbar_closed_form(p0, T):
    """Four-bar positions by trigonometry (law of cosines at the rocker pivot and a
    rigid rotation of the coupler triangle), independent of the oracle's algebra.
    Returns (positions [T,5,2], acos argument [T])."""
    A0, A, B0, B, P = p0
    th = 2 * np.pi * np.arange(T) / T
    u = A - A0
    At = A0 + np.stack([np.cos(th) * u[0] - np.sin(th) * u[1], np.sin(th) * u[0] + np.cos(th) * u[1]], -1)
    b = np.linalg.norm(B - A)   # coupler
    c = np.linalg.norm(B - B0)  # rocker
    w = At - B0
    delta = np.linalg.norm(w, axis=-1)
    arg = (c * c + delta * delta - b * b) / (2 * c * delta)
    # branch: orientation of (A, B0, B) at t = 0
    sgn = np.sign((A - B0)[0] * (B - B0)[1] - (A - B0)[1] * (B - B0)[0])
    psi = np.arctan2(w[:, 1], w[:, 0]) + sgn * np.arccos(np.clip(arg, -1, 1))
    Bt = B0 + c * np.stack([np.cos(psi), np.sin(psi)], -1)
    ang = np.arctan2(*(Bt - At).T[::-1]) - math.atan2(*(B - A)[::-1])
    v = P - A
    Pt = At + np.stack([np.cos(ang) * v[0] - np.sin(ang) * v[1], np.sin(ang) * v[0] + np.cos(ang) * v[1]], -1)
    X = np.stack([np.broadcast_to(A0, At.shape), At, np.broadcast_to(B0, At.shape), Bt, Pt], 1)
    return X, arg


def test_fourbar_matches_trigonometric_solution(fourbars):
    f, r = fourbars
    L = bbox_diag(f.pos, f.n_joints)
    checked = 0
    for m in range(f.B):
        X, arg = fourbar_closed_form(f.pos[m], T)
        bad = np.abs(arg) > 1
        lock_cf = int(np.argmax(bad)) if bad.any() else -1
        margin = np.min(np.abs(np.abs(arg) - 1)) < 1e-9
        if not margin:
            assert r.lock_step[m] == lock_cf
        stop = T if r.lock_step[m] < 0 else r.lock_step[m]
        good = np.abs(np.abs(arg[:stop]) - 1) > 1e-6
        if good.any():
            d = np.abs(r.traj[m].transpose(1, 0, 2)[:stop][good] - X[:stop][good]).max()
            assert d <= 1e-9 * L[m]
            checked += 1
    assert checked > 0.9 * f.B


def test_full_rotation_criterion(fourbars):
    """Crank a, ground g, coupler b, rocker c: the crank turns fully iff the diagonal
    range [|g - a|, g + a] lies inside [|b - c|, b + c].  Sampling at T steps can
    only miss a lock window, never invent one."""
    f, r = fourbars
    agree = 0
    for m in range(f.B):
        A0, A, B0, B, _ = f.pos[m]
        a, g = np.linalg.norm(A - A0), np.linalg.norm(B0 - A0)
        b, c = np.linalg.norm(B - A), np.linalg.norm(B - B0)
        full = (g + a <= b + c) and (abs(g - a) >= abs(b - c))
        if full:
            assert r.valid[m] == 1
        agree += int(full) == int(r.valid[m])
    assert agree >= 0.995 * f.B
    assert 0.05 < r.valid.mean() < 0.95


def test_fourbar_margin_indicator_closed_form(fourbars):
    """The margin indicator q of each dyad is sin^2 of the angle at the joint it solves,
    which the law of cosines gives independently of the oracle's algebra.  For the
    four-bar, dyad 0 solves the rocker joint B (coupler b = |B - A|, rocker c = |B - B0|,
    diagonal delta(t) = |A(t) - B0|): q0 = 1 - cos^2 with cos = (b^2 + c^2 - delta^2) /
    (2 b c), negative exactly when the triangle cannot close.  Dyad 1 solves the coupler
    point P on the rigid triangle (A, B, P): q1 is constant.  min_disc = min over the
    steps before the lock of min(q0, q1) (+inf if the lock is at step 0); min_abs_q also
    takes |q0| of the locking step, where dyad 1 is not reached."""
    f, r = fourbars
    th = 2 * np.pi * np.arange(T) / T
    locked = 0
    for m in range(f.B):
        A0, A, B0, B, P = f.pos[m].astype(np.float64)
        u = A - A0
        At = A0 + np.stack([np.cos(th) * u[0] - np.sin(th) * u[1], np.sin(th) * u[0] + np.cos(th) * u[1]], -1)
        b, c = np.linalg.norm(B - A), np.linalg.norm(B - B0)
        delta = np.linalg.norm(At - B0, axis=-1)
        q0 = 1 - ((b * b + c * c - delta * delta) / (2 * b * c)) ** 2
        pa, pb = np.linalg.norm(P - A), np.linalg.norm(P - B)
        q1 = 1 - ((pa * pa + pb * pb - b * b) / (2 * pa * pb)) ** 2
        scale = ((b * b + c * c + delta * delta) ** 2 / (4 * b * b * c * c)).max() + 1.0 / (pa * pb) ** 2
        lk = int(r.lock_step[m])
        stop = T if lk < 0 else lk
        if stop == 0:
            assert r.min_disc[m] == np.inf
            md, ab = np.inf, np.inf
        else:
            md = min(q0[:stop].min(), q1)
            ab = min(np.abs(q0[:stop]).min(), abs(q1))
            assert abs(r.min_disc[m] - md) <= 1e-12 * scale
        if lk >= 0:
            locked += 1
            assert q0[lk] <= 1e-12 * scale  # the lock is the triangle failing to close
            ab = min(ab, abs(q0[lk]))
        assert abs(r.min_abs_q[m] - ab) <= 1e-12 * scale
    assert 0.05 * f.B < locked < 0.95 * f.B


def test_margin_indicator_from_positions(oracle_lib, dyads):
    """On general candidates: q of dyad (k; i, j) at a solved step equals
    cross(p_i - p_k, p_j - p_k)^2 / (r1^2 r2^2), with the positions of the (separately
    pinned) trajectories and the link lengths taken from the initial positions.  At the
    locking step the failing dyad's q comes from the law of cosines on its parents'
    distance.  min_disc and min_abs_q must be these minima: over the dyads of the steps
    before the lock, and for min_abs_q also the dyads of the locking step up to and
    including the failing one."""
    batch, r = dyads
    checked = locks = 0
    for m in range(min(batch.B, 600)):
        if r.status[m] != 0:
            continue
        n = batch.n_joints[m]
        p0 = batch.pos[m].astype(np.float64)
        P = oracle_lib.plan(n, batch.adj[m], batch.jtype[m], p0)
        lk = int(r.lock_step[m])
        stop = T if lk < 0 else lk
        tr = r.traj[m]
        md = ab = np.inf
        for d in range(P.n_dyads):
            k, i, j = P.k[d], P.i[d], P.j[d]
            r1, r2 = ((p0[k] - p0[i]) ** 2).sum(), ((p0[k] - p0[j]) ** 2).sum()
            if stop:
                a, b = tr[i, :stop] - tr[k, :stop], tr[j, :stop] - tr[k, :stop]
                q = (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]) ** 2 / (r1 * r2)
                md = min(md, q.min())
                ab = min(ab, np.abs(q).min())
        if lk >= 0:
            locks += 1
            out, locked, _, _, q_lock = oracle_lib.solve_at(P, p0, 2 * math.pi * lk / T)
            assert locked
            for d in range(P.n_dyads):
                k, i, j = P.k[d], P.i[d], P.j[d]
                r1, r2 = math.dist(p0[k], p0[i]), math.dist(p0[k], p0[j])
                if np.isnan(out[k]).any():  # the failing dyad
                    dl = math.dist(out[i], out[j])
                    q = 1 - ((r1 * r1 + r2 * r2 - dl * dl) / (2 * r1 * r2)) ** 2
                    assert q <= 1e-12 and abs(q - q_lock) <= 1e-12 * (r1 * r1 + r2 * r2 + dl * dl) ** 2 / (r1 * r2) ** 2
                    ab = min(ab, abs(q))
                    break
                a, b = out[i] - out[k], out[j] - out[k]
                ab = min(ab, (a[0] * b[1] - a[1] * b[0]) ** 2 / (r1 * r1 * r2 * r2))
        assert r.min_disc[m] == md or abs(r.min_disc[m] - md) <= 1e-9
        assert r.min_abs_q[m] == ab or abs(r.min_abs_q[m] - ab) <= 1e-9
        checked += 1
    assert checked > 300 and locks > 100


def solve_branch(p0, i_j_k, signs, theta, pivot, motor, fixed):
    """Positions at crank angle theta for given branch signs, by trigonometry."""
    pos = p0.copy()
    u = p0[motor] - p0[pivot]
    pos[motor] = p0[pivot] + [math.cos(theta) * u[0] - math.sin(theta) * u[1],
                              math.sin(theta) * u[0] + math.cos(theta) * u[1]]
    for (i, j, k), s in zip(i_j_k, signs):
        r1 = np.linalg.norm(p0[k] - p0[i])
        r2 = np.linalg.norm(p0[k] - p0[j])
        w = pos[j] - pos[i]
        d = np.linalg.norm(w)
        cosb = (d * d + r1 * r1 - r2 * r2) / (2 * d * r1)
        if not (-1 < cosb < 1):
            return None
        al = math.atan2(w[1], w[0]) + s * math.acos(cosb)
        pos[k] = pos[i] + r1 * np.array([math.cos(al), math.sin(al)])
    return pos


def test_brute_force_branches(oracle_lib):
    b = I.dyad_batch(400, 5, 7, seed=11)
    checked = 0
    for m in range(b.B):
        n = b.n_joints[m]
        p0 = b.pos[m].astype(np.float64)
        P = oracle_lib.plan(n, b.adj[m], b.jtype[m], p0)
        nd = P.n_dyads
        if nd > 4:
            continue
        ijk = [(P.i[d], P.j[d], P.k[d]) for d in range(nd)]
        fixed = [a for a in range(n) if b.jtype[m, a] == 0]
        combos = [tuple(1 - 2 * ((c >> d) & 1) for d in range(nd)) for c in range(2 ** nd)]
        hits = [s for s in combos
                if (x := solve_branch(p0, ijk, s, 0.0, P.pivot, P.motor, fixed)) is not None
                and np.abs(x[:n] - p0[:n]).max() < 1e-9]
        assert len(hits) == 1
        for t in range(1, 40):
            th = 2 * math.pi * t / 40
            out, locked, qmin, *_ = oracle_lib.solve_at(P, p0, th)
            if locked:
                break
            mine = solve_branch(p0, ijk, hits[0], th, P.pivot, P.motor, fixed)
            assert np.abs(out[:n] - mine[:n]).max() < 1e-9
            if qmin > 1e-2:
                # continuity: a small further turn lands on the branch nearest to this one
                th2 = th + 1e-4
                nxt, lk2, *_ = oracle_lib.solve_at(P, p0, th2)
                assert not lk2
                cands = [x for s in combos if (x := solve_branch(p0, ijk, s, th2, P.pivot, P.motor, fixed)) is not None]
                dist = [np.abs(x[:n] - out[:n]).max() for x in cands]
                assert np.abs(nxt[:n] - cands[int(np.argmin(dist))][:n]).max() < 1e-9
            checked += 1
    assert checked > 500


def test_special_cases(oracle_lib):
    rng = np.random.default_rng(3)
    # joint 3 on two ground joints: stationary; joint 4 on pivot + crank: circle with the crank
    edges = [(0, 1), (0, 3), (2, 3), (0, 4), (1, 4), (1, 5), (3, 5)]
    for _ in range(20):
        adj, jt, pos = mech(6, edges, [0, 2, 0, 1, 1, 1], pos=rng.random((6, 2)))
        batch = I.MechBatch(np.array([6], np.int32), adj[None], jt[None], pos[None])
        r = oracle_lib.simulate(batch, 64)
        stop = 64 if r.lock_step[0] < 0 else r.lock_step[0]
        tr = r.traj[0]
        assert np.abs(tr[3, :stop] - pos[3]).max() < 1e-12
        th = 2 * np.pi * np.arange(stop) / 64
        v = pos[4] - pos[0]
        circ = pos[0] + np.stack([np.cos(th) * v[0] - np.sin(th) * v[1], np.sin(th) * v[0] + np.cos(th) * v[1]], -1)
        assert np.abs(tr[4, :stop] - circ).max() < 1e-12
    # no simple joints: the crank alone never locks, the coupler is the actuated joint
    adj, jt, pos = mech(3, [(0, 1)], [0, 2, 0])
    batch = I.MechBatch(np.array([3], np.int32), adj[None], jt[None], pos[None])
    r = oracle_lib.simulate(batch, 8)
    assert r.valid[0] == 1 and np.allclose(r.path[0], r.traj[0, 1])


def test_unsimulated_mechanisms(oracle_lib):
    adj, jt, pos = mech(5, FOURBAR_E, [0, 1, 0, 1, 1])
    batch = I.MechBatch(np.array([5], np.int32), adj[None], jt[None], pos[None])
    r = oracle_lib.simulate(batch, 8)
    assert r.status[0] == 4 and r.valid[0] == 0 and r.lock_step[0] == -2 and np.isnan(r.traj).all()


def test_threads_do_not_change_results(oracle_lib):
    b = I.dyad_batch(500, 6, 10, seed=2)
    r1 = oracle_lib.simulate(b, 50, threads=1)
    r8 = oracle_lib.simulate(b, 50, threads=8)
    assert np.array_equal(r1.traj, r8.traj, equal_nan=True)
    assert np.array_equal(r1.lock_step, r8.lock_step)


# -------------------------------------------------------------------- normalisation

def test_normalize_properties_and_invariance(oracle_lib, fourbars):
    f, r = fourbars
    curves = r.path[r.valid == 1][:300]
    out = oracle_lib.normalize(curves)
    x, y = out[..., 0], out[..., 1]
    assert np.abs(x.mean(1)).max() < 1e-12 and np.abs(y.mean(1)).max() < 1e-12
    assert np.abs(np.sqrt((x * x + y * y).mean(1)) - 1).max() < 1e-12
    assert np.abs((x * y).mean(1)).max() < 1e-12
    assert ((x * x).mean(1) >= (y * y).mean(1) - 1e-12).all()
    assert ((x ** 3).sum(1) >= -1e-12).all()
    # principal axis from a library SVD of the centred curve
    for k in range(min(50, len(curves))):
        c = curves[k] - curves[k].mean(0)
        _, s, vt = np.linalg.svd(c, full_matrices=False)
        if s[0] - s[1] > 1e-6 * s[0]:
            ax = vt[0]
            rot = np.stack([c @ ax, c @ np.array([-ax[1], ax[0]])], -1) / np.sqrt((c ** 2).sum(1).mean())
            if (rot[:, 0] ** 3).sum() < 0:
                rot = -rot
            assert np.abs(rot - out[k]).max() < 1e-9
    # similarity invariance
    rng = np.random.default_rng(0)
    for k in range(min(100, len(curves))):
        a = rng.uniform(0, 2 * np.pi)
        R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        moved = rng.uniform(0.2, 5) * curves[k] @ R.T + rng.normal(size=2)
        o2 = oracle_lib.normalize(moved[None])[0]
        lam = np.linalg.eigvalsh(np.cov(out[k].T))
        if lam[1] - lam[0] > 1e-6 and abs((out[k, :, 0] ** 3).sum()) > 1e-6:
            assert np.abs(o2 - out[k]).max() < 1e-9


def test_normalize_ellipse_and_degenerate(oracle_lib):
    s = 2 * np.pi * np.arange(200) / 200
    e = np.stack([3 * np.cos(s), 1 * np.sin(s)], -1)
    a = 0.7
    R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    out = oracle_lib.normalize((e @ R.T + [4, -2])[None])[0]
    rms = np.sqrt((e ** 2).sum(1).mean())
    # an ellipse is symmetric: sum x^3 = 0 picks either orientation; compare up to sign
    ref = e / rms
    assert min(np.abs(out - ref).max(), np.abs(out + ref).max()) < 1e-12
    z = oracle_lib.normalize(np.ones((1, 200, 2)))
    assert (z == 0).all()


# -------------------------------------------------------------------------- chamfer

def test_chamfer_against_cdist(oracle_lib):
    rng = np.random.default_rng(4)
    for _ in range(20):
        P = rng.normal(size=(rng.integers(1, 60), 2))
        Q = rng.normal(size=(rng.integers(1, 60), 2))
        D = cdist(P, Q)
        ref = D.min(1).mean() + D.min(0).mean()
        assert oracle_lib.chamfer(P, Q) == pytest.approx(ref, rel=1e-13)
        assert oracle_lib.chamfer(P, Q) == pytest.approx(oracle_lib.chamfer(Q, P), rel=1e-13)
        assert oracle_lib.chamfer(P, P) == 0.0


def test_chamfer_topk_exact_copy_ranks_first(oracle_lib):
    rng = np.random.default_rng(5)
    db = rng.normal(size=(300, 50, 2))
    q = db[[17, 200]].copy()
    idx, dist = oracle_lib.chamfer_topk(q, db, 5)
    assert idx[0, 0] == 17 and idx[1, 0] == 200 and dist[0, 0] == 0 and dist[1, 0] == 0
    d = oracle_lib.chamfer_many(q[0], db)
    ref = np.argsort(d, kind="stable")[:5]
    assert np.array_equal(idx[0], ref)
    assert (np.diff(dist, axis=1) >= 0).all()


def test_topk_ties_go_to_lower_index(oracle_lib):
    d = np.array([3.0, 1.0, 2.0, 1.0, 1.0, 0.5])
    idx, dist = oracle_lib.topk(d, 4)
    assert list(idx) == [5, 1, 3, 4]


# ---- the paper's max-distance-line normalisation (Sec. "Dataset Curation & Processing")

def _similar(c, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 2 * np.pi)
    R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    return rng.uniform(0.2, 5) * c @ R.T + rng.normal(size=2) * 3


def test_maxline_circle_ellipse_segment(oracle_lib):
    O = oracle_lib
    s = np.linspace(0, 2 * np.pi, 200, endpoint=False)
    circle = np.stack([3 + 2 * np.cos(s), -1 + 2 * np.sin(s)], -1)
    ellipse = _similar(np.stack([3 * np.cos(s), np.sin(s)], -1), 1)
    u = np.linspace(0, 1, 50)
    segment = np.stack([0.3 + 2 * u, -0.2 + 1.5 * u], -1)
    out, pair, var = O.normalize_maxline(np.stack([circle, ellipse, segment[np.arange(200) % 50]]))
    # circle: diameter 1 centred in the box, every point 0.5 from the centre
    assert abs(out[0, :, 0].min()) < 1e-12 and abs(out[0, :, 0].max() - 1) < 1e-12
    assert np.abs(np.hypot(out[0, :, 0] - 0.5, out[0, :, 1] - 0.5) - 0.5).max() < 1e-3
    assert var[0] < 1e-12
    # ellipse 3:1: major axis horizontal with length 1, minor axis 1/3, centred
    assert abs(np.ptp(out[1, :, 0]) - 1) < 1e-12 and abs(np.ptp(out[1, :, 1]) - 1 / 3) < 1e-3
    assert abs(out[1, :, 1].min() + out[1, :, 1].max() - 1) < 1e-12
    assert var[1] > 5e-4  # not a circle by the paper's threshold
    # segment: horizontal, length 1, at mid-height; its ends are the pair, in index order
    assert np.abs(out[2, :, 1] - 0.5).max() < 1e-12 and abs(out[2, :, 0].min()) < 1e-12
    assert tuple(pair[2]) == (0, 49) and out[2, 0, 0] < out[2, 49, 0]


def test_maxline_pair_is_the_farthest_pair(oracle_lib):
    O = oracle_lib
    from scipy.spatial.distance import pdist, squareform
    rng = np.random.default_rng(4)
    curves = rng.normal(size=(20, 60, 2))
    out, pair, _ = O.normalize_maxline(curves)
    for m in range(20):
        D = squareform(pdist(curves[m]))
        a, b = pair[m]
        assert a < b and abs(D[a, b] - D.max()) <= 1e-12 * D.max()
        # the pair becomes a horizontal line of length 1 from a to b; the box is centred
        assert abs(out[m, b, 0] - out[m, a, 0] - 1) < 1e-12 and abs(out[m, b, 1] - out[m, a, 1]) < 1e-12
        lo, hi = out[m].min(0), out[m].max(0)
        assert np.abs((lo + hi) / 2 - 0.5).max() < 1e-12
        assert np.abs(squareform(pdist(out[m])) - D / D.max()).max() < 1e-12  # a similarity


def test_maxline_similarity_invariance_and_mirror(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(5)
    c = rng.normal(size=(80, 2))
    ref, pr, vr = O.normalize_maxline(c[None])
    for seed in range(5):
        out, pair, var = O.normalize_maxline(_similar(c, seed)[None])
        assert np.array_equal(pair, pr)
        assert np.abs(out - ref).max() < 1e-9 and abs(var[0] - vr[0]) < 1e-12
    mir = c * np.array([-1.0, 1.0])
    out, pair, _ = O.normalize_maxline(mir[None])
    assert np.array_equal(pair, pr)
    assert np.abs(out[0, :, 0] - ref[0, :, 0]).max() < 1e-9
    assert np.abs(out[0, :, 1] - (1 - ref[0, :, 1])).max() < 1e-9


def test_maxline_degenerate_and_imposed_pair(oracle_lib):
    O = oracle_lib
    same = np.full((1, 30, 2), 0.7)
    out, _, var = O.normalize_maxline(same)
    assert np.all(out == 0.5) and var[0] == 0
    rng = np.random.default_rng(6)
    c = rng.normal(size=(3, 40, 2))
    out, pair, var = O.normalize_maxline(c)
    out2, pair2, var2 = O.normalize_maxline(c, pairs=pair)
    assert np.array_equal(out, out2) and np.array_equal(pair, pair2) and np.array_equal(var, var2)


def test_first_under_scan_order(oracle_lib):
    """The paper's retrieval: the first k curves below the threshold in scan order. A copy
    of the query placed first in the scan is returned first at distance 0; a threshold
    above every distance returns the first k curves of the scan whatever their
    distances; one below every distance returns none; hits come in scan order."""
    O = oracle_lib
    rng = np.random.default_rng(8)
    s = np.linspace(0, 2 * np.pi, 40, endpoint=False)
    db = np.stack([np.stack([np.cos(s) * a, np.sin(s)], -1) for a in rng.uniform(0.5, 2, 30)])
    q = db[17].copy()
    order = rng.permutation(30)
    order = np.concatenate([[17], order[order != 17]])  # curve 17 is scanned first
    idx, dist = O.chamfer_first_under(q[None], db, order, 0.3, 3)
    assert idx[0, 0] == 17 and dist[0, 0] == 0.0
    d = O.chamfer_many(q, db)
    found = idx[0][idx[0] >= 0]
    assert np.all(d[found] < 0.3)
    pos = [int(np.nonzero(order == i)[0][0]) for i in found]
    assert pos == sorted(pos)
    skipped = order[:pos[-1]]  # every curve scanned before the last hit and not returned is >= 0.3
    assert np.all(d[np.setdiff1d(skipped, found)] >= 0.3)
    idx, _ = O.chamfer_first_under(q[None], db, order, 1e9, 5)
    assert np.array_equal(idx[0], order[:5])
    idx, dist = O.chamfer_first_under(q[None], db, order, 0.0, 3)
    assert np.all(idx == -1) and np.all(np.isinf(dist))


def test_splitmix64_published_outputs(oracle_lib):
    """The keep draws' generator against the published splitmix64 sequence started at 0."""
    z = oracle_lib.splitmix64(0, np.arange(3))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_curation_flags(oracle_lib):
    """The paper's curation on a hand-built four-bar: the crank tip (linked to the
    ground pivot) is an arc and, tracing a full circle, a circle too; the rocker joint
    (linked to the second pivot) is an arc but not a circle; the coupler point is
    neither and is always kept; fixed joints have no path; with keep rate 0 nothing
    flagged is kept and with keep rate 1 everything is."""
    O = oracle_lib
    from paper_2208_14567_gb300 import inputs as I
    fb = I.fourbar_batch(1)
    fb.pos[0] = np.array([[0.0, 0.0], [0.3, 0.0], [1.0, 0.0], [0.8, 0.7], [0.5, 0.9]])
    r = O.simulate(fb, 200, traj=True, path=False)
    assert r.valid[0] == 1
    c0 = O.curate_paths(r.traj, None, fb, keep_rate=0.0)
    f = c0["flags"][0]
    assert f[0] == 0 and f[2] == 0                      # fixed joints
    assert f[1] == 1 | 2 | 4                            # crank tip: arc and circle, removed
    assert f[3] & 2 and not f[3] & 4 and not f[3] & 8   # rocker: arc, removed
    assert f[4] == 1 | 8                                # coupler point: kept
    assert c0["circ_var"][0, 1] < 1e-12 and c0["circ_var"][0, 4] > 5e-4
    assert list(c0["kept_index"]) == [4]
    c1 = O.curate_paths(r.traj, None, fb, keep_rate=1.0)
    assert list(c1["kept_index"]) == [1, 3, 4]
    n0, _, _ = O.normalize_maxline(r.traj[0, 4][None])
    assert np.array_equal(c1["kept_paths"][2], n0[0])
