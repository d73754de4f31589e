"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  * plan: statuses, solve order and parents bit-exact; lengths within 1e-14 relative;
    host and device builders bit-identical;
  * valid / lock_step: identical, except mechanisms whose oracle margin indicator
    min |q| over the evaluated dyads is <= MARGIN (counted and printed);
  * positions: LINKS_MIXED within 1e-5 of the bounding-box diagonal L at every step
    both sides simulated; LINKS_PLAIN_F64 within 1e-9 L where the oracle's
    min_disc > 1e-8 and within 1e-5 L elsewhere;
  * NaN exactly from the locking step on and for padding joints.
"""
import numpy as np
import pytest

from conftest import bbox_diag
from oracle import oracle as O
from paper_2208_14567_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 1e-9
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_14567_gb300 import links
    links.lib()
    return links


def sim_for(batch, L):
    from paper_2208_14567_gb300.api import Simulator
    return Simulator(max(batch.B, 1), batch.nmax)


def run(batch, T, precision, out_mode, L, host_build=False, out_capacity=None, builder=0):
    from paper_2208_14567_gb300.api import to_device
    s = sim_for(batch, L)
    try:
        if builder:
            L.links_set_tuning(s.ctx, batch.nmax, L.TUNE_BUILDER, builder)
        if host_build:
            st = s.build_host(batch)
        else:
            st = s.build(to_device(batch)).cpu().numpy()
        o = s.simulate(T, precision, out_mode, out_capacity=out_capacity)
        s.sync()
        if out_mode == L.OUT_VALID_ONLY:  # copy back only the written rows
            rows = min(int(o.n_out[0]), o.traj.shape[0])
            o.traj, o.path = o.traj[:rows], o.path[:rows]
        res = {k: (None if v is None else v.cpu().numpy()) for k, v in o.__dict__.items()}
        res["status"] = st
        return res
    finally:
        s.close()


def check_flags(res, ref, label):
    margin = ~(ref.min_abs_q > MARGIN)
    mism = (res["valid"] != ref.valid) | (res["lock_step"] != ref.lock_step)
    bad = mism & ~margin
    print(f"[{label}] mechanisms {len(ref.valid)} valid {ref.valid.mean():.4f} margin cases {int(margin.sum())} "
          f"flag mismatches in margin {int((mism & margin).sum())}")
    assert not bad.any(), f"{int(bad.sum())} flag mismatches outside the margin, e.g. {np.nonzero(bad)[0][:5]}"
    return mism


def check_positions(batch, traj, path, ref, lock_gpu, tol, label, tight=None):
    Ld = bbox_diag(batch.pos, batch.n_joints)
    T = traj.shape[2]
    B, nm = batch.B, batch.nmax
    lr = np.where(ref.lock_step < 0, T, np.maximum(ref.lock_step, 0))
    lg = np.where(lock_gpu < 0, T, np.maximum(lock_gpu, 0))
    stop = np.minimum(lr, lg)
    tmask = np.arange(T)[None, :] < stop[:, None]
    jmask = np.arange(nm)[None, :] < batch.n_joints[:, None]
    ok = ref.status == 0
    err = np.abs(traj.astype(np.float64) - ref.traj).max(-1)  # [B, nm, T]
    m = ok[:, None, None] & jmask[:, :, None] & tmask[:, None, :]
    e = np.where(ok, np.where(m, err, 0.0).max((1, 2)) / np.where(ok, Ld, 1.0), 0.0)
    assert np.isfinite(e[ok]).all()
    print(f"[{label}] max position error / L = {e.max():.3e}")
    lim = np.full(B, tol) if tight is None else tight
    assert (e <= lim).all(), f"worst mechanism {int(e.argmax())}: {e.max():.3e}"
    # NaN from the GPU's lock step on (its own flags), and for padding joints
    gl = np.where(lock_gpu < 0, T, np.maximum(lock_gpu, 0))
    after = np.arange(T)[None, :] >= gl[:, None]
    nanm = (after[:, None, :] & jmask[:, :, None]) | ~jmask[:, :, None] | ~ok[:, None, None]
    assert np.isnan(traj[nanm]).all()
    assert not np.isnan(traj[~nanm]).any()
    # the path is the coupler joint's trajectory
    perr = np.abs(path.astype(np.float64) - ref.path).max(-1)
    pm = ok[:, None] & tmask
    assert (np.where(ok, np.where(pm, perr, 0).max(1) / np.where(ok, Ld, 1.0), 0.0) <= lim).all()


def tight_f64(ref, B):
    return np.where(ref.min_disc > 1e-8, 1e-9, TOL_MIXED)


# ------------------------------------------------------------------------------- plan

def planted_bad(batch):
    """Copy of a batch with every status code planted in the first rows."""
    b = I.MechBatch(batch.n_joints.copy(), batch.adj.copy(), batch.jtype.copy(), batch.pos.copy())
    b.n_joints[0] = 1                       # BAD_SIZE
    b.jtype[1, 3] = 5                       # BAD_TYPE
    b.adj[2, 3, 4] = 1 - b.adj[2, 3, 4]     # BAD_ADJ (asymmetric)
    b.jtype[3, b.jtype[3] == 2] = 1         # NO_MOTOR
    m = int(np.nonzero(b.jtype[4] == 2)[0][0])
    for a in range(b.nmax):
        if b.jtype[4, a] == 0:
            b.adj[4, m, a] = b.adj[4, a, m] = 0  # NO_PIVOT
    b.adj[5, :, :] = 0                       # every simple joint dangling -> NOT_DYAD_SOLVABLE
    m = int(np.nonzero(b.jtype[5] == 2)[0][0])
    f = int(np.nonzero(b.jtype[5] == 0)[0][0])
    b.adj[5, m, f] = b.adj[5, f, m] = 1
    n = b.n_joints[6]                        # extra link -> OVERCONSTRAINED
    for x in range(n):
        for y in range(x + 1, n):
            if not b.adj[6, x, y] and not (b.jtype[6, x] == 0 and b.jtype[6, y] == 0):
                b.adj[6, x, y] = b.adj[6, y, x] = 1
                break
        else:
            continue
        break
    return b


@pytest.mark.parametrize("n_lo,n_hi,nmax,f64,builder", [(6, 8, 8, False, 0), (5, 8, 8, True, 0), (6, 8, 8, False, 2),
                                                         (5, 8, 8, True, 2), (6, 16, 16, False, 0),
                                                         (6, 20, 20, True, 0), (6, 20, 20, False, 0),
                                                         (3, 6, 32, False, 0), (5, 15, 15, False, 0)])
def test_device_and_host_plans_simulate_identically(L, n_lo, n_hi, nmax, f64, builder):
    """The device builders (a thread per mechanism for n_max <= 8; the warp-flat builder,
    a lane per mechanism for the search and a lane per dyad for the geometry, for larger
    n_max or when chosen) and the host builder give the same plans: every output of a
    mixed simulation on them is the same to the bit, the planted ill-formed mechanisms
    included.  n_max 15 reads the adjacency bytewise (rows not whole words)."""
    batch = planted_bad(I.dyad_batch(4000, n_lo, n_hi, seed=n_hi + nmax, permute=True, nmax=nmax,
                                     pos_dtype=np.float64 if f64 else np.float32))
    a = run(batch, 64, L.MIXED, L.OUT_FULL, L, host_build=False, builder=builder)
    b = run(batch, 64, L.MIXED, L.OUT_FULL, L, host_build=True)
    for k in ("status", "valid", "lock_step", "min_disc", "traj", "path"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    print(f"[plans n={n_lo}-{n_hi} n_max={nmax} {'f64' if f64 else 'f32'}] valid {a['valid'].mean():.3f} "
          f"statuses {sorted(set(a['status'].tolist()))}")


@pytest.mark.parametrize("n_lo,n_hi,nmax,f64", [(6, 8, 8, False), (6, 20, 20, True), (6, 20, 20, False),
                                              (3, 6, 32, False), (5, 15, 15, False)])
def test_mask_build_equals_byte_build(L, n_lo, n_hi, nmax, f64):
    """links_plan_build_masks (the adjacency as neighbour bit masks) and links_plan_build
    (uint8 matrix) give the same plans: statuses and every output of a mixed simulation
    identical to the bit, the planted ill-formed mechanisms included."""
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = planted_bad(I.dyad_batch(4000, n_lo, n_hi, seed=7 * nmax, permute=True, nmax=nmax,
                                     pos_dtype=np.float64 if f64 else np.float32))
    res = []
    for masks in (False, True):
        with Simulator(batch.B, batch.nmax) as s:
            st = s.build(to_device(batch, masks=masks))
            o = s.simulate(64, L.MIXED, L.OUT_FULL)
            s.sync()
            res.append({"status": st.cpu().numpy(),
                        **{k: getattr(o, k).cpu().numpy() for k in ("valid", "lock_step", "min_disc", "traj", "path")}})
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k], equal_nan=True), k
    assert len(set(res[0]["status"].tolist())) >= 7


def test_plan_matches_oracle_device_and_host(L):
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = planted_bad(I.dyad_batch(3000, 6, 16, seed=2, permute=True, nmax=20))
    with Simulator(batch.B, batch.nmax) as s:
        st_dev = s.build(to_device(batch)).cpu().numpy()
        topo_d, len_d = L.links_plan_export(s.plan, 0, batch.B)
        st_host = s.build_host(batch)
        topo_h, len_h = L.links_plan_export(s.plan, 0, batch.B)
    assert np.array_equal(st_dev, st_host)
    assert np.array_equal(topo_d, topo_h)
    assert np.array_equal(len_d, len_h, equal_nan=True)
    seen = set()
    for m in range(batch.B):
        P = O.plan(batch.n_joints[m], batch.adj[m], batch.jtype[m], batch.pos[m].astype(np.float64))
        assert st_dev[m] == P.status
        seen.add(P.status)
        if P.status:
            continue
        t = topo_d[m]
        assert (t[2], t[3], t[4], t[5]) == (P.motor, P.pivot, P.coupler, P.n_dyads)
        for d in range(P.n_dyads):
            k, i, j = t[6 + 3 * d: 9 + 3 * d]
            exp = (P.i[d], P.j[d]) if P.s[d] > 0 else (P.j[d], P.i[d])
            assert (k, i, j) == (P.k[d], *exp)
            r1, r2 = (P.r1sq[d], P.r2sq[d]) if P.s[d] > 0 else (P.r2sq[d], P.r1sq[d])
            assert abs(len_d[m, 2 * d] - r1) <= 1e-14 * r1 and abs(len_d[m, 2 * d + 1] - r2) <= 1e-13 * max(r2, r1)
    assert seen == set(range(8))


# ------------------------------------------------------------------------ simulation

def test_plain_f64_fourbars_full(L):
    """4096 random four-bars, FP64 inputs, FULL output (the plain-method configuration)."""
    batch = I.fourbar_batch(4096, seed=0)
    ref = O.simulate(batch, 200)
    res = run(batch, 200, L.PLAIN_F64, L.OUT_FULL, L)
    check_flags(res, ref, "f64 four-bars")
    check_positions(batch, res["traj"], res["path"], ref, res["lock_step"], TOL_MIXED, "f64 four-bars",
                    tight=tight_f64(ref, batch.B))
    assert np.abs(res["min_disc"][ref.valid == 1] - ref.min_disc[ref.valid == 1]).max() < 1e-6


@pytest.mark.parametrize("case", ["fourbar", "dyad6-8", "dyad6-20-permuted", "dyad-host-build"])
def test_mixed_full_matches_oracle(L, case):
    if case == "fourbar":
        batch = I.fourbar_batch(4096, seed=1)
    elif case == "dyad6-8":
        batch = I.dyad_batch(6000, 6, 8, seed=3)
    else:
        batch = I.dyad_batch(4000, 6, 20, seed=4, permute=True)
    T = 200
    ref = O.simulate(batch, T)
    res = run(batch, T, L.MIXED, L.OUT_FULL, L, host_build=case == "dyad-host-build")
    check_flags(res, ref, case)
    check_positions(batch, res["traj"], res["path"], ref, res["lock_step"], TOL_MIXED, case)
    # min_disc comes from the FP32 screen (double-word on rescued steps): absolute error
    ok = (ref.status == 0) & (ref.lock_step != 0) & (res["lock_step"] == ref.lock_step)
    dq = np.abs(res["min_disc"][ok] - ref.min_disc[ok])
    print(f"[{case}] max |min_disc - oracle| = {dq.max():.3e}")
    assert (dq <= 1e-4 + 1e-3 * ref.min_disc[ok]).all()


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_valid_only_rows(L, precision):
    p = L.MIXED if precision == "mixed" else L.PLAIN_F64
    batch = I.dyad_batch(5000, 6, 10, seed=5)
    full = run(batch, 128, p, L.OUT_FULL, L)
    vo = run(batch, 128, p, L.OUT_VALID_ONLY, L)
    idx = np.nonzero(full["valid"])[0]
    n = int(vo["n_out"][0])
    assert n == len(idx) and np.array_equal(vo["out_index"][:n], idx)
    assert np.array_equal(vo["traj"][:n], full["traj"][idx], equal_nan=True)
    assert np.array_equal(vo["path"][:n], full["path"][idx], equal_nan=True)
    assert np.array_equal(vo["valid"], full["valid"]) and np.array_equal(vo["lock_step"], full["lock_step"])
    # capacity below the number of valid rows: only the first rows are written
    cap = max(1, n // 3)
    part = run(batch, 128, p, L.OUT_VALID_ONLY, L, out_capacity=cap)
    assert int(part["n_out"][0]) == n
    assert np.array_equal(part["out_index"][:cap], idx[:cap])
    assert np.array_equal(part["traj"][:cap], full["traj"][idx[:cap]], equal_nan=True)


def test_emit_census(L):
    """links_emit_census: the emit computes every step before the lock of each row it
    writes; the double-word recomputations are a subset, in steps and dyad-steps; the
    census is deterministic and writes no output."""
    import torch
    from paper_2208_14567_gb300.api import to_device
    batch = I.dyad_batch(3000, 6, 10, seed=9)
    T = 64
    s = sim_for(batch, L)
    try:
        st = s.build(to_device(batch)).cpu().numpy()
        nd = batch.n_joints - (batch.jtype[:, :batch.nmax] == 0).sum(1) - 1
        ok = st == 0
        for mode in (L.OUT_FULL, L.OUT_VALID_ONLY):
            o = s.simulate(T, L.MIXED, mode)
            s.sync()
            traj0 = o.traj.clone()
            cap = o.traj.shape[0]
            args = (o.lock_step, o.out_index, cap)
            w = L.links_emit_census(s.ctx, s.plan, T, mode, *args)
            assert w == L.links_emit_census(s.ctx, s.plan, T, mode, *args)
            assert torch.allclose(o.traj, traj0, rtol=0, atol=0, equal_nan=True)  # nothing written
            lock = o.lock_step.cpu().numpy().astype(np.int64)
            if mode == L.OUT_FULL:
                steps = np.where(lock < 0, T, lock)[ok]
                dyads = (np.where(lock < 0, T, lock) * nd)[ok]
            else:
                v = o.valid.cpu().numpy().astype(bool)
                steps = np.full(v.sum(), T)
                dyads = T * nd[v]
            assert w["steps"] == steps.sum()
            assert 0 <= w["double_word_steps"] <= w["steps"] and 0 <= w["double_word_dyads"] <= dyads.sum()
            print(f"mode {mode}: {w}")
        with pytest.raises(L.LinksError):
            L.links_emit_census(s.ctx, s.plan, 0, L.OUT_FULL, o.lock_step)
    finally:
        s.close()


def check_rows_against_oracle(batch, got, T, label):
    """A LINKS_MIXED result with VALID_ONLY rows (got: numpy outputs) against the FP64
    oracle on the same inputs: valid flags equal outside the margin; every row within
    TOL_MIXED of the oracle's trajectory and coupler path where the oracle calls the
    mechanism valid; every rejected mechanism's lock step a step at which the oracle's
    solver locks (or whose smallest |q| lies inside the margin), no earlier than the
    oracle's first lock."""
    ref = O.simulate(batch, T)
    margin = ~(ref.min_abs_q > MARGIN)
    ok = ref.status == 0
    bad = (got["valid"] != ref.valid) & ~margin
    assert not bad.any(), f"{int(bad.sum())} flag mismatches outside the margin"
    n = int(got["n_out"][0])
    rows = got["out_index"][:n]
    Ld = bbox_diag(batch.pos, batch.n_joints)
    worst = 0.0
    for r, b in enumerate(rows):
        if ref.valid[b] != 1:
            continue
        nj = batch.n_joints[b]
        e = np.abs(got["traj"][r, :nj].astype(np.float64) - ref.traj[b, :nj]).max() / Ld[b]
        ep = np.abs(got["path"][r].astype(np.float64) - ref.path[b]).max() / Ld[b]
        worst = max(worst, e, ep)
    assert worst <= TOL_MIXED, f"max position error / L {worst:.3e}"
    rej = np.nonzero(ok & (got["valid"] == 0))[0]
    checked = 0
    for b in rej:
        ls = int(got["lock_step"][b])
        assert ls >= 0
        if not margin[b]:
            assert ls >= ref.lock_step[b] >= 0
        P = O.plan(batch.n_joints[b], batch.adj[b], batch.jtype[b], batch.pos[b].astype(np.float64))
        _, locked, _, qabs, _ = O.solve_at(P, batch.pos[b].astype(np.float64), 2 * np.pi * ls / T)
        assert locked or qabs <= MARGIN, (b, ls)
        checked += 1
    print(f"[{label}] oracle: rows {n}, max position error / L {worst:.2e}, rejected lock steps checked {checked}, "
          f"margin cases {int(margin.sum())}")


@pytest.mark.parametrize("case", ["dyad6-8", "dyad6-20"])
def test_two_stage_screen(L, case):
    """links_simulate_two_stage: the coarse grid's angles are fine-grid angles, so the
    valid flags, the valid rows and their outputs equal the single-stage run; rejected
    mechanisms carry a fine-grid locking step no earlier than the first one.  Then the
    two-stage result itself against the oracle (flags, rows, and each rejected
    mechanism's lock step an oracle locking angle)."""
    import torch
    from paper_2208_14567_gb300.api import to_device
    batch = I.dyad_batch(5000, 6, 8, seed=21) if case == "dyad6-8" else I.dyad_batch(4000, 6, 20, seed=22, nmax=20)
    T, T_low = 200, 50
    s = sim_for(batch, L)
    try:
        st = s.build(to_device(batch)).cpu().numpy()
        one = s.simulate(T, L.MIXED, L.OUT_VALID_ONLY)
        s.sync()
        ref = {k: (None if v is None else v.cpu().numpy().copy()) for k, v in one.__dict__.items()}
        n_low = torch.zeros(1, dtype=torch.int32, device="cuda")
        two = s.simulate_two_stage(T, T_low, n_low_valid=n_low)
        s.sync()
        got = {k: (None if v is None else v.cpu().numpy()) for k, v in two.__dict__.items()}
        n = int(ref["n_out"][0])
        assert int(got["n_out"][0]) == n and np.array_equal(got["valid"], ref["valid"])
        assert np.array_equal(got["out_index"][:n], ref["out_index"][:n])
        assert np.array_equal(got["traj"][:n], ref["traj"][:n], equal_nan=True)
        assert np.array_equal(got["path"][:n], ref["path"][:n], equal_nan=True)
        v = ref["valid"] == 1
        assert np.array_equal(got["lock_step"][v], ref["lock_step"][v])
        assert np.array_equal(got["min_disc"][v], ref["min_disc"][v])
        rej = (st == 0) & ~v
        assert (got["lock_step"][rej] >= ref["lock_step"][rej]).all()
        coarse = got["lock_step"][rej] != ref["lock_step"][rej]
        assert (got["lock_step"][rej][coarse] % (T // T_low) == 0).all()
        nl = int(n_low.item())
        assert nl >= n
        print(f"[{case}] valid {n}, valid on {T_low} positions {nl}: false-valid rate {(nl - n) / max(nl, 1):.4f}")
        check_rows_against_oracle(batch, got, T, f"two-stage {case}")
        with pytest.raises(L.LinksError):
            s.simulate_two_stage(T, 60)
    finally:
        s.close()


@pytest.mark.parametrize("n", [6, 8, 10, 12, 15, 20])
def test_paper_generator_matches_oracle(L, n):
    """Candidates of the paper's own generator (topologies by the J operator under the
    paper's rules; joints uniform in the unit box, then standardised by a similarity to
    the ground pivot at (0.5, 0.5) and a horizontal actuator arm of 0.05): eight
    topologies x 300 position samples of n joints, LINKS_MIXED FULL against the oracle --
    flags outside the margin, positions within 1e-5 L at every step, min_disc as in the
    generic tests."""
    batch = I.paper_batch(8, 300, n, seed=500 + n)
    T = 200
    ref = O.simulate(batch, T)
    res = run(batch, T, L.MIXED, L.OUT_FULL, L)
    assert np.array_equal(res["status"], ref.status) and (ref.status == 0).all()
    check_flags(res, ref, f"paper n={n}")
    check_positions(batch, res["traj"], res["path"], ref, res["lock_step"], TOL_MIXED, f"paper n={n}")
    ok = (ref.lock_step != 0) & (res["lock_step"] == ref.lock_step)
    dq = np.abs(res["min_disc"][ok] - ref.min_disc[ok])
    assert (dq <= 1e-4 + 1e-3 * ref.min_disc[ok]).all()


@pytest.mark.parametrize("n", [6, 8, 12])
def test_paper_topology_million_samples_emit_agrees_with_screen(L, n):
    """One topology of the paper's generator with 1M standardised position samples,
    VALID_ONLY rows: the emit's double-word chain never finds a lock on a step the
    screen passed (the device error word stays clear, so the sync succeeds), and 1500
    sampled valid rows match the oracle within 1e-5 L at every step."""
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = I.paper_batch(1, 1_000_000, n, seed=100 + n)
    T = 200
    with Simulator(batch.B, batch.nmax) as s:
        s.build(to_device(batch))
        o = s.simulate(T, L.MIXED, L.OUT_VALID_ONLY)
        s.sync()
        nv = int(o.n_out[0])
        assert nv > 0
        rng = np.random.default_rng(n)
        pick = np.sort(rng.choice(nv, size=min(nv, 1500), replace=False))
        idx = o.out_index[:nv].cpu().numpy()[pick]
        traj = o.traj[:nv].cpu().numpy()[pick]
        path = o.path[:nv].cpu().numpy()[pick]
    sub = batch.take(idx)
    ref = O.simulate(sub, T)
    assert (ref.valid == 1).sum() >= len(idx) - 2  # margin cases only
    Ld = bbox_diag(sub.pos, sub.n_joints)
    keep = ref.valid == 1
    e = np.abs(traj[:, :n].astype(np.float64) - ref.traj[:, :n]).max((1, 2, 3)) / Ld
    ep = np.abs(path.astype(np.float64) - ref.path).max((1, 2)) / Ld
    worst = max(e[keep].max(), ep[keep].max())
    assert worst <= TOL_MIXED, worst
    print(f"[paper topology n={n} 1M] valid {nv} max position error / L {worst:.2e}")


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_packed_rows_equal_valid_only_rows(L, precision):
    """links_simulate_packed against LINKS_OUT_VALID_ONLY on the same plan: the same
    rows, n_out, out_index and paths; each packed row's n joints bit-identical to the
    padded row's first n joints, at joint offsets equal to the prefix sums of n with the
    total at row_offset[rows]; nothing written past the rows' joints."""
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = I.dyad_batch(6000, 6, 12, seed=31)
    T = 77
    prec = L.MIXED if precision == "mixed" else L.PLAIN_F64
    with Simulator(batch.B, batch.nmax) as s:
        s.build(to_device(batch))
        a = s.simulate(T, prec, L.OUT_VALID_ONLY)
        p = s.alloc_packed(T, prec)
        p.traj.fill_(123.0)
        s.simulate_packed(T, prec, out=p)
        s.sync()
        n = int(a.n_out[0])
        assert int(p.n_out[0]) == n and n > 0
        idx = a.out_index[:n].cpu().numpy()
        assert np.array_equal(p.out_index[:n].cpu().numpy(), idx)
        assert np.array_equal(p.path[:n].cpu().numpy(), a.path[:n].cpu().numpy(), equal_nan=True)
        for k in ("valid", "lock_step", "min_disc"):
            assert np.array_equal(getattr(p, k).cpu().numpy(), getattr(a, k).cpu().numpy(), equal_nan=True), k
        nj = batch.n_joints[idx].astype(np.int64)
        offs = np.concatenate([[0], np.cumsum(nj)])
        assert np.array_equal(p.row_offset[:n + 1].cpu().numpy(), offs)
        tp, ta = p.traj.cpu().numpy(), a.traj[:n].cpu().numpy()
    want = np.concatenate([ta[r, :nj[r]] for r in range(n)])
    assert np.array_equal(tp[:offs[n]], want)
    assert (tp[offs[n]:] == 123.0).all()
    print(f"[packed {precision}] rows {n} joint rows {offs[n]} of {n * batch.nmax} padded")


def test_packed_rows_capacities(L):
    """Row capacity below the valid count (rows = out_capacity, the total over those rows)
    and a trajectory capacity that ends inside a row: rows that fit entirely are written,
    the others keep the sentinel, and every row's path is written."""
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = I.dyad_batch(5000, 6, 8, seed=32)
    T = 40
    with Simulator(batch.B, batch.nmax) as s:
        s.build(to_device(batch))
        a = s.simulate(T, L.MIXED, L.OUT_VALID_ONLY)
        s.sync()
        nv = int(a.n_out[0])
        cap = nv // 2
        idx = a.out_index[:cap].cpu().numpy()
        nj = batch.n_joints[idx].astype(np.int64)
        offs = np.concatenate([[0], np.cumsum(nj)])
        k = cap // 3
        tcap = int(offs[k]) + 1  # ends inside row k
        p = s.alloc_packed(T, L.MIXED, out_capacity=cap, traj_capacity=tcap)
        p.traj.fill_(123.0)
        s.simulate_packed(T, L.MIXED, out=p)
        s.sync()
        assert int(p.n_out[0]) == nv
        assert np.array_equal(p.row_offset.cpu().numpy(), offs)
        tp, ta = p.traj.cpu().numpy(), a.traj[:cap].cpu().numpy()
        assert np.array_equal(p.path.cpu().numpy(), a.path[:cap].cpu().numpy(), equal_nan=True)
    want = np.concatenate([ta[r, :nj[r]] for r in range(k)])
    assert np.array_equal(tp[:offs[k]], want)
    assert (tp[offs[k]:] == 123.0).all()
    with Simulator(4, 8) as s:
        with pytest.raises(L.LinksError):
            L.links_simulate_packed(s.ctx, s.plan, T, L.MIXED, None, 0, None, None, None, None, None, None, 0)


@pytest.mark.parametrize("T", [1, 7, 33, 64])
def test_ragged_steps_and_statuses(L, T):
    batch = planted_bad(I.dyad_batch(700, 6, 12, seed=6, permute=True))
    ref = O.simulate(batch, T)
    for p in (L.MIXED, L.PLAIN_F64):
        res = run(batch, T, p, L.OUT_FULL, L)
        assert np.array_equal(res["status"], ref.status)
        bad = ref.status != 0
        assert (res["valid"][bad] == 0).all() and (res["lock_step"][bad] == -2).all()
        assert np.isnan(res["min_disc"][bad]).all()
        check_flags(res, ref, f"T={T}")
        check_positions(batch, res["traj"], res["path"], ref, res["lock_step"], TOL_MIXED, f"T={T}")


def test_empty_single_and_largest_mechanisms(L):
    from paper_2208_14567_gb300.api import Simulator, to_device
    empty = I.dyad_batch(1, 6, 6, seed=0).slice(0, 0)
    with Simulator(4, 6) as s:
        s.build(to_device(empty))
        o = s.simulate(16, L.MIXED, L.OUT_VALID_ONLY)
        s.sync()
        assert int(o.n_out[0]) == 0
    one = I.dyad_batch(1, 7, 7, seed=9)
    ref = O.simulate(one, 50)
    res = run(one, 50, L.MIXED, L.OUT_FULL, L)
    check_positions(one, res["traj"], res["path"], ref, res["lock_step"], TOL_MIXED, "B=1")
    big = I.dyad_batch(200, 32, 32, seed=10, nmax=32)   # n_max = LINKS_MAX_JOINTS
    ref = O.simulate(big, 40)
    for p in (L.MIXED, L.PLAIN_F64):
        res = run(big, 40, p, L.OUT_FULL, L)
        check_flags(res, ref, "n=32")
        check_positions(big, res["traj"], res["path"], ref, res["lock_step"], TOL_MIXED, "n=32")
    # only the crank: never locks, the coupler is the actuated joint
    adj = np.zeros((1, 3, 3), np.uint8)
    adj[0, 0, 1] = adj[0, 1, 0] = 1
    crank = I.MechBatch(np.array([3], np.int32), adj, np.array([[0, 2, 0]], np.int8),
                        np.array([[[0.5, 0.5], [0.6, 0.5], [0.1, 0.9]]], np.float32))
    ref = O.simulate(crank, 20)
    res = run(crank, 20, L.MIXED, L.OUT_FULL, L)
    assert res["valid"][0] == 1 and np.abs(res["path"][0] - ref.path[0]).max() < 1e-6


def test_too_large_batch_is_rejected(L):
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = I.dyad_batch(10, 6, 6, seed=0)
    with Simulator(5, 6) as s:
        with pytest.raises(L.LinksError) as e:
            s.build(to_device(batch))
        assert e.value.status == L.ECAPACITY


def test_graph_replay_and_determinism(L):
    from paper_2208_14567_gb300.api import Simulator, to_device
    a = I.dyad_batch(3000, 6, 8, seed=11)
    b = I.dyad_batch(3000, 6, 8, seed=12)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with Simulator(3000, 8, stream=stream) as s:
            db = to_device(a)
            out = s.alloc(200, L.MIXED, L.OUT_VALID_ONLY)
            status = torch.empty(3000, dtype=torch.int32, device="cuda")
            L.links_prepare(s.ctx, 200)
            L.links_capture_begin(s.ctx)
            s.build(db, status)
            s.simulate(200, L.MIXED, L.OUT_VALID_ONLY, out=out)
            g = L.links_capture_end(s.ctx)
            results = []
            for src in (a, b, a):
                for dst, x in zip((db.n_joints, db.adj, db.jtype, db.pos), (src.n_joints, src.adj, src.jtype, src.pos)):
                    dst.copy_(torch.from_numpy(np.ascontiguousarray(x)))
                L.links_graph_launch(s.ctx, g)
                s.sync()
                n = int(out.n_out[0])
                results.append((out.valid.cpu().numpy(), out.traj[:n].cpu().numpy()))
            L.links_graph_free(g)
    direct = run(b, 200, L.MIXED, L.OUT_VALID_ONLY, L)
    n = int(direct["n_out"][0])
    assert np.array_equal(results[1][0], direct["valid"])
    assert np.array_equal(results[1][1], direct["traj"][:n], equal_nan=True)
    assert np.array_equal(results[0][0], results[2][0])
    assert np.array_equal(results[0][1], results[2][1], equal_nan=True)


@pytest.mark.slow
def test_full_size_one_million_candidates(L):
    """1M candidates of 6-8 joints, T = 200, LINKS_MIXED with VALID_ONLY rows: the
    launch configuration bench.py times.  Flags of all 1M against the oracle,
    trajectories of 3000 sampled valid rows."""
    batch = I.dyad_batch(1 << 20, 6, 8, seed=0)
    ref = O.simulate(batch, 200, traj=False, path=False)
    res = run(batch, 200, L.MIXED, L.OUT_VALID_ONLY, L)
    check_flags(res, ref, "1M mixed")
    n = int(res["n_out"][0])
    assert np.array_equal(res["out_index"][:n], np.nonzero(res["valid"])[0])
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(n, size=min(3000, n), replace=False))
    sub = batch.take(res["out_index"][rows])
    rs = O.simulate(sub, 200)
    check_positions(sub, res["traj"][rows], res["path"][rows], rs, np.full(len(rows), -1, np.int16),
                    TOL_MIXED, "1M sampled rows")
    f64 = run(batch, 200, L.PLAIN_F64, L.OUT_VALID_ONLY, L)
    check_flags(f64, ref, "1M f64")


@pytest.mark.parametrize("nmax", [8, 12, 20])
def test_every_kernel_shape_gives_the_same_outputs(L, nmax, tmp_path):
    """The shape table (links_set_tuning): every screen shape (lanes, steps per lane, CTAs
    per SM) and emit shape (shared or thread-local double-word slots, CTAs per SM) gives
    the same flags, lock steps, minimum discriminants, rows and trajectories to the bit;
    the autotuner's table survives a save and a load into another context; out-of-range
    values and files tuned on another device are refused."""
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = I.dyad_batch(6000, 6, nmax, seed=70 + nmax, permute=True, nmax=nmax)
    T = 96
    db = to_device(batch)
    shapes = [dict(screen_lanes=8), dict(screen_lanes=16, screen_steps=1), dict(screen_lanes=32, screen_ctas=1),
              dict(screen_lanes=8, screen_steps=2 if nmax <= 16 else 1, screen_ctas=2),
              dict(screen_lanes=16, screen_defer=1), dict(screen_lanes=8, screen_defer=1, screen_steps=1),
              dict(emit_dws=0), dict(emit_dws=1, emit_ctas=1), dict(emit_dws=0, emit_ctas=2)]
    ref = None
    with Simulator(batch.B, nmax) as s:
        for sh in shapes:
            for k in L.TUNE_KEYS:
                L.links_set_tuning(s.ctx, nmax, L.TUNE_KEYS[k], -1 if k == "emit_dws" else (8 if k == "screen_lanes" else 0))
            for k, v in sh.items():
                L.links_set_tuning(s.ctx, nmax, L.TUNE_KEYS[k], v)
            s.build(db)
            o = s.simulate(T, L.MIXED, L.OUT_VALID_ONLY)
            s.sync()
            n = int(o.n_out[0])
            got = [o.valid.cpu().numpy(), o.lock_step.cpu().numpy(), o.min_disc.cpu().numpy(),
                   o.out_index[:n].cpu().numpy(), o.traj[:n].cpu().numpy(), o.path[:n].cpu().numpy()]
            if ref is None:
                ref = got
            else:
                for a, b in zip(ref, got):
                    assert np.array_equal(a, b, equal_nan=True), sh
        lanes = L.links_autotune(s.ctx, s.plan, T)
        table = L.tuning_table(s.ctx, nmax)
        assert table["screen_lanes"] == lanes
        path = str(tmp_path / "tuning.txt")
        L.links_tuning_save(s.ctx, path)
        with pytest.raises(L.LinksError):
            L.links_set_tuning(s.ctx, nmax, L.TUNE_SCREEN_LANES, 12)
        with pytest.raises(L.LinksError):
            L.links_set_tuning(s.ctx, 20, L.TUNE_SCREEN_STEPS, 2)
        with pytest.raises(L.LinksError):
            L.links_set_tuning(s.ctx, nmax, 17, 0)
    with Simulator(batch.B, nmax) as s2:
        L.links_tuning_load(s2.ctx, path)
        assert L.tuning_table(s2.ctx, nmax) == table
        text = open(path).read().splitlines()
        other = str(tmp_path / "other.txt")
        with open(other, "w") as f:
            f.write("links-tuning 2 sms 7 device some other GPU\n" + "\n".join(text[1:]) + "\n")
        with pytest.raises(L.LinksError):
            L.links_tuning_load(s2.ctx, other)
    print(f"[shapes n_max={nmax}] autotuned {table}")


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_every_screen_lane_count_matches_oracle(L, lanes):
    from paper_2208_14567_gb300.api import Simulator, to_device
    batch = I.dyad_batch(3000, 6, 20, seed=40 + lanes, permute=True)
    ref = O.simulate(batch, 200)
    with Simulator(batch.B, batch.nmax) as s:
        L.links_set_screen_lanes(s.ctx, batch.nmax, lanes)
        s.build(to_device(batch))
        o = s.simulate(200, L.MIXED, L.OUT_FULL)
        s.sync()
        res = {"valid": o.valid.cpu().numpy(), "lock_step": o.lock_step.cpu().numpy()}
        traj, path = o.traj.cpu().numpy(), o.path.cpu().numpy()
    check_flags(res, ref, f"lanes={lanes}")
    check_positions(batch, traj, path, ref, res["lock_step"], TOL_MIXED, f"lanes={lanes}")


@pytest.mark.slow
def test_config3_four_million_graph_autotuned(L):
    """4M dyad-built candidates of 6-20 joints in one persistent screen launch under a
    captured CUDA graph (plan build + simulate), lanes per mechanism autotuned; flags
    of all 4M against the oracle and the plain FP64 kernel, 2000 sampled valid rows
    against the oracle."""
    from paper_2208_14567_gb300.api import Simulator, to_device
    B, T = 4 * 1024 * 1024, 200
    batch = I.dyad_batch(B, 6, 20, seed=3, nmax=20)
    ref = O.simulate(batch, T, traj=False, path=False)
    n_valid = int(ref.valid.sum())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with Simulator(B, 20, stream=stream) as s:
            db = to_device(batch)
            status = torch.empty(B, dtype=torch.int32, device="cuda")
            s.build(db, status)
            lanes = L.links_autotune(s.ctx, s.plan, T)
            out = s.alloc(T, L.MIXED, L.OUT_VALID_ONLY, out_capacity=n_valid + 4096)
            L.links_prepare(s.ctx, T)
            L.links_capture_begin(s.ctx)
            s.build(db, status)
            s.simulate(T, L.MIXED, L.OUT_VALID_ONLY, out=out)
            g = L.links_capture_end(s.ctx)
            L.links_graph_launch(s.ctx, g)
            s.sync()
            L.links_graph_free(g)
            res = {"valid": out.valid.cpu().numpy(), "lock_step": out.lock_step.cpu().numpy()}
            n = int(out.n_out[0])
            idx = out.out_index[:n].cpu().numpy()
            rows = np.sort(np.random.default_rng(1).choice(n, size=min(2000, n), replace=False))
            traj = out.traj[torch.from_numpy(rows).cuda()].cpu().numpy()
            path = out.path[torch.from_numpy(rows).cuda()].cpu().numpy()
            del out
            f = s.simulate(T, L.PLAIN_F64, L.OUT_VALID_ONLY, traj=False, path=False)
            s.sync()
            f64 = {"valid": f.valid.cpu().numpy(), "lock_step": f.lock_step.cpu().numpy()}
    print(f"[config 3] lanes per mechanism chosen by the autotuner: {lanes}")
    check_flags(res, ref, "4M mixed (graph)")
    check_flags(f64, ref, "4M plain f64")
    assert np.array_equal(idx, np.nonzero(res["valid"])[0])
    sub = batch.take(idx[rows])
    rs = O.simulate(sub, T)
    check_positions(sub, traj, path, rs, np.full(len(rows), -1, np.int16), TOL_MIXED, "4M sampled rows")
