"""Parity of the path stage (normalisation, chamfer top-k) with the FP64 oracle.

Curves are coupler paths of valid four-bars simulated by the oracle (never by the
CUDA path), under random similarity transforms, plus degenerate cases.

Tolerances:
  * normalise: |gpu - oracle| <= 2e-5 (curves have unit RMS radius) where the
    oracle's principal-axis gap (lambda1 - lambda2)/(lambda1 + lambda2) >= 1e-3 and
    |mean x^3| >= 1e-3; otherwise (axis or sign ill-determined) the per-point radii
    must agree to 2e-5 (the rotation-invariant content);
  * chamfer top-k: every returned distance equals the oracle's CD of that pair to
    1e-5 relative; the returned set is the oracle's top-k up to near-ties at the
    boundary (a returned index's oracle CD <= the oracle's k-th CD + 1e-5 rel).
"""
import numpy as np
import pytest

from oracle import oracle as O
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


@pytest.fixture(scope="module")
def ctx(L):
    c = L.links_create(0, torch.cuda.current_stream())
    yield c
    L.links_destroy(c)


def coupler_curves(n, T, seed):
    f = I.fourbar_batch(5 * n + 64, seed=seed)
    r = O.simulate(f, T, traj=False, path=True)
    return r.path[r.valid == 1][:n]


def transformed(curves, seed):
    rng = np.random.default_rng(seed)
    out = np.empty_like(curves)
    for m in range(len(curves)):
        a = rng.uniform(0, 2 * np.pi)
        R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        out[m] = rng.uniform(0.3, 3) * curves[m] @ R.T + rng.normal(size=2)
    return out


def gpu_normalize(L, ctx, curves32):
    x = torch.from_numpy(np.ascontiguousarray(curves32)).cuda()
    y = torch.empty_like(x)
    L.links_normalize(ctx, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def margin_mask(ref):
    x, y = ref[..., 0], ref[..., 1]
    sxx, syy = (x * x).mean(1), (y * y).mean(1)
    gap = (sxx - syy) / np.maximum(sxx + syy, 1e-300)
    s3 = np.abs((x ** 3).mean(1))
    return (gap < 1e-3) | (s3 < 1e-3)


@pytest.mark.parametrize("T", [200, 7, 33, 256, 1000])
def test_normalize_matches_oracle(L, ctx, T):
    base = coupler_curves(400, T, seed=T)
    curves = transformed(base, seed=T).astype(np.float32)
    s = np.linspace(0, 2 * np.pi, T, endpoint=False)
    special = np.stack([
        np.stack([np.cos(s), np.sin(s)], -1) * 2 + 1,            # circle: isotropic
        np.stack([3 * np.cos(s), np.sin(s)], -1),                 # ellipse: sum x^3 = 0
        np.full((T, 2), 0.25),                                    # one point: zeros
    ]).astype(np.float32)
    curves = np.concatenate([curves, special])
    ref = O.normalize(curves.astype(np.float64))
    out = gpu_normalize(L, ctx, curves)
    mg = margin_mask(ref)
    mg[-1] = False
    ok = ~mg
    err = np.abs(out[ok] - ref[ok]).max()
    print(f"[T={T}] curves {len(curves)} margin {int(mg.sum())} max |gpu - oracle| {err:.2e}")
    assert err <= 2e-5
    assert mg.sum() <= 0.05 * len(curves) + 2
    rad_g = np.linalg.norm(out[mg], axis=-1)
    rad_r = np.linalg.norm(ref[mg], axis=-1)
    assert np.abs(rad_g - rad_r).max() <= 2e-5
    assert (out[-1] == 0).all()


def test_normalize_in_place_and_empty(L, ctx):
    curves = transformed(coupler_curves(50, 200, 3), 4).astype(np.float32)
    x = torch.from_numpy(curves).cuda()
    ref = gpu_normalize(L, ctx, curves)
    L.links_normalize(ctx, x, x)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), ref)
    e = torch.empty((0, 200, 2), dtype=torch.float32, device="cuda")
    L.links_normalize(ctx, e, e)


def gpu_topk(L, ctx, q32, db32, k):
    q = torch.from_numpy(np.ascontiguousarray(q32)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(db32)).cuda()
    idx = torch.empty((q.shape[0], k), dtype=torch.int32, device="cuda")
    dist = torch.empty((q.shape[0], k), dtype=torch.float32, device="cuda")
    L.links_chamfer_topk(ctx, q, d, k, idx, dist)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


def check_topk(q, db, idx, dist, k, label):
    rel = 1e-5
    worst = 0.0
    for a in range(len(q)):
        ref = O.chamfer_many(q[a].astype(np.float64), db.astype(np.float64))
        ridx, rd = O.topk(ref, k)
        got = idx[a]
        assert (got >= 0).all()
        assert (np.diff(dist[a]) >= 0).all()
        worst = max(worst, float(np.abs(dist[a] - ref[got]).max() / max(rd[-1], 1e-12)))
        assert np.allclose(dist[a], ref[got], rtol=rel, atol=1e-7)
        assert (ref[got] <= rd[-1] * (1 + rel) + 1e-7).all()
        assert len(set(got.tolist())) == k
    print(f"[{label}] queries {len(q)} db {len(db)} max relative distance error {worst:.2e}")


@pytest.mark.parametrize("T,M,Q,k", [(200, 3000, 24, 10), (37, 1500, 9, 5), (64, 100, 17, 32), (256, 700, 5, 1)])
def test_chamfer_topk_matches_oracle(L, ctx, T, M, Q, k):
    curves = O.normalize(coupler_curves(M + Q, T, seed=100 + T)).astype(np.float32)
    db, held = curves[:M], curves[M:M + Q]
    q = I.perturb_curves(held, 0.02, seed=T)
    q = O.normalize(q.astype(np.float64)).astype(np.float32)
    q[0] = db[M // 2]  # an exact copy must come first, at distance 0
    idx, dist = gpu_topk(L, ctx, q, db, k)
    assert idx[0, 0] == M // 2 and dist[0, 0] == 0.0
    check_topk(q, db, idx, dist, k, f"T={T} M={M} Q={Q} k={k}")


def test_chamfer_ties_and_small_database(L, ctx):
    T = 50
    base = O.normalize(coupler_curves(6, T, seed=7)).astype(np.float32)
    db = np.concatenate([base, base[:3]])  # indices 6, 7, 8 duplicate 0, 1, 2
    idx, dist = gpu_topk(L, ctx, base[:3], db, 12)
    for a in range(3):
        assert idx[a, 0] == a and idx[a, 1] == a + 6 and dist[a, 1] == 0.0  # tie -> lower index first
        assert (idx[a, 9:] == -1).all() and np.isinf(dist[a, 9:]).all()    # only 9 curves exist
    idx, dist = gpu_topk(L, ctx, base[:2], db[:0], 4)
    assert (idx == -1).all() and np.isinf(dist).all()


def test_chamfer_rejects_bad_sizes(L, ctx):
    q = torch.zeros((2, 300, 2), dtype=torch.float32, device="cuda")
    idx = torch.empty((2, 4), dtype=torch.int32, device="cuda")
    dist = torch.empty((2, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(L.LinksError):
        L.links_chamfer_topk(ctx, q, q, 4, idx, dist)  # T > 256
    q = torch.zeros((2, 200, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(L.LinksError):
        L.links_chamfer_topk(ctx, q, q, 33, idx, dist)  # k > 32


@pytest.mark.parametrize("T,M,Q,k", [(200, 20000, 40, 10), (64, 5000, 33, 32), (13, 3000, 9, 3), (2, 2000, 7, 5)])
def test_chamfer_pruning_changes_nothing(L, ctx, T, M, Q, k):
    """The lower-bound pruning only skips curves that cannot enter the top-k, so the
    pruned and the exhaustive search agree bit for bit, near-duplicates included."""
    curves = O.normalize(coupler_curves(M // 4 + Q, T, seed=300 + T)).astype(np.float32)
    base, held = curves[:M // 4], curves[M // 4:]
    # the database: each curve 4 times, three of them slightly perturbed (near-ties)
    db = np.concatenate([base] + [I.perturb_curves(base, s, seed=s_i) for s_i, s in enumerate((1e-6, 1e-4, 1e-2))])
    db = db[np.random.default_rng(T).permutation(len(db))].astype(np.float32)
    q = np.concatenate([I.perturb_curves(held, 0.02, seed=T), db[:3]]).astype(np.float32)
    L.links_set_chamfer_prune(ctx, False)
    idx0, dist0 = gpu_topk(L, ctx, q, db, k)
    L.links_set_chamfer_prune(ctx, True)
    idx1, dist1 = gpu_topk(L, ctx, q, db, k)
    assert np.array_equal(idx0, idx1) and np.array_equal(dist0, dist1)
    sel = np.random.default_rng(T).choice(len(q), 6, replace=False)
    check_topk(q[sel], db, idx1[sel], dist1[sel], k, f"pruned T={T} M={len(db)}")
    assert L.lib().links_set_chamfer_prune(ctx, 2) == L.EINVAL


@pytest.mark.parametrize("T", [200, 7, 33, 256])
def test_normalize_maxline_matches_oracle(L, ctx, T):
    """The paper's normalisation: the pair the kernel finds (float32) is a farthest pair up
    to float rounding, and with that pair imposed the oracle's normalised curve and
    circle statistic match."""
    base = coupler_curves(300, T, seed=50 + T)
    curves = transformed(base, seed=T).astype(np.float32)
    s = np.linspace(0, 2 * np.pi, T, endpoint=False)
    special = np.stack([
        np.stack([np.cos(s), np.sin(s)], -1) * 2 + 1,                        # circle
        np.stack([0.3 + 2 * np.linspace(0, 1, T), -0.2 + np.linspace(0, 1, T)], -1),  # segment
        np.full((T, 2), 0.25),                                               # one point
    ]).astype(np.float32)
    curves = np.concatenate([curves, special])
    x = torch.from_numpy(curves).cuda()
    y = torch.empty_like(x)
    pair = torch.empty((len(curves), 2), dtype=torch.int32, device="cuda")
    var = torch.empty(len(curves), dtype=torch.float32, device="cuda")
    L.links_normalize_maxline(ctx, x, y, pair, var)
    torch.cuda.synchronize()
    out, pr, vr = y.cpu().numpy(), pair.cpu().numpy(), var.cpu().numpy()
    c64 = curves.astype(np.float64)
    _, opair, _ = O.normalize_maxline(c64)
    ref, _, rvar = O.normalize_maxline(c64, pairs=pr)
    dist = lambda c, pq: np.hypot(*(c[pq[1]] - c[pq[0]]))
    for m in range(len(curves) - 1):
        assert pr[m, 0] < pr[m, 1] and dist(c64[m], pr[m]) >= dist(c64[m], opair[m]) * (1 - 1e-5)
    err = np.abs(out - ref).max()
    print(f"[T={T}] curves {len(curves)} same pair as the oracle {np.mean((pr == opair).all(1)):.3f} "
          f"max |gpu - oracle| {err:.2e} max |var - oracle| {np.abs(vr - rvar).max():.2e}")
    assert err <= 2e-5 and np.abs(vr - rvar).max() <= 2e-6
    assert (out[-1] == 0.5).all()
    if T % 2 == 0:  # antipodal points: a circle of diameter 1 about the box centre
        assert vr[-3] < 1e-6
    with pytest.raises(L.LinksError):
        L.links_normalize_maxline(ctx, x, x)


def gpu_first(L, ctx, q32, db32, order, thr, k):
    q = torch.from_numpy(np.ascontiguousarray(q32)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(db32)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(order, dtype=np.int32)).cuda()
    idx = torch.empty((q.shape[0], k), dtype=torch.int32, device="cuda")
    dist = torch.empty((q.shape[0], k), dtype=torch.float32, device="cuda")
    L.links_chamfer_first_under(ctx, q, d, o, thr, k, idx, dist)
    L.links_sync(ctx)
    return idx.cpu().numpy(), dist.cpu().numpy()


def check_first(q, db, order, thr, k, idx, dist, label):
    """Indices bit-exact with the oracle (the decision at the threshold is taken on the
    FP64 distance); distances within 1e-5 relative."""
    ridx, rdist = O.chamfer_first_under(q.astype(np.float64), db.astype(np.float64), order, thr, k)
    assert np.array_equal(idx, ridx), (label, idx, ridx)
    hit = ridx >= 0
    assert np.allclose(dist[hit], rdist[hit], rtol=1e-5, atol=1e-7)
    assert np.isinf(dist[~hit]).all()
    print(f"[{label}] queries {len(q)} db {len(db)} hits {int(hit.sum())} of {hit.size}")


@pytest.mark.parametrize("T,M,Q,k", [(200, 3000, 24, 3), (37, 1500, 9, 5), (13, 700, 17, 32), (256, 400, 5, 1)])
def test_chamfer_first_under_matches_oracle(L, ctx, T, M, Q, k):
    """The paper's retrieval (first k under a cut-off in a shuffled scan) against the
    oracle, at cut-offs from none to all of the database; pruning on and off agree."""
    curves = O.normalize(coupler_curves(M + Q, T, seed=500 + T)).astype(np.float32)
    db, held = curves[:M], curves[M:M + Q]
    q = O.normalize(I.perturb_curves(held, 0.02, seed=T).astype(np.float64)).astype(np.float32)
    q[0] = db[M // 3]
    order = np.random.default_rng(T).permutation(M)
    order = np.concatenate([[M // 3], order[order != M // 3]])  # the copy is scanned first
    d0 = O.chamfer_many(q[1].astype(np.float64), db.astype(np.float64))
    for thr in (0.0, float(np.quantile(d0, 0.002)), float(np.quantile(d0, 0.05)), float(np.quantile(d0, 0.5)),
                float("inf")):
        for prune in (True, False):
            L.links_set_chamfer_prune(ctx, prune)
            idx, dist = gpu_first(L, ctx, q, db, order, thr, k)
            if prune:
                ref = (idx, dist)
            else:
                assert np.array_equal(ref[0], idx) and np.array_equal(ref[1], dist)
        check_first(q, db, order, thr, k, idx, dist, f"T={T} M={M} thr={thr:.3g}")
        if thr > 0:  # the exact copy is the first hit, at distance 0
            assert idx[0, 0] == M // 3 and dist[0, 0] == 0.0
    L.links_set_chamfer_prune(ctx, True)


def test_chamfer_first_under_threshold_band(L, ctx):
    """Cut-offs placed exactly at the FP64 distance of a pair (a miss: the test is CD <
    threshold) and just above it (a hit): the FP32 distance sits inside its rounding
    band, so the FP64 recomputation decides, as the oracle does."""
    T, M = 64, 500
    curves = O.normalize(coupler_curves(M + 4, T, seed=77)).astype(np.float32)
    db, q = curves[:M], curves[M:M + 4]
    order = np.random.default_rng(5).permutation(M)
    for a in range(4):
        d = O.chamfer_many(q[a].astype(np.float64), db.astype(np.float64))
        # the curve scanned first that has no nearer curve scanned before it
        j = int(order[0])
        for thr in (float(d[j]), float(np.nextafter(d[j], np.inf))):
            idx, dist = gpu_first(L, ctx, q[a:a + 1], db, order, thr, 1)
            check_first(q[a:a + 1], db, order, thr, 1, idx, dist, f"band query {a} thr={thr!r}")
            assert (idx[0, 0] == j) == (thr > d[j])


def test_chamfer_first_under_partial_scan_and_errors(L, ctx):
    """A scan over part of the database (L < M, repeats allowed), an empty scan, and an
    order entry out of range (skipped, raised on the device error word)."""
    T, M = 50, 600
    curves = O.normalize(coupler_curves(M + 3, T, seed=9)).astype(np.float32)
    db, q = curves[:M], curves[M:]
    rng = np.random.default_rng(1)
    order = np.concatenate([rng.choice(M, 150, replace=False), rng.choice(M, 50)])
    thr = float(np.quantile(O.chamfer_many(q[0].astype(np.float64), db.astype(np.float64)), 0.3))
    idx, dist = gpu_first(L, ctx, q, db, order, thr, 8)
    check_first(q, db, order, thr, 8, idx, dist, "partial scan")
    idx, dist = gpu_first(L, ctx, q, db, order[:0], thr, 4)
    assert (idx == -1).all() and np.isinf(dist).all()
    bad = order.copy()
    bad[3] = M + 5
    with pytest.raises(L.LinksError) as e:
        gpu_first(L, ctx, q, db, bad, thr, 4)
    assert e.value.status == L.EDEVICE
    L.links_sync(ctx)  # the error word was cleared
    qq = torch.zeros((2, T, 2), dtype=torch.float32, device="cuda")
    o = torch.zeros(4, dtype=torch.int32, device="cuda")
    idx = torch.empty((2, 4), dtype=torch.int32, device="cuda")
    dist = torch.empty((2, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(L.LinksError):
        L.links_chamfer_first_under(ctx, qq, qq, o, float("nan"), 4, idx, dist)
    with pytest.raises(L.LinksError):
        L.links_chamfer_first_under(ctx, qq, qq, o, 0.1, 33, idx, dist)


def test_chamfer_first_under_full_size_sampled(L, ctx):
    """The scan at the retrieval benchmark's size (1M curves of 200 points, pruning on, the
    bench's chunking), checked on sampled queries: over the scan prefix up to the k-th
    hit (at most 4000 positions), the oracle's hits are exactly the kernel's."""
    T, M, Q, k = 200, 1_000_000, 32, 3
    db = I.fourier_curves(M, T, seed=21)
    q = np.concatenate([I.perturb_curves(db[:Q // 2], 0.05, seed=22), I.fourier_curves(Q // 2, T, seed=23)])
    order = np.random.default_rng(24).permutation(M)
    sample = db[order[:2000]].astype(np.float64)
    thr = float(np.quantile(O.chamfer_many(q[Q // 2].astype(np.float64), sample), 0.002))
    idx, dist = gpu_first(L, ctx, q, db, order, thr, k)
    rng = np.random.default_rng(25)
    for a in sorted(set(rng.choice(Q, 5, replace=False).tolist()) | {0, Q // 2}):
        hits = idx[a][idx[a] >= 0]
        pos = np.array([int(np.nonzero(order == h)[0][0]) for h in hits], dtype=np.int64)
        end = int(pos[-1]) + 1 if len(hits) == k else M
        end = min(end, 4000)
        pre = order[:end]
        d = O.chamfer_many(q[a].astype(np.float64), db[pre].astype(np.float64))
        ref = pre[d < thr][:k]
        assert np.array_equal(hits[:len(ref)], ref), (a, hits, ref)
        assert np.all(pos[len(ref):] >= end)
        dd = O.chamfer_many(q[a].astype(np.float64), db[hits].astype(np.float64))
        assert np.all(dd < thr) and np.allclose(dist[a][:len(hits)], dd, rtol=1e-5, atol=1e-7)
        print(f"[full size] query {a}: hits {hits.tolist()} at positions {pos.tolist()}")


def test_chamfer_topk_full_size_sampled(L, ctx):
    """The top-10 at the retrieval benchmark's size (1024 noisy queries against 1M
    normalised curves of 200 points, pruning on): at this size the shared k-th distance
    is tight and the prune and early-exit paths run as in the benchmark.  Sampled queries
    are checked against the oracle's exhaustive chamfer distances over all 1M curves."""
    T, M, Q, k = 200, 1_000_000, 1024, 10
    db = O.normalize(I.fourier_curves(M, T, seed=31).astype(np.float64)).astype(np.float32)
    held = O.normalize(I.fourier_curves(Q, T, seed=32).astype(np.float64)).astype(np.float32)
    q = O.normalize(I.perturb_curves(held, 0.02, seed=33).astype(np.float64)).astype(np.float32)
    q[1] = db[777_777]  # an exact copy ranks first at distance 0
    idx, dist = gpu_topk(L, ctx, q, db, k)
    assert idx[1, 0] == 777_777 and dist[1, 0] == 0.0
    sel = sorted({0, Q - 1} | set(np.random.default_rng(34).choice(Q, 2, replace=False).tolist()))
    check_topk(q[sel], db, idx[sel], dist[sel], k, "full size 1024 x 1M")


@pytest.mark.parametrize("n_lo,n_hi,T,keep", [(6, 8, 200, 0.005), (5, 12, 64, 0.3), (6, 10, 33, 1.0)])
def test_curation_matches_oracle(L, ctx, n_lo, n_hi, T, keep):
    """The paper's curation of every moving joint's path, on the oracle's trajectories of
    valid candidates (valid-only rows, so row r is mechanism row_index[r]): path and arc
    flags bit-exact; the normalising pair a farthest pair up to float rounding; with it
    imposed, the oracle's circle statistic within 2e-6 and the circle flag equal (a
    statistic within 1e-6 of the threshold may go either way); kept flags exactly as
    the keep rule gives from the flags and the splitmix64 draws; the kept list in order
    and its normalised paths within 2e-5."""
    batch = I.dyad_batch(1500, n_lo, n_hi, seed=T + n_hi, nmax=n_hi)
    res = O.simulate(batch, T, traj=True, path=False)
    rows = np.nonzero(res.valid == 1)[0].astype(np.int32)
    traj = res.traj[rows].astype(np.float32)
    R, n_max = traj.shape[0], traj.shape[1]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    flags = torch.empty((R, n_max), dtype=torch.uint8, device="cuda")
    cv = torch.empty((R, n_max), dtype=torch.float32, device="cuda")
    pair = torch.empty((R, n_max, 2), dtype=torch.int32, device="cuda")
    cap = R * n_max
    kidx = torch.empty(cap, dtype=torch.int32, device="cuda")
    kpaths = torch.empty((cap, T, 2), dtype=torch.float32, device="cuda")
    nk = torch.empty(1, dtype=torch.int32, device="cuda")
    L.links_curate_paths(ctx, dev(traj), dev(rows), dev(batch.n_joints.astype(np.int32)), dev(batch.adj),
                         dev(batch.jtype), flags, nk, keep_rate=keep, seed=99, circ_var=cv, pair=pair,
                         kept_index=kidx, kept_paths=kpaths)
    L.links_sync(ctx)
    f, v, pr = flags.cpu().numpy(), cv.cpu().numpy(), pair.cpu().numpy()
    n_kept = int(nk.item())
    ref = O.curate_paths(traj.astype(np.float64), rows, batch, keep_rate=keep, seed=99, pairs=pr)
    assert np.array_equal(f & 3, ref["flags"] & 3)
    _, opair, _ = O.normalize_maxline(traj.reshape(R * n_max, T, 2)[(f.reshape(-1) & 1) != 0].astype(np.float64))
    c64 = traj.reshape(R * n_max, T, 2)[(f.reshape(-1) & 1) != 0].astype(np.float64)
    gp = pr.reshape(-1, 2)[(f.reshape(-1) & 1) != 0]
    d = lambda c, pq: np.hypot(*(c[pq[1]] - c[pq[0]]))
    for m in range(len(c64)):
        assert d(c64[m], gp[m]) >= d(c64[m], opair[m]) * (1 - 1e-5)
    has = (f & 1) != 0
    assert np.abs(v[has] - ref["circ_var"][has]).max() <= 2e-6
    near = np.abs(ref["circ_var"] - 5e-4) <= 1e-6
    assert np.array_equal((f & 4)[~near], (ref["flags"] & 4)[~near])
    b = rows[:, None].astype(np.uint64) * np.uint64(n_max) + np.arange(n_max, dtype=np.uint64)[None, :]
    u = (O.splitmix64(99, b) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    want = has & (((f & 6) == 0) | (u < keep))
    assert np.array_equal((f & 8) != 0, want)
    kl = np.nonzero(want.reshape(-1))[0]
    assert n_kept == len(kl) and np.array_equal(kidx.cpu().numpy()[:n_kept], kl)
    err = np.abs(kpaths.cpu().numpy()[:n_kept] - ref["kept_paths"]).max() if n_kept else 0.0
    assert err <= 2e-5
    arcs, circles = int(((f & 2) != 0).sum()), int(((f & 4) != 0).sum())
    print(f"[curation n={n_lo}-{n_hi} T={T}] rows {R} paths {int(has.sum())} arcs {arcs} circles {circles} "
          f"kept {n_kept} near-threshold {int((near & has).sum())} max path err {err:.2e}")


def test_curation_bad_row_and_sizes(L, ctx):
    """A row index out of range gives that row no paths and raises the device error word;
    bad sizes are refused."""
    batch = I.dyad_batch(64, 6, 6, seed=3)
    res = O.simulate(batch, 50, traj=True, path=False)
    traj = torch.from_numpy(np.nan_to_num(res.traj).astype(np.float32)).cuda()
    rows = torch.arange(64, dtype=torch.int32, device="cuda")
    rows[5] = 64
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    flags = torch.empty((64, 6), dtype=torch.uint8, device="cuda")
    nk = torch.empty(1, dtype=torch.int32, device="cuda")
    L.links_curate_paths(ctx, traj, rows, dev(batch.n_joints.astype(np.int32)), dev(batch.adj), dev(batch.jtype),
                         flags, nk)
    with pytest.raises(L.LinksError) as e:
        L.links_sync(ctx)
    assert e.value.status == L.EDEVICE
    assert (flags[5].cpu().numpy() == 0).all()
    with pytest.raises(L.LinksError):
        L.links_curate_paths(ctx, traj, rows, dev(batch.n_joints.astype(np.int32)), dev(batch.adj),
                             dev(batch.jtype), flags, nk, circle_var=float("nan"))


def test_curation_and_scan_edge_cases(L, ctx):
    """Empty inputs and one-point paths: no rows curate to nothing; paths of one point are
    circles of variance 0 (the oracle agrees); a scan with no queries or a k larger than
    the database returns -1 past the hits."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    batch = I.dyad_batch(16, 6, 6, seed=4)
    nk = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    empty = torch.empty((0, 6, 5, 2), dtype=torch.float32, device="cuda")
    L.links_curate_paths(ctx, empty, None, dev(batch.n_joints.astype(np.int32)), dev(batch.adj), dev(batch.jtype),
                         torch.empty((0, 6), dtype=torch.uint8, device="cuda"), nk)
    L.links_sync(ctx)
    assert int(nk.item()) == 0
    res = O.simulate(batch, 1, traj=True, path=False)
    traj = res.traj.astype(np.float32)
    flags = torch.empty((16, 6), dtype=torch.uint8, device="cuda")
    cv = torch.empty((16, 6), dtype=torch.float32, device="cuda")
    L.links_curate_paths(ctx, dev(traj), None, dev(batch.n_joints.astype(np.int32)), dev(batch.adj),
                         dev(batch.jtype), flags, nk, circ_var=cv, keep_rate=0.0)
    L.links_sync(ctx)
    ref = O.curate_paths(traj.astype(np.float64), None, batch, keep_rate=0.0)
    f = flags.cpu().numpy()
    assert np.array_equal(f, ref["flags"])
    assert (cv.cpu().numpy() == 0).all() and ((f & 1) == 0).sum() + ((f & 4) != 0).sum() == f.size
    T = 20
    db = O.normalize(coupler_curves(5, T, seed=8)).astype(np.float32)
    q = db[:2].copy()
    idx, dist = gpu_first(L, ctx, q, db, np.arange(5), float("inf"), 8)
    assert np.array_equal(idx[:, :5], np.tile(np.arange(5), (2, 1))) and (idx[:, 5:] == -1).all()
    assert np.isinf(dist[:, 5:]).all()
    idx, dist = gpu_first(L, ctx, q[:0], db, np.arange(5), 1.0, 3)
    assert idx.shape == (0, 3)
