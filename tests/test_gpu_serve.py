"""Continuous-batching serving (the request loop runs on the device): results are the
same alone and in the mix, match the batch path and the oracle, and admission /
timeouts behave (host-side fault injection: paused admission, a full queue, an
oversized request, a poll that times out, a device barrier whose wait runs out)."""
import time

import numpy as np
import pytest

from conftest import bbox_diag
from oracle import oracle as O
from paper_2208_14567_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 100
NMAX = 20


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_14567_gb300 import links
    links.lib()
    return links


class Out:
    def __init__(self, n):
        self.valid = np.zeros(n, np.uint8)
        self.lock = np.zeros(n, np.int16)
        self.md = np.zeros(n, np.float32)
        self.idx = np.full(n, -1, np.int32)
        self.paths = np.zeros((n, T, 2), np.float32)


def make_requests(pool, sizes):
    reqs, off = [], 0
    for n in sizes:
        reqs.append(pool.slice(off, off + n))
        off += n
    return reqs


def submit(L, ctx, batch, out):
    r = L.make_request(np.ascontiguousarray(batch.n_joints), np.ascontiguousarray(batch.adj),
                       np.ascontiguousarray(batch.jtype), np.ascontiguousarray(batch.pos), out.valid, out.lock,
                       out.md, out.idx, out.paths)
    while True:
        try:
            return L.links_serve_submit(ctx, r), r
        except L.LinksError as e:
            if e.status != L.EBUSY:
                raise
            time.sleep(1e-4)


def wait(L, ctx, ticket, limit_s=60.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        res = L.links_serve_poll(ctx, ticket, 10000)
        if res is not None:
            return res
    raise AssertionError("request did not finish")


def test_alone_equals_mix_equals_batch_path(L):
    pool = I.dyad_batch(30000, 6, 20, seed=31, nmax=NMAX, permute=True)
    rng = np.random.default_rng(0)
    sizes = np.clip(np.exp(rng.uniform(0, np.log(5000), 40)).astype(int), 1, 5000)
    sizes = sizes[np.cumsum(sizes) <= pool.B]
    reqs = make_requests(pool, sizes)
    ctx = L.links_create(0, torch.cuda.current_stream())
    try:
        L.links_serve_start(ctx, 256 << 20, 8, NMAX, T)
        alone = []
        for b in reqs:  # one at a time
            o = Out(b.B)
            t, keep = submit(L, ctx, b, o)
            res = wait(L, ctx, t)
            assert res.status == 0
            alone.append((o, res.n_valid))
        mix, tickets = [], []
        for b in reqs:  # all at once: they share passes
            o = Out(b.B)
            t, keep = submit(L, ctx, b, o)
            mix.append(o)
            tickets.append((t, keep))
        results = [wait(L, ctx, t) for t, _ in tickets]
        L.links_serve_stop(ctx)
    finally:
        L.links_destroy(ctx)
    for (oa, na), om, rm in zip(alone, mix, results):
        assert rm.status == 0 and rm.n_valid == na
        assert np.array_equal(oa.valid, om.valid) and np.array_equal(oa.lock, om.lock)
        assert np.array_equal(oa.md, om.md, equal_nan=True)
        assert np.array_equal(oa.idx[:na], om.idx[:na])
        assert np.array_equal(oa.paths[:na], om.paths[:na])
    # the batch path on the concatenated requests gives the same flags and rows
    from paper_2208_14567_gb300.api import Simulator, to_device
    allb = pool.slice(0, int(sizes.sum()))
    with Simulator(allb.B, NMAX) as s:
        s.build(to_device(allb))
        o = s.simulate(T, L.MIXED, L.OUT_VALID_ONLY, traj=False, path=True)
        p = o.path[:int(o.n_out[0])].clone()
        L.links_normalize(s.ctx, p, p)
        s.sync()
        valid = o.valid.cpu().numpy()
        paths = p.cpu().numpy()
    assert np.array_equal(np.concatenate([m.valid for m in mix]), valid)
    rows = np.concatenate([m.paths[:r.n_valid] for m, r in zip(mix, results)])
    assert np.array_equal(rows, paths)
    # and the oracle: flags (outside the margin) and normalised paths
    ref = O.simulate(allb, T, traj=False, path=True)
    margin = ~(ref.min_abs_q > 1e-9)
    assert not ((valid != ref.valid) & ~margin).any()
    refp = O.normalize(ref.path[ref.valid == 1])
    same = (valid == ref.valid)[ref.valid == 1]
    x = refp[same]
    g = paths[(ref.valid == 1)[valid == 1]]
    # positions carry up to 1e-5 L of error (L = bounding-box diagonal of the
    # mechanism); normalisation divides by the path's RMS radius r, so the error of a
    # normalised point is about 1e-5 L / r, and the rotation adds that over the gap of
    # the principal axes.  Compare points where axis and sign are well determined, and
    # the rotation-invariant radii everywhere.
    Lb = bbox_diag(allb.pos, allb.n_joints)[ref.valid == 1][same]
    raw = ref.path[ref.valid == 1][same]
    rms = np.sqrt(((raw - raw.mean(1, keepdims=True)) ** 2).sum(-1).mean(1))
    amp = 1e-5 * Lb / rms
    sxx, syy = (x[..., 0] ** 2).mean(1), (x[..., 1] ** 2).mean(1)
    gap = (sxx - syy) / (sxx + syy)
    s3 = np.abs((x[..., 0] ** 3).mean(1))
    ok = (gap > 100 * amp) & (s3 > 100 * amp)
    err = np.abs(g - x).max(axis=(1, 2))
    assert (err[ok] <= amp[ok] * (4 + 4 / gap[ok])).all()
    rerr = np.abs(np.linalg.norm(g, axis=-1) - np.linalg.norm(x, axis=-1)).max(1)
    assert (rerr <= 4 * amp).all()
    print(f"serve: {len(reqs)} requests, {allb.B} candidates, {int(valid.sum())} valid, "
          f"max normalised path error {err[ok].max():.2e} ({int(ok.sum())} well-conditioned), "
          f"max error / (1e-5 L / r) {(err[ok] / (amp[ok] * (1 + 1 / gap[ok]))).max():.2f}")


def test_overload_many_small_requests_behind_a_large_one(L):
    """Offered load above what one pass at a time can absorb: a large request occupies
    the GPU while 200 small requests arrive one by one, each of which can open a pass of
    its own.  Every request's flags, valid indices and normalised paths must equal the
    batch path's on the same candidates (the serving loop must not mix up the results
    of passes that are in flight together)."""
    pool = I.dyad_batch(80000, 6, 20, seed=35, nmax=NMAX, permute=True)
    rng = np.random.default_rng(3)
    sizes = [60000] + list(rng.integers(1, 40, 200))
    sizes = np.array(sizes)[np.cumsum(sizes) <= pool.B]
    reqs = make_requests(pool, sizes)
    ctx = L.links_create(0, torch.cuda.current_stream())
    outs, tickets = [], []
    try:
        L.links_serve_start(ctx, 1 << 30, 512, NMAX, T)
        for b in reqs:
            o = Out(b.B)
            t, keep = submit(L, ctx, b, o)
            outs.append(o)
            tickets.append((t, keep))
            time.sleep(2e-5)
        results = [wait(L, ctx, t) for t, _ in tickets]
        stats = L.links_serve_stats(ctx)
        L.links_serve_stop(ctx)
    finally:
        L.links_destroy(ctx)
    # the request loop ran on the device: many passes per launch of its kernel
    assert stats["kernel_launches"] < stats["passes"]
    print(f"overload: {stats}")
    from paper_2208_14567_gb300.api import Simulator, to_device
    allb = pool.slice(0, int(sizes.sum()))
    with Simulator(allb.B, NMAX) as s:
        s.build(to_device(allb))
        o = s.simulate(T, L.MIXED, L.OUT_VALID_ONLY, traj=False, path=True)
        p = o.path[:int(o.n_out[0])].clone()
        L.links_normalize(s.ctx, p, p)
        s.sync()
        valid = o.valid.cpu().numpy()
        lock = o.lock_step.cpu().numpy()
        paths = p.cpu().numpy()
    off = row = 0
    for b, o, r in zip(reqs, outs, results):
        assert r.status == 0
        v = valid[off:off + b.B]
        assert np.array_equal(o.valid, v) and np.array_equal(o.lock, lock[off:off + b.B])
        n = int(v.sum())
        assert r.n_valid == n
        assert np.array_equal(o.idx[:n], np.nonzero(v)[0])
        assert np.array_equal(o.paths[:n], paths[row:row + n])
        off += b.B
        row += n
    print(f"overload: {len(reqs)} requests, {off} candidates, {row} valid rows")


def test_admission_timeout_and_refusals(L):
    pool = I.dyad_batch(4000, 6, 12, seed=32, nmax=12)
    ctx = L.links_create(0, torch.cuda.current_stream())
    try:
        per = 12 * 12 + 12 + 96 + 4 + 64 + 32 + 16 * 12 * 2 + 48 * 10 + 4 + 15 + T * 8
        L.links_serve_start(ctx, per * 1000, 2, 12, T)
        big = pool.slice(0, 1500)
        with pytest.raises(L.LinksError) as e:  # can never fit the arena
            submit(L, ctx, big, Out(big.B))
        assert e.value.status == L.ECAPACITY
        L.links_serve_pause(ctx, True)
        outs = [Out(600) for _ in range(3)]
        parts = [pool.slice(600 * i, 600 * (i + 1)) for i in range(3)]
        keep = []
        t0 = L.links_serve_submit(ctx, L.make_request(*req_arrays(parts[0]), outs[0].valid, outs[0].lock)); keep.append(parts[0])
        t1 = L.links_serve_submit(ctx, L.make_request(*req_arrays(parts[1]), outs[1].valid, outs[1].lock)); keep.append(parts[1])
        with pytest.raises(L.LinksError) as e:  # queue of 2 is full while admission is held
            L.links_serve_submit(ctx, L.make_request(*req_arrays(parts[2]), outs[2].valid, outs[2].lock))
        assert e.value.status == L.EBUSY
        assert L.links_serve_poll(ctx, t0, 2000) is None  # forced timeout: nothing admitted
        L.links_serve_pause(ctx, False)
        r0, r1 = wait(L, ctx, t0), wait(L, ctx, t1)  # 600 + 600 > 1000: the second waits for memory
        assert r0.status == 0 and r1.status == 0
        assert r1.admit_ms >= r0.done_ms - 1.0
        with pytest.raises(L.LinksError):
            L.links_serve_poll(ctx, t0, 0)  # released ticket
        L.links_serve_stop(ctx)
    finally:
        L.links_destroy(ctx)
    ref = O.simulate(pool.slice(0, 1200), T, traj=False, path=False)
    margin = ~(ref.min_abs_q > 1e-9)
    got = np.concatenate([outs[0].valid, outs[1].valid])
    assert not ((got != ref.valid) & ~margin).any()


def test_device_loop_barrier_timeout_is_reported_and_recovered(L):
    """Fault injection on the host side: one grid barrier of the next pass waits for a
    block that does not exist.  The wait gives up after 200 ms, the serving kernel returns,
    the request completes with LINKS_EDEVICE, and the next request is served normally
    (same flags and paths as the batch path)."""
    pool = I.dyad_batch(3000, 6, 12, seed=36, nmax=NMAX)
    a, b = pool.slice(0, 1500), pool.slice(1500, 3000)
    ctx = L.links_create(0, torch.cuda.current_stream())
    try:
        L.links_serve_start(ctx, 64 << 20, 8, NMAX, T)
        L.links_serve_inject_stall(ctx, 200)
        oa = Out(a.B)
        t, keep = submit(L, ctx, a, oa)
        with pytest.raises(L.LinksError) as e:
            wait(L, ctx, t)
        assert e.value.status == L.EDEVICE
        ob = Out(b.B)
        t, keep = submit(L, ctx, b, ob)
        rb = wait(L, ctx, t)
        assert rb.status == 0
        with pytest.raises(L.LinksError):
            L.links_serve_inject_stall(ctx, 0)
        L.links_serve_stop(ctx)
    finally:
        L.links_destroy(ctx)
    from paper_2208_14567_gb300.api import Simulator, to_device
    with Simulator(b.B, NMAX) as s:
        s.build(to_device(b))
        o = s.simulate(T, L.MIXED, L.OUT_VALID_ONLY, traj=False, path=True)
        n = int(o.n_out[0])
        p = o.path[:n].clone()
        L.links_normalize(s.ctx, p, p)
        s.sync()
        assert np.array_equal(o.valid.cpu().numpy(), ob.valid) and rb.n_valid == n
        assert np.array_equal(p.cpu().numpy(), ob.paths[:n])


def req_arrays(b):
    return (np.ascontiguousarray(b.n_joints), np.ascontiguousarray(b.adj), np.ascontiguousarray(b.jtype),
            np.ascontiguousarray(b.pos))


def test_malformed_requests(L):
    ctx = L.links_create(0, torch.cuda.current_stream())
    try:
        with pytest.raises(L.LinksError) as e:
            L.links_serve_submit(ctx, L.Request())
        assert e.value.status == L.ESTATE  # not started
        L.links_serve_start(ctx, 64 << 20, 4, 8, T)
        with pytest.raises(L.LinksError) as e:
            L.links_serve_submit(ctx, L.Request())  # empty
        assert e.value.status == L.EINVAL
        b = I.dyad_batch(50, 6, 8, seed=33)
        b.jtype[3, 1] = 1  # no actuated joint -> per-candidate status, not a failure
        o = Out(50)
        t, keep = submit(L, ctx, b, o)
        r = wait(L, ctx, t)
        assert r.status == 0 and o.lock[3] == -2 and o.valid[3] == 0
        L.links_serve_stop(ctx)
    finally:
        L.links_destroy(ctx)
