"""ctypes wrapper of the plain FP64 oracle (``links_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product package.  Batches are split
into contiguous ranges that run on a thread pool (ctypes releases the GIL during
the C call), so the oracle uses every host core.

Top-k selection is a library sort (numpy ``lexsort``): ascending distance, ties to
the lower database index (the exact top-k reading of the retrieval case study).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "links_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liblinks_oracle.so")

MAXJ = 64
STATUS = {0: "OK", 1: "BAD_SIZE", 2: "BAD_TYPE", 3: "BAD_ADJ", 4: "NO_MOTOR", 5: "NO_PIVOT",
          6: "NOT_DYAD_SOLVABLE", 7: "OVERCONSTRAINED"}


class Plan(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n", ctypes.c_int32), ("motor", ctypes.c_int32),
                ("pivot", ctypes.c_int32), ("n_dyads", ctypes.c_int32), ("coupler", ctypes.c_int32),
                ("k", ctypes.c_int32 * MAXJ), ("i", ctypes.c_int32 * MAXJ),
                ("j", ctypes.c_int32 * MAXJ), ("s", ctypes.c_int32 * MAXJ),
                ("r1sq", ctypes.c_double * MAXJ), ("r2sq", ctypes.c_double * MAXJ)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _OUT)
    return _OUT


_lib = None


def _bind(L):
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int
    L.lo_plan.argtypes = [i32, i32, P, P, P, ctypes.POINTER(Plan)]
    L.lo_plan.restype = i32
    L.lo_solve_at.argtypes = [ctypes.POINTER(Plan), i32, P, ctypes.c_double, P, P, P, P]
    L.lo_solve_at.restype = i32
    L.lo_simulate.argtypes = [i64, i64, i32, P, P, P, P, i32, P, P, P, P, P, P, P]
    L.lo_simulate.restype = None
    L.lo_normalize.argtypes = [i64, i64, i32, P, P]
    L.lo_normalize.restype = None
    L.lo_normalize_maxline.argtypes = [i32, P, P, P, P, P]
    L.lo_normalize_maxline.restype = None
    L.lo_chamfer.argtypes = [i32, P, i32, P]
    L.lo_chamfer.restype = ctypes.c_double
    L.lo_chamfer_many.argtypes = [i32, P, i64, i64, i32, P, P]
    L.lo_chamfer_many.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def compile_variant(src_text: str, out_path: str):
    """Compile a modified copy of the oracle source (used by the mutation tests)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-D_DEFAULT_SOURCE",
                    "-o", out_path, src, "-lm"], check=True)
    return _bind(ctypes.CDLL(out_path))


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def n_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())


def _ranges(n: int, parts: int, min_chunk: int = 1):
    parts = max(1, min(parts, (n + min_chunk - 1) // min_chunk))
    edges = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(edges[i]), int(edges[i + 1])) for i in range(parts) if edges[i + 1] > edges[i]]


def _run_parallel(fn, n: int, threads: int | None, min_chunk: int = 64):
    threads = n_threads() if threads is None else threads
    rs = _ranges(n, threads * 4, min_chunk)
    if threads <= 1 or len(rs) <= 1:
        for r in rs:
            fn(*r)
        return
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda r: fn(*r), rs))


def plan(n: int, adj: np.ndarray, jtype: np.ndarray, pos: np.ndarray) -> Plan:
    """Solve order of one mechanism (adj [nmax,nmax], jtype [nmax], pos [nmax,2])."""
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    jtype = np.ascontiguousarray(jtype, dtype=np.int8)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    P = Plan()
    lib().lo_plan(int(n), adj.shape[0], _ptr(adj), _ptr(jtype), _ptr(pos), ctypes.byref(P))
    return P


def solve_at(P: Plan, pos0: np.ndarray, theta: float):
    """Joint positions at crank angle theta -> (out [nmax,2], locked, q_min, q_abs_min, q_lock)."""
    pos0 = np.ascontiguousarray(pos0, dtype=np.float64)
    out = np.empty_like(pos0)
    qm, qa, ql = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    locked = lib().lo_solve_at(ctypes.byref(P), pos0.shape[0], _ptr(pos0), float(theta), _ptr(out),
                               ctypes.byref(qm), ctypes.byref(qa), ctypes.byref(ql))
    return out, bool(locked), qm.value, qa.value, ql.value


class SimResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def simulate(batch, T: int, *, traj: bool = True, path: bool = True, threads: int | None = None):
    """Plan and simulate every mechanism of a MechBatch in FP64.

    Returns status [B] int32, valid [B] uint8, lock_step [B] int16 (-1 none, -2 not
    simulated), min_disc [B] (min q over the steps before the lock), min_abs_q [B]
    (min |q| over every dyad evaluated, the margin indicator), traj [B,nmax,T,2] and
    path [B,T,2] (NaN from the lock on) when requested.
    """
    B, nmax = batch.B, batch.nmax
    nj = np.ascontiguousarray(batch.n_joints, dtype=np.int32)
    adj = np.ascontiguousarray(batch.adj, dtype=np.uint8)
    jt = np.ascontiguousarray(batch.jtype, dtype=np.int8)
    pos = np.ascontiguousarray(batch.pos, dtype=np.float64)
    tr = np.empty((B, nmax, T, 2)) if traj else None
    pa = np.empty((B, T, 2)) if path else None
    valid = np.empty(B, np.uint8)
    lock = np.empty(B, np.int16)
    mind = np.empty(B)
    mabs = np.empty(B)
    st = np.empty(B, np.int32)
    L = lib()

    def run(b0, b1):
        L.lo_simulate(b0, b1, nmax, _ptr(nj), _ptr(adj), _ptr(jt), _ptr(pos), T, _ptr(tr), _ptr(pa),
                      _ptr(valid), _ptr(lock), _ptr(mind), _ptr(mabs), _ptr(st))

    _run_parallel(run, B, threads)
    return SimResult(status=st, valid=valid, lock_step=lock, min_disc=mind, min_abs_q=mabs,
                     traj=tr, path=pa)


def normalize(curves: np.ndarray, threads: int | None = None) -> np.ndarray:
    c = np.ascontiguousarray(curves, dtype=np.float64)
    M, T = c.shape[0], c.shape[1]
    out = np.empty_like(c)
    L = lib()
    _run_parallel(lambda a, b: L.lo_normalize(a, b, T, _ptr(c), _ptr(out)), M, threads)
    return out


def normalize_maxline(curves: np.ndarray, pairs: np.ndarray | None = None):
    """The paper's normalisation (lo_normalize_maxline) of [M, T, 2] curves.
    -> (normalised [M, T, 2], pair [M, 2] int32, circle variance [M]).  ``pairs`` [M, 2]
    imposes the pair of each curve instead of the maximum-distance search."""
    c = np.ascontiguousarray(curves, dtype=np.float64)
    M, T = c.shape[0], c.shape[1]
    out = np.empty_like(c)
    pair = np.zeros((M, 2), dtype=np.int32)
    var = np.zeros(M, dtype=np.float64)
    pin = None if pairs is None else np.ascontiguousarray(pairs, dtype=np.int32)
    L = lib()
    for m in range(M):
        L.lo_normalize_maxline(T, _ptr(c[m]), _ptr(out[m]), None if pin is None else _ptr(pin[m]),
                               _ptr(pair[m]), _ptr(var[m:]))
    return out, pair, var


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Output idx (from 0) of splitmix64 started at ``seed`` (Steele, Lea and Flood,
    OOPSLA 2014, with Vigna's published constants), as uint64."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) \
            * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def curate_paths(traj: np.ndarray, row_index, batch, circle_var: float = 5e-4, keep_rate: float = 0.005,
                 seed: int = 0, pairs: np.ndarray | None = None):
    """The paper's dataset curation (Sec. "Dataset Curation & Processing") of the joint
    paths traj [R, n_max, T, 2] (row r of mechanism row_index[r], or r if None): every
    moving joint's path is normalised (normalize_maxline); it is an arc when the joint is
    linked to a fixed joint, a circle when its circle variance is below circle_var; arcs
    and circles are kept only when the keep draw of (b, j), output b * n_max + j of
    splitmix64(seed) as a double in [0, 1), is below keep_rate.  ``pairs`` [R, n_max, 2]
    imposes the normalising pairs.
    -> dict(flags [R, n_max] uint8: 1 path, 2 arc, 4 circle, 8 kept; circ_var [R, n_max];
            pair [R, n_max, 2]; kept_index (r * n_max + j, increasing); kept_paths)."""
    R, n_max, T = traj.shape[0], traj.shape[1], traj.shape[2]
    rows = np.arange(R) if row_index is None else np.asarray(row_index, dtype=np.int64)
    flags = np.zeros((R, n_max), np.uint8)
    cv = np.zeros((R, n_max))
    pair = np.zeros((R, n_max, 2), np.int32)
    normed = np.zeros((R, n_max, T, 2))
    for r in range(R):
        b = int(rows[r])
        n = int(batch.n_joints[b])
        for j in range(n):
            if batch.jtype[b, j] == 0:
                continue  # a fixed joint does not move
            out, pr, var = normalize_maxline(traj[r, j][None], None if pairs is None else pairs[r, j][None])
            normed[r, j], pair[r, j], cv[r, j] = out[0], pr[0], var[0]
            arc = any(batch.adj[b, j, k] and batch.jtype[b, k] == 0 for k in range(n))
            circle = var[0] < circle_var
            u = float(splitmix64(seed, np.uint64(b * n_max + j)) >> np.uint64(11)) * 2.0 ** -53
            kept = not (arc or circle) or u < keep_rate
            flags[r, j] = 1 | (2 if arc else 0) | (4 if circle else 0) | (8 if kept else 0)
    kept_index = np.nonzero((flags.reshape(-1) & 8) != 0)[0]
    return dict(flags=flags, circ_var=cv, pair=pair, kept_index=kept_index,
                kept_paths=normed.reshape(R * n_max, T, 2)[kept_index])


def chamfer(p: np.ndarray, q: np.ndarray) -> float:
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().lo_chamfer(p.shape[0], _ptr(p), q.shape[0], _ptr(q))


def chamfer_many(query: np.ndarray, db: np.ndarray, threads: int | None = None) -> np.ndarray:
    """Chamfer distance from one query curve to every database curve (FP64)."""
    q = np.ascontiguousarray(query, dtype=np.float64)
    d = np.ascontiguousarray(db, dtype=np.float64)
    M, T = d.shape[0], d.shape[1]
    out = np.empty(M)
    L = lib()
    _run_parallel(lambda a, b: L.lo_chamfer_many(q.shape[0], _ptr(q), a, b, T, _ptr(d), _ptr(out)),
                  M, threads, min_chunk=16)
    return out


def topk(dist: np.ndarray, k: int):
    """Exact top-k of a distance vector: ascending, ties to the lower index."""
    order = np.lexsort((np.arange(dist.shape[0]), dist))[:k]
    return order.astype(np.int64), dist[order]


def chamfer_topk(queries: np.ndarray, db: np.ndarray, k: int, threads: int | None = None):
    idx = np.empty((queries.shape[0], k), np.int64)
    dist = np.empty((queries.shape[0], k))
    for qi in range(queries.shape[0]):
        d = chamfer_many(queries[qi], db, threads)
        idx[qi], dist[qi] = topk(d, k)
    return idx, dist


def first_under(dist: np.ndarray, order: np.ndarray, threshold: float, k: int):
    """The paper's retrieval (Sec. "A Case Study of Mechanism Retrieval"): going through
    the database in the shuffled order ``order`` (order[r] = the curve looked at r-th),
    the first k curves whose distance is below the threshold.
    -> (indices [<= k] in scan order, their distances)."""
    hits = order[dist[order] < threshold][:k]
    return hits.astype(np.int64), dist[hits]


def chamfer_first_under(queries: np.ndarray, db: np.ndarray, order: np.ndarray, threshold: float, k: int,
                        threads: int | None = None):
    """first_under of each query's chamfer distances; -1 / inf past the hits found."""
    idx = np.full((queries.shape[0], k), -1, np.int64)
    dist = np.full((queries.shape[0], k), np.inf)
    for qi in range(queries.shape[0]):
        i, d = first_under(chamfer_many(queries[qi], db, threads), order, threshold, k)
        idx[qi, :len(i)], dist[qi, :len(i)] = i, d
    return idx, dist
