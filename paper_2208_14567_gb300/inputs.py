"""Seeded synthetic inputs for the linkage-simulation hot path.

Test and benchmark infrastructure shared by the CUDA path and the oracle.  This
module only draws random numbers and lays them out in the paper's mechanism
representation (Sec. "Mechanism Representation": an n x n 0/1 adjacency matrix
plus, per joint, a type -- 0 fixed, 1 simple, 2 actuated -- and an initial
position).  It contains none of the method's arithmetic: no solve order, no
kinematics, no normalisation and no distances.

Random numbers come from one counter-based generator: the splitmix64 finaliser
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; the constants of Vigna's published splitmix64) applied to
``key + (counter + 1) * golden_gamma``.  Every draw is addressed by
(seed, stream, counter), so results do not depend on batch order, array sizes
or library versions.

Workload recipes (the paper's dataset is not available; these stand in for it):

* ``fourbar_batch``: random four-bar mechanisms with a coupler point.  Joint 0 is
  the ground pivot of the crank, joint 1 the crank tip (actuated), joint 2 the
  second ground pivot, joint 3 the rocker joint (linked to 1 and 2), joint 4 the
  coupler point (linked to 1 and 3).  Positions are uniform in [0,1]^2
  (Sec. "Finding Valid Initial Positions", bounding-box rule), kept in float64.
* ``dyad_batch``: candidates grown from the paper's initial mechanism (ground
  joint 0, actuated joint 1 on the crank 0-1, floating ground joint 2;
  Sec. "1-DOF Operator", "Initialization") by repeated joint operators: with
  probability 1/4 the fixed-node operator N_g (one third of the probability of
  N_s, Sec. "Generating Valid Topologies") while fewer than ``ground_max``
  ground joints exist and the joint is not the last one; otherwise N_s, a new
  simple joint linked to two distinct existing joints that are not both fixed.
  The joint count is uniform on [n_lo, n_hi].  Positions are uniform in
  [0,1]^2, drawn in float64 and rounded once to float32; both the CUDA path and
  the oracle consume the rounded values.
* ``perturb_curves``: query curves = stored curves + N(0, sigma^2) per
  coordinate (Box-Muller from the same generator).
* ``fourier_curves``: closed curves from a random Fourier series of 4 harmonics
  (coefficient h uniform on [-1, 1] / h^1.5 per coordinate), a database of path
  shapes of any size drawn without simulating anything.
* ``poisson_requests``: request arrival times with exponential gaps and
  candidate counts log-uniform on [1, c_max].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

FIXED, SIMPLE, MOTOR, PAD = 0, 1, 2, -1


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-addressed splitmix64 stream: draw ``i`` is a pure function of (seed, tag, i)."""

    def __init__(self, seed: int, tag: int):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        t = np.array([tag & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        self.key = _mix(_mix(s + _GAMMA) ^ (t * _STREAM_MUL))[0]

    def u64(self, idx) -> np.ndarray:
        idx = np.asarray(idx, dtype=np.uint64)
        return _mix(self.key + (idx + np.uint64(1)) * _GAMMA)

    def uniform(self, idx) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# Stream tags (one per purpose, so that changing one recipe leaves the others alone).
_T_NJ, _T_GROUND, _T_PAIR, _T_POS, _T_PERM, _T_NOISE, _T_ARRIVE, _T_COUNT, _T_SHAPE = range(1, 10)


@dataclass
class MechBatch:
    """B mechanisms padded to ``nmax`` joints (the paper's representation)."""

    n_joints: np.ndarray  # int32 [B]
    adj: np.ndarray       # uint8 [B, nmax, nmax], symmetric, zero diagonal, zero padding
    jtype: np.ndarray     # int8  [B, nmax]; 0 fixed, 1 simple, 2 actuated, -1 padding
    pos: np.ndarray       # float32 or float64 [B, nmax, 2]; zero padding

    @property
    def B(self) -> int:
        return int(self.n_joints.shape[0])

    @property
    def nmax(self) -> int:
        return int(self.adj.shape[1])

    def slice(self, lo: int, hi: int) -> "MechBatch":
        return MechBatch(self.n_joints[lo:hi], self.adj[lo:hi], self.jtype[lo:hi], self.pos[lo:hi])

    def take(self, idx) -> "MechBatch":
        idx = np.asarray(idx)
        return MechBatch(self.n_joints[idx], self.adj[idx], self.jtype[idx], self.pos[idx])

    def masks(self, chunk: int = 1 << 18) -> np.ndarray:
        """The adjacency as neighbour bit masks, uint32 [B, nmax]: bit c of row a set
        when adj[a, c] is nonzero (the input of links_plan_build_masks)."""
        B, n = self.B, self.nmax
        out = np.zeros((B, n), dtype=np.uint32)
        for lo in range(0, B, chunk):
            bits = np.packbits(self.adj[lo:lo + chunk] != 0, axis=-1, bitorder="little")  # [b, n, ceil(n/8)]
            words = np.zeros(bits.shape[:2] + (4,), dtype=np.uint8)
            words[..., :bits.shape[-1]] = bits
            out[lo:lo + chunk] = words.view("<u4")[..., 0]
        return out


def _positions(st: Stream, B: int, nmax: int, n_joints: np.ndarray, dtype) -> np.ndarray:
    b = np.arange(B, dtype=np.uint64)[:, None, None]
    j = np.arange(nmax, dtype=np.uint64)[None, :, None]
    c = np.arange(2, dtype=np.uint64)[None, None, :]
    u = st.uniform(b * np.uint64(2 * 64) + j * np.uint64(2) + c)
    u[np.arange(nmax)[None, :] >= n_joints[:, None]] = 0.0
    return u.astype(dtype)


def fourbar_batch(B: int, seed: int = 0, pos_dtype=np.float64) -> MechBatch:
    """Random four-bar linkages with a coupler point (5 joints); see the module docstring."""
    nmax = 5
    n = np.full(B, 5, dtype=np.int32)
    adj = np.zeros((B, nmax, nmax), dtype=np.uint8)
    for a, c in ((0, 1), (1, 3), (2, 3), (1, 4), (3, 4)):
        adj[:, a, c] = 1
        adj[:, c, a] = 1
    jt = np.tile(np.array([FIXED, MOTOR, FIXED, SIMPLE, SIMPLE], dtype=np.int8), (B, 1))
    pos = _positions(Stream(seed, _T_POS + 100), B, nmax, n, pos_dtype)
    return MechBatch(n, adj, jt, pos)


def dyad_batch(B: int, n_lo: int, n_hi: int, seed: int = 0, *, ground_max: int = 3,
               p_ground: float = 0.25, nmax: int | None = None, permute: bool = False,
               pos_dtype=np.float32, tag: int = 0) -> MechBatch:
    """Candidates built by sequential dyad addition from the paper's initial mechanism.

    ``permute`` relabels the joints of each candidate by a random permutation (the
    representation then no longer lists joints in solve order).  ``tag`` separates
    independent workloads drawn with the same seed.
    """
    if not (3 <= n_lo <= n_hi):
        raise ValueError("need 3 <= n_lo <= n_hi")
    nmax = n_hi if nmax is None else nmax
    if nmax < n_hi or nmax > 64:
        raise ValueError("nmax must be in [n_hi, 64]")
    base = tag * 1000
    st_n, st_g = Stream(seed, base + _T_NJ), Stream(seed, base + _T_GROUND)
    st_p, st_pos = Stream(seed, base + _T_PAIR), Stream(seed, base + _T_POS)
    bidx = np.arange(B, dtype=np.uint64)
    span = n_hi - n_lo + 1
    n = (n_lo + np.floor(st_n.uniform(bidx) * span)).astype(np.int32)
    n = np.minimum(n, n_hi)

    jt = np.full((B, nmax), PAD, dtype=np.int8)
    jt[:, 0], jt[:, 1], jt[:, 2] = FIXED, MOTOR, FIXED
    isfix = np.zeros((B, nmax), dtype=bool)
    isfix[:, 0] = isfix[:, 2] = True
    adj = np.zeros((B, nmax, nmax), dtype=np.uint8)
    adj[:, 0, 1] = adj[:, 1, 0] = 1
    nfix = np.full(B, 2, dtype=np.int32)
    max_attempts = 64
    flat = adj.reshape(-1)
    for k in range(3, n_hi):
        live = np.nonzero(k < n)[0]
        if live.size == 0:
            break
        ul = live.astype(np.uint64)
        ug = st_g.uniform(ul * np.uint64(64) + np.uint64(k))
        ground = (k < n[live] - 1) & (nfix[live] < ground_max) & (ug < p_ground)
        g_idx, s_idx = live[ground], live[~ground]
        jt[g_idx, k] = FIXED
        isfix[g_idx, k] = True
        nfix[g_idx] += 1
        jt[s_idx, k] = SIMPLE
        pi = np.zeros(s_idx.size, dtype=np.int64)
        pj = np.zeros(s_idx.size, dtype=np.int64)
        todo = np.arange(s_idx.size)
        for att in range(max_attempts):
            if todo.size == 0:
                break
            rows_t = s_idx[todo]
            ctr = (rows_t.astype(np.uint64) * np.uint64(64) + np.uint64(k)) * np.uint64(2 * max_attempts) \
                + np.uint64(2 * att)
            i = np.minimum(np.floor(st_p.uniform(ctr) * k).astype(np.int64), k - 1)
            j = np.minimum(np.floor(st_p.uniform(ctr + np.uint64(1)) * (k - 1)).astype(np.int64), k - 2)
            j = j + (j >= i)
            ok = ~(isfix[rows_t, i] & isfix[rows_t, j])
            pi[todo[ok]], pj[todo[ok]] = i[ok], j[ok]
            todo = todo[~ok]
        # Deterministic fallback (probability < 3^-64): link to the actuated joint 1 and joint 0.
        pi[todo], pj[todo] = 0, 1
        rowbase = s_idx.astype(np.int64) * nmax * nmax
        for a, c in ((k, pi), (k, pj)):
            flat[rowbase + a * nmax + c] = 1
            flat[rowbase + c * nmax + a] = 1

    pos = _positions(st_pos, B, nmax, n, np.float64).astype(pos_dtype)
    batch = MechBatch(n, adj, jt, pos)
    if permute:
        batch = _permute(batch, Stream(seed, base + _T_PERM))
    return batch


def topology_rules(batch: MechBatch) -> tuple[np.ndarray, np.ndarray]:
    """The paper's topology rules (Sec. "Dataset Features & Statistics", rules of topology creation)
    for candidates built by ``dyad_batch`` without permutation, where joint k's parents
    are its neighbours of lower index and the last joint is the last one solved:

    * irreducible: the last joint depends, through its parents, on every joint;
    * the last joint is not linked to a fixed joint.

    Returns the two boolean masks [B]."""
    B, nmax = batch.B, batch.nmax
    n = batch.n_joints
    rows = np.arange(B)
    anc = np.zeros((B, nmax), dtype=np.uint64)
    anc[:, 0] = 1
    anc[:, 1] = 3  # the actuated joint turns about joint 0
    lower = np.tril(np.ones((nmax, nmax), dtype=bool), -1)
    for k in range(2, nmax):
        live = k < n
        fixed = batch.jtype[:, k] == FIXED
        par = (batch.adj[:, k, :] != 0) & lower[k][None, :]  # neighbours of lower index
        dep = np.bitwise_or.reduce(np.where(par, anc, np.uint64(0)), axis=1)
        anc[:, k] = np.where(live, np.uint64(1) << np.uint64(k), 0) | np.where(live & ~fixed, dep, 0)
    last = n - 1
    full = (np.uint64(1) << n.astype(np.uint64)) - np.uint64(1)
    irreducible = anc[rows, last] == full
    isfix = batch.jtype == FIXED
    linked = (batch.adj[rows, last, :] != 0) & isfix
    return irreducible, ~linked.any(axis=1)


def paper_topologies(K: int, n: int, seed: int = 0, *, ground_max: int = 3, p_ground: float = 0.25) -> MechBatch:
    """K topologies of n joints from the J operator that meet the paper's topology rules
    (``topology_rules``).  The operator's pairs are drawn with the heuristic the rules
    suggest: the first parent of a new joint is a joint that no joint depends on yet
    (fixed ones first), so that at the end only the last joint is left without
    dependants; candidates that still break a rule are drawn again."""
    if n < 5:
        raise ValueError("need n >= 5 for a topology with a free final joint")
    st = Stream(seed, 700 + _T_PAIR)
    adj = np.zeros((K, n, n), dtype=np.uint8)
    jt = np.full((K, n), PAD, dtype=np.int8)
    for t in range(K):
        for attempt in range(1000):
            u = st.uniform(np.uint64(t) * np.uint64(1 << 20) + np.uint64(attempt) * np.uint64(1 << 10)
                           + np.arange(4 * n, dtype=np.uint64))
            a = np.zeros((n, n), dtype=np.uint8)
            typ = np.full(n, SIMPLE, dtype=np.int8)
            typ[0], typ[1], typ[2] = FIXED, MOTOR, FIXED
            a[0, 1] = a[1, 0] = 1
            sinks = [2, 1]  # joints nothing depends on yet, fixed ones first
            nfix = 2
            for k in range(3, n):
                r = u[4 * k: 4 * k + 4]
                if k < n - 2 and nfix < ground_max and r[0] < p_ground:
                    typ[k] = FIXED
                    nfix += 1
                    sinks.insert(0, k)
                    continue
                i = sinks[0]
                cand = [c for c in range(k) if c != i and not (typ[c] == FIXED and typ[i] == FIXED)]
                if k == n - 1:  # the last joint: no fixed parent
                    cand = [c for c in cand if typ[c] != FIXED]
                j = cand[min(int(r[1] * len(cand)), len(cand) - 1)] if cand else i
                a[k, i] = a[i, k] = a[k, j] = a[j, k] = 1
                sinks = [c for c in sinks if c not in (i, j)] + [k]
            trial = MechBatch(np.array([n], dtype=np.int32), a[None], typ[None], np.zeros((1, n, 2)))
            irr, free = topology_rules(trial)
            if irr[0] and free[0]:
                adj[t], jt[t] = a, typ
                break
        else:
            raise RuntimeError("no topology met the rules in 1000 draws")
    return MechBatch(np.full(K, n, dtype=np.int32), adj, jt, np.zeros((K, n, 2)))


def paper_batch(n_topologies: int, samples: int, n: int, seed: int = 0) -> MechBatch:
    """The paper's own candidates (Sec. "Dataset Features & Statistics"; Sec. "Finding
    Valid Initial Positions"): ``n_topologies`` topologies of n joints meeting the topology
    rules (``paper_topologies``), each with ``samples`` random initial positions: every
    joint drawn uniformly in the unit square (bounding-box rule), then standardised as
    the paper's invariance rules say -- the mechanism translated so that the actuator's
    ground joint is at (0.5, 0.5), rotated so that the actuator arm points along +x and
    scaled so that it has length 0.05 (actuated joint at (0.55, 0.5)).  A draw whose
    standardised joints leave the unit square is drawn again (up to 16 times; the last
    draw is kept).  The standardisation is a similarity, so it leaves each candidate's
    validity as drawn.  Candidates are topology-major."""
    t = paper_topologies(n_topologies, n, seed)
    rep = np.repeat(np.arange(n_topologies), samples)
    B = rep.size
    out = np.zeros((B, n, 2))
    todo = np.arange(B)
    for attempt in range(16):
        p = _positions(Stream(seed, 900 + _T_POS + 1000 * attempt), B, n, t.n_joints[rep], np.float64)[todo]
        c = p[:, 1] - p[:, 0]
        ln = np.hypot(c[:, 0], c[:, 1])
        ln = np.where(ln > 0, ln, 1.0)
        cs, sn = c[:, 0] / ln, c[:, 1] / ln
        d = p - p[:, :1]
        x = (cs[:, None] * d[..., 0] + sn[:, None] * d[..., 1]) * (0.05 / ln)[:, None]
        y = (-sn[:, None] * d[..., 0] + cs[:, None] * d[..., 1]) * (0.05 / ln)[:, None]
        q = np.stack([0.5 + x, 0.5 + y], -1)
        out[todo] = q
        inside = ((q >= 0) & (q <= 1)).all(axis=(1, 2))
        todo = todo[~inside]
        if todo.size == 0:
            break
    out[:, 0] = (0.5, 0.5)
    out[:, 1] = (0.55, 0.5)
    return MechBatch(t.n_joints[rep].copy(), np.ascontiguousarray(t.adj[rep]), np.ascontiguousarray(t.jtype[rep]),
                     out.astype(np.float32))


def _permute(batch: MechBatch, st: Stream) -> MechBatch:
    B, nmax = batch.B, batch.nmax
    key = st.uniform(np.arange(B, dtype=np.uint64)[:, None] * np.uint64(64)
                     + np.arange(nmax, dtype=np.uint64)[None, :])
    key[np.arange(nmax)[None, :] >= batch.n_joints[:, None]] = 2.0  # padding stays at the end
    perm = np.argsort(key, axis=1, kind="stable")  # new label r holds old joint perm[:, r]
    rows = np.arange(B)[:, None]
    jt = batch.jtype[rows, perm]
    pos = batch.pos[rows, perm]
    adj = batch.adj[rows[:, :, None], perm[:, :, None], perm[:, None, :]]
    return MechBatch(batch.n_joints.copy(), np.ascontiguousarray(adj), np.ascontiguousarray(jt),
                     np.ascontiguousarray(pos))


def perturb_curves(curves: np.ndarray, sigma: float, seed: int = 0, tag: int = 0) -> np.ndarray:
    """curves + N(0, sigma^2) per coordinate (Box-Muller), same shape, float32."""
    st = Stream(seed, tag * 1000 + _T_NOISE)
    size = curves.size
    h = (size + 1) // 2
    idx = np.arange(h, dtype=np.uint64) * np.uint64(2)
    u1 = 1.0 - st.uniform(idx)  # (0, 1]
    u2 = st.uniform(idx + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])[:size]
    return (curves.astype(np.float64) + sigma * z.reshape(curves.shape)).astype(np.float32)


def fourier_curves(M: int, T: int, seed: int = 0, harmonics: int = 4) -> np.ndarray:
    """[M, T, 2] float32 closed curves sampled at T equally spaced parameters."""
    st = Stream(seed, _T_SHAPE)
    H = harmonics
    c = st.uniform(np.arange(M * H * 4, dtype=np.uint64)).reshape(M, H, 4) * 2.0 - 1.0
    c /= (np.arange(1, H + 1, dtype=np.float64) ** 1.5)[None, :, None]
    ang = 2.0 * np.pi * np.arange(T, dtype=np.float64) / T
    hs = np.arange(1, H + 1, dtype=np.float64)[:, None] * ang[None, :]  # [H, T]
    cs, sn = np.cos(hs), np.sin(hs)
    out = np.empty((M, T, 2), np.float32)
    for lo in range(0, M, 65536):
        cc = c[lo:lo + 65536]
        out[lo:lo + 65536, :, 0] = cc[:, :, 0] @ cs + cc[:, :, 1] @ sn
        out[lo:lo + 65536, :, 1] = cc[:, :, 2] @ cs + cc[:, :, 3] @ sn
    return out


def poisson_requests(n_req: int, rate_hz: float, c_max: int, seed: int = 0, tag: int = 0):
    """Arrival times (s, cumulative exponential gaps) and log-uniform counts on [1, c_max]."""
    sa, sc = Stream(seed, tag * 1000 + _T_ARRIVE), Stream(seed, tag * 1000 + _T_COUNT)
    i = np.arange(n_req, dtype=np.uint64)
    gaps = -np.log(1.0 - sa.uniform(i)) / rate_hz
    counts = np.floor(np.exp(sc.uniform(i) * np.log(c_max + 1.0))).astype(np.int64)
    counts = np.clip(counts, 1, c_max)
    return np.cumsum(gaps), counts
