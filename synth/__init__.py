"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *makes inputs*: undirected edge lists, their symmetric CSR
form, and batch updates (edge deletions and insertions).  It holds none of the
method's arithmetic (no degrees, no communities, no modularity), so it can
feed both the CPU oracle and the GPU library without coupling them.

Workload shapes follow the paper's evaluation (Sections 5.1.3 and 5.1.4):
undirected graphs with unit weights, random batch updates made of 80%
insertions between uniformly chosen vertex pairs and 20% deletions of
uniformly chosen existing edges, and temporal streams loaded 90% as a base
graph with the rest replayed as batches.

Every generator takes an explicit integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "EdgeList",
    "sbm",
    "planted_partition",
    "rmat",
    "to_csr",
    "random_batch",
    "BatchStream",
    "temporal_pa_stream",
    "temporal_pa_stream_vec",
    "temporal_edges",
    "window_batch",
    "graph_stats",
    "log_uniform_int",
    "EdgePool",
    "poisson_requests",
    "planted_group_params",
    "planted_group_member",
    "planted_group",
]


@dataclass
class EdgeList:
    """Undirected simple graph: each edge once with u < v, u32 weights."""

    n: int
    u: np.ndarray  # uint32
    v: np.ndarray  # uint32
    w: np.ndarray  # uint32

    @property
    def m(self) -> int:
        return int(self.u.shape[0])


def _dedupe_first(lo: np.ndarray, hi: np.ndarray):
    """Distinct (lo, hi) pairs, kept in order of first appearance."""
    key = (lo.astype(np.uint64) << np.uint64(32)) | hi.astype(np.uint64)
    _, first = np.unique(key, return_index=True)
    first.sort()
    return lo[first], hi[first]


def _distinct_pairs(rng, draw, count: int):
    """Draw `count` distinct undirected pairs (u < v) using draw(k) -> (a, b)."""
    los = np.zeros(0, np.int64)
    his = np.zeros(0, np.int64)
    while los.shape[0] < count:
        need = count - los.shape[0]
        a, b = draw(int(need * 1.1) + 64)
        keep = a != b
        a, b = a[keep], b[keep]
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        los, his = _dedupe_first(np.concatenate([los, lo]), np.concatenate([his, hi]))
    return los[:count], his[:count]


def sbm(n: int, blocks: int, p_in: float, p_out: float, seed: int) -> EdgeList:
    """Stochastic block model with equal blocks; each pair is an edge with
    probability p_in (same block) or p_out (different blocks); unit weights.

    The edge counts are drawn as binomials over the pair counts and the
    pairs as distinct uniform samples, which is the same distribution as
    independent Bernoulli trials per pair."""
    rng = np.random.default_rng(seed)
    s = n // blocks
    assert s * blocks == n, "blocks must divide n"
    pairs_in = blocks * (s * (s - 1) // 2)
    pairs_all = n * (n - 1) // 2
    k_in = int(rng.binomial(pairs_in, p_in))
    k_out = int(rng.binomial(pairs_all - pairs_in, p_out))

    def draw_in(k):
        blk = rng.integers(0, blocks, k)
        return blk * s + rng.integers(0, s, k), blk * s + rng.integers(0, s, k)

    def draw_out(k):
        a = rng.integers(0, n, k)
        b = rng.integers(0, n, k)
        same = (a // s) == (b // s)
        b[same] = a[same]  # rejected as a == b below
        return a, b

    lo1, hi1 = _distinct_pairs(rng, draw_in, k_in)
    lo2, hi2 = _distinct_pairs(rng, draw_out, k_out)
    u = np.concatenate([lo1, lo2]).astype(np.uint32)
    v = np.concatenate([hi1, hi2]).astype(np.uint32)
    return EdgeList(n, u, v, np.ones(u.shape[0], np.uint32))


def planted_partition(n: int, blocks: int, mu: float, mean_degree: float,
                      w_max: int, seed: int) -> EdgeList:
    """Planted partition with mixing mu: a fraction mu of each vertex's
    expected degree leaves its block.  Equal blocks (the last ones absorb the
    remainder), weights uniform in 1..w_max."""
    rng = np.random.default_rng(seed)
    base = n // blocks
    sizes = np.full(blocks, base, np.int64)
    sizes[: n - base * blocks] += 1
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    block_of = np.repeat(np.arange(blocks), sizes)
    k_in = int(round(n * (1.0 - mu) * mean_degree / 2.0))
    k_out = int(round(n * mu * mean_degree / 2.0))
    # intra pairs: pick a block with probability proportional to its pair count
    pair_w = (sizes * (sizes - 1)).astype(np.float64)
    pair_w /= pair_w.sum()

    def draw_in(k):
        blk = rng.choice(blocks, size=k, p=pair_w)
        return (starts[blk] + rng.integers(0, sizes[blk]),
                starts[blk] + rng.integers(0, sizes[blk]))

    def draw_out(k):
        a = rng.integers(0, n, k)
        b = rng.integers(0, n, k)
        same = block_of[a] == block_of[b]
        b[same] = a[same]
        return a, b

    lo1, hi1 = _distinct_pairs(rng, draw_in, k_in)
    lo2, hi2 = _distinct_pairs(rng, draw_out, k_out)
    u = np.concatenate([lo1, lo2]).astype(np.uint32)
    v = np.concatenate([hi1, hi2]).astype(np.uint32)
    w = rng.integers(1, w_max + 1, u.shape[0]).astype(np.uint32)
    return EdgeList(n, u, v, w)


def rmat(scale: int, n_edges: int, seed: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, chunk: int = 1 << 23) -> EdgeList:
    """R-MAT graph on 2**scale vertices: recursive quadrant choice with
    probabilities (a, b, c, 1-a-b-c), no noise, then a seeded random vertex
    permutation.  Self-loops are dropped and the undirected pair (min, max)
    deduplicated; draws continue until n_edges distinct edges exist, and the
    first n_edges in order of first appearance are kept.  Unit weights."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    perm = rng.permutation(n).astype(np.int64)
    keys = np.zeros(0, np.uint64)
    ab, abc = a + b, a + b + c
    while keys.shape[0] < n_edges:
        want = int((n_edges - keys.shape[0]) * 1.25) + 1024
        parts = []
        for off in range(0, want, chunk):
            k = min(chunk, want - off)
            u = np.zeros(k, np.int64)
            v = np.zeros(k, np.int64)
            for _ in range(scale):
                r = rng.random(k)
                ubit = r >= ab
                vbit = ((r >= a) & (r < ab)) | (r >= abc)
                u = (u << 1) | ubit
                v = (v << 1) | vbit
            u = perm[u]
            v = perm[v]
            keep = u != v
            u, v = u[keep], v[keep]
            lo, hi = np.minimum(u, v), np.maximum(u, v)
            parts.append((lo.astype(np.uint64) << np.uint64(32)) | hi.astype(np.uint64))
        allk = np.concatenate([keys] + parts)
        _, first = np.unique(allk, return_index=True)
        first.sort()
        keys = allk[first]
    keys = keys[:n_edges]
    u = (keys >> np.uint64(32)).astype(np.uint32)
    v = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return EdgeList(n, u, v, np.ones(u.shape[0], np.uint32))


def to_csr(g: EdgeList):
    """Symmetric CSR (both arcs of every edge), rows sorted by neighbour.

    Returns (offsets uint64[n+1], indices uint32[2m], weights uint32[2m])."""
    src = np.concatenate([g.u, g.v]).astype(np.uint64)
    dst = np.concatenate([g.v, g.u]).astype(np.uint64)
    w = np.concatenate([g.w, g.w])
    key = (src << np.uint64(32)) | dst
    uniform = w.size == 0 or bool(np.all(w == w[0]))
    if uniform:
        key.sort()
        ws = np.full(key.shape[0], w[0] if w.size else 1, np.uint32)
    else:
        order = np.argsort(key, kind="stable")
        key = key[order]
        ws = w[order]
    rows = (key >> np.uint64(32)).astype(np.int64)
    idx = (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    counts = np.bincount(rows, minlength=g.n)
    off = np.zeros(g.n + 1, np.uint64)
    np.cumsum(counts, out=off[1:])
    return off, idx, ws.astype(np.uint32)


def random_batch(n: int, edges: EdgeList, n_ins: int, n_del: int, seed: int):
    """One random batch update: n_ins insertions between uniformly chosen
    vertex pairs (i != j, weight 1) and n_del deletions of distinct existing
    edges chosen uniformly (weight 0 = remove the whole edge).

    Returns (dels uint32[n_del, 3], ins uint32[n_ins, 3]) with rows (u, v, w)."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(edges.m, size=n_del, replace=False) if n_del else np.zeros(0, np.int64)
    dels = np.stack([edges.u[pick], edges.v[pick], np.zeros(n_del, np.uint32)], 1)
    a = rng.integers(0, n, n_ins)
    b = rng.integers(0, n - 1, n_ins)
    b = b + (b >= a)  # uniform over j != i
    ins = np.stack([a, b, np.ones(n_ins, np.int64)], 1)
    return dels.astype(np.uint32).reshape(-1, 3), ins.astype(np.uint32).reshape(-1, 3)


class BatchStream:
    """Consecutive random batch updates on an evolving graph.

    Deletions draw base-graph edges without replacement across the whole
    stream, so each one still exists when its batch arrives; insertions are
    uniform vertex pairs (an insertion of an existing edge adds weight)."""

    def __init__(self, edges: EdgeList, seed: int):
        self.n = edges.n
        self.edges = edges
        self.rng = np.random.default_rng(seed)
        self.order = self.rng.permutation(edges.m)
        self.pos = 0

    def next(self, size: int, frac_ins: float = 0.8, w_max: int = 1):
        """Insertion weights are 1, or uniform in 1..w_max when w_max > 1."""
        n_ins = int(round(size * frac_ins))
        n_del = size - n_ins
        if self.pos + n_del > self.order.shape[0]:
            raise ValueError("stream ran out of base edges to delete")
        pick = self.order[self.pos:self.pos + n_del]
        self.pos += n_del
        dels = np.stack([self.edges.u[pick], self.edges.v[pick],
                         np.zeros(n_del, np.uint32)], 1).astype(np.uint32)
        a = self.rng.integers(0, self.n, n_ins)
        b = self.rng.integers(0, self.n - 1, n_ins)
        b = b + (b >= a)
        w = self.rng.integers(1, w_max + 1, n_ins) if w_max > 1 else np.ones(n_ins, np.int64)
        ins = np.stack([a, b, w], 1).astype(np.uint32)
        return dels.reshape(-1, 3), ins.reshape(-1, 3)


def temporal_pa_stream(n: int, steps: int, p_repeat: float, seed: int):
    """Temporal preferential-attachment interaction stream.

    Vertex k arrives at step k * (steps // n).  At each step, with
    probability p_repeat an earlier interaction (chosen uniformly) repeats;
    otherwise a source (the newest vertex on its arrival step, else a
    uniformly chosen arrived vertex) connects to a target chosen with
    probability proportional to (degree + 1) among arrived vertices; self
    pairs are redrawn.  Returns (src, dst) uint32 arrays of length `steps`,
    in time order.  Degree-proportional choice uses the classic urn: a list
    holding each vertex once plus once per incident interaction."""
    rng = np.random.default_rng(seed)
    gap = max(1, steps // n)
    src = np.zeros(steps, np.uint32)
    dst = np.zeros(steps, np.uint32)
    # urn capacity: one slot per vertex + two per interaction
    urn = np.zeros(n + 2 * steps, np.uint32)
    urn_len = 0
    arrived = 0
    # pre-draw the random numbers in blocks to keep the Python loop cheap
    block = 1 << 16
    t = 0
    while t < steps:
        k = min(block, steps - t)
        r_rep = rng.random(k)
        r_a = rng.random(k)
        r_b = rng.random(k)
        r_c = rng.random(k)
        for q in range(k):
            step = t + q
            newest = -1
            while arrived < n and arrived * gap <= step:
                urn[urn_len] = arrived
                urn_len += 1
                newest = arrived
                arrived += 1
            if arrived < 2:
                # not enough vertices yet: pair the first two (forced arrival)
                while arrived < 2:
                    urn[urn_len] = arrived
                    urn_len += 1
                    arrived += 1
            if step > 0 and r_rep[q] < p_repeat:
                e = int(r_a[q] * step)
                s, d = src[e], dst[e]
            else:
                s = newest if newest >= 0 else int(r_a[q] * arrived)
                d = int(urn[int(r_b[q] * urn_len)])
                tries = 0
                while d == s:
                    tries += 1
                    x = (r_c[q] * 7919.0 * tries) % 1.0
                    d = int(urn[int(x * urn_len)])
                    if tries > 64:
                        d = (s + 1) % arrived
                        break
            src[step], dst[step] = s, d
            urn[urn_len] = s
            urn[urn_len + 1] = d
            urn_len += 2
        t += k
    return src, dst


def _temporal_draws(n: int, steps: int, p_repeat: float, seed: int, vertex_weight: int | None):
    """The random choices of temporal_pa_stream_vec, one entry per step:
    (direct source, repeat flag, repeated step, urn position of the target,
    vertices arrived, vertex weight in the urn)."""
    rng = np.random.default_rng(seed)
    T = int(steps)
    gap = max(1, T // n)
    delta = int(vertex_weight) if vertex_weight else max(1, (2 * T) // n)
    t = np.arange(T, dtype=np.int64)
    arrived = np.minimum(n, t // gap + 2)
    newest = t // gap + 1                      # vertex arriving at step t (if any)
    is_arrival = (t % gap == 0) & (newest < n)
    src_direct = np.where(is_arrival, newest, (rng.random(T) * arrived).astype(np.int64))
    repeat = (rng.random(T) < p_repeat) & ~is_arrival & (t > 0)
    s_rep = (rng.random(T) * t).astype(np.int64)          # earlier step repeated (t >= 1)
    r = (rng.random(T) * (delta * arrived + 2 * t)).astype(np.int64)  # urn position of the target
    return src_direct, repeat, s_rep, r, arrived, delta


def temporal_pa_stream_vec(n: int, steps: int, p_repeat: float, seed: int, vertex_weight: int | None = None):
    """Temporal preferential-attachment interaction stream for large sizes
    (tens of millions of steps), generated with array operations.

    Vertices 0 and 1 arrive at step 0 and vertex k >= 2 at step
    (k - 1) * gap, gap = max(1, steps // n).  At each step t:
      - on vertex k's arrival step the newcomer k is the source and draws a
        target; at t = 0 the source is vertex 1;
      - otherwise, with probability p_repeat, an earlier interaction chosen
        uniformly among steps [0, t) repeats (its source and target);
      - otherwise a uniformly chosen arrived vertex is the source and draws
        a target.
    A target is drawn uniformly from the urn holding each arrived vertex
    `vertex_weight` times (default: the mean number of interactions per
    vertex, 2 * steps / n) plus both endpoints of every earlier step, i.e.
    with probability proportional to (interactions so far + vertex_weight).
    With weight 1 and arrivals rare against interactions the urn condenses:
    the first vertices end up holding a fixed fraction of all interactions;
    a weight near the mean degree gives a heavy tail instead (largest
    degree about 32,000 interactions at 2 million vertices and 30 million
    steps).  An urn entry that is the endpoint of an earlier step is a
    pointer to that step's value; pointers always lead to earlier steps, so
    all values are resolved by pointer jumping.  A draw that lands on the
    source itself yields a self pair, which the stream keeps and the graph
    builders drop.  Returns (src, dst) uint32 arrays of length `steps`, in
    time order."""
    T = int(steps)
    src_direct, repeat, s_rep, r, arrived, delta = _temporal_draws(n, T, p_repeat, seed, vertex_weight)
    # slots 2t (source of step t) and 2t + 1 (target): a direct vertex id
    # (ptr < 0) or a pointer to an earlier slot
    ptr = np.full(2 * T, -1, np.int64)
    val = np.zeros(2 * T, np.int64)
    val[0::2] = src_direct
    ptr[0::2] = np.where(repeat, 2 * s_rep, -1)
    on_vertex = r < delta * arrived
    ptr[1::2] = np.where(repeat, 2 * s_rep + 1, np.where(on_vertex, -1, r - delta * arrived))
    val[1::2] = np.where(on_vertex, r // delta, 0)
    del src_direct, repeat, s_rep, r, arrived, on_vertex
    todo = np.flatnonzero(ptr >= 0)
    while todo.size:
        p = ptr[todo]
        pp = ptr[p]                            # read before this round's writes
        ready = pp < 0
        done_idx = todo[ready]
        val[done_idx] = val[p[ready]]
        ptr[done_idx] = -1
        wait = todo[~ready]
        ptr[wait] = pp[~ready]                 # jump
        todo = wait
    return val[0::2].astype(np.uint32), val[1::2].astype(np.uint32)


def temporal_edges(src: np.ndarray, dst: np.ndarray, n: int) -> EdgeList:
    """Collapse a temporal interaction list into an undirected weighted graph
    (weight = multiplicity of the pair); self pairs are dropped."""
    keep = src != dst
    src, dst = src[keep], dst[keep]
    lo = np.minimum(src, dst).astype(np.uint64)
    hi = np.maximum(src, dst).astype(np.uint64)
    key = (lo << np.uint64(32)) | hi
    uk, cnt = np.unique(key, return_counts=True)
    u = (uk >> np.uint64(32)).astype(np.uint32)
    v = (uk & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return EdgeList(n, u, v, cnt.astype(np.uint32))


def window_batch(src: np.ndarray, dst: np.ndarray, start: int, end: int, size: int):
    """One sliding-window batch of a temporal stream whose window holds
    interactions [start, end): insert interactions [end, end + size) with
    weight 1 each, expire the `size` oldest, [start, start + size), as
    deletions of one unit per interaction grouped by pair.  Self pairs are
    dropped on both sides.  Returns (deletions, insertions) as (k, 3) uint32
    arrays of (u, v, w)."""
    ins = np.stack([src[end:end + size], dst[end:end + size], np.ones(size, np.uint32)], 1)
    ins = ins[ins[:, 0] != ins[:, 1]]
    s, d = src[start:start + size], dst[start:start + size]
    keep = s != d
    lo, hi = np.minimum(s[keep], d[keep]), np.maximum(s[keep], d[keep])
    key, cnt = np.unique((lo.astype(np.uint64) << np.uint64(32)) | hi, return_counts=True)
    dels = np.stack([(key >> np.uint64(32)).astype(np.uint32), (key & np.uint64(0xFFFFFFFF)).astype(np.uint32),
                     cnt.astype(np.uint32)], 1)
    return dels, ins


def graph_stats(g: EdgeList) -> dict:
    deg = np.bincount(np.concatenate([g.u, g.v]).astype(np.int64), minlength=g.n)
    return {"n": g.n, "m": g.m, "max_deg": int(deg.max()) if g.n else 0,
            "mean_deg": float(2 * g.m / g.n) if g.n else 0.0,
            "isolated": int((deg == 0).sum())}


def log_uniform_int(rng, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


class EdgePool:
    """The edges a graph holds as a request stream evolves it, as unit-weight
    entries: each base edge and each inserted edge is one entry (a pair
    inserted twice has two).  A deletion removes a uniformly chosen entry and
    one unit of weight, so every generated deletion is valid; two entries of
    the same pair drawn for one batch become one deletion of weight 2.
    Insertions join uniform vertex pairs with weight 1."""

    def __init__(self, edges: EdgeList, seed: int):
        self.n = edges.n
        self.rng = np.random.default_rng(seed)
        cap = max(1024, edges.m * 2)
        self.u = np.zeros(cap, np.int64)
        self.v = np.zeros(cap, np.int64)
        self.u[:edges.m] = edges.u
        self.v[:edges.m] = edges.v
        self.size = edges.m

    def _grow(self, extra):
        if self.size + extra > self.u.shape[0]:
            cap = max(self.u.shape[0] * 2, self.size + extra)
            self.u = np.resize(self.u, cap)
            self.v = np.resize(self.v, cap)

    def next(self, size: int, frac_ins: float = 0.8):
        n_ins = int(round(size * frac_ins))
        n_del = min(size - n_ins, self.size)
        idx = np.unique(self.rng.integers(0, self.size, n_del)) if n_del else np.zeros(0, np.int64)
        lo = np.minimum(self.u[idx], self.v[idx])
        hi = np.maximum(self.u[idx], self.v[idx])
        key, cnt = np.unique((lo << 32) | hi, return_counts=True)
        dels = np.stack([key >> 32, key & 0xFFFFFFFF, cnt], 1).astype(np.uint32)
        # remove the drawn entries: the surviving entries of the last len(idx)
        # slots move into the holes below the new end
        k = idx.shape[0]
        end = self.size - k
        holes = idx[idx < end]
        tail = np.arange(end, self.size)
        keep = tail[~np.isin(tail, idx, assume_unique=True)]
        self.u[holes] = self.u[keep]
        self.v[holes] = self.v[keep]
        self.size = end
        a = self.rng.integers(0, self.n, n_ins)
        b = self.rng.integers(0, self.n - 1, n_ins)
        b = b + (b >= a)
        self._grow(n_ins)
        self.u[self.size:self.size + n_ins] = a
        self.v[self.size:self.size + n_ins] = b
        self.size += n_ins
        ins = np.stack([a, b, np.ones(n_ins, np.int64)], 1).astype(np.uint32)
        return dels.reshape(-1, 3), ins.reshape(-1, 3)


def poisson_requests(num_graphs: int, rate: float, duration: float, size_lo: int, size_hi: int,
                     seed: int):
    """Arrival times (seconds) of a Poisson stream of `rate` requests per
    second over `duration`, each for a uniformly chosen graph, with a batch
    size log-uniform in [size_lo, size_hi] edges."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        g = int(rng.integers(0, num_graphs))
        size = int(round(math.exp(rng.uniform(math.log(size_lo), math.log(size_hi)))))
        out.append((t, g, size))
    return out


def planted_group_params(count: int, n_lo: float, n_hi: float, seed: int):
    """Per graph (n, blocks, mu, seed) of `planted_group`, drawn in order:
    n log-uniform in [n_lo, n_hi], blocks log-uniform in [20, 2000] (at most
    n / 32, so blocks keep room for their internal edges), mu uniform in
    [0.1, 0.5]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = log_uniform_int(rng, n_lo, n_hi)
        blocks = max(2, min(log_uniform_int(rng, 20, 2000), n // 32))
        mu = float(rng.uniform(0.1, 0.5))
        out.append((n, blocks, mu, int(rng.integers(1 << 31))))
    return out


def planted_group_member(k: int, count: int, n_lo: float, n_hi: float, seed: int, mean_degree: float = 16.0,
                         w_max: int = 16):
    """Graph k of `planted_group(count, n_lo, n_hi, seed)` alone, with its
    CSR: (EdgeList, (n, offsets, indices, weights)).  A module-level function,
    so that worker processes can build the graphs of a group in parallel."""
    n, blocks, mu, gseed = planted_group_params(count, n_lo, n_hi, seed)[k]
    g = planted_partition(n, blocks, mu, mean_degree, w_max, gseed)
    return g, (g.n, *to_csr(g))


def planted_group(count: int, n_lo: float, n_hi: float, seed: int, mean_degree: float = 16.0,
                  w_max: int = 16):
    """Independent planted-partition graphs of uneven size (parameters from
    `planted_group_params`), weights uniform in 1..w_max.  Returns a list of
    (EdgeList, {"n", "blocks", "mu"})."""
    out = []
    for n, blocks, mu, gseed in planted_group_params(count, n_lo, n_hi, seed):
        g = planted_partition(n, blocks, mu, mean_degree, w_max, gseed)
        out.append((g, {"n": n, "blocks": blocks, "mu": round(mu, 4)}))
    return out
