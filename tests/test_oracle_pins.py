"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: Newman's
all-pairs modularity in exact rationals, brute-force re-evaluation of every
candidate move, recomputation from scratch, closed forms and special cases.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from tests.exact import dense_matrix, edges_of, move, newman_q, random_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make(oracle_mod, n, off, idx, w, loops=False):
    return oracle_mod.Oracle(n, off, idx, w, allow_self_loops=loops)


def q_fraction(o):
    q, num, den = o.modularity()
    return q, Fraction(num, den) if den else Fraction(0)


# ---------------------------------------------------------------------------
# Eq. 1 -- modularity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_modularity_equals_newman_all_pairs(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 12))
    off, idx, w = random_graph(rng, n, 0.45, wmax=5)
    if len(idx) == 0:
        pytest.skip("empty graph")
    o = make(oracle_mod, n, off, idx, w)
    A = dense_matrix(n, off, idx, w)
    for _ in range(4):
        C = rng.integers(0, n, n).astype(np.uint32)
        o.set_membership(C)
        q, qf = q_fraction(o)
        assert qf == newman_q(A, list(C))
        assert abs(q - float(qf)) <= 1e-15
        assert Fraction(-1, 2) <= qf <= 1  # range stated in Section 3.2


def test_modularity_special_cases(oracle_mod):
    # one community: Q = 0
    rng = np.random.default_rng(5)
    off, idx, w = random_graph(rng, 9, 0.5, wmax=3)
    o = make(oracle_mod, 9, off, idx, w)
    o.set_membership(np.zeros(9, np.uint32))
    assert q_fraction(o)[1] == 0
    # singletons on a simple graph: Q = -sum K_i^2 / (2m)^2
    o.set_membership(np.arange(9, dtype=np.uint32))
    K, _, m2 = o.weights()
    assert q_fraction(o)[1] == -Fraction(int((K.astype(object) ** 2).sum()), m2 * m2)
    # two disjoint equal cliques, each its own community: Q = 1/2
    edges = [(a, b, 1) for a, b in itertools.combinations(range(4), 2)]
    edges += [(a + 4, b + 4, 1) for a, b in itertools.combinations(range(4), 2)]
    g = synth.EdgeList(8, np.array([e[0] for e in edges], np.uint32),
                       np.array([e[1] for e in edges], np.uint32), np.ones(len(edges), np.uint32))
    off, idx, w = synth.to_csr(g)
    o = make(oracle_mod, 8, off, idx, w)
    o.set_membership(np.array([0, 0, 0, 0, 4, 4, 4, 4], np.uint32))
    assert q_fraction(o)[1] == Fraction(1, 2)


# ---------------------------------------------------------------------------
# Eq. 2 -- delta-modularity equals the recomputed difference of Eq. 1
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("loops", [False, True])
def test_delta_modularity_matches_q_difference(oracle_mod, seed, loops):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 10))
    off, idx, w = random_graph(rng, n, 0.5, wmax=4, self_loops=loops)
    if len(idx) == 0:
        pytest.skip("empty graph")
    o = make(oracle_mod, n, off, idx, w, loops)
    A = dense_matrix(n, off, idx, w)
    C = list(rng.integers(0, n, n))
    o.set_membership(np.array(C, np.uint32))
    _, _, m2 = o.weights()
    q0 = newman_q(A, C)
    for i in range(n):
        for c in range(n):
            if c == C[i]:
                continue
            num = o.delta_q_num(i, c)  # 2m^2 * dQ = (m2^2 / 2) * dQ
            assert Fraction(2 * num, m2 * m2) == newman_q(A, move(C, i, c)) - q0


# The appendix's correctness argument lists how one vertex migration i: d -> c
# changes every other vertex v's delta-modularity (its cases 17-28; nothing
# else changes: K and m stay, Sigma_d loses K_i and Sigma_c gains it).  In
# numerator units N = 2m^2 dQ, with m2 = 2m, w = w_iv and the communities
# named by their role (v's own first, then the target):
#   17  d, neighbour, -> c    +2 m2 w - 2 K_i K_v
#   18  d, neighbour, -> b    +m2 w - K_i K_v
#   19  c, neighbour, -> d    -2 m2 w + 2 K_i K_v
#   20  c, neighbour, -> b    -m2 w + K_i K_v
#   21  b, neighbour, -> d    -m2 w + K_i K_v
#   22  b, neighbour, -> c    +m2 w - K_i K_v
#   23  d, non-neighbour, -> c   -2 K_i K_v  (printed with +: case 17 at w = 0
#                                             and Eq. 2 both give -)
#   24  d, non-neighbour, -> b   -K_i K_v
#   25  c, non-neighbour, -> d   +2 K_i K_v
#   26  c, non-neighbour, -> b   +K_i K_v
#   27  b, non-neighbour, -> d   +K_i K_v
#   28  b, non-neighbour, -> c   -K_i K_v
MIGRATION_CASES = {
    ("d", True, "c"): (17, lambda m2, w, ki, kv: 2 * m2 * w - 2 * ki * kv),
    ("d", True, "b"): (18, lambda m2, w, ki, kv: m2 * w - ki * kv),
    ("c", True, "d"): (19, lambda m2, w, ki, kv: -2 * m2 * w + 2 * ki * kv),
    ("c", True, "b"): (20, lambda m2, w, ki, kv: -m2 * w + ki * kv),
    ("b", True, "d"): (21, lambda m2, w, ki, kv: -m2 * w + ki * kv),
    ("b", True, "c"): (22, lambda m2, w, ki, kv: m2 * w - ki * kv),
    ("d", False, "c"): (23, lambda m2, w, ki, kv: -2 * ki * kv),
    ("d", False, "b"): (24, lambda m2, w, ki, kv: -ki * kv),
    ("c", False, "d"): (25, lambda m2, w, ki, kv: 2 * ki * kv),
    ("c", False, "b"): (26, lambda m2, w, ki, kv: ki * kv),
    ("b", False, "d"): (27, lambda m2, w, ki, kv: ki * kv),
    ("b", False, "c"): (28, lambda m2, w, ki, kv: -ki * kv),
}


def test_vertex_migration_changes_neighbour_gains_as_the_appendix_states(oracle_mod):
    """Cases 17-28 of the appendix, exactly: for random weighted graphs and
    memberships, move one vertex i from d to c and compare every other
    vertex's change in 2m^2 dQ with the case it falls in."""
    seen = set()
    for seed in range(12):
        rng = np.random.default_rng(700 + seed)
        n = 24
        off, idx, w = random_graph(rng, n, 0.35, wmax=3)
        A = dense_matrix(n, off, idx, w)
        C = rng.integers(0, 4, n).astype(np.uint32)
        C[:4] = [0, 1, 2, 3]  # every label used
        o = make(oracle_mod, n, off, idx, w)
        o.set_membership(C)
        K, _, m2 = o.weights()
        i = int(rng.integers(4, n))
        d = int(C[i])
        c = int(rng.choice([x for x in range(4) if x != d]))
        before = {(v, y): o.delta_q_num(v, y) for v in range(n) if v != i for y in range(4) if y != C[v]}
        C2 = C.copy()
        C2[i] = c
        o.set_membership(C2)
        assert o.weights()[2] == m2
        for (v, y), n0 in before.items():
            role = lambda x: "d" if x == d else "c" if x == c else "b"
            if role(int(C[v])) == "b" and role(y) == "b":
                assert o.delta_q_num(v, y) == n0  # between two bystander communities: unchanged
                continue
            case, delta = MIGRATION_CASES[(role(int(C[v])), A[i][v] > 0, role(y))]
            assert o.delta_q_num(v, y) - n0 == delta(m2, A[i][v], int(K[i]), int(K[v])), (case, v, y)
            seen.add(case)
    assert seen == set(range(17, 29))


# ---------------------------------------------------------------------------
# Alg. 5 -- local-moving decisions against brute force
# ---------------------------------------------------------------------------

def substep_class(i, k):
    return ((i * 0x9E3779B1) & 0xFFFFFFFF) * k >> 32


def brute_force_iteration(A, C, F, R, k):
    """One local-moving iteration by exhaustive search over neighbour
    communities with exact Q recomputation; same schedule as the oracle."""
    n = len(A)
    C = list(C)
    F = list(F)
    Fnext = [0] * n
    S = Fraction(0)
    m2 = sum(sum(r) for r in A)
    for sub in range(k):
        snap = list(C)
        size = [snap.count(c) for c in range(n)]
        q0 = newman_q(A, snap)
        moves = []
        for i in range(n):
            if not F[i] or substep_class(i, k) != sub:
                continue
            F[i] = 0
            if not R[i]:
                continue
            d = snap[i]
            cands = sorted({snap[j] for j in range(n) if j != i and A[i][j] > 0} - {d})
            best, gain = None, None
            for c in cands:
                g = newman_q(A, move(snap, i, c)) - q0
                if gain is None or g > gain:
                    best, gain = c, g
            if best is None or gain <= 0:
                continue
            if size[d] == 1 and size[best] == 1 and best > d:
                continue
            moves.append((i, best, gain))
        for i, c, g in moves:
            C[i] = c
            S += g
            for j in range(n):
                if j != i and A[i][j] > 0 and R[j]:
                    Fnext[j] = 1
    return C, Fnext, S * m2 * m2 / 2


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("k", [1, 4])
@pytest.mark.parametrize("kind", ["weighted", "unit", "loops"])
def test_move_iteration_matches_brute_force(oracle_mod, seed, k, kind):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(4, 12))
    off, idx, w = random_graph(rng, n, 0.4, wmax=1 if kind == "unit" else 3,
                               self_loops=kind == "loops")
    if len(idx) == 0:
        pytest.skip("empty graph")
    o = make(oracle_mod, n, off, idx, w, kind == "loops")
    o.set_options(substeps=k)
    A = dense_matrix(n, off, idx, w)
    C = list(rng.integers(0, max(2, n // 2), n))
    F = list((rng.random(n) < 0.8).astype(np.uint8))
    R = list((rng.random(n) < 0.85).astype(np.uint8))
    o.set_membership(np.array(C, np.uint32))
    Fo, moved, dq = o.move_iteration(np.array(F, np.uint8), np.array(R, np.uint8))
    Cexp, Fexp, Sexp = brute_force_iteration(A, C, F, R, k)
    assert list(o.membership()) == Cexp
    assert list(Fo) == Fexp
    assert Fraction(dq) == Sexp
    # Sigma after the iteration equals recomputation from the new membership
    K, S, _ = o.weights()
    exp = np.zeros(n, np.int64)
    np.add.at(exp, np.array(Cexp, np.int64), K)
    assert np.array_equal(S, exp)


def test_tie_break_smallest_community(oracle_mod):
    # vertex 0 links equally to communities 3 and 5 of equal totals: it joins 3
    e = [(0, 1), (0, 2), (1, 3), (2, 5), (3, 4), (5, 6)]
    g = synth.EdgeList(7, np.array([a for a, _ in e], np.uint32),
                       np.array([b for _, b in e], np.uint32), np.ones(len(e), np.uint32))
    off, idx, w = synth.to_csr(g)
    o = make(oracle_mod, 7, off, idx, w)
    o.set_options(substeps=1)
    o.set_membership(np.array([0, 5, 3, 3, 3, 5, 5], np.uint32)[[0, 2, 1, 3, 4, 5, 6]])
    C = o.membership()
    assert C[1] != C[2]
    F = np.zeros(7, np.uint8)
    F[0] = 1
    o.move_iteration(F, np.ones(7, np.uint8))
    assert o.membership()[0] == min(C[1], C[2])


def test_singleton_swap_guard(oracle_mod):
    # two singletons joined by a heavy edge would swap forever under plain
    # synchronous moves; the minimum-label guard lets only the larger id move
    g = synth.EdgeList(4, np.array([0, 2], np.uint32), np.array([1, 3], np.uint32),
                       np.array([5, 1], np.uint32))
    off, idx, w = synth.to_csr(g)
    o = make(oracle_mod, 4, off, idx, w)
    o.set_options(substeps=1)
    o.set_membership(np.arange(4, dtype=np.uint32))
    o.move_iteration(np.ones(4, np.uint8), np.ones(4, np.uint8))
    assert list(o.membership()) == [0, 0, 2, 2]


# ---------------------------------------------------------------------------
# Alg. 7 -- incremental K and Sigma equal recomputation from scratch
# ---------------------------------------------------------------------------

def recompute(o):
    off, idx, w = o.graph()
    K = np.add.reduceat(w.astype(np.int64), off[:-1].astype(np.int64)) if len(w) else None
    deg = np.diff(off.astype(np.int64))
    Kr = np.zeros(o.n, np.int64)
    rows = np.repeat(np.arange(o.n), deg)
    np.add.at(Kr, rows, w.astype(np.int64))
    C = o.membership()
    Sr = np.zeros(o.n, np.int64)
    np.add.at(Sr, C.astype(np.int64), Kr)
    return Kr, Sr, int(w.astype(np.int64).sum())


def weighted_batch(rng, o, n_ins, n_del, wmax=3):
    off, idx, w = o.graph()
    edges = edges_of(o.n, off, idx, w)
    pick = rng.choice(len(edges), size=min(n_del, len(edges)), replace=False)
    dels = []
    for p in pick:
        u, v, wt = edges[p]
        mode = rng.integers(0, 3)
        wd = 0 if mode == 0 else int(rng.integers(1, wt + 1))
        dels.append((v, u, wd) if rng.random() < 0.5 else (u, v, wd))
    ins = []
    for _ in range(n_ins):
        a = int(rng.integers(0, o.n))
        b = int(rng.integers(0, o.n - 1))
        b += b >= a
        ins.append((a, b, int(rng.integers(1, wmax + 1))))
    if ins and rng.random() < 0.5:
        ins.append(ins[0])  # the same pair twice: weights add
    return np.array(dels, np.uint32).reshape(-1, 3), np.array(ins, np.uint32).reshape(-1, 3)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_incremental_weights_equal_recomputation(oracle_mod, mode):
    rng = np.random.default_rng(7 + mode)
    g = synth.planted_partition(600, 12, 0.3, 8, 4, 9)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    o.static()
    for _ in range(6):
        d, i = weighted_batch(rng, o, 40, 15)
        assert o.apply_batch(d, i) == 0
        K, S, m2 = o.weights()
        Kr, Sr, m2r = recompute(o)  # against C^{t-1}
        assert np.array_equal(K, Kr) and np.array_equal(S, Sr) and m2 == m2r
        o.update(mode)
        K, S, m2 = o.weights()
        Kr, Sr, m2r = recompute(o)  # against C^t
        assert np.array_equal(K, Kr) and np.array_equal(S, Sr) and m2 == m2r
        assert S.sum() == m2 and K.sum() == m2  # sum Sigma_c = 2m


@pytest.mark.parametrize("seed", range(3))
def test_several_batches_before_one_update(oracle_mod, seed):
    """R19: batches applied one after another before a single update are
    each applied against C^{t-1} and marked together (Alg. 1 over every arc
    of every batch).  When the batches do not touch the same edge, that is
    one batch holding all of them: the same K, Sigma, 2m, initial frontier,
    and the same update result."""
    rng = np.random.default_rng(40 + seed)
    g = synth.planted_partition(800, 16, 0.3, 8, 4, 11 + seed)
    off, idx, w = synth.to_csr(g)
    a = oracle_mod.Oracle(g.n, off, idx, w)
    b = oracle_mod.Oracle(g.n, off, idx, w)
    a.static()
    b.static()
    base = edges_of(g.n, off, idx, w)
    pick = rng.choice(len(base), 60, replace=False)
    dels = [(base[p][0], base[p][1], 0 if k % 3 else int(rng.integers(1, base[p][2] + 1)))
            for k, p in enumerate(pick)]
    gone = {(min(u, v), max(u, v)) for u, v, _ in dels}
    ins = []
    while len(ins) < 90:
        u = int(rng.integers(0, g.n))
        v = int(rng.integers(0, g.n - 1))
        v += v >= u
        if (min(u, v), max(u, v)) not in gone:  # a whole-weight deletion after an insertion
            ins.append((u, v, int(rng.integers(1, 4))))  # would depend on the order
    batches = [(dels[:30], ins[:50]), (dels[30:], ins[50:])]  # no edge deleted twice
    for d, i in batches:
        assert a.apply_batch(np.array(d, np.uint32), np.array(i, np.uint32)) == 0
    assert b.apply_batch(np.array(dels, np.uint32), np.array(ins, np.uint32)) == 0
    for x, y in zip(a.weights(), b.weights()):
        assert np.array_equal(x, y)
    Fa, Ra = a.mark(2)
    Fb, Rb = b.mark(2)
    assert np.array_equal(Fa, Fb) and np.array_equal(Ra, Rb) and Fa.any()
    a.update(2)
    b.update(2)
    assert np.array_equal(a.membership(), b.membership())
    assert a.modularity()[1:] == b.modularity()[1:]
    assert a.stats()["affected_initial"] == int(Fa.sum())


def test_batch_graph_semantics(oracle_mod):
    # deletions first (w = 0 removes the whole edge, w > 0 decrements), then
    # insertions (add weight, or create the edge)
    g = synth.EdgeList(5, np.array([0, 1, 2], np.uint32), np.array([1, 2, 3], np.uint32),
                       np.array([4, 2, 1], np.uint32))
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(5, off, idx, w)
    o.static()
    assert o.apply_batch([(1, 0, 1), (2, 1, 0)], [(2, 1, 3), (3, 4, 2), (4, 3, 1)]) == 0
    off2, idx2, w2 = o.graph()
    got = set(edges_of(5, off2, idx2, w2))
    assert got == {(0, 1, 3), (1, 2, 3), (2, 3, 1), (3, 4, 3)}


def test_batch_errors_leave_state_unchanged(oracle_mod):
    g = synth.sbm(200, 4, 0.2, 0.01, 3)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    with pytest.raises(oracle_mod.OracleError):
        o.update(2)  # before static
    assert o.apply_batch([], [(0, 1, 1)]) == -7
    o.static()
    before = (o.graph(), o.weights(), o.membership())
    u, v = int(g.u[0]), int(g.v[0])
    absent = next((a, b) for a in range(g.n) for b in range(a + 1, g.n)
                  if b not in set(idx[int(off[a]):int(off[a + 1])]))
    cases = [
        ([], [(0, 0, 1)], -1),                       # self-loop
        ([], [(0, g.n, 1)], -1),                     # vertex out of range
        ([], [(0, 1, 0)], -1),                       # zero insertion weight
        ([(u, v, 0), (v, u, 0)], [], -1),            # same edge deleted twice
        ([absent + (0,)], [], -2),                   # absent edge
        ([(u, v, 2)], [], -2),                       # more weight than present
        ([], [(u, v, 0xFFFFFFFF)], -3),              # u32 weight overflow
        ([absent + (0,)], [(0, 0, 1)], -1),          # invalid wins over not-found
    ]
    for d, i, code in cases:
        assert o.apply_batch(np.array(d, np.uint32).reshape(-1, 3),
                             np.array(i, np.uint32).reshape(-1, 3)) == code
        after = (o.graph(), o.weights(), o.membership())
        for x, y in zip(before[0] + before[1][:2] + (before[2],),
                        after[0] + after[1][:2] + (after[2],)):
            assert np.array_equal(x, y)
        assert before[1][2] == after[1][2]


def test_two_m_limit(oracle_mod):
    # 2m (the sum of all arc weights) must stay below 2^32
    g = synth.EdgeList(3, np.array([0], np.uint32), np.array([1], np.uint32),
                       np.array([0x80000000], np.uint32))
    off, idx, w = synth.to_csr(g)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(3, off, idx, w)  # 2m = 2^32
    g.w[:] = 0x7FFFFFFF
    off, idx, w = synth.to_csr(g)
    oracle_mod.Oracle(3, off, idx, w)  # 2m = 2^32 - 2 is accepted
    g.w[:] = 0x3FFFFFFF
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(3, off, idx, w)
    o.static()
    assert o.apply_batch([], [(1, 2, 0x40000001)]) == -3  # 2m would reach 2^32
    assert o.apply_batch([], [(1, 2, 0x40000000)]) == 0   # 2m = 2^32 - 2


# ---------------------------------------------------------------------------
# Alg. 6 -- aggregation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("loops", [False, True])
def test_aggregation_preserves_weight_and_modularity(oracle_mod, seed, loops):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(4, 12))
    off, idx, w = random_graph(rng, n, 0.45, wmax=4, self_loops=loops)
    if len(idx) == 0:
        pytest.skip("empty graph")
    o = make(oracle_mod, n, off, idx, w, loops)
    C = rng.integers(0, n, n).astype(np.uint32)
    o.set_membership(C)
    soff, sidx, sw = o.aggregate()
    nv = len(soff) - 1
    assert nv == len(set(C.tolist()))
    A = dense_matrix(n, off, idx, w)
    S = dense_matrix(nv, soff, sidx, sw)
    assert sum(map(sum, S)) == sum(map(sum, A))  # total weight preserved
    assert all(S[a][b] == S[b][a] for a in range(nv) for b in range(nv))  # symmetric
    # renumbering by ascending old label
    ren = {c: r for r, c in enumerate(sorted(set(C.tolist())))}
    for a in range(nv):
        for b in range(nv):
            exp = sum(A[i][j] for i in range(n) for j in range(n)
                      if ren[int(C[i])] == a and ren[int(C[j])] == b)
            assert S[a][b] == exp
    # Q of the super graph with singletons equals Q of G under C
    assert newman_q(S, list(range(nv))) == newman_q(A, [ren[int(c)] for c in C])


# ---------------------------------------------------------------------------
# Alg. 1-3 -- marking of initially affected vertices
# ---------------------------------------------------------------------------

def four_case_graph(oracle_mod):
    # communities A = {0..3}, B = {4..7}, X = {8, 9, 10}
    e = [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 7), (3, 4), (0, 7), (8, 9), (9, 10)]
    g = synth.EdgeList(11, np.array([a for a, _ in e], np.uint32),
                       np.array([b for _, b in e], np.uint32), np.ones(len(e), np.uint32))
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(11, off, idx, w)
    o.set_membership(np.array([0, 0, 0, 0, 4, 4, 4, 4, 8, 8, 8], np.uint32))
    # deletion inside A, deletion across A-B, insertion across A-B,
    # insertion inside B
    assert o.apply_batch([(0, 1, 0), (3, 4, 0)], [(2, 5, 1), (4, 6, 1)]) == 0
    return o


def test_dynamic_frontier_marking_rules(oracle_mod):
    o = four_case_graph(oracle_mod)
    F, R = o.mark(2)
    assert set(np.flatnonzero(F)) == {0, 1, 2, 5}  # both endpoints, two rules
    assert R.all()


def test_naive_dynamic_marks_everything(oracle_mod):
    o = four_case_graph(oracle_mod)
    F, R = o.mark(0)
    assert F.all() and R.all()


def test_delta_screening_marking(oracle_mod):
    o = four_case_graph(oracle_mod)
    F, R = o.mark(1)
    # intra deletion (0,1) flags community A; insertion (2,5) flags B via the
    # best community of both sources; X stays untouched
    assert set(np.flatnonzero(F)) == set(range(8))
    assert np.array_equal(F, R)


def test_delta_screening_best_community(oracle_mod):
    # source 0 (community 0) gets insertions to communities 5 and 9; the
    # better one by 2m*H[c] - K_0*Sigma_c is the heavier link
    e = [(0, 1), (5, 6), (9, 10), (10, 11), (6, 7), (2, 3)]
    g = synth.EdgeList(12, np.array([a for a, _ in e], np.uint32),
                       np.array([b for _, b in e], np.uint32), np.ones(len(e), np.uint32))
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(12, off, idx, w)
    C = np.array([0, 0, 2, 2, 4, 5, 5, 5, 8, 9, 9, 9], np.uint32)
    o.set_membership(C)
    assert o.apply_batch([], [(0, 5, 1), (0, 9, 3)]) == 0
    F, _ = o.mark(1)
    marked = set(np.flatnonzero(F))
    assert {9, 10, 11}.issubset(marked)        # community of the best link
    assert {0, 1, 5, 6}.issubset(marked)        # sources (both ends) and neighbours
    assert 7 not in marked                      # community 5 itself is not flagged
    assert not {2, 3, 4, 8} & marked


@pytest.mark.parametrize("intra", [1, 6])
def test_delta_screening_choice_is_best_delta_modularity(oracle_mod, intra):
    """When all of a source's cross-community links are the inserted ones,
    H[c] = K_{i->c}, so the DS choice (Alg. 3) must be the neighbour community
    with the largest exact dQ of moving the source (Eq. 2, recomputed from
    Eq. 1).  The source's own degree K_i decides between a small community
    with one new link and a large one with two: intra = 1 picks the large one,
    intra = 6 the small one."""
    e = [(0, 1 + k) for k in range(intra)]               # source 0 and its community
    e += [(10, 11), (11, 12)]                            # community 10: path
    e += [(20 + k, 21 + k) for k in range(7)]            # community 20: path ...
    e += [(a, b) for a in range(23, 28) for b in range(a + 2, 28)]  # ... and chords
    e += [(a, b) for a in range(30, 41) for b in range(a + 1, 41)]  # filler clique
    n = 41
    g = synth.EdgeList(n, np.array([a for a, _ in e], np.uint32),
                       np.array([b for _, b in e], np.uint32), np.ones(len(e), np.uint32))
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(n, off, idx, w)
    C = np.arange(n, dtype=np.uint32)
    C[: intra + 1] = 0
    C[10:13] = 10
    C[20:28] = 20
    C[30:41] = 30
    o.set_membership(C)
    assert o.apply_batch([], [(0, 10, 1), (0, 20, 1), (0, 21, 1)]) == 0
    off2, idx2, w2 = o.graph()
    A = dense_matrix(n, off2, idx2, w2)
    q0 = newman_q(A, list(C))
    gains = {c: newman_q(A, move(list(C), 0, c)) - q0 for c in (10, 20)}
    best = 20 if gains[20] > gains[10] else 10
    assert best == (20 if intra == 1 else 10)  # the case is built to flip
    far = {10: {12}, 20: set(range(23, 28))}   # members no source is adjacent to
    marked = set(np.flatnonzero(o.mark(1)[0]))
    assert far[best] <= marked
    assert not far[30 - best] & marked
    assert not set(range(30, 41)) & marked


def test_figure3_initial_frontier(oracle_mod):
    """Fig. 3 (Section 4.1.1): deletion (1,2) inside the red community and
    insertion (4,12) across red/blue make {1, 2, 4, 12} the initial frontier;
    in the first iteration vertex 2 moves to green, marking 8 and 10."""
    path = os.path.join(GOLDEN, "fig3_frontier.txt")
    rows = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            key, _, val = line.partition(":")
            rows[key.strip()] = [int(x) for x in val.split()]
    n = rows["n"][0]
    ed = np.array(rows["edges"], np.uint32).reshape(-1, 3)
    g = synth.EdgeList(n, ed[:, 0], ed[:, 1], ed[:, 2])
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(n, off, idx, w)
    o.set_membership(np.array(rows["membership"], np.uint32))
    assert o.apply_batch(np.array(rows["delete"], np.uint32).reshape(-1, 3),
                         np.array(rows["insert"], np.uint32).reshape(-1, 3)) == 0
    F, R = o.mark(2)
    assert set(np.flatnonzero(F)) == set(rows["initial_frontier"])
    o.set_options(substeps=1)
    F1, moved, _ = o.move_iteration(F, R)
    v, c = rows["first_move"]
    assert o.membership()[v] == c and moved[v]
    assert set(rows["first_marked"]).issubset(set(np.flatnonzero(F1)))


# ---------------------------------------------------------------------------
# Alg. 4 -- driver: tolerance, mode equivalences, empty batch
# ---------------------------------------------------------------------------

def test_iteration_tolerance_is_exact(oracle_mod):
    g = synth.sbm(2000, 20, 0.05, 0.002, 12)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    o.static()
    _, _, m2 = o.weights()
    tr = o.trace()
    tau = Fraction(1, 100)
    for t, (_, _, s) in enumerate(tr):
        converged = Fraction(s, m2 * m2 // 2) <= tau  # sum dQ = S / (2 m^2)
        if t < len(tr) - 1:
            assert not converged
        else:
            assert converged or len(tr) == 20


@pytest.mark.parametrize("mode,n,blocks,mu,size,several", [
    ("static", 1500, 15, 0.3, 0, True), (0, 1500, 15, 0.3, 1500, True), (1, 1500, 15, 0.3, 1500, True),
    (2, 1500, 15, 0.3, 1500, True),
    (1, 3000, 150, 0.2, 60, False), (2, 3000, 150, 0.2, 60, False),  # DS marks 2/3 of the vertices here
])
def test_first_pass_replays_as_single_iterations(oracle_mod, mode, n, blocks, mu, size, several):
    """Pass 0 of Alg. 4 repeats Alg. 5's iteration from the initial frontier
    until sum dQ <= tau (exactly: 100 S <= 2m^2) or 20 iterations.  Replaying
    it one iteration at a time -- the single iteration is pinned by brute
    force above; community sizes are recounted from scratch before each --
    gives the driver's trace (vertices processed, movers and S of every
    iteration), its iteration count, and its counts of initially and ever
    affected vertices."""
    g = synth.planted_partition(n, blocks, mu, 10, 3, 5)
    off, idx, w = synth.to_csr(g)
    a = oracle_mod.Oracle(g.n, off, idx, w)
    b = oracle_mod.Oracle(g.n, off, idx, w)
    if mode == "static":
        a.static()
        b.set_membership(np.arange(g.n, dtype=np.uint32))  # singletons, K and Sigma from scratch
        F = np.ones(g.n, np.uint8)
        R = np.ones(g.n, np.uint8)
    else:
        a.static()
        b.static()
        d, i = synth.BatchStream(g, 3).next(size, w_max=3)
        assert a.apply_batch(d, i) == 0 and b.apply_batch(d, i) == 0
        a.update(mode)
        F, R = b.mark(mode)
    _, _, m2 = b.weights()
    initial = int(F.sum())
    ever = np.zeros(g.n, bool)
    trace = []
    for _ in range(20):
        ever |= F.astype(bool)
        processed = int(F.sum())
        F, moved, S = b.move_iteration(F, R)
        trace.append((processed, int(moved.sum()), S))
        assert (S > 0) == (moved.sum() > 0)  # every move gains
        if 100 * S <= m2 * m2 // 2:
            break
    st = a.stats()
    assert a.trace() == trace
    assert st["iterations"][0] == len(trace)
    assert st["affected_initial"] == initial and st["affected_ever"] == int(ever.sum())
    if mode in ("static", 0):
        assert initial == g.n
    if mode == 1 and not several:
        assert 0 < int(R.sum()) < g.n  # a proper affected range
    assert (len(trace) > 1) == several  # > 1: the carry-over between iterations is exercised


@pytest.mark.parametrize("case", ["static", "df"])
def test_later_passes_are_louvain_on_the_aggregated_graph(oracle_mod, case):
    """Alg. 4's passes compose: after the first pass, Louvain continues on
    the aggregated graph G' from singletons with every vertex unprocessed and
    the tolerance dropped once.  So the full run's membership equals the
    first pass's membership (renumbered ascending) looked up in a separate
    run of static Louvain on G' whose tolerance starts at tau / 10, and the
    two runs have the same Sigma, modularity and later-pass iteration counts."""
    if case == "static":
        g = synth.planted_partition(3000, 60, 0.4, 8, 4, 6)
    else:
        g = synth.planted_partition(2000, 40, 0.3, 8, 3, 5)
    off, idx, w = synth.to_csr(g)
    full = oracle_mod.Oracle(g.n, off, idx, w)
    first = oracle_mod.Oracle(g.n, off, idx, w)
    if case == "static":
        first.set_options(max_passes=1)
        full.static()
        first.static()
    else:
        full.static()
        first.static()
        d, i = synth.BatchStream(g, 3).next(5000, w_max=3)
        assert full.apply_batch(d, i) == 0 and first.apply_batch(d, i) == 0
        first.set_options(max_passes=1)
        full.update(2)
        first.update(2)
    st = full.stats()
    assert st["passes"] >= 3 and first.stats()["iterations"] == st["iterations"][:1]
    C0 = first.membership()
    soff, sidx, sw = first.aggregate()
    nv = len(soff) - 1
    ren = np.zeros(g.n, np.int64)
    labels = np.unique(C0)
    ren[labels] = np.arange(labels.shape[0])
    sup = oracle_mod.Oracle(nv, soff, sidx, sw.astype(np.uint32), allow_self_loops=True)
    sup.set_options(max_passes=9, tau_den=1000)
    sup.static()
    assert np.array_equal(full.membership(), sup.membership()[ren[C0]])
    assert sup.stats()["iterations"] == st["iterations"][1:]
    _, Sf, m2f = full.weights()
    _, Ss, m2s = sup.weights()
    assert m2f == m2s and np.array_equal(Sf[:nv], Ss) and not Sf[nv:].any()
    assert full.modularity()[1:] == sup.modularity()[1:]


def test_tolerance_drops_per_pass(oracle_mod):
    """Alg. 4 divides the iteration tolerance by TOLERANCE_DROP after every
    pass: the first pass is the same whatever the drop, and a tighter
    second-pass tolerance (drop 10) makes the second pass iterate longer
    than no drop (drop 1) on the same first-pass result."""
    for g in (synth.sbm(3000, 30, 0.05, 0.002, 8), synth.planted_partition(3000, 30, 0.35, 10, 4, 8)):
        off, idx, w = synth.to_csr(g)
        its = {}
        for drop in (10, 1):
            o = oracle_mod.Oracle(g.n, off, idx, w)
            o.set_options(tolerance_drop=drop)
            o.static()
            its[drop] = o.stats()["iterations"]
        assert its[10][0] == its[1][0]
        assert its[10][1] > its[1][1]


def test_aggregation_tolerance_rule(oracle_mod):
    """Alg. 4's tau_agg test: after a pass of more than one iteration the
    graph is aggregated and another pass runs unless the communities are
    more than tau_agg of its vertices.  A clustered graph shrinks to a few
    percent, so static Louvain runs a second pass at tau_agg = 0.8 and stops
    after the first at tau_agg = 0 (every ratio exceeds it)."""
    g = synth.sbm(2000, 20, 0.05, 0.001, 8)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    o.static()
    st = o.stats()
    assert st["iterations"][0] > 1 and st["passes"] >= 2
    o2 = oracle_mod.Oracle(g.n, off, idx, w)
    o2.set_options(tau_agg=0.0)
    o2.static()
    st2 = o2.stats()
    assert st2["iterations"][0] > 1 and st2["passes"] == 1


def test_static_equals_nd_from_singletons(oracle_mod):
    g = synth.sbm(1500, 15, 0.06, 0.003, 21)
    off, idx, w = synth.to_csr(g)
    a = oracle_mod.Oracle(g.n, off, idx, w)
    a.static()
    b = oracle_mod.Oracle(g.n, off, idx, w)
    b.set_membership(np.arange(g.n, dtype=np.uint32))
    b.update(0)
    assert np.array_equal(a.membership(), b.membership())


def test_df_with_everything_affected_equals_nd(oracle_mod):
    g = synth.sbm(1500, 15, 0.06, 0.003, 22)
    off, idx, w = synth.to_csr(g)
    d, i = synth.random_batch(g.n, g, 40, 10, 5)
    a = oracle_mod.Oracle(g.n, off, idx, w)
    a.static()
    a.apply_batch(d, i)
    b = oracle_mod.Oracle(g.n, off, idx, w)
    b.static()
    b.apply_batch(d, i)
    a.update(0)
    ones = np.ones(g.n, np.uint8)
    b.louvain_from(ones, ones)  # DF marking replaced by "all affected"
    assert np.array_equal(a.membership(), b.membership())


def test_empty_batch_leaves_state_unchanged(oracle_mod):
    g = synth.sbm(1000, 10, 0.08, 0.004, 23)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    o.static()
    before = (o.membership(), o.weights())
    o.apply_batch([], [])
    o.update(2)
    assert np.array_equal(before[0], o.membership())
    assert np.array_equal(before[1][0], o.weights()[0])
    assert np.array_equal(before[1][1], o.weights()[1])
    assert o.stats()["iterations"] == [1] and o.stats()["affected_ever"] == 0


def test_planted_partition_sanity(oracle_mod):
    # not a parity pin: Louvain should find most of the planted structure
    g = synth.sbm(10000, 50, 0.02, 0.0002, 1)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    o.static()
    q_static = o.modularity()[0]
    o.set_membership(np.repeat(np.arange(50), 200).astype(np.uint32))
    q_planted = o.modularity()[0]
    assert 0.6 < q_planted < 0.7
    assert q_static > q_planted - 0.15


# ---------------------------------------------------------------------------
# Cross-checks against an independent implementation (networkx)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_modularity_matches_networkx(oracle_mod, seed):
    """Eq. 1 against networkx's modularity (Newman's definition, written
    independently) on weighted graphs without self-loops, for random and
    planted memberships."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.community import modularity
    rng = np.random.default_rng(100 + seed)
    g = synth.planted_partition(400, 8, 0.2 + 0.1 * seed, 8, 9, 50 + seed)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_weighted_edges_from(zip(g.u.tolist(), g.v.tolist(), g.w.tolist()))
    for C in (rng.integers(0, 20, g.n), np.arange(g.n) // 50, np.zeros(g.n, np.int64)):
        C = C.astype(np.uint32)
        o.set_membership(C)
        parts = {}
        for v, c in enumerate(C.tolist()):
            parts.setdefault(c, set()).add(v)
        q_nx = modularity(G, list(parts.values()), weight="weight")
        assert abs(o.modularity()[0] - q_nx) <= 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_exact_helper_matches_networkx(seed):
    """The exact all-pairs Q that several pins use as their reference agrees
    with networkx's modularity on random weighted graphs with self-loops.
    A self-loop arc of weight w counts once in K_i and in sigma_c here
    (R1, R2); networkx counts a self-loop twice in a degree, so it gets the
    loop with weight w / 2."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.community import modularity
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(5, 14))
    off, idx, w = random_graph(rng, n, 0.4, wmax=5, self_loops=True)
    if len(idx) == 0:
        pytest.skip("empty graph")
    A = dense_matrix(n, off, idx, w)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for i in range(n):
        for j in range(i, n):
            if A[i][j]:
                G.add_edge(i, j, weight=A[i][j] / 2 if i == j else A[i][j])
    for C in (rng.integers(0, 3, n), np.arange(n), np.zeros(n, np.int64)):
        parts = {}
        for v, c in enumerate(C.tolist()):
            parts.setdefault(c, set()).add(v)
        q_nx = modularity(G, list(parts.values()), weight="weight")
        assert abs(float(newman_q(A, list(C))) - q_nx) <= 1e-12


def test_static_louvain_quality_near_networkx(oracle_mod):
    """Sanity, not parity: the oracle's static Louvain (fixed schedule)
    reaches a modularity close to networkx's Louvain on a planted partition
    (both heuristics; different orders give nearby local optima)."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.community import louvain_communities, modularity
    g = synth.sbm(3000, 30, 0.05, 0.002, 5)
    off, idx, w = synth.to_csr(g)
    o = oracle_mod.Oracle(g.n, off, idx, w)
    o.static()
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_weighted_edges_from(zip(g.u.tolist(), g.v.tolist(), g.w.tolist()))
    q_nx = modularity(G, louvain_communities(G, weight="weight", seed=1), weight="weight")
    assert abs(o.modularity()[0] - q_nx) < 0.02
