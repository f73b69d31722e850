"""Exact (rational) restatements of the paper's definitions, used to pin the
oracle.  Plain Python over tiny graphs; no code shared with the oracle.

Conventions (Section 3): each undirected edge is stored as two arcs (i, j)
and (j, i); a self-loop is one arc (i, i).  K_i is the sum of the weights of
the arcs leaving i, and 2m the sum of all arc weights.
"""
from fractions import Fraction

import numpy as np


def dense_matrix(n, off, idx, w):
    """A[i][j] = weight of arc (i, j) (0 if absent), as Python ints."""
    A = [[0] * n for _ in range(n)]
    for i in range(n):
        for k in range(int(off[i]), int(off[i + 1])):
            A[i][int(idx[k])] += int(w[k])
    return A


def newman_q(A, C):
    """Newman-Girvan modularity over all ordered vertex pairs:
    Q = 1/(2m) sum_{i,j} [A_ij - K_i K_j / (2m)] delta(C_i, C_j)."""
    n = len(A)
    K = [sum(row) for row in A]
    m2 = sum(K)
    if m2 == 0:
        return Fraction(0)
    q = Fraction(0)
    for i in range(n):
        for j in range(n):
            if C[i] == C[j]:
                q += Fraction(A[i][j]) - Fraction(K[i] * K[j], m2)
    return q / m2


def move(C, i, c):
    D = list(C)
    D[i] = c
    return D


def random_graph(rng, n, p, wmax=1, self_loops=False):
    """Random undirected graph as symmetric CSR (rows sorted)."""
    arcs = {}
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                wt = int(rng.integers(1, wmax + 1))
                arcs[(i, j)] = wt
                arcs[(j, i)] = wt
        if self_loops and rng.random() < 0.3:
            arcs[(i, i)] = int(rng.integers(1, wmax + 1))
    keys = sorted(arcs)
    off = np.zeros(n + 1, np.uint64)
    idx = np.array([j for (_, j) in keys], np.uint32)
    ww = np.array([arcs[k] for k in keys], np.uint32)
    for (i, _) in keys:
        off[i + 1] += 1
    off = np.cumsum(off).astype(np.uint64)
    return off, idx, ww


def edges_of(n, off, idx, w):
    """Undirected edge list (i < j) with weights from a symmetric CSR."""
    out = []
    for i in range(n):
        for k in range(int(off[i]), int(off[i + 1])):
            j = int(idx[k])
            if i < j:
                out.append((i, j, int(w[k])))
    return out
