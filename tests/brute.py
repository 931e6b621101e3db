"""Brute-force references used to pin the oracle (small inputs only)."""
from __future__ import annotations

import itertools

import numpy as np


def k_pattern_dense(n, rowptr, col, w_pairs=()) -> np.ndarray:
    """Boolean pattern of J^T J + W + I (symmetric), from the definition."""
    P = np.eye(n, dtype=bool)
    for r in range(len(rowptr) - 1):
        cs = col[rowptr[r]:rowptr[r + 1]]
        P[np.ix_(cs, cs)] = True
    for i, j in w_pairs:
        P[i, j] = P[j, i] = True
    return P


def symbolic_elimination(P: np.ndarray):
    """Fill pattern of the Cholesky factor by eliminating the graph of P column
    by column: after column j, all of its lower neighbours become pairwise
    adjacent. Returns (parent, colcount incl. diagonal, list of row sets)."""
    n = P.shape[0]
    F = np.tril(P.copy())
    parent = np.full(n, -1, dtype=np.int64)
    cols = []
    for j in range(n):
        rows = np.flatnonzero(F[j + 1:, j]) + j + 1
        cols.append(rows)
        if rows.size:
            parent[j] = rows[0]
            F[np.ix_(rows, rows)] = True
            F[:] = np.tril(F)
    counts = np.array([1 + len(r) for r in cols], dtype=np.int64)
    return parent, counts, cols


def vertex_enumeration_lp(A, b, c, l, u, tol=1e-9):
    """Exact optimum of min c^T x, A x >= b, l <= x <= u by enumerating every
    vertex (n active constraints out of m + 2n)."""
    m, n = A.shape
    G = np.vstack([A, np.eye(n), -np.eye(n)])
    h = np.concatenate([b, l, -u])
    best = np.inf
    bestx = None
    for act in itertools.combinations(range(G.shape[0]), n):
        M = G[list(act)]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, h[list(act)])
        if np.all(G @ x - h >= -tol * (1 + np.abs(h))):
            v = float(c @ x)
            if v < best:
                best, bestx = v, x
    return best, bestx
