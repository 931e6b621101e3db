"""Pins of the CPU oracle against brute force, library routines and the
algebra of the paper's Newton system (3). CPU only."""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import gen
import oracle
from tests import brute


def _lp_cases():
    yield "grid3", gen.grid_lp(3, seed=5), gen.nd_order_grid3d(3, leaf=4)
    yield "grid4x3x5", gen.grid_lp(4, 3, 5, seed=6), gen.nd_order_grid3d(4, 3, 5, leaf=8)
    lp = gen.random_lp(60, 40, 4, seed=7)
    yield "random60", lp, gen.lp_ordering(lp)
    lp = gen.random_lp(45, 70, 3, seed=8)
    yield "random45_id", lp, None


def _tri_rows(n):
    rowptr = np.arange(0, 2 * (n - 1) + 1, 2, dtype=np.int64)
    col = np.array([[i, i + 1] for i in range(n - 1)], dtype=np.int32).ravel()
    return rowptr, col


def _fundamental_starts(parent, counts):
    n = len(parent)
    nchild = np.bincount(parent[parent >= 0], minlength=n)
    starts = [0]
    for j in range(1, n):
        join = parent[j - 1] == j and nchild[j] == 1 and counts[j] == counts[j - 1] - 1
        if not join:
            starts.append(j)
    return starts


def _check_symbolic(n, rowptr, col, perm):
    S = oracle.analyze(n, len(rowptr) - 1, rowptr, col, perm)
    P = brute.k_pattern_dense(n, rowptr, col)
    # final ordering is a permutation
    assert sorted(S.perm.tolist()) == list(range(n))
    Pf = P[np.ix_(S.perm, S.perm)]
    parent, counts, cols = brute.symbolic_elimination(Pf)
    np.testing.assert_array_equal(S.parent, parent)
    np.testing.assert_array_equal(S.colcount, counts)
    for j in range(n):
        np.testing.assert_array_equal(S.li[S.lp[j]:S.lp[j + 1]], cols[j])
    assert S.nnz_l == counts.sum()
    assert S.flops == float((counts.astype(float) ** 2).sum())
    # the final numbering is a postorder: each subtree is the contiguous range ending at its root
    size = np.ones(n, dtype=np.int64)
    for j in range(n):
        if parent[j] >= 0:
            assert parent[j] > j
            size[parent[j]] += size[j]
    for j in range(n):
        desc = [k for k in range(n) if _is_desc(parent, k, j)]
        assert desc == list(range(j - size[j] + 1, j + 1))
    # postordering keeps the fill of the given ordering
    Pg = P if perm is None else P[np.ix_(perm, perm)]
    _, counts_given, _ = brute.symbolic_elimination(Pg)
    assert counts_given.sum() == counts.sum()
    # supernodes: contiguous, chains in the etree, coarsening of the fundamental partition
    sup = S.super
    assert sup[0] == 0 and sup[-1] == n and np.all(np.diff(sup) > 0)
    fstarts = set(_fundamental_starts(parent, counts))
    assert set(sup[:-1].tolist()) <= fstarts
    for s in range(S.nsuper):
        c0, c1 = sup[s], sup[s + 1]
        for j in range(c0, c1 - 1):
            assert parent[j] == j + 1
        # row structure = union of the column structures minus the block's own columns
        union = sorted(set(int(i) for j in range(c0, c1) for i in cols[j] if i >= c1))
        assert S.sri[S.srp[s]:S.srp[s + 1]].tolist() == union
        assert len(union) == counts[c1 - 1] - 1
        # explicit zeros obey the amalgamation bound
        ncol, nrow = c1 - c0, len(union)
        nz = ncol * (ncol + 1) // 2 + ncol * nrow
        z = nz - int(counts[c0:c1].sum())
        assert z >= 0
        if z > 0:
            assert (ncol <= 4 or (ncol <= 16 and 10 * z <= 8 * nz) or (ncol <= 48 and 10 * z <= nz)
                    or 20 * z <= nz)
        # supernode parent and level
        p = S.sparent[s]
        if parent[c1 - 1] < 0:
            assert p == -1
        else:
            assert sup[p] <= parent[c1 - 1] < sup[p + 1]
    kids = [[] for _ in range(S.nsuper)]
    for s in range(S.nsuper):
        if S.sparent[s] >= 0:
            kids[S.sparent[s]].append(s)
    for s in range(S.nsuper):
        want = 0 if not kids[s] else 1 + max(S.slevel[c] for c in kids[s])
        assert S.slevel[s] == want
    return S


def _is_desc(parent, k, j):
    while k != -1:
        if k == j:
            return True
        k = parent[k]
    return False


@pytest.mark.parametrize("case", list(_lp_cases()), ids=lambda c: c[0])
def test_symbolic_matches_brute_force(case):
    _, lp, perm = case
    _check_symbolic(lp.n, lp.rowptr, lp.col, perm)


def test_symbolic_special_cases():
    n = 12
    rp, col = _tri_rows(n)
    S = _check_symbolic(n, rp, col, None)
    # tridiagonal: chain etree, no fill
    assert S.parent.tolist() == list(range(1, n)) + [-1]
    assert S.nnz_l == 2 * n - 1
    # one dense row: a single supernode holding every column
    S = _check_symbolic(n, np.array([0, n], np.int64), np.arange(n, dtype=np.int32), None)
    assert S.nsuper == 1 and S.nnz_l == n * (n + 1) // 2
    # arrow: every variable coupled to the last one only -> star etree, no fill
    rp = np.arange(0, 2 * (n - 1) + 1, 2, dtype=np.int64)
    col = np.array([[i, n - 1] for i in range(n - 1)], dtype=np.int32).ravel()
    S = _check_symbolic(n, rp, col, None)
    assert np.all(S.parent[:-1] == n - 1) and S.nnz_l == 2 * n - 1
    # diagonal only (empty J): n roots, no fill
    S = _check_symbolic(n, np.zeros(1, np.int64), np.zeros(0, np.int32), None)
    assert np.all(S.parent == -1) and S.nnz_l == n


def _random_D(m, seed):
    return 10.0 ** gen.uniform(seed, m, -4.0, 4.0)


@pytest.mark.parametrize("case", list(_lp_cases()), ids=lambda c: c[0])
def test_assemble_factor_solve(case):
    _, lp, perm = case
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _random_D(lp.m, 3)
    dextra = gen.uniform(4, lp.n, 0.0, 2.0)
    kval = oracle.assemble(S, lp.m, lp.rowptr, lp.col, lp.val, D, dextra, 1e-8)
    K = oracle.k_dense(S, kval)
    A = lp.dense_A()
    Kref = A.T @ np.diag(D) @ A + np.diag(dextra) + 1e-8 * np.eye(lp.n)
    np.testing.assert_allclose(K, Kref, rtol=1e-13, atol=1e-13 * np.abs(Kref).max())
    lval, bad = oracle.factor(S, kval)
    assert bad == 0
    L = oracle.l_dense(S, lval)
    Kf = K[np.ix_(S.perm, S.perm)]
    Lref = np.linalg.cholesky(Kf)
    np.testing.assert_allclose(L, Lref, rtol=0, atol=1e-12 * np.abs(Lref).max())
    assert np.linalg.norm(L @ L.T - Kf) <= 1e-13 * np.linalg.norm(Kf)
    b = gen.normal(5, lp.n)
    x = oracle.solve(S, lval, b)
    assert np.linalg.norm(Kref @ x - b) <= 1e-10 * np.linalg.norm(b) * np.linalg.cond(Kref) ** 0.5
    np.testing.assert_allclose(x, np.linalg.solve(Kref, b), rtol=1e-8, atol=1e-10)
    scale = np.abs(Kref).sum(1).max() * np.abs(x).max()
    np.testing.assert_allclose(oracle.kmatvec(S, kval, x), Kref @ x, rtol=0, atol=1e-14 * scale)


def test_factor_reports_first_bad_pivot():
    n = 10
    rp = np.zeros(1, np.int64)
    col = np.zeros(0, np.int32)
    S = oracle.analyze(n, 0, rp, col, None)
    dextra = np.ones(n)
    dextra[6] = -1.0
    dextra[8] = -1.0
    kval = oracle.assemble(S, 0, rp, col, np.zeros(0), np.zeros(0), dextra, 0.0)
    _, bad = oracle.factor(S, kval)
    assert bad == 7  # 1 + first failing column (identity ordering, diagonal matrix)


def _newton_dense(lp, x, s, lam, w, dp, dd):
    """Full regularised Newton system (3), unknowns (d_x, d_s, -d_lambda)."""
    n = lp.n
    A = lp.dense_A()
    J = np.vstack([A, np.eye(n), -np.eye(n)])
    mt = J.shape[0]
    g = J @ x - np.concatenate([lp.b, lp.l, -lp.u])
    M = np.zeros((n + 2 * mt, n + 2 * mt))
    M[:n, :n] = dp * np.eye(n)
    M[:n, n + mt:] = J.T
    M[n:n + mt, n:n + mt] = np.diag(lam / s)
    M[n:n + mt, n + mt:] = -np.eye(mt)
    M[n + mt:, :n] = J
    M[n + mt:, n:n + mt] = -np.eye(mt)
    M[n + mt:, n + mt:] = -dd * np.eye(mt)
    rhs = -np.concatenate([lp.c - J.T @ lam, lam - w / s, g - s])
    sol = np.linalg.solve(M, rhs)
    return sol[:n], sol[n:n + mt], -sol[n + mt:]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_condensed_direction_equals_full_newton_system(seed):
    lp = gen.random_lp(12, 9, 3, seed=20 + seed)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None)
    mt = lp.m + 2 * lp.n
    x = gen.uniform(seed + 30, lp.n, 0.5, 9.5)
    s = gen.uniform(seed + 31, mt, 0.01, 3.0)
    lam = gen.uniform(seed + 32, mt, 0.01, 3.0)
    w = gen.uniform(seed + 33, mt, 0.0, 0.5)
    for dp, dd in [(1e-8, 1e-8), (1e-2, 1e-3)]:
        dx, ds, dl = oracle.lp_direction(S, lp, x, s, lam, w, dp, dd)
        rx, rs, rl = _newton_dense(lp, x, s, lam, w, dp, dd)
        for a, r in [(dx, rx), (ds, rs), (dl, rl)]:
            np.testing.assert_allclose(a, r, rtol=1e-7, atol=1e-9 * np.abs(r).max())


@pytest.mark.parametrize("seed", range(6))
def test_tiny_lp_vertex_enumeration(seed):
    n, m = 3 + seed % 2, 4 + seed % 3
    lp = gen.random_lp(n, m, 2, seed=100 + seed)
    best, _ = brute.vertex_enumeration_lp(lp.dense_A(), lp.b, lp.c, lp.l, lp.u)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None)
    r = oracle.ipm_lp(S, lp, tol=1e-10)
    assert r["status"] == 0
    assert abs(r["objective"] - best) <= 1e-6 * max(1.0, abs(best))
    assert np.all(r["s"] > 0) and np.all(r["lam"] > 0)


def _dual_objective(lp, lam):
    m, n = lp.m, lp.n
    return float(lp.b @ lam[:m] + lp.l @ lam[m:m + n] - lp.u @ lam[m + n:])


def test_small_lp_matches_highs():
    lp = gen.random_lp(2000, 1000, 5, seed=0)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, gen.lp_ordering(lp))
    r = oracle.ipm_lp(S, lp, tol=1e-8)
    assert r["status"] == 0 and r["kkt"] <= 1e-8
    A = sp.csr_matrix((lp.val, lp.col, lp.rowptr), shape=(lp.m, lp.n))
    h = so.linprog(lp.c, A_ub=-A, b_ub=-lp.b, bounds=list(zip(lp.l, lp.u)), method="highs")
    assert h.status == 0
    assert abs(r["objective"] - h.fun) <= 1e-6 * abs(h.fun)
    # duality gap equals s^T lambda up to the residuals at the returned point
    gap = r["objective"] - _dual_objective(lp, r["lam"])
    assert abs(gap - r["s"] @ r["lam"]) <= 1e-6 * max(1.0, abs(r["objective"]))
    assert np.all(r["s"] > 0) and np.all(r["lam"] > 0)


def test_grid_lp_matches_highs():
    g = 6
    lp = gen.grid_lp(g, seed=1)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, gen.nd_order_grid3d(g))
    r = oracle.ipm_lp(S, lp, tol=1e-8)
    assert r["status"] == 0
    A = sp.csr_matrix((lp.val, lp.col, lp.rowptr), shape=(lp.m, lp.n))
    h = so.linprog(lp.c, A_ub=-A, b_ub=-lp.b, bounds=list(zip(lp.l, lp.u)), method="highs")
    assert abs(r["objective"] - h.fun) <= 1e-6 * abs(h.fun)
