"""Pins of the oracle's augmented (4) and dual condensed (6) formulations and
of its LDL^T, against the mathematics (CPU only).

- LDL^T: L D L^T rebuilds K; on an SPD matrix with every sign +1 it is the
  Cholesky factor of numpy rescaled (L_chol = L diag(sqrt d)); on the
  quasi-definite augmented matrix the pivot signs follow the blocks for any
  ordering (strong factorizability, Sec. 2); a planted wrong sign is reported
  at the first column of that sign.
- The dual condensed matrix equals D_G^{-1} + A H^{-1} A^T formed densely.
- Both directions equal the dense solution of the full Newton system (3), and
  the oracle's primal-condensed direction (5) on larger sparse problems."""
import numpy as np
import pytest

import gen
import oracle
from oracle import forms
from tests.test_oracle import _newton_dense


def _point(lp, seed):
    mt = lp.m + int(np.isfinite(lp.l).sum()) + int(np.isfinite(lp.u).sum())
    x = gen.uniform(seed, lp.n, 0.5, 9.5)
    s = 10.0 ** gen.uniform(seed + 1, mt, -2.0, 1.0)
    lam = 10.0 ** gen.uniform(seed + 2, mt, -2.0, 1.0)
    w = gen.uniform(seed + 3, mt, 0.0, 0.5)
    return x, s, lam, w


def _rand_perm(n, seed):
    return np.argsort(gen.uniform(seed, n, 0.0, 1.0)).astype(np.int32)


def test_ldlt_of_spd_matrix_is_rescaled_cholesky():
    lp = gen.random_lp(30, 20, 3, seed=3)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, gen.lp_ordering(lp))
    D = 10.0 ** gen.uniform(4, lp.m, -1.0, 1.0)
    kval = oracle.assemble(S, lp.m, lp.rowptr, lp.col, lp.val, D, None, 0.5)
    lval, dval, bad = oracle.factor_ldlt(S, kval, np.ones(lp.n, np.int8))
    assert bad == 0 and np.all(dval > 0)
    L = oracle.l_dense(S, lval)
    np.testing.assert_allclose(np.diag(L), 1.0)
    C = np.linalg.cholesky(oracle.k_dense(S, kval, final=True))
    np.testing.assert_allclose(L * np.sqrt(dval)[None, :], C, rtol=0, atol=1e-12 * np.abs(C).max())


@pytest.mark.parametrize("pseed", [0, 1, 2])
def test_ldlt_of_augmented_matrix_any_ordering(pseed):
    lp = gen.random_lp(14, 9, 3, seed=11)
    x, s, lam, _ = _point(lp, 40)
    perm = _rand_perm(lp.n + lp.m, 50 + pseed)
    S, kval, sign = forms.augmented_system(lp, s, lam, x, 1e-8, 1e-8, perm)
    lval, dval, bad = oracle.factor_ldlt(S, kval, sign)
    assert bad == 0
    # pivot signs follow the blocks (final numbering -> original variable)
    np.testing.assert_array_equal(np.sign(dval), sign[S.perm])
    L = oracle.l_dense(S, lval)
    K = oracle.k_dense(S, kval, final=True)
    np.testing.assert_allclose(L @ np.diag(dval) @ L.T, K, rtol=0, atol=1e-12 * np.abs(K).max())
    b = gen.normal(60 + pseed, lp.n + lp.m)
    xs = oracle.solve_ldlt(S, lval, dval, b)
    np.testing.assert_allclose(xs, np.linalg.solve(oracle.k_dense(S, kval), b), rtol=1e-9,
                               atol=1e-12 * np.abs(xs).max())


def test_ldlt_reports_first_pivot_of_the_wrong_sign():
    lp = gen.random_lp(14, 9, 3, seed=12)
    x, s, lam, _ = _point(lp, 41)
    S, kval, sign = forms.augmented_system(lp, s, lam, x, 1e-8, 1e-8, None)
    bad_sign = sign.copy()
    bad_sign[lp.n + 4] = 1  # a multiplier variable declared positive
    _, _, bad = oracle.factor_ldlt(S, kval, bad_sign)
    # every other pivot has its block's sign: the planted variable's column fails
    assert bad == int(np.flatnonzero(S.perm == lp.n + 4)[0]) + 1


def test_dual_condensed_matrix_is_the_dense_product():
    lp = gen.random_lp(20, 12, 4, seed=13)
    x, s, lam, _ = _point(lp, 42)
    S, kval, _ = forms.dual_system(lp, s, lam, x, 1e-6, 1e-8)
    _, D, hdiag, _, _ = forms.reduced_terms(lp, x, s, lam, np.zeros(len(s)), 1e-6, 1e-8)
    A = lp.dense_A()
    want = np.diag(1.0 / D[:lp.m]) + A @ np.diag(1.0 / hdiag) @ A.T
    got = oracle.k_dense(S, kval)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forms_equal_full_newton_system(seed):
    lp = gen.random_lp(12, 9, 3, seed=20 + seed)
    x, s, lam, w = _point(lp, 70 + 4 * seed)
    for dp, dd in [(1e-8, 1e-8), (1e-2, 1e-3)]:
        rx, rs, rl = _newton_dense(lp, x, s, lam, w, dp, dd)
        for fn in (forms.dual_direction, forms.augmented_direction):
            dx, ds, dl = fn(lp, x, s, lam, w, dp, dd)
            for a, r in [(dx, rx), (ds, rs), (dl, rl)]:
                np.testing.assert_allclose(a, r, rtol=1e-7, atol=1e-9 * np.abs(r).max())


@pytest.mark.parametrize("case", ["random200", "grid5"])
def test_forms_equal_primal_condensed_direction(case):
    if case == "grid5":
        lp, perm = gen.grid_lp(5, seed=3), gen.nd_order_grid3d(5)
        perm_aug = np.concatenate([[p, lp.n + p] for p in perm]).astype(np.int32)
        perm_dual = perm
    else:
        lp = gen.random_lp(200, 120, 5, seed=14)
        perm, perm_dual, perm_aug = gen.lp_ordering(lp), None, None
    x, s, lam, w = _point(lp, 90)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    px, ps, pl = oracle.lp_direction(S, lp, x, s, lam, w)
    for fn, pm in ((forms.dual_direction, perm_dual), (forms.augmented_direction, perm_aug)):
        dx, ds, dl = fn(lp, x, s, lam, w, 1e-8, 1e-8, pm)
        for a, r in [(dx, px), (ds, ps), (dl, pl)]:
            np.testing.assert_allclose(a, r, rtol=1e-8, atol=1e-10 * np.abs(r).max())


def test_augmented_direction_with_a_full_hessian():
    """A QP whose Hessian is not diagonal (the dual form needs a diagonal one):
    the augmented direction still equals the primal-condensed one."""
    lp = gen.random_lp(16, 10, 3, seed=15)
    n = lp.n
    # W = B B^T + I (positive definite, dense lower triangle)
    B = gen.normal(16, n * 3).reshape(n, 3)
    Wd = B @ B.T + np.eye(n)
    wp = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for j in range(n):
        rows += list(range(j, n))
        vals += list(Wd[j:, j])
        wp[j + 1] = len(rows)
    W = (wp, np.array(rows, np.int32), np.array(vals))
    x, s, lam, w = _point(lp, 91)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None, W[0], W[1])
    px, ps, pl = oracle.lp_direction(S, lp, x, s, lam, w, W=W)
    dx, ds, dl = forms.augmented_direction(lp, x, s, lam, w, 1e-8, 1e-8, None, W)
    for a, r in [(dx, px), (ds, ps), (dl, pl)]:
        np.testing.assert_allclose(a, r, rtol=1e-8, atol=1e-10 * np.abs(r).max())
