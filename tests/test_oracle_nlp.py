"""Pins of the FP64 grid-NLP oracle (no GPU).

* the Jacobian and the Hessian of the Lagrangian against central differences;
* without the cubic term and with v free, the interior-point solution equals
  the equality-constrained QP solved by one sparse linear system;
* the barrier parameter never increases; at the solution the slacks and
  multipliers stay positive, h(x) = 0 and v is inside its bounds.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import nlp as ON


def _S(P):
    return oracle.analyze(P.n, P.m, P.rowptr, P.col, gen.nd_order_grid_nlp(P.N), P.wp, P.wi)


def test_pattern_rows():
    P = gen.grid_nlp(5)
    NN = 25
    assert P.rowptr[-1] == 2 * (5 * NN - 4 * 5 + NN)  # 5-point stencil entries + v, twice
    for r in (0, 7, NN - 1, NN + 12):
        cols = P.col[P.rowptr[r]:P.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0) and cols[-1] == NN + r % NN


def test_jacobian_and_hessian_match_finite_differences():
    P = gen.grid_nlp(6, seed=9)
    rng = np.random.default_rng(1)
    x = rng.normal(0, 0.5, P.n)
    lam = rng.uniform(0.1, 2.0, 4 * 36)
    f, h, jv, grad = ON.evaluate(P, x)
    rows = np.repeat(np.arange(P.m), np.diff(P.rowptr))
    eps = 1e-6
    for e in rng.choice(jv.size, 40, replace=False):
        r, c = rows[e], P.col[e]
        xp, xm = x.copy(), x.copy()
        xp[c] += eps
        xm[c] -= eps
        hp = ON.h_rows(ON.evaluate(P, xp)[1])[r]
        hm = ON.h_rows(ON.evaluate(P, xm)[1])[r]
        assert jv[e] == pytest.approx((hp - hm) / (2 * eps), rel=1e-6, abs=1e-4)
    # gradient of f
    for c in rng.choice(P.n, 10, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[c] += eps
        xm[c] -= eps
        assert grad[c] == pytest.approx((ON.evaluate(P, xp)[0] - ON.evaluate(P, xm)[0]) / (2 * eps),
                                        rel=1e-6, abs=1e-6)
    # Hessian of L = f - lambda^T g: diagonal, from differences of grad L
    w = ON.hessian_diag(P, x, lam)

    def grad_L(z):
        _, hz, jz, gz = ON.evaluate(P, z)
        return gz - ON.jt_full(P, jz, lam)

    for c in rng.choice(P.n, 10, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[c] += eps
        xm[c] -= eps
        col = (grad_L(xp) - grad_L(xm)) / (2 * eps)
        assert w[c] == pytest.approx(col[c], rel=1e-5, abs=1e-4)
        off = np.delete(col, c)
        assert np.max(np.abs(off)) < 1e-4 * max(1.0, abs(col[c]))


def test_without_cubic_term_matches_equality_qp():
    P = gen.grid_nlp(10, seed=4, cubic=0, v_bounded=0)
    res = ON.ipm_grid_nlp(_S(P), P, tol=1e-9, max_iter=100)
    f_ref, u_ref, v_ref = ON.equality_qp_solution(P)
    assert res["status"] == 0
    assert res["objective"] == pytest.approx(f_ref, rel=1e-7)
    assert np.max(np.abs(res["x"][:100] - u_ref)) < 1e-5 * max(1.0, np.max(np.abs(u_ref)))


def test_general_problem_invariants():
    P = gen.grid_nlp(10, seed=6)
    res = ON.ipm_grid_nlp(_S(P), P, tol=1e-8, max_iter=200)
    assert res["status"] == 0 and res["kkt"] <= 1e-8
    assert np.all(np.diff(res["mu"]) <= 0.0)
    assert np.all(res["s"] > 0) and np.all(res["lam"] > 0)
    x = res["x"]
    _, h, _, _ = ON.evaluate(P, x)
    assert np.max(np.abs(h)) < 1e-6 * (P.N + 1) ** 2
    assert np.all(x[100:] >= -1 - 1e-8) and np.all(x[100:] <= 1 + 1e-8)
