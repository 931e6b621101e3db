"""Pins of the oracle's QP path (W != 0): the condensed direction against the
full Newton system (3) with a Hessian, and an MPC instance whose bounds are
inactive against the textbook finite-horizon LQR (Riccati) solution."""
import numpy as np
import pytest

import gen
import oracle


def _lower_csc(Wd):
    n = Wd.shape[0]
    cp, ri, vv = [0], [], []
    for j in range(n):
        for i in range(j, n):
            if Wd[i, j] != 0.0:
                ri.append(i)
                vv.append(Wd[i, j])
        cp.append(len(ri))
    return np.array(cp, np.int64), np.array(ri, np.int32), np.array(vv)


@pytest.mark.parametrize("seed", [0, 1])
def test_qp_direction_equals_full_newton_system(seed):
    lp = gen.random_lp(10, 8, 3, seed=40 + seed)
    n = lp.n
    G = gen.normal(50 + seed, n * n).reshape(n, n)
    Wd = G @ G.T / n + np.eye(n)
    Wd[np.abs(Wd) < 0.3] = 0.0  # sparse-ish but symmetric
    Wd = (Wd + Wd.T) / 2 + n * np.eye(n)
    W = _lower_csc(Wd)
    S = oracle.analyze(n, lp.m, lp.rowptr, lp.col, None, W[0], W[1])
    mt = lp.m + 2 * n
    x = gen.uniform(60 + seed, n, 0.5, 9.5)
    s = gen.uniform(61 + seed, mt, 0.01, 3.0)
    lam = gen.uniform(62 + seed, mt, 0.01, 3.0)
    w = gen.uniform(63 + seed, mt, 0.0, 0.5)
    dp, dd = 1e-8, 1e-8
    dx, ds, dl = oracle.lp_direction(S, lp, x, s, lam, w, dp, dd, W=W)
    A = lp.dense_A()
    J = np.vstack([A, np.eye(n), -np.eye(n)])
    g = J @ x - np.concatenate([lp.b, lp.l, -lp.u])
    M = np.zeros((n + 2 * mt, n + 2 * mt))
    M[:n, :n] = Wd + dp * np.eye(n)
    M[:n, n + mt:] = J.T
    M[n:n + mt, n:n + mt] = np.diag(lam / s)
    M[n:n + mt, n + mt:] = -np.eye(mt)
    M[n + mt:, :n] = J
    M[n + mt:, n:n + mt] = -np.eye(mt)
    M[n + mt:, n + mt:] = -dd * np.eye(mt)
    rhs = -np.concatenate([lp.c + Wd @ x - J.T @ lam, lam - w / s, g - s])
    sol = np.linalg.solve(M, rhs)
    for got, want in [(dx, sol[:n]), (ds, sol[n:n + mt]), (dl, -sol[n + mt:])]:
        np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9 * np.abs(want).max())


def lqr_cost(A, B, Q, R, x0):
    """Finite-horizon LQR by the backward Riccati recursion: cost-to-go
    V_k(x) = x^T P_k x / 2 with P_T = Q, gain K_k = (R + B^T P B)^{-1} B^T P A,
    P_k = Q_k + A^T P A - A^T P B K_k (Q_0 = 0: x_0 is not a decision)."""
    T = A.shape[0]
    Qm, Rm = np.diag(Q), np.diag(R)
    P = Qm.copy()
    for k in range(T - 1, -1, -1):
        Ak, Bk = A[k], B[k]
        K = np.linalg.solve(Rm + Bk.T @ P @ Bk, Bk.T @ P @ Ak)
        P = (Qm if k > 0 else 0.0 * Qm) + Ak.T @ P @ Ak - Ak.T @ P @ Bk @ K
    return 0.5 * x0 @ P @ x0


@pytest.mark.parametrize("inst", [0, 1])
def test_mpc_with_inactive_bounds_matches_lqr(inst):
    mb = gen.mpc_batch(2, seed=11, t_min=6, t_max=12)
    A, B, Q, R, x0 = mb.instance(inst)
    lp, W = gen.mpc_instance_qp(A, B, Q, R, x0, u_max=1e3, x_max=1e3)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None, W[0], W[1])
    r = oracle.ipm_lp(S, lp, tol=1e-9, W=W)
    assert r["status"] == 0
    want = lqr_cost(A, B, Q, R, x0)
    assert abs(r["objective"] - want) <= 1e-6 * max(1.0, abs(want))


def test_mpc_with_active_bounds_invariants():
    mb = gen.mpc_batch(1, seed=12, t_min=8, t_max=8)
    A, B, Q, R, x0 = mb.instance(0)
    lp, W = gen.mpc_instance_qp(A, B, Q, R, 3.0 * x0, u_max=0.2, x_max=5.0)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None, W[0], W[1])
    r = oracle.ipm_lp(S, lp, tol=1e-8, W=W)
    assert r["status"] == 0 and r["kkt"] <= 1e-8
    z = r["x"]
    assert np.all(np.abs(z[[k * 16 + j for k in range(8) for j in range(4)]]) <= 0.2 + 1e-6)
    # bounds bite: the unconstrained LQR optimum is strictly cheaper
    assert r["objective"] > lqr_cost(A, B, Q, R, 3.0 * x0) * (1 + 1e-6)
