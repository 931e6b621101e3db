"""FP64 CPU oracle of the interior-point method on the grid NLP.

TEST INFRASTRUCTURE ONLY: the product never imports this module.

Problem (gen.GridNLP): min f(x) = 1/2 ||u - u_t||^2 + alpha/2 ||v||^2 subject to
the rows of g(x) = [h(x); -h(x); v - v_lo; v_hi - v] >= 0 with
h(x) = -Lap_h u + c3 u^3 - v (the equality as a pair of inequalities, Sec. 2
problem statement). Each iteration follows the primal-dual method of Sec. 2:
the Newton system (3) at (x, s, lambda) with complementarity target mu,
condensed to Eq. (5) with W = Hessian of L = f - lambda^T (g - s):
    W_uu = 1 - 6 c3 u (lambda^+ - lambda^-),   W_vv = alpha.
The Newton step of the NLP at x is the step of the local quadratic model, so
the condensed solve reuses the oracle's LP/QP direction with b = J x - h(x)
(making J x - b = h) and c = grad f - W x (making c + W x = grad f).

Rules of this oracle (the paper names an interior-point method without fixing
them for nonconvex problems; both sides implement exactly these):
  * start x = 0, s = max(g, 1), lambda = 1, mu = 0.1;
  * barrier update (monotone): when max(primal, dual, max|s lambda - mu|)
    (scaled as the KKT residual) <= 10 mu, mu <- max(tol / 10, min(0.2 mu, mu^1.5));
  * step: tau = max(0.99, 1 - mu); one common alpha = min(alpha_s, alpha_lambda)
    from the fraction to the boundary; backtracking (halving, at most 10 times)
    on phi = f - mu sum ln s + nu ||g(x) - s||_1 with the Armijo factor 1e-4
    along the one-sided directional derivative D phi = grad f . dx - mu sum
    ds / s + nu D||g - s||_1, where D||g - s||_1 = sum sign(g - s) (J dx - ds)
    over rows with g != s plus |J dx - ds| over the others (the step solves
    the regularised system (3), which leaves delta_d d_lambda in g - s: on the
    rows of an equality pair, whose slacks both stay positive, that is all
    of g - s, so the linear model's -||g - s||_1 would promise a decrease no
    step can give), allowing for rounding 10 eps |phi| (a direction with
    D phi >= 0 takes the full alpha);
    nu = max(nu, ||lambda + d_lambda||_inf + 1);
  * inertia: a non-positive pivot raises delta_p by 100x (from 1e-8) and refactors.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from . import oracle as _o

MU0 = 0.1
KAPPA_MU, THETA_MU, KAPPA_EPS = 0.2, 1.5, 10.0
ARMIJO, MAX_HALVINGS = 1e-4, 10
EPS = float(np.finfo(np.float64).eps)  # rounding allowance of the merit comparison


def _pattern_derivs(P):
    """Per J entry: 0 centre u, 1 neighbour u, 2 v (pattern order)."""
    NN = P.N * P.N
    rows = np.repeat(np.arange(P.m), np.diff(P.rowptr))
    grid_row = rows % NN
    kind = np.where(P.col >= NN, 2, np.where(P.col == grid_row, 0, 1))
    sign = np.where(rows < NN, 1.0, -1.0)
    return kind, sign, grid_row


def evaluate(P, x):
    """f, h (N^2), J values (pattern order), grad f at x."""
    N, NN = P.N, P.N * P.N
    hinv2 = float((N + 1) ** 2)
    u = x[:NN].reshape(N, N)  # [iy, ix]
    v = x[NN:].reshape(N, N)
    nb = np.zeros_like(u)
    nb[1:, :] += u[:-1, :]
    nb[:-1, :] += u[1:, :]
    nb[:, 1:] += u[:, :-1]
    nb[:, :-1] += u[:, 1:]
    h = (4.0 * u - nb) * hinv2 + P.cubic * u ** 3 - v
    ut = P.ut.reshape(N, N)
    f = 0.5 * np.sum((u - ut) ** 2) + 0.5 * P.alpha * np.sum(v ** 2)
    grad = np.concatenate([(u - ut).ravel(), P.alpha * v.ravel()])
    kind, sign, grid_row = _pattern_derivs(P)
    uf = u.ravel()
    d = np.where(kind == 0, 4.0 * hinv2 + 3.0 * P.cubic * uf[grid_row] ** 2,
                 np.where(kind == 1, -hinv2, -1.0))
    return float(f), h.ravel(), sign * d, grad


def hessian_diag(P, x, lam):
    NN = P.N * P.N
    u = x[:NN]
    return np.concatenate([1.0 - 6.0 * P.cubic * u * (lam[:NN] - lam[NN:2 * NN]),
                           np.full(NN, P.alpha)])


def g_full(P, x, h):
    NN = P.N * P.N
    parts = [h, -h]
    if P.v_bounded:
        parts += [x[NN:] - P.v_lo, P.v_hi - x[NN:]]
    return np.concatenate(parts)


def jt_full(P, jv, y):
    """J^T y for all rows (general rows, then v - v_lo (+e), then v_hi - v (-e))."""
    NN, m = P.N * P.N, P.m
    rows = np.repeat(np.arange(m), np.diff(P.rowptr))
    out = np.zeros(P.n)
    np.add.at(out, P.col, jv * y[rows])
    if P.v_bounded:
        out[NN:] += y[m:m + NN] - y[m + NN:m + 2 * NN]
    return out


def ipm_grid_nlp(S, P, tol=1e-6, max_iter=200, delta_p=1e-8, delta_d=1e-8, ir_max=3,
                 log=None) -> dict:
    """Returns objective, kkt, iterations, status (0 converged, 7 iteration
    limit), mu history and the final x, s, lambda."""
    n, m = P.n, P.m
    x = np.zeros(n)
    f, h, jv, grad = evaluate(P, x)
    g = g_full(P, x, h)
    s = np.maximum(g, 1.0)
    lam = np.ones_like(s)
    mt = s.size
    mu = MU0
    bscale = 1.0
    if P.v_bounded:
        bscale = max(1.0, abs(P.v_lo), abs(P.v_hi))
    cscale = max(1.0, float(np.max(np.abs(grad))))
    nu = 0.0
    mus, status, it = [], 7, 0
    wp, wi = P.wp, P.wi
    lp = SimpleNamespace(n=n, m=m, rowptr=P.rowptr, col=P.col, val=None, b=None, c=None,
                         l=P.l, u=P.u)
    for it in range(max_iter + 1):
        f, h, jv, grad = evaluate(P, x)
        g = g_full(P, x, h)
        rd = grad - jt_full(P, jv, lam)
        fs = max(1.0, abs(f))
        primal, dual = float(np.max(np.abs(g - s))), float(np.max(np.abs(rd)))
        kkt = max(primal / bscale, dual / cscale, float(np.max(np.abs(s * lam))) / fs)
        mus.append(mu)
        if log is not None:
            log.append((it, f, kkt, mu))
        if kkt <= tol:
            status = 0
            break
        if it == max_iter:
            break
        if max(primal / bscale, dual / cscale, float(np.max(np.abs(s * lam - mu))) / fs) <= KAPPA_EPS * mu:
            mu = max(tol / 10.0, min(KAPPA_MU * mu, mu ** THETA_MU))
        wv = hessian_diag(P, x, lam)
        jx = np.zeros(m)
        rows = np.repeat(np.arange(m), np.diff(P.rowptr))
        np.add.at(jx, rows, jv * x[P.col])
        lp.val, lp.b, lp.c = jv, jx - h_rows(h), grad - wv * x
        dp = delta_p
        for _ in range(12):
            try:
                dx, ds, dl = _o.lp_direction(S, lp, x, s, lam, np.full(mt, mu), dp, delta_d,
                                             ir_max, W=(wp, wi, wv))
                break
            except ArithmeticError:
                dp = dp * 100.0 if dp > 0 else 1e-8
        else:
            status = 6
            break
        tau = max(0.99, 1.0 - mu)
        a_s = min(1.0, tau * np.min(-s[ds < 0] / ds[ds < 0])) if np.any(ds < 0) else 1.0
        a_l = min(1.0, tau * np.min(-lam[dl < 0] / dl[dl < 0])) if np.any(dl < 0) else 1.0
        alpha = min(a_s, a_l)
        nu = max(nu, float(np.max(np.abs(lam + dl))) + 1.0)
        viol = float(np.sum(np.abs(g - s)))
        phi0 = f - mu * float(np.sum(np.log(s))) + nu * viol
        jdx = g_full(P, dx, _jv_times(P, jv, dx)) + _bound_offsets(P)
        r, t = g - s, jdx - ds
        dtheta = float(np.sum(np.where(r > 0, t, np.where(r < 0, -t, np.abs(t)))))
        dphi = float(grad @ dx) - mu * float(np.sum(ds / s)) + nu * dtheta
        if dphi < 0.0:
            for _ in range(MAX_HALVINGS):
                xt, st = x + alpha * dx, s + alpha * ds
                ft, ht, _, _ = evaluate(P, xt)
                phit = ft - mu * float(np.sum(np.log(st))) + nu * float(np.sum(np.abs(g_full(P, xt, ht) - st)))
                if phit <= phi0 + ARMIJO * alpha * dphi + 10.0 * EPS * abs(phi0):
                    break
                alpha *= 0.5
        x, s, lam = x + alpha * dx, s + alpha * ds, lam + alpha * dl
    f, h, jv, grad = evaluate(P, x)
    return dict(objective=f, kkt=kkt, iterations=it, status=status, mu=np.array(mus), x=x, s=s,
                lam=lam)


def _jv_times(P, jv, d):
    """J_h d (the linearisation of h, pattern order values)."""
    rows = np.repeat(np.arange(P.m), np.diff(P.rowptr))
    out = np.zeros(P.m)
    np.add.at(out, rows, jv * d[P.col])
    return out[:P.N * P.N]


def _bound_offsets(P):
    """g_full is affine in x on the bound rows: g_full(P, d, J_h d) carries the
    bounds' constants, which the linear term J d must not; this undoes them."""
    NN = P.N * P.N
    if not P.v_bounded:
        return np.zeros(P.m)
    return np.concatenate([np.zeros(P.m), np.full(NN, P.v_lo), np.full(NN, -P.v_hi)])


def h_rows(h):
    """Values of the general rows [h; -h]."""
    return np.concatenate([h, -h])


def equality_qp_solution(P):
    """Without the cubic term and with v free, the problem is the equality-
    constrained QP min 1/2||u - u_t||^2 + alpha/2 ||Lap_h u||^2 (v = -Lap_h u):
    (I + alpha A^T A) u = u_t with A = -Lap_h, one sparse solve."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    N = P.N
    hinv2 = float((N + 1) ** 2)
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.identity(N)
    A = (sp.kron(I, T) + sp.kron(T, I)) * hinv2
    u = spla.spsolve((sp.identity(N * N) + P.alpha * (A.T @ A)).tocsc(), P.ut)
    v = A @ u
    f = 0.5 * float(np.sum((u - P.ut) ** 2)) + 0.5 * P.alpha * float(np.sum(v ** 2))
    return f, u, v
