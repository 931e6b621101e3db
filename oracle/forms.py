"""Oracle of the augmented (4) and dual condensed (6) formulations of the
Newton system (3) (test infrastructure only, like the rest of ``oracle/``).

Sec. 3 ("Condensed KKT Systems") derives three systems from (3): the augmented
system (4), obtained by eliminating d_s; the primal condensed system (5),
eliminating d_lambda from (4); and the dual condensed system (6) ("normal
equations"), eliminating d_x from (4) when W + delta_p I is easy to invert.
Every one of them gives the same Newton direction. This module computes the
direction through (4) and through (6) for the LP/QP of ``oracle.ipm_lp``
(general rows A x >= b, bounds l <= x <= u, optional Hessian W), with the
oracle's own symbolic analysis, assembly, Cholesky and a plain LDL^T.

Reading taken (the paper writes (4) and (6) for g without splitting its
rows): the bound rows have Jacobian rows +-e_i, so their part of J^T D J is
diagonal; they are folded into the (1,1) block H = W + delta_p I + D_l + D_u
and only the m general rows keep a multiplier block. With q = g_G - w_G /
lambda_G (general rows) and
    r~ = grad f - J^T lambda + J_B^T D_B (g_B - w_B / lambda_B)   (B: bound rows),
(4) reads  [H, A^T; A, -D_G^{-1}] [d_x; y] = -[r~; q],  y = -d_lambda_G,
and (6) reads  (D_G^{-1} + A H^{-1} A^T) y = q - A H^{-1} r~,
              d_x = -H^{-1} (r~ + A^T y),
which needs H diagonal (W diagonal or absent). Both give the d_x of (5);
d_lambda and d_s then follow from rows 2-3 of (3) as in ``lp_direction``.

The augmented matrix is symmetric quasi-definite (H positive definite,
-D_G^{-1} negative definite), so LDL^T exists without pivoting for every
ordering, with d_j > 0 on the first n variables and < 0 on the last m
(strong factorizability, Sec. 2). The dual condensed matrix is SPD.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o


def _rows(lp):
    lidx = np.flatnonzero(np.isfinite(lp.l))
    uidx = np.flatnonzero(np.isfinite(lp.u))
    return lidx, uidx


def _amul(lp, v):
    """A v for the CSR matrix A of the general rows (plain loops over rows)."""
    out = np.zeros(lp.m)
    for r in range(lp.m):
        a, b = lp.rowptr[r], lp.rowptr[r + 1]
        out[r] = np.dot(lp.val[a:b], v[lp.col[a:b]])
    return out


def _atmul(lp, v):
    """A^T v."""
    out = np.zeros(lp.n)
    for r in range(lp.m):
        a, b = lp.rowptr[r], lp.rowptr[r + 1]
        out[lp.col[a:b]] += lp.val[a:b] * v[r]
    return out


def _wmul(W, x):
    out = np.zeros(len(x))
    if W is None:
        return out
    wp, wi, wv = W
    for j in range(len(x)):
        for e in range(wp[j], wp[j + 1]):
            i = wi[e]
            out[i] += wv[e] * x[j]
            if i != j:
                out[j] += wv[e] * x[i]
    return out


def reduced_terms(lp, x, s, lam, w, delta_p, delta_d, W=None):
    """g, D, the diagonal of H (with W's diagonal), r~ and q (see the module text)."""
    m, n = lp.m, lp.n
    lidx, uidx = _rows(lp)
    nl = len(lidx)
    g = np.concatenate([_amul(lp, x) - lp.b, x[lidx] - lp.l[lidx], lp.u[uidx] - x[uidx]])
    D = 1.0 / (delta_d + s / lam)
    hdiag = np.full(n, float(delta_p))
    np.add.at(hdiag, lidx, D[m:m + nl])
    np.add.at(hdiag, uidx, D[m + nl:])
    if W is not None:
        wp, wi, wv = W
        for j in range(n):
            for e in range(wp[j], wp[j + 1]):
                if wi[e] == j:
                    hdiag[j] += wv[e]
    t = D * (g - w / lam) - lam  # per row: D (g - w / lambda) - lambda
    t[:m] = -lam[:m]             # general rows keep only - lambda in r~
    rt = lp.c + _wmul(W, x) + _atmul(lp, t[:m])
    np.add.at(rt, lidx, t[m:m + nl])
    np.subtract.at(rt, uidx, t[m + nl:])
    q = g[:m] - w[:m] / lam[:m]
    return g, D, hdiag, rt, q


def _recover(lp, x, s, lam, w, g, D, dx):
    """Rows 2-3 of (3): d_lambda = D (w / lambda - g - J d_x), d_s."""
    lidx, uidx = _rows(lp)
    jdx = np.concatenate([_amul(lp, dx), dx[lidx], -dx[uidx]])
    dl = D * (w / lam - g - jdx)
    ds = -s + w / lam - (s / lam) * dl
    return ds, dl


def transpose_pattern(lp):
    """CSR of A^T (n rows, m columns), entries ascending, and the index of each
    entry's value in A's CSR order."""
    counts = np.bincount(lp.col, minlength=lp.n)
    tp = np.zeros(lp.n + 1, np.int64)
    tp[1:] = np.cumsum(counts)
    ti = np.empty(len(lp.col), np.int32)
    src = np.empty(len(lp.col), np.int64)
    fill = tp[:-1].copy()
    for r in range(lp.m):
        for e in range(lp.rowptr[r], lp.rowptr[r + 1]):
            j = lp.col[e]
            ti[fill[j]] = r
            src[fill[j]] = e
            fill[j] += 1
    return tp, ti, src


def dual_system(lp, s, lam, x, delta_p, delta_d, perm=None, W=None):
    """Symbolic analysis and values of K6 = D_G^{-1} + A H^{-1} A^T (order m),
    assembled by the oracle as W' + J'^T D' J' with J' = A^T (n x m), D' =
    1 / diag(H) and W' = diag(D_G^{-1})."""
    m = lp.m
    tp, ti, src = transpose_pattern(lp)
    w = np.zeros(len(s))
    _, D, hdiag, _, _ = reduced_terms(lp, x, s, lam, w, delta_p, delta_d, W)
    wp = np.arange(m + 1, dtype=np.int64)
    wi = np.arange(m, dtype=np.int32)
    S = _o.analyze(m, lp.n, tp, ti, perm, wp, wi)
    kval = _o.assemble(S, lp.n, tp, ti, lp.val[src], 1.0 / hdiag, None, 0.0, wp, wi, 1.0 / D[:m])
    return S, kval, (tp, ti, src, wp, wi)


def augmented_pattern(lp, W=None):
    """Lower CSC pattern of the augmented matrix (order n + m): column j < n
    holds W's rows of column j with the diagonal always present, then rows
    n + i for A_ij != 0; column n + i only its diagonal."""
    n, m = lp.n, lp.m
    tp, ti, src = transpose_pattern(lp)
    cols_r, cols_src = [], []
    for j in range(n):
        rows = {j: ("d", -1)}
        if W is not None:
            wp, wi, _ = W
            for e in range(wp[j], wp[j + 1]):
                rows[int(wi[e])] = ("w", e)
        for e in range(tp[j], tp[j + 1]):
            rows[n + int(ti[e])] = ("a", int(src[e]))
        order = sorted(rows)
        cols_r.append(order)
        cols_src.append([rows[r] for r in order])
    for i in range(m):
        cols_r.append([n + i])
        cols_src.append([("g", i)])
    cp = np.zeros(n + m + 1, np.int64)
    cp[1:] = np.cumsum([len(c) for c in cols_r])
    ri = np.array([r for c in cols_r for r in c], np.int32)
    srcs = [t for c in cols_src for t in c]
    return cp, ri, srcs


def augmented_system(lp, s, lam, x, delta_p, delta_d, perm=None, W=None):
    """Symbolic analysis and values of the augmented matrix (4) with the bound
    rows folded into H; returns (S, kval, sign) with sign +1 on the n primal
    and -1 on the m multiplier variables (original numbering)."""
    n, m = lp.n, lp.m
    w = np.zeros(len(s))
    _, D, hdiag, _, _ = reduced_terms(lp, x, s, lam, w, delta_p, delta_d, W)
    cp, ri, srcs = augmented_pattern(lp, W)
    vals = np.empty(len(srcs))
    for k, (kind, e) in enumerate(srcs):
        if kind == "w":
            vals[k] = W[2][e]
        elif kind == "a":
            vals[k] = lp.val[e]
        elif kind == "g":
            vals[k] = -1.0 / D[e]
        else:
            vals[k] = 0.0
    # the diagonal of the first n columns: + delta_p + D_l + D_u (hdiag minus W's diagonal)
    wdiag = np.zeros(n)
    if W is not None:
        wp, wi, wv = W
        for j in range(n):
            for e in range(wp[j], wp[j + 1]):
                if wi[e] == j:
                    wdiag[j] += wv[e]
    for j in range(n):
        vals[cp[j]] += hdiag[j] - wdiag[j]  # the diagonal is the first entry of column j
    S = _o.analyze(n + m, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), perm, cp, ri)
    kval = _o.assemble(S, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                       np.zeros(0), None, 0.0, cp, ri, vals)
    sign = np.concatenate([np.ones(n, np.int8), -np.ones(m, np.int8)])
    return S, kval, sign


def _refine(S, kval, solve, rhs, ir_max=3):
    x = solve(rhs)
    bn = np.abs(rhs).max()
    for _ in range(ir_max):
        r = rhs - _o.kmatvec(S, kval, x)
        if bn == 0 or np.abs(r).max() <= 1e-14 * bn:
            break
        x = x + solve(r)
    return x


def dual_direction(lp, x, s, lam, w, delta_p=1e-8, delta_d=1e-8, perm=None, W=None):
    """(d_x, d_s, d_lambda) through the dual condensed system (6) (see the
    module text); perm orders the m rows."""
    g, D, hdiag, rt, q = reduced_terms(lp, x, s, lam, w, delta_p, delta_d, W)
    S, kval, _ = dual_system(lp, s, lam, x, delta_p, delta_d, perm, W)
    lval, bad = _o.factor(S, kval)
    if bad:
        raise ArithmeticError(f"non-positive pivot at column {bad - 1}")
    u = rt / hdiag
    y = _refine(S, kval, lambda b: _o.solve(S, lval, b), q - _amul(lp, u))
    dx = -(rt + _atmul(lp, y)) / hdiag
    ds, dl = _recover(lp, x, s, lam, w, g, D, dx)
    return dx, ds, dl


def augmented_direction(lp, x, s, lam, w, delta_p=1e-8, delta_d=1e-8, perm=None, W=None):
    """(d_x, d_s, d_lambda) through the augmented system (4) and LDL^T (see
    the module text); perm orders the n + m unknowns (d_x then y)."""
    g, D, hdiag, rt, q = reduced_terms(lp, x, s, lam, w, delta_p, delta_d, W)
    S, kval, sign = augmented_system(lp, s, lam, x, delta_p, delta_d, perm, W)
    lval, dval, bad = _o.factor_ldlt(S, kval, sign)
    if bad:
        raise ArithmeticError(f"pivot of the wrong sign at column {bad - 1}")
    z = _refine(S, kval, lambda b: _o.solve_ldlt(S, lval, dval, b), -np.concatenate([rt, q]))
    dx = z[:lp.n]
    ds, dl = _recover(lp, x, s, lam, w, g, D, dx)
    return dx, ds, dl
