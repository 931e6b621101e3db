"""Degenerate and edge inputs of the interior-point path against closed forms
and the oracle: no general rows (bounds only), one variable, an empty row, a
dense row (one wide front), free variables, and a non-positive pivot."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_16094_gb300 as gb  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _solve(n, m, rowptr, col, val, b, c, l, u, prec=0, tol=1e-8):
    o = gb.default_options(precision=prec, tol=tol, max_iter=200, storage_fp64=1)
    ctx = gb.IpmContext(n, m, rowptr, col, l, u, options=o)
    ctx.kkt_analyze(None)
    ctx.ipm_set_workspace()
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
    lam = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
    res = ctx.ipm_solve(dev(val if len(val) else np.zeros(1)), dev(b if len(b) else np.zeros(1)),
                        dev(c), x, s, lam)
    return res, x.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 4])
def test_bounds_only(prec):
    """m = 0: min c^T x on [0, 10]^n has x_i = 0 for c_i > 0 and 10 for c_i < 0."""
    n = 300
    c = gen.normal(5, n)
    res, x = _solve(n, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0),
                    c, np.zeros(n), np.full(n, 10.0), prec=prec)
    assert res.status == 0
    want = np.where(c > 0, 0.0, 10.0)
    assert res.objective == pytest.approx(float(c @ want), rel=1e-7, abs=1e-7)
    assert np.max(np.abs(x - want)) < 1e-5


def test_one_variable():
    """min x s.t. 2 x >= 3, 0 <= x <= 10: x = 1.5."""
    res, x = _solve(1, 1, np.array([0, 1]), np.array([0], np.int32), np.array([2.0]),
                    np.array([3.0]), np.array([1.0]), np.zeros(1), np.full(1, 10.0))
    assert res.status == 0 and x[0] == pytest.approx(1.5, abs=1e-7)


def test_empty_row_and_unbounded_above_match_oracle():
    """A row without entries (0 >= b, b < 0) and variables without upper
    bounds (costs positive, so the optimum stays finite) against the oracle."""
    lp = gen.random_lp(60, 40, 4, seed=17)
    rowptr = lp.rowptr.copy()
    col, val = lp.col.copy(), lp.val.copy()
    # empty row 7: drop its entries, make it trivially feasible
    s0, e0 = rowptr[7], rowptr[8]
    col = np.delete(col, np.arange(s0, e0))
    val = np.delete(val, np.arange(s0, e0))
    rowptr[8:] -= e0 - s0
    b = lp.b.copy()
    b[7] = -1.0
    l, u = lp.l.copy(), lp.u.copy()
    u[5:15] = np.inf  # no upper bound
    res, x = _solve(lp.n, lp.m, rowptr, col, val, b, lp.c, l, u)
    lp2 = gen.LP(lp.n, lp.m, rowptr, col, val, b, lp.c, l, u, lp.x0)
    S = oracle.analyze(lp.n, lp.m, rowptr, col, None)
    ref = oracle.ipm_lp(S, lp2, tol=1e-8)
    assert res.status == 0 and ref["status"] == 0
    assert res.objective == pytest.approx(ref["objective"], rel=1e-6)


def test_dense_row_gives_one_wide_front():
    """One row touching all 700 variables: K is dense (one front wider than
    several 128-blocks with a ragged tail); the IPM matches the oracle."""
    n = 700
    lp = gen.random_lp(n, 200, 3, seed=19)
    rows = [lp.col[lp.rowptr[r]:lp.rowptr[r + 1]] for r in range(lp.m)]
    vals = [lp.val[lp.rowptr[r]:lp.rowptr[r + 1]] for r in range(lp.m)]
    rows.append(np.arange(n, dtype=np.int32))
    vals.append(np.ones(n))
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    col = np.concatenate(rows).astype(np.int32)
    val = np.concatenate(vals)
    b = np.concatenate([lp.b, [float(n)]])  # sum x >= n (x0 ~ U(1,9) keeps it feasible)
    lp2 = gen.LP(n, lp.m + 1, rowptr, col, val, b, lp.c, lp.l, lp.u, lp.x0)
    for prec in (0, 4):
        res, x = _solve(n, lp.m + 1, rowptr, col, val, b, lp.c, lp.l, lp.u, prec=prec)
        S = oracle.analyze(n, lp.m + 1, rowptr, col, None)
        ref = oracle.ipm_lp(S, lp2, tol=1e-8)
        assert res.status == 0 and ref["status"] == 0
        assert res.objective == pytest.approx(ref["objective"], rel=1e-6)


def test_unbounded_lp_is_not_reported_optimal():
    """Variables without lower bounds whose costs make the LP unbounded: the
    iterates diverge and the solve must end in an error, as the oracle's does."""
    lp = gen.random_lp(60, 40, 4, seed=17)
    l = lp.l.copy()
    l[:5] = -np.inf
    res, _ = _solve(lp.n, lp.m, lp.rowptr, lp.col, lp.val, lp.b, lp.c, l, lp.u)
    lp2 = gen.LP(lp.n, lp.m, lp.rowptr, lp.col, lp.val, lp.b, lp.c, l, lp.u, lp.x0)
    ref = oracle.ipm_lp(oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None), lp2, tol=1e-8)
    assert ref["status"] != 0
    assert res.status != 0
