"""FP64 factorisation with its dense updates on the tensor cores (Ozaki slices,
options.fp64_tc) against the CPU oracle's FP64 left-looking Cholesky and the
FP64 FMA-pipe factor of the same matrix.

The fronts span several 64-column windows with ragged tails (15^3: a
450-column top separator; 22^3: ~970 columns, where the last block columns
have fewer row tiles than the launch wants CTAs, so their K ranges are split
over CTAs and summed with atomics); D spans up to eight decades so that the
windows' exponents differ widely."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402
from tests.test_gpu_parity import PROBLEMS, _oracle_K, _problem, _state, dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    oracle.build()


def _ctx(lp, perm, **opt):
    o = gb.default_options(storage_fp64=1, **opt)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
    info = ctx.kkt_analyze(perm)
    ctx.ipm_set_workspace()
    return ctx, info


def _entries(S, n):
    cols = np.repeat(np.arange(n), np.diff(S.lp) + 1).astype(np.int32)
    rows = np.empty_like(cols)
    for j in range(n):
        b = S.lp[j] + j
        rows[b] = j
        rows[b + 1: b + 1 + S.lp[j + 1] - S.lp[j]] = S.li[S.lp[j]:S.lp[j + 1]]
    return rows, cols


@pytest.mark.parametrize("spread", [1.0, 4.0])
@pytest.mark.parametrize("name", PROBLEMS)
def test_fp64_tc_factor_matches_oracle(name, spread):
    """Entries within 1e-12 of the oracle's (relative to their column's largest
    entry), or, where D spans eight decades and any two FP64 factorisations of
    K differ by more (the pivots amplify rounding), no further from the oracle
    than 4x the FMA-pipe FP64 factor is; backward error 1e-13 either way."""
    lp, perm = _problem(name)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 2, spread=spread)
    Kv = _oracle_K(S, lp, D, 1e-8)
    lval, obad = oracle.factor(S, Kv)
    assert obad == 0
    rows, cols = _entries(S, lp.n)
    colmax = np.zeros(lp.n)
    np.maximum.at(colmax, cols, np.abs(lval))
    err = []
    for tc in (0, 1):
        ctx, info = _ctx(lp, perm, fp64_tc=tc)
        ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
        st, bad = ctx.kkt_factor(gb.IPM_FP64)
        assert st == 0 and bad == -1
        got = ctx.kkt_factor_entries(rows, cols)
        err.append(np.max(np.abs(got - lval) / colmax[cols]))
    print(name, spread, "max entry error (column-relative): FMA %.2e, tensor cores %.2e" % tuple(err))
    assert err[1] <= max(1e-12, 4 * err[0]), err
    L = np.zeros((lp.n, lp.n))
    L[rows, cols] = got
    K = oracle.k_dense(S, Kv, final=True)
    assert np.linalg.norm(L @ L.T - K) <= 1e-13 * np.linalg.norm(K)


def test_fp64_tc_matches_oracle_with_split_updates():
    """22^3 grid: the top front's late block columns take the split-K path;
    the entries are no further from the oracle's than the FMA-pipe FP64
    factor's are (4x, or 1e-12 relative to their column)."""
    lp = gen.grid_lp(22, seed=5)
    perm = gen.nd_order_grid3d(22)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 7, spread=3.0)
    lval, obad = oracle.factor(S, _oracle_K(S, lp, D, 1e-8))
    assert obad == 0
    rows, cols = _entries(S, lp.n)
    colmax = np.zeros(lp.n)
    np.maximum.at(colmax, cols, np.abs(lval))
    err = []
    for tc in (0, 1):
        ctx, info = _ctx(lp, perm, fp64_tc=tc)
        assert info.max_ncol > 900
        ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
        st, bad = ctx.kkt_factor(gb.IPM_FP64)
        assert st == 0 and bad == -1
        got = ctx.kkt_factor_entries(rows, cols)
        err.append(np.max(np.abs(got - lval) / colmax[cols]))
    print("22^3 max entry error (column-relative): FMA %.2e, tensor cores %.2e" % tuple(err))
    assert err[1] <= max(1e-12, 4 * err[0]), err


def test_fp64_tc_solve_and_refinement():
    lp, perm = _problem("grid15")
    ctx, info = _ctx(lp, perm, fp64_tc=1)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 3, spread=3.0)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    ctx.kkt_factor(gb.IPM_FP64)
    b = gen.normal(4, lp.n)
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    K = oracle.k_dense(S, _oracle_K(S, lp, D, 1e-8))
    ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_NONE)
    r = np.linalg.norm(K @ x.cpu().numpy() - b) / np.linalg.norm(b)
    assert r <= 1e-10


@pytest.mark.parametrize("name", ["grid15", "random600"])
def test_fp64_tc_ipm_matches_oracle(name):
    lp, perm = _problem(name)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    ref = oracle.ipm_lp(S, lp, tol=1e-8)
    assert ref["status"] == 0
    mt = lp.m + 2 * lp.n
    iters = []
    for tc in (0, 1):
        ctx, info = _ctx(lp, perm, precision=gb.IPM_FP64, tol=1e-8, fp64_tc=tc)
        x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        s = torch.empty(mt, dtype=torch.float64, device="cuda")
        lam = torch.empty(mt, dtype=torch.float64, device="cuda")
        res = ctx.ipm_solve(dev(lp.val), dev(lp.b), dev(lp.c), x, s, lam)
        assert res.status == 0 and res.kkt <= 1e-8, res.as_dict()
        assert abs(res.objective - ref["objective"]) <= 1e-6 * abs(ref["objective"])
        iters.append(res.iterations)
    assert abs(iters[1] - iters[0]) <= 1


def test_fp64_tc_needs_analysis_with_the_option():
    """Turning fp64_tc on after kkt_analyze sized no slices: the factor refuses."""
    lp, perm = _problem("grid7x9x5")
    ctx, info = _ctx(lp, perm, fp64_tc=0)
    D = _state(lp, 2)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    ctx.ipm_set_options(gb.default_options(storage_fp64=1, fp64_tc=1))
    with pytest.raises(gb.IpmError) as e:
        ctx.kkt_factor(gb.IPM_FP64)
    assert e.value.status == 10  # IPM_ERR_UNSUPPORTED


def test_fp64_tc_nan_reaches_a_pivot():
    """A NaN in K (one D entry) propagates through the slices (its window's
    exponent marks it) into a pivot: the factor reports a failed pivot, as the
    FMA-pipe FP64 factor does, instead of hiding it."""
    lp, perm = _problem("grid15")
    D = _state(lp, 2)
    D[lp.m // 2] = np.nan
    bads = []
    for tc in (0, 1):
        ctx, info = _ctx(lp, perm, fp64_tc=tc)
        ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
        st, bad = ctx.kkt_factor(gb.IPM_FP64, raise_on_error=False)
        assert st == 5 and bad >= 0, (tc, st, bad)  # IPM_ERR_NOT_SPD
        bads.append(bad)
    # a failed pivot of the tensor-core factor is redone on the FMA pipe, which decides
    assert bads[0] == bads[1]
