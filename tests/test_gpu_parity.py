"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Sizes span several factor/solve blocks (64 wide) with ragged tails: the 15^3
grid has a 450-column top separator (7 blocks, last one 2 wide)."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    oracle.build()


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _problem(name):
    if name == "grid15":
        lp = gen.grid_lp(15, seed=11)
        return lp, gen.nd_order_grid3d(15)
    if name == "grid7x9x5":
        lp = gen.grid_lp(7, 9, 5, seed=12)
        return lp, gen.nd_order_grid3d(7, 9, 5)
    if name == "random600":
        lp = gen.random_lp(600, 300, 5, seed=13)
        return lp, gen.lp_ordering(lp)
    raise KeyError(name)


PROBLEMS = ["grid15", "grid7x9x5", "random600"]


def _ctx(lp, perm, **opt):
    o = gb.default_options(**opt)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
    info = ctx.kkt_analyze(perm)
    ctx.ipm_set_workspace()
    return ctx, info


def _state(lp, seed, spread=1.0):
    mt = lp.m + 2 * lp.n
    D = 10.0 ** gen.uniform(seed, mt, -spread, spread)
    return D


def _oracle_K(S, lp, D, delta_p):
    m, n = lp.m, lp.n
    dextra = D[m:m + n] + D[m + n:]
    return oracle.assemble(S, m, lp.rowptr, lp.col, lp.val, D[:m], dextra, delta_p)


@pytest.mark.parametrize("name", PROBLEMS)
def test_assembly_matches_oracle(name):
    lp, perm = _problem(name)
    ctx, info = _ctx(lp, perm)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 1, spread=4.0)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    got = ctx.kkt_export_assembled()
    want = _oracle_K(S, lp, D, 1e-8)
    # bound on the rounding of a sum of products: a few ulps of the sum of |terms|
    absK = oracle.assemble(S, lp.m, lp.rowptr, lp.col, np.abs(lp.val), D[:lp.m],
                           D[lp.m:lp.m + lp.n] + D[lp.m + lp.n:], 1e-8)
    assert np.all(np.abs(got - want) <= 8 * np.finfo(float).eps * absK)


@pytest.mark.parametrize("name", PROBLEMS)
def test_fp64_factor_matches_oracle(name):
    lp, perm = _problem(name)
    ctx, info = _ctx(lp, perm)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 2, spread=1.0)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    st, bad = ctx.kkt_factor(gb.IPM_FP64)
    assert st == 0 and bad == -1
    lval, obad = oracle.factor(S, _oracle_K(S, lp, D, 1e-8))
    assert obad == 0
    cols = np.repeat(np.arange(lp.n), np.diff(S.lp) + 1).astype(np.int32)
    rows = np.empty_like(cols)
    for j in range(lp.n):
        b = S.lp[j] + j
        rows[b] = j
        rows[b + 1: b + 1 + S.lp[j + 1] - S.lp[j]] = S.li[S.lp[j]:S.lp[j + 1]]
    got = ctx.kkt_factor_entries(rows, cols)
    scale = np.abs(lval).max()
    np.testing.assert_allclose(got, lval, rtol=0, atol=1e-12 * scale)
    # an entry outside the structure of column 0 reads as zero
    struct0 = set(S.li[S.lp[0]:S.lp[1]].tolist())
    outside = [r for r in range(1, lp.n) if r not in struct0][:3]
    assert np.all(ctx.kkt_factor_entries(np.array(outside), np.zeros(len(outside))) == 0.0)
    # ||L L^T - K||_F / ||K||_F from the extracted factor
    L = np.zeros((lp.n, lp.n))
    L[rows, cols] = got
    K = oracle.k_dense(S, _oracle_K(S, lp, D, 1e-8), final=True)
    assert np.linalg.norm(L @ L.T - K) <= 1e-13 * np.linalg.norm(K)


@pytest.mark.parametrize("name", PROBLEMS)
@pytest.mark.parametrize("prec", [gb.IPM_FP64, gb.IPM_FP32])
def test_solve_with_refinement(name, prec):
    lp, perm = _problem(name)
    ctx, info = _ctx(lp, perm, storage_fp64=1)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 3, spread=3.0)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    ctx.kkt_factor(prec)
    b = gen.normal(4, lp.n)
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    K = oracle.k_dense(S, _oracle_K(S, lp, D, 1e-8))
    if prec == gb.IPM_FP64:
        ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_NONE)
        r = np.linalg.norm(K @ x.cpu().numpy() - b) / np.linalg.norm(b)
        assert r <= 1e-10
    info = ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_IR)
    xs = x.cpu().numpy()
    assert info.rel_residual <= 1e-10
    assert np.abs(K @ xs - b).max() <= 1e-10 * np.abs(b).max() * 4
    np.testing.assert_allclose(xs, np.linalg.solve(K, b), rtol=1e-6,
                               atol=1e-8 * np.abs(xs).max())


@pytest.mark.parametrize("name", PROBLEMS)
def test_newton_direction_matches_oracle(name):
    lp, perm = _problem(name)
    ctx, info = _ctx(lp, perm)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    mt = lp.m + 2 * lp.n
    x = gen.uniform(21, lp.n, 0.5, 9.5)
    s = gen.uniform(22, mt, 0.01, 3.0)
    lam = gen.uniform(23, mt, 0.01, 3.0)
    w = gen.uniform(24, mt, 0.0, 0.2)
    out = [torch.empty(k, dtype=torch.float64, device="cuda") for k in (lp.n, mt, mt)]
    ctx.ipm_newton_direction(dev(lp.val), dev(lp.b), dev(lp.c), dev(x), dev(s), dev(lam), dev(w),
                             *out)
    want = oracle.lp_direction(S, lp, x, s, lam, w, 1e-8, 1e-8)
    for g, wv in zip(out, want):
        np.testing.assert_allclose(g.cpu().numpy(), wv, rtol=1e-8, atol=1e-10 * np.abs(wv).max())


def test_not_spd_reports_first_column():
    lp, perm = _problem("grid7x9x5")
    ctx, info = _ctx(lp, perm)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 5, spread=0.5)
    # two variables get a large negative bound-row weight
    for v in (S.perm[40], S.perm[200]):
        D[lp.m + v] = -1e4
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    st, bad = ctx.kkt_factor(gb.IPM_FP64, raise_on_error=False)
    _, obad = oracle.factor(S, _oracle_K(S, lp, D, 1e-8))
    assert st == 5
    assert obad > 0 and bad == obad - 1


@pytest.mark.parametrize("name,prec,tol", [("random600", gb.IPM_FP64, 1e-8),
                                           ("grid15", gb.IPM_FP64, 1e-8),
                                           ("grid15", gb.IPM_FP32, 1e-6)])
def test_ipm_matches_oracle(name, prec, tol):
    lp, perm = _problem(name)
    ctx, info = _ctx(lp, perm, precision=prec, tol=tol, storage_fp64=1 if prec == 0 else 0)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    ref = oracle.ipm_lp(S, lp, tol=tol)
    assert ref["status"] == 0
    mt = lp.m + 2 * lp.n
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")
    res = ctx.ipm_solve(dev(lp.val), dev(lp.b), dev(lp.c), x, s, lam)
    assert res.status == 0, res.as_dict()
    assert res.kkt <= tol
    assert abs(res.objective - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    xs, ss, ls = x.cpu().numpy(), s.cpu().numpy(), lam.cpu().numpy()
    assert np.all(ss > 0) and np.all(ls > 0)
    assert abs(lp.c @ xs - res.objective) <= 1e-9 * abs(res.objective)


def test_small_lp_workload():
    """n=2000, m=1000, 5 nonzeros per row, FP64, tol 1e-8 (the small random LP)."""
    lp = gen.random_lp(2000, 1000, 5, seed=0)
    perm = gen.lp_ordering(lp)
    ctx, info = _ctx(lp, perm, precision=gb.IPM_FP64, tol=1e-8)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    ref = oracle.ipm_lp(S, lp, tol=1e-8)
    mt = lp.m + 2 * lp.n
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")
    res = ctx.ipm_solve(dev(lp.val), dev(lp.b), dev(lp.c), x, s, lam)
    assert res.status == 0 and res.kkt <= 1e-8
    assert abs(res.objective - ref["objective"]) <= 1e-6 * abs(ref["objective"])


def test_solve_problem_matches_ipm_solve():
    """ipm_solve_problem with an LP description gives ipm_solve's result bit
    for bit (the same path), and refuses an unknown kind."""
    lp = gen.grid_lp(8, seed=41)
    perm = gen.nd_order_grid3d(8)
    out = []
    for use_struct in (False, True):
        ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                            options=gb.default_options(precision=gb.IPM_TF32X3, storage_fp64=0,
                                                       tol=1e-8))
        ctx.kkt_analyze(perm)
        ctx.ipm_set_workspace()
        x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        s = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        lam = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        jv, b, c = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (lp.val, lp.b, lp.c))
        if use_struct:
            res = ctx.ipm_solve_problem(x, s, lam, jvals=jv, b=b, c=c)
            p = gb.ProblemDesc()
            p.kind = 7
            assert ctx._lib.ipm_solve_problem(ctx.handle, gb.C.byref(p), gb._dp(x), gb._dp(s),
                                              gb._dp(lam), None) == 1
        else:
            res = ctx.ipm_solve(jv, b, c, x, s, lam)
        assert res.status == 0
        out.append((res.objective, res.iterations, x.cpu().numpy()))
        ctx.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_cg_escalation_moves_to_split_tf32_and_matches_oracle():
    """cg_escalate: a TF32 factor whose iteration needs more CG steps than the
    limit moves ipm_solve to the split TF32 for the rest (counted once in
    fp64_fallbacks), and the solve still reaches the oracle's optimum; with the
    limit off the same TF32 solve never escalates on CG steps."""
    G = 14
    lp = gen.grid_lp(G, seed=43)
    perm = gen.nd_order_grid3d(G)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None)
    ref = oracle.ipm_lp(S, lp, tol=1e-8)
    out = {}
    for esc in (0, 2):
        ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                            options=gb.default_options(precision=gb.IPM_TF32, storage_fp64=0,
                                                       tol=1e-8, fallback_fp64=1,
                                                       cg_escalate=esc))
        ctx.kkt_analyze(perm)
        ctx.ipm_set_workspace()
        x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        s = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        lam = torch.empty(ctx.m_tot, dtype=torch.float64, device="cuda")
        jv, b, c = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (lp.val, lp.b, lp.c))
        res = ctx.ipm_solve(jv, b, c, x, s, lam)
        out[esc] = res
        assert res.status == 0, res.as_dict()
        assert res.objective == pytest.approx(ref["objective"], rel=1e-6)
        ctx.close()
    assert out[2].fp64_fallbacks == 1
    assert out[2].pcg_steps < out[0].pcg_steps


@pytest.mark.parametrize("where", ["c", "jvals"])
def test_nan_in_the_data_is_reported(where):
    """A NaN in c makes the objective and the KKT residual NaN: ipm_solve stops
    with IPM_ERR_NUMERIC at once instead of factoring. A NaN in J's values
    reaches K (its row's slack starts at max(g, 1) = 1): the solve fails
    (a NaN pivot or residual), it never reports an optimum."""
    lp, perm = _problem("grid7x9x5")
    ctx, info = _ctx(lp, perm, precision=gb.IPM_FP64, storage_fp64=1, tol=1e-8)
    c, val = lp.c.copy(), lp.val.copy()
    (c if where == "c" else val)[3] = np.nan
    mt = lp.m + 2 * lp.n
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")
    res = ctx.ipm_solve(dev(val), dev(lp.b), dev(c), x, s, lam)
    if where == "c":
        assert res.status == 6, res.as_dict()  # IPM_ERR_NUMERIC
        assert res.factorizations == 0
    else:
        assert res.status != 0, res.as_dict()
