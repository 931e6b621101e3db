"""Grid NLP on the GPU against the FP64 oracle (same rules: monotone barrier,
common step with merit backtracking, inertia by regularisation)."""
import numpy as np
import pytest

import gen
import oracle
from oracle import nlp as ON

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_16094_gb300 as gb  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _solve(P, precision=0, tol=1e-8, **kw):
    o = gb.default_options(precision=precision, tol=tol, max_iter=200,
                           storage_fp64=1, **kw)
    G = gb.GridNLP(P.N, perm=gen.nd_order_grid_nlp(P.N), alpha=P.alpha, v_lo=P.v_lo, v_hi=P.v_hi,
                   cubic=P.cubic, v_bounded=P.v_bounded, options=o)
    n, mt = G.pat["n"], G.ctx.m_tot
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")
    res = G.ipm_solve_grid_nlp(dev(P.ut), x, s, lam)
    return res, x.cpu().numpy(), s.cpu().numpy(), lam.cpu().numpy()


def _oracle(P, tol=1e-8):
    S = oracle.analyze(P.n, P.m, P.rowptr, P.col, gen.nd_order_grid_nlp(P.N), P.wp, P.wi)
    return ON.ipm_grid_nlp(S, P, tol=tol, max_iter=200)


@pytest.mark.parametrize("N", [16, 23])
def test_fp64_matches_oracle(N):
    P = gen.grid_nlp(N, seed=31)
    res, x, s, lam = _solve(P)
    ref = _oracle(P)
    assert res.status == 0 and ref["status"] == 0
    assert res.kkt <= 1e-8
    assert res.objective == pytest.approx(ref["objective"], rel=1e-6)
    # the equality pairs make the interior degenerate (both slacks vanish), so a
    # KKT residual of 1e-8 pins x only loosely; the objective is the contract
    assert np.max(np.abs(x - ref["x"])) <= 1e-3 * max(1.0, np.max(np.abs(ref["x"])))
    assert np.all(s > 0) and np.all(lam > 0)
    assert abs(res.iterations - ref["iterations"]) <= 2


def test_fp64_tensor_core_factor_matches_oracle():
    """FP64 factorisations with the updates on the tensor cores (fp64_tc): the
    grid NLP's K spans many decades within a row, and a pivot the slices make
    non-positive is redone on the FMA pipe before delta_p is raised, so the
    regularisations stay those of the FMA-pipe FP64 solve and the optimum is the oracle's."""
    P = gen.grid_nlp(40, seed=35)
    out = []
    for tc in (0, 1):
        res, x, s, lam = _solve(P, tol=1e-7, fp64_tc=tc)
        assert res.status == 0 and res.kkt <= 1e-7, res.as_dict()
        out.append(res)
    ref = _oracle(P, tol=1e-7)
    assert out[1].objective == pytest.approx(ref["objective"], rel=1e-6)
    assert out[1].regularizations <= out[0].regularizations + 2
    assert out[0].fp64_tc_rechecks == 0


def test_without_cubic_term_matches_equality_qp():
    P = gen.grid_nlp(20, seed=32, cubic=0, v_bounded=0)
    res, x, _, _ = _solve(P, tol=1e-9)
    f_ref, u_ref, _ = ON.equality_qp_solution(P)
    assert res.status == 0
    assert res.objective == pytest.approx(f_ref, rel=1e-7)
    assert np.max(np.abs(x[:400] - u_ref)) < 1e-5 * max(1.0, np.max(np.abs(u_ref)))


def test_split_tf32_factor_matches_oracle():
    P = gen.grid_nlp(40, seed=33)
    res, x, _, _ = _solve(P, precision=4, tol=1e-6, fallback_fp64=1)
    ref = _oracle(P, tol=1e-6)
    assert res.status == 0 and res.kkt <= 1e-6
    assert res.objective == pytest.approx(ref["objective"], rel=1e-6)


def test_bf16_factor_with_fallback_matches_oracle():
    """BF16 factors with the FP64 fallback: a step after which the KKT residual
    grows tenfold is taken back and redone in FP64, so the solve still reaches
    the oracle's optimum."""
    P = gen.grid_nlp(40, seed=34)
    res, x, s, lam = _solve(P, precision=gb.IPM_BF16, tol=1e-6, fallback_fp64=1)
    ref = _oracle(P, tol=1e-6)
    assert res.status == 0 and res.kkt <= 1e-6
    assert res.objective == pytest.approx(ref["objective"], rel=1e-6)
    assert np.all(s > 0) and np.all(lam > 0)


def test_callback_nlp_matches_grid_path():
    """ipm_solve_nlp with the problem given by callbacks (here the oracle's FP64
    evaluation of the grid NLP, copied to the device) reaches the optimum of
    the library's own grid-NLP path and of the oracle; a failing callback ends
    the solve with IPM_ERR_NUMERIC."""
    P = gen.grid_nlp(16, seed=35)
    o = gb.default_options(precision=0, tol=1e-8, max_iter=200, storage_fp64=1)
    G = gb.GridNLP(P.N, perm=gen.nd_order_grid_nlp(P.N), alpha=P.alpha, v_lo=P.v_lo, v_hi=P.v_hi,
                   cubic=P.cubic, v_bounded=P.v_bounded, options=o)
    n, mt = G.pat["n"], G.ctx.m_tot
    m = G.pat["m"]

    def bufs():
        return (torch.empty(n, dtype=torch.float64, device="cuda"),
                torch.empty(mt, dtype=torch.float64, device="cuda"),
                torch.empty(mt, dtype=torch.float64, device="cuda"))

    x1, s1, l1 = bufs()
    r1 = G.ipm_solve_grid_nlp(dev(P.ut), x1, s1, l1)

    def ev(x, f, grad, g, jv):
        fx, h, jvals, gr = ON.evaluate(P, x.cpu().numpy())
        f.copy_(torch.tensor([fx], dtype=torch.float64))
        grad.copy_(torch.as_tensor(gr))
        g.copy_(torch.as_tensor(ON.h_rows(h)))
        jv.copy_(torch.as_tensor(jvals))

    def hs(x, lam, wv):
        wv.copy_(torch.as_tensor(ON.hessian_diag(P, x.cpu().numpy(), lam.cpu().numpy()[:m])))

    x2, s2, l2 = bufs()
    r2 = G.ctx.ipm_solve_nlp(ev, hs, x2, s2, l2)
    ref = _oracle(P)
    assert r1.status == 0 and r2.status == 0, (r1.as_dict(), r2.as_dict())
    assert r2.kkt <= 1e-8
    # a KKT residual of 1e-8 fixes the objective to about that relative accuracy
    # (the evaluations differ in rounding: numpy on the host against the kernels)
    assert r2.objective == pytest.approx(r1.objective, rel=1e-7)
    assert r2.objective == pytest.approx(ref["objective"], rel=1e-6)
    assert abs(r2.iterations - r1.iterations) <= 2

    def bad(x, f, grad, g, jv):
        raise RuntimeError("evaluation failed")

    x3, s3, l3 = bufs()
    assert G.ctx.ipm_solve_nlp(bad, hs, x3, s3, l3).status == 6  # IPM_ERR_NUMERIC


def test_rejects_foreign_pattern():
    lp = gen.grid_lp(4, seed=1)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u)
    ctx.kkt_analyze(None)
    ctx.ipm_set_workspace()
    G = gb.ipm_grid_nlp_pattern(4)
    x = torch.zeros(lp.n, dtype=torch.float64, device="cuda")
    s = torch.zeros(ctx.m_tot, dtype=torch.float64, device="cuda")
    st = ctx._lib.ipm_solve_grid_nlp(ctx.handle, gb.C.byref(G["params"]), gb._dp(x), gb._dp(x),
                                     gb._dp(s), gb._dp(s), None)
    assert st == 1  # IPM_ERR_ARG
