"""The dual condensed (6) and augmented (4) formulations on the GPU against the
oracle (oracle/forms.py), element by element, through the C ABI.

Per formulation: the assembled system matrix, the factor (Cholesky of (6);
the signed pivot-free factor L S L^T of the quasi-definite (4), compared with
the oracle's L D L^T as L |D|^{1/2}), refined solves, the Newton direction
(equal to the primal condensed one of (5)), and whole interior-point solves
(objective within 1e-6 of the oracle's, KKT residual within tolerance)."""
import numpy as np
import pytest

import gen
import oracle
from oracle import forms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402

FORM = {"dual": gb.IPM_FORM_DUAL, "augmented": gb.IPM_FORM_AUGMENTED}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    oracle.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _problem(name, form):
    if name == "grid7x9x5":
        lp = gen.grid_lp(7, 9, 5, seed=12)
        nd = gen.nd_order_grid3d(7, 9, 5)
    elif name == "grid12":
        lp = gen.grid_lp(12, seed=21)
        nd = gen.nd_order_grid3d(12)
    else:  # random LP, natural ordering
        lp = gen.random_lp(600, 300, 5, seed=13)
        return lp, None
    if form == "dual":
        return lp, nd
    return lp, np.concatenate([[p, lp.n + p] for p in nd]).astype(np.int32)


def _point(lp, seed, spread=1.0):
    mt = lp.m + 2 * lp.n
    x = gen.uniform(seed, lp.n, 0.5, 9.5)
    s = 10.0 ** gen.uniform(seed + 1, mt, -spread, spread)
    lam = 10.0 ** gen.uniform(seed + 2, mt, -spread, spread)
    return x, s, lam


def _ctx(lp, perm, form, **opt):
    o = gb.default_options(formulation=FORM[form], **opt)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
    info = ctx.kkt_analyze(perm)
    ctx.ipm_set_workspace()
    return ctx, info


def _assemble(ctx, lp, s, lam, dp=1e-8, dd=1e-8):
    D = 1.0 / (dd + s / lam)
    ctx.kkt_assemble(dev(lp.val), dev(D), dp)
    return D


def _oracle_system(form, lp, s, lam, x, perm):
    if form == "dual":
        S, kval, _ = forms.dual_system(lp, s, lam, x, 1e-8, 1e-8, perm)
        return S, kval, None
    return forms.augmented_system(lp, s, lam, x, 1e-8, 1e-8, perm)


@pytest.mark.parametrize("form", ["dual", "augmented"])
@pytest.mark.parametrize("name", ["grid7x9x5", "random600"])
def test_assembly_matches_oracle(form, name):
    lp, perm = _problem(name, form)
    ctx, info = _ctx(lp, perm, form)
    x, s, lam = _point(lp, 3, spread=2.0)
    _assemble(ctx, lp, s, lam)
    got = ctx.kkt_export_assembled()
    S, kval, _ = _oracle_system(form, lp, s, lam, x, perm)
    assert got.size == kval.size
    np.testing.assert_allclose(got, kval, rtol=1e-13, atol=1e-15 * np.abs(kval).max())


def _factor_entries(ctx, S, n):
    cols = np.repeat(np.arange(n), np.diff(S.lp) + 1).astype(np.int32)
    rows = np.empty_like(cols)
    for j in range(n):
        b = S.lp[j] + j
        rows[b] = j
        rows[b + 1: b + 1 + S.lp[j + 1] - S.lp[j]] = S.li[S.lp[j]:S.lp[j + 1]]
    return rows, cols, ctx.kkt_factor_entries(rows, cols)


@pytest.mark.parametrize("prec,tc", [(gb.IPM_FP64, 0), (gb.IPM_FP32, 0), (gb.IPM_FP64, 1)],
                         ids=["fp64", "fp32", "fp64_tc"])
@pytest.mark.parametrize("form", ["dual", "augmented"])
@pytest.mark.parametrize("name", ["grid7x9x5", "random600"])
def test_factor_matches_oracle(form, name, prec, tc):
    """fp64_tc: the SPD system of (6) takes the tensor-core FP64 updates; the
    signed LDL^T of (4) keeps the FMA path."""
    lp, perm = _problem(name, form)
    ctx, info = _ctx(lp, perm, form, storage_fp64=1, fp64_tc=tc)
    x, s, lam = _point(lp, 4)
    _assemble(ctx, lp, s, lam)
    st, bad = ctx.kkt_factor(prec)
    assert st == 0 and bad == -1 and ctx.ipm_last_perturbed() == 0
    S, kval, sign = _oracle_system(form, lp, s, lam, x, perm)
    n = S.n
    rows, cols, got = _factor_entries(ctx, S, n)
    if form == "dual":
        lval, bad = oracle.factor(S, kval)
        want = lval
    else:  # L S L^T with L = L_ldl |d|^{1/2} (column scaling)
        lval, dval, bad = oracle.factor_ldlt(S, kval, sign)
        want = lval * np.sqrt(np.abs(dval))[cols]
    assert bad == 0
    tol = 1e-11 if prec == gb.IPM_FP64 else 2e-4
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("form", ["dual", "augmented"])
@pytest.mark.parametrize("name", ["grid7x9x5", "random600"])
def test_refined_solve(form, name):
    lp, perm = _problem(name, form)
    ctx, info = _ctx(lp, perm, form, storage_fp64=0)
    x, s, lam = _point(lp, 5, spread=2.0)
    _assemble(ctx, lp, s, lam)
    ctx.kkt_factor(gb.IPM_FP32)
    S, kval, _ = _oracle_system(form, lp, s, lam, x, perm)
    b = gen.normal(6, S.n)
    xs = torch.empty(S.n, dtype=torch.float64, device="cuda")
    si = ctx.kkt_solve(dev(b), xs, gb.IPM_REFINE_IR)
    r = oracle.kmatvec(S, kval, xs.cpu().numpy()) - b
    assert si.rel_residual <= 1e-10 and np.abs(r).max() <= 4e-10 * np.abs(b).max()


@pytest.mark.parametrize("form", ["dual", "augmented"])
@pytest.mark.parametrize("name", ["grid7x9x5", "random600"])
def test_newton_direction_matches_oracle(form, name):
    lp, perm = _problem(name, form)
    ctx, info = _ctx(lp, perm, form, storage_fp64=1)
    x, s, lam = _point(lp, 7, spread=1.5)
    mt = lp.m + 2 * lp.n
    w = gen.uniform(8, mt, 0.0, 0.5)
    dx, ds, dl = (torch.empty(k, dtype=torch.float64, device="cuda") for k in (lp.n, mt, mt))
    ctx.ipm_newton_direction(dev(lp.val), dev(lp.b), dev(lp.c), dev(x), dev(s), dev(lam), dev(w),
                             dx, ds, dl)
    fn = forms.dual_direction if form == "dual" else forms.augmented_direction
    rx, rs, rl = fn(lp, x, s, lam, w, 1e-8, 1e-8, perm)
    Sp = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None)
    px, ps, pl = oracle.lp_direction(Sp, lp, x, s, lam, w)  # the primal condensed (5)
    for a, r, p in [(dx, rx, px), (ds, rs, ps), (dl, rl, pl)]:
        a = a.cpu().numpy()
        np.testing.assert_allclose(a, r, rtol=1e-8, atol=1e-10 * np.abs(r).max())
        np.testing.assert_allclose(a, p, rtol=1e-8, atol=1e-10 * np.abs(p).max())


CASES = [("dual", gb.IPM_FP64), ("dual", gb.IPM_TF32X3), ("augmented", gb.IPM_FP64),
         ("augmented", gb.IPM_FP32)]


@pytest.mark.parametrize("form,prec", CASES, ids=[f"{f}-{p}" for f, p in CASES])
@pytest.mark.parametrize("name", ["grid12", "random600"])
def test_ipm_matches_oracle(form, prec, name):
    lp, perm = _problem(name, form)
    # the FP32 LDL^T of the quasi-definite system loses accuracy as the
    # multiplier block spans more decades: it falls back to FP64 when a solve
    # misses its tolerance
    fb = form == "augmented" and prec == gb.IPM_FP32
    ctx, info = _ctx(lp, perm, form, precision=prec,
                     storage_fp64=1 if (prec == gb.IPM_FP64 or fb) else 0, tol=1e-8,
                     fallback_fp64=1 if fb else 0)
    Sp = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None)
    ref = oracle.ipm_lp(Sp, lp, tol=1e-8)
    mt = lp.m + 2 * lp.n
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")
    res = ctx.ipm_solve(dev(lp.val), dev(lp.b), dev(lp.c), x, s, lam)
    assert res.status == 0, res.as_dict()
    assert res.kkt <= 1e-8
    assert abs(res.objective - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    if fb:  # the FP32 factor carried the early iterations itself
        assert res.fp64_fallbacks <= 1 and res.factorizations > res.fp64_fallbacks + 2


def test_augmented_rejects_tensor_core_precisions():
    lp, perm = _problem("grid7x9x5", "augmented")
    ctx, info = _ctx(lp, perm, "augmented", storage_fp64=0)
    x, s, lam = _point(lp, 9)
    _assemble(ctx, lp, s, lam)
    st, _ = ctx.kkt_factor(gb.IPM_TF32X3, raise_on_error=False)
    assert st == 10  # IPM_ERR_UNSUPPORTED: the signed factor runs in FP64 or FP32
