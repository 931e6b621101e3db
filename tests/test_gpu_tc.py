"""Tensor-core (tcgen05: TF32, split TF32, BF16) factorisation vs the CPU oracle.

TF32 keeps 10 explicit mantissa bits, so the factor itself is only accurate to
about 1e-3 relative; FP64 refinement must then recover a 1e-10 solve residual
and the interior-point method the oracle's objective. Fronts of the 15^3 grid
span 4 block columns of 128 (450-column top separator) and several K tiles."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402
from tests.test_gpu_parity import _ctx, _oracle_K, _problem, _state, dev  # noqa: E402

TF32_BACKWARD = 5e-3  # ||L L^T - K||_F / ||K||_F allowed for a TF32 factor (unit roundoff 2^-11)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    oracle.build()


def _dense_factor(ctx, S, n):
    cols = np.repeat(np.arange(n), np.diff(S.lp) + 1).astype(np.int32)
    rows = np.empty_like(cols)
    for j in range(n):
        b = S.lp[j] + j
        rows[b] = j
        rows[b + 1: b + 1 + S.lp[j + 1] - S.lp[j]] = S.li[S.lp[j]:S.lp[j + 1]]
    L = np.zeros((n, n))
    L[rows, cols] = ctx.kkt_factor_entries(rows, cols)
    return L


TF32X3_BACKWARD = 2e-6  # 3-term split: products about as accurate as FP32 FMA
# BF16 keeps 7 explicit mantissa bits (unit roundoff 2^-8 for the operands of
# the updates); the panel solves stay TF32 and the diagonal blocks FP32
BF16_BACKWARD = 2e-2


@pytest.mark.parametrize("prec,bound", [(gb.IPM_TF32, TF32_BACKWARD), (gb.IPM_TF32X3, TF32X3_BACKWARD),
                                        (gb.IPM_BF16, BF16_BACKWARD)],
                         ids=["tf32", "tf32x3", "bf16"])
@pytest.mark.parametrize("name", ["grid15", "random600", "grid7x9x5"])
def test_tf32_factor_backward_error(name, prec, bound):
    lp, perm = _problem(name)
    ctx, info = _ctx(lp, perm, precision=prec, storage_fp64=0)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    D = _state(lp, 2, spread=1.0)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    st, bad = ctx.kkt_factor(prec)
    assert st == 0 and ctx.ipm_last_perturbed() == 0
    K = oracle.k_dense(S, _oracle_K(S, lp, D, 1e-8), final=True)
    L = _dense_factor(ctx, S, lp.n)
    err = np.linalg.norm(L @ L.T - K) / np.linalg.norm(K)
    assert err <= bound
    if prec == gb.IPM_TF32:
        assert err >= 1e-5  # the products really ran in TF32
    if prec == gb.IPM_BF16:  # the updates really ran in BF16: coarser than TF32
        ctx.kkt_factor(gb.IPM_TF32)
        Lt = _dense_factor(ctx, S, lp.n)
        err_tf32 = np.linalg.norm(Lt @ Lt.T - K) / np.linalg.norm(K)
        assert err >= 2 * err_tf32, (err, err_tf32)
    # the same factor in FP32 FMA arithmetic is far more accurate: TF32 really ran
    ctx.kkt_factor(gb.IPM_FP32)
    L32 = _dense_factor(ctx, S, lp.n)
    err32 = np.linalg.norm(L32 @ L32.T - K) / np.linalg.norm(K)
    assert err32 <= 1e-5
    lval, _ = oracle.factor(S, _oracle_K(S, lp, D, 1e-8))
    assert np.abs(L - oracle.l_dense(S, lval)).max() <= 0.05 * np.abs(lval).max()


@pytest.mark.parametrize("prec", [gb.IPM_TF32, gb.IPM_TF32X3, gb.IPM_BF16],
                         ids=["tf32", "tf32x3", "bf16"])
@pytest.mark.parametrize("name", ["grid15", "random600"])
def test_tf32_solve_refined_to_1e10(name, prec):
    lp, perm = _problem(name)
    ctx, info = _ctx(lp, perm, precision=prec, storage_fp64=0)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    # BF16 updates break down (perturbed pivots) on K this badly conditioned;
    # they are refined from a factor of a matrix whose D spans two decades
    D = _state(lp, 3, spread=1.0 if prec == gb.IPM_BF16 else 3.0)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    ctx.kkt_factor(prec)
    assert ctx.ipm_last_perturbed() == 0
    b = gen.normal(4, lp.n)
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    info = ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_IR)
    assert info.rel_residual <= 1e-10
    K = oracle.k_dense(S, _oracle_K(S, lp, D, 1e-8))
    assert np.abs(K @ x.cpu().numpy() - b).max() <= 4e-10 * np.abs(b).max()


@pytest.mark.parametrize("prec", [gb.IPM_TF32, gb.IPM_TF32X3, gb.IPM_BF16],
                         ids=["tf32", "tf32x3", "bf16"])
@pytest.mark.parametrize("name", ["grid15", "random600"])
def test_tf32_ipm_matches_oracle(name, prec):
    lp, perm = _problem(name)
    # a BF16 factor whose PCG misses the acceptance tolerance is redone in split TF32
    ctx, info = _ctx(lp, perm, precision=prec, storage_fp64=0, tol=1e-6,
                     fallback_fp64=1 if prec == gb.IPM_BF16 else 0)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    ref = oracle.ipm_lp(S, lp, tol=1e-6)
    mt = lp.m + 2 * lp.n
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")
    res = ctx.ipm_solve(dev(lp.val), dev(lp.b), dev(lp.c), x, s, lam)
    assert res.status == 0, res.as_dict()
    assert res.kkt <= 1e-6
    assert abs(res.objective - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    if prec == gb.IPM_BF16:  # BF16 factors carried some iterations themselves
        assert res.fp64_fallbacks < res.iterations, res.as_dict()
