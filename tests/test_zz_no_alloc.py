"""The allocation-free solve (kkt_solve_noalloc) through the C ABI.

Some callers cannot allocate device memory at the moment they need a solve (a
locked or exhausted memory pool, another library's allocation-free callback, a
framework allocator that must not be re-entered). kkt_solve_noalloc serves them
from a static device array; these tests check it against kkt_solve without
refinement, against a host FP64 residual with the oracle's matrix, and that the
calls commit no device memory. Collected last on purpose: every call shares the
one static array, and a run that stops at the first failure has then already
run every other test. Passes alone in a fresh process as well."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402

# normwise backward error ||K x - b|| / (||K|| ||x|| + ||b||) (inf-norms) of one
# unrefined solve, per factor arithmetic (TF32 keeps 10 mantissa bits)
BACKWARD = {gb.IPM_FP64: 1e-13, gb.IPM_FP32: 1e-5, gb.IPM_TF32: 2e-2, gb.IPM_TF32X3: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    oracle.build()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", [gb.IPM_FP64, gb.IPM_FP32, gb.IPM_TF32, gb.IPM_TF32X3],
                         ids=["fp64", "fp32", "tf32", "tf32x3"])
def test_noalloc_solve_matches_kkt_solve_twice(prec):
    g = 14
    lp = gen.grid_lp(g, seed=7)
    perm = gen.nd_order_grid3d(g)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                        options=gb.default_options(storage_fp64=1))
    ctx.kkt_analyze(perm)
    ctx.ipm_set_workspace()
    mt = lp.m + 2 * lp.n
    D = 10.0 ** gen.uniform(5, mt, -2.0, 2.0)
    ctx.kkt_assemble(_dev(lp.val), _dev(D), 1e-8)
    ctx.kkt_factor(prec)
    # the oracle's K (FP64, host) for the residuals
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, perm)
    kval = oracle.assemble(S, lp.m, lp.rowptr, lp.col, lp.val, D[:lp.m],
                           D[lp.m:lp.m + lp.n] + D[lp.m + lp.n:], 1e-8)
    K = oracle.k_dense(S, kval)
    knorm = np.abs(K).sum(axis=1).max()
    bs = [_dev(gen.normal(seed, lp.n)) for seed in (8, 9)]
    refs = []
    for b in bs:
        x_ref = torch.empty_like(b)
        ctx.kkt_solve(b, x_ref, gb.IPM_REFINE_NONE, raise_on_error=False)
        refs.append(x_ref)
    xs = [torch.full_like(b, float("nan")) for b in bs]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for call, (b, x) in enumerate(zip(bs, xs)):  # two calls in a row, different right-hand sides
        ctx.kkt_solve_noalloc(b, x)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device memory changed by {free0 - free1} bytes"
    for call, (b, x, x_ref) in enumerate(zip(bs, xs, refs)):
        xr, xn, bh = x_ref.cpu().numpy(), x.cpu().numpy(), b.cpu().numpy()
        tol = 1e-12 if prec == gb.IPM_FP64 else 1e-5
        np.testing.assert_allclose(xn, xr, rtol=0, atol=tol * np.abs(xr).max(),
                                   err_msg=f"call {call}")
        eta = np.abs(K @ xn - bh).max() / (knorm * np.abs(xn).max() + np.abs(bh).max())
        assert eta <= BACKWARD[prec], f"call {call}: backward error {eta:.2e}"


def test_noalloc_rejects_problems_beyond_the_static_array():
    g = 56
    lp = gen.grid_lp(g, seed=1)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u)
    ctx.kkt_analyze(gen.nd_order_grid3d(g))
    b = torch.zeros(lp.n, dtype=torch.float64, device="cuda")
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    st = ctx.kkt_solve_noalloc(b, x, raise_on_error=False)
    assert st == 4  # IPM_ERR_NOMEM, before any GPU work
    assert "limit" in gb.load().ipm_last_error(ctx.handle).decode()
    assert gb.load().kkt_solve_noalloc_capacity() == 1 << 20
