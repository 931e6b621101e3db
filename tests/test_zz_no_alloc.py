"""The allocation-free solve (kkt_solve_noalloc) against kkt_solve without
refinement, through the C ABI. Collected last on purpose: it shares one static
device array across calls, and a run that stops at the first failure has then
already run every other test. Passes alone in a fresh process as well."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", [gb.IPM_FP64, gb.IPM_FP32])
def test_noalloc_solve_matches_kkt_solve_twice(prec):
    lp = gen.grid_lp(14, seed=7)
    perm = gen.nd_order_grid3d(14)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                        options=gb.default_options(storage_fp64=1))
    ctx.kkt_analyze(perm)
    ctx.ipm_set_workspace()
    mt = lp.m + 2 * lp.n
    D = 10.0 ** gen.uniform(5, mt, -2.0, 2.0)
    ctx.kkt_assemble(_dev(lp.val), _dev(D), 1e-8)
    ctx.kkt_factor(prec)
    for call, seed in enumerate((8, 9)):  # two calls in a row, different right-hand sides
        b = _dev(gen.normal(seed, lp.n))
        x_ref = torch.empty_like(b)
        ctx.kkt_solve(b, x_ref, gb.IPM_REFINE_NONE, raise_on_error=False)
        x = torch.full_like(b, float("nan"))
        ctx.kkt_solve_noalloc(b, x)
        torch.cuda.synchronize()
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        tol = 1e-12 if prec == gb.IPM_FP64 else 1e-5
        np.testing.assert_allclose(xn, xr, rtol=0, atol=tol * np.abs(xr).max(),
                                   err_msg=f"call {call}")


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
