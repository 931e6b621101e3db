"""The bounded waits of the persistent solve run out, and the context recovers.

An abandoned task (the test hook of kkt_test_solve_timeout: the first or the
second forward task of the solve's order) stands in for a result that never
arrives; with a short poll limit the tasks waiting for it give up, record the
timeout, and the launch drains. Nothing faults or hangs: the kernel ends, kkt_solve reports
IPM_ERR_TIMEOUT, and the next solves are correct."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402

IPM_ERR_TIMEOUT = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("withheld", [0, 1])
def test_solve_barrier_timeout_is_reported_and_recovered(withheld):
    G = 12
    lp = gen.grid_lp(G, seed=2)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                        options=gb.default_options(precision=gb.IPM_TF32X3, storage_fp64=0))
    ctx.kkt_analyze(gen.nd_order_grid3d(G))
    ctx.ipm_set_workspace()
    mt = lp.m + 2 * lp.n
    D = 10.0 ** gen.uniform(gen.stream_seed(3, 1), mt, -1.0, 1.0)
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    ctx.kkt_factor(gb.IPM_TF32X3)
    A = sp.csr_matrix((lp.val, lp.col, lp.rowptr), shape=(lp.m, lp.n))
    K = A.T @ sp.diags(D[:lp.m]) @ A + sp.diags(D[lp.m:lp.m + lp.n] + D[lp.m + lp.n:] + 1e-8)
    b = gen.normal(4, lp.n)
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")

    ctx.kkt_test_solve_timeout(spins=2000, withheld_task=withheld)
    st = ctx._lib.kkt_solve(ctx.handle, gb._dp(dev(b)), gb._dp(x), 1, gb.IPM_REFINE_NONE, None)
    torch.cuda.synchronize()  # the launch ended: the stream drains
    assert st == IPM_ERR_TIMEOUT
    assert "bounded wait" in ctx._lib.ipm_last_error(ctx.handle).decode()

    # the next solves run to the FP64 target
    for _ in range(2):
        si = ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_IR)
        r = np.abs(K @ x.cpu().numpy() - b).max() / np.abs(b).max()
        assert si.rel_residual <= 1e-10 and r <= 1e-9
