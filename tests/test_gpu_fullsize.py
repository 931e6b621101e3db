"""Parity at the benchmark's full sizes, in the configuration bench.py times
(100^3 grid LP, split-TF32 factor stored in FP32; the 4096-instance MPC batch),
on sampled outputs the definitions give one by one and on properties that
hold at any size (residuals recomputed on the host in FP64)."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_16094_gb300 as gb  # noqa: E402

G = 100


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def grid100():
    lp = gen.grid_lp(G, seed=1)
    o = gb.default_options(precision=gb.IPM_TF32X3, storage_fp64=0, tol=1e-6)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u, options=o)
    ctx.kkt_analyze(gen.nd_order_grid3d(G))
    ctx.ipm_set_workspace()
    A = sp.csr_matrix((lp.val, lp.col, lp.rowptr), shape=(lp.m, lp.n))
    D = 10.0 ** gen.uniform(gen.stream_seed(77, 1), lp.m + 2 * lp.n, -2.0, 2.0)
    dex = D[lp.m:lp.m + lp.n] + D[lp.m + lp.n:]
    K = (A.T @ sp.diags(D[:lp.m]) @ A + sp.diags(dex + 1e-8)).tocsr()
    absK = (abs(A).T @ sp.diags(D[:lp.m]) @ abs(A) + sp.diags(dex + 1e-8)).tocsr()
    yield dict(lp=lp, ctx=ctx, A=A, D=D, K=K, absK=absK)
    ctx.close()


def test_assembly_sampled_entries(grid100):
    """K entries in the original lower pattern (column-major, diagonal first)
    against A^T D A + diag on 20000 sampled entries."""
    d = grid100
    lp, ctx, K, absK = d["lp"], d["ctx"], d["K"], d["absK"]
    ctx.kkt_assemble(dev(lp.val), dev(d["D"]), 1e-8)
    got = ctx.kkt_export_assembled()
    Kl = sp.tril(K).tocsc()
    Kl.sort_indices()
    # pattern order: per column j the diagonal, then the rows below in ascending order
    assert got.size == Kl.nnz
    cols = np.repeat(np.arange(lp.n), np.diff(Kl.indptr))
    rows = Kl.indices
    assert np.all(rows[Kl.indptr[:-1]] == np.arange(lp.n))  # diagonal first
    idx = gen.splitmix64(91, 20000) % np.uint64(got.size)
    idx = idx.astype(np.int64)
    want = np.asarray(K[rows[idx], cols[idx]]).ravel()
    bound = 8 * np.finfo(float).eps * np.asarray(absK[rows[idx], cols[idx]]).ravel()
    assert np.all(np.abs(got[idx] - want) <= bound)


def test_split_tf32_factor_solve_residual_on_host(grid100):
    """The bench configuration: factor in split TF32, solve with FP64
    refinement; the residual recomputed on the host in FP64 meets 1e-9."""
    d = grid100
    lp, ctx, K = d["lp"], d["ctx"], d["K"]
    ctx.kkt_assemble(dev(lp.val), dev(d["D"]), 1e-8)
    st, bad = ctx.kkt_factor(gb.IPM_TF32X3)
    assert st == 0 and bad == -1
    b = gen.normal(92, lp.n)
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    info = ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_IR)
    xs = x.cpu().numpy()
    r = np.abs(K @ xs - b).max() / np.abs(b).max()
    assert info.rel_residual <= 1e-10 and r <= 1e-9, (info.rel_residual, r)
    # one unrefined solve has the normwise backward error of a split-TF32
    # factor (near FP32 rounding): a dropped or doubled update of the
    # super-step schedule would leave errors of the size of the entries
    info0 = ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_NONE, raise_on_error=False)
    x0 = x.cpu().numpy()
    knorm = abs(K).sum(axis=1).max()
    eta = np.abs(K @ x0 - b).max() / (knorm * np.abs(x0).max() + np.abs(b).max())
    assert eta <= 1e-5, eta
    assert info0.rel_residual < 1e-2
    assert ctx.ipm_last_perturbed() == 0


def test_newton_direction_satisfies_condensed_system(grid100):
    """At an interior iterate of the bench problem, the direction solves Eq. (5)
    and recovers d_lambda, d_s as Eq. (3) prescribes (checked on the host)."""
    d = grid100
    lp, ctx, A = d["lp"], d["ctx"], d["A"]
    n, m, mt = lp.n, lp.m, lp.m + 2 * lp.n
    x = gen.uniform(gen.stream_seed(93, 1), n, 0.5, 9.5)
    s = 10.0 ** gen.uniform(gen.stream_seed(93, 2), mt, -1.0, 1.0)
    lam = 10.0 ** gen.uniform(gen.stream_seed(93, 3), mt, -1.0, 1.0)
    w = np.full(mt, 0.1)
    dx, ds, dl = (torch.empty(k, dtype=torch.float64, device="cuda") for k in (n, mt, mt))
    ctx.ipm_newton_direction(dev(lp.val), dev(lp.b), dev(lp.c), dev(x), dev(s), dev(lam), dev(w),
                             dx, ds, dl)
    dx, ds, dl = dx.cpu().numpy(), ds.cpu().numpy(), dl.cpu().numpy()
    # g and J over all rows: general rows, x - l, u - x
    g = np.concatenate([A @ x - lp.b, x - lp.l, lp.u - x])
    Jdx = np.concatenate([A @ dx, dx, -dx])
    D = 1.0 / (1e-8 + s / lam)
    # rows 2-3 of the Newton system (3)
    np.testing.assert_allclose(dl, D * (w / lam - g - Jdx), rtol=1e-9, atol=1e-12 * np.abs(dl).max())
    np.testing.assert_allclose(ds, -s + w / lam - (s / lam) * dl, rtol=1e-9,
                               atol=1e-12 * np.abs(ds).max())
    # row 1: grad f - J^T (lambda + d_lambda) = 0 up to the linear-solve residual
    def JT(v):
        return A.T @ v[:m] + v[m:m + n] - v[m + n:]
    r1 = lp.c - JT(lam + dl)
    scale = np.abs(lp.c).max() + np.abs(JT(np.abs(lam + dl))).max()
    assert np.abs(r1).max() <= 1e-8 * scale


def test_mpc_full_batch_converges_and_samples_match_oracle():
    """All 4096 instances of the benchmark batch converge in the autotuned launch
    shape; six sampled instances match the oracle's objective."""
    mb = gen.mpc_batch(4096, seed=3)
    b = gb.BatchedMPC(mb)
    cfg, _ = b.ipm_mpc_autotune(precision=gb.IPM_FP32, tol=1e-8)
    b.ipm_solve_batched(precision=gb.IPM_FP32, instances_per_cta=cfg.instances_per_cta,
                        ctas=cfg.ctas, tol=1e-8, max_iter=100)
    torch.cuda.synchronize()
    st = b.status.cpu().numpy()
    assert np.all(st == 0), np.flatnonzero(st)
    assert float(b.kkt.max().item()) <= 1e-8
    obj = b.obj.cpu().numpy()
    for i in (gen.splitmix64(94, 6) % np.uint64(4096)).astype(np.int64):
        lp, W = gen.mpc_instance_qp(*mb.instance(int(i)), u_max=mb.u_max, x_max=mb.x_max)
        S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None, W[0], W[1])
        ref = oracle.ipm_lp(S, lp, tol=1e-8, W=W)
        assert ref["status"] == 0
        assert obj[i] == pytest.approx(ref["objective"], rel=1e-6), int(i)
