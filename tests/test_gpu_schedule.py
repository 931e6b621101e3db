"""The tensor-core factorisation at the benchmark's schedule, against the
definition of Eq. (5).

On the grid LPs the relaxed amalgamation gives a root supernode of 1,680
(24^3), 3,008 (32^3) and 4,720 (40^3) columns: several 512-column super-steps,
and on the root level the update of the next super-step runs ahead on the
second stream. A factor that dropped or doubled such an update would leave
L L^T - K of the size of the entries it missed; a correct split-TF32 factor has
a backward error near FP32 rounding, a plain TF32 factor near 2^-11 and a
factor with BF16 updates near 2^-8.

K is built on the host from its definition (A^T diag(D_A) A + diag(D_l + D_u)
+ delta I, scipy, FP64) and permuted to the factor's final numbering."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402

SUPER = 512  # columns per super-step of the tensor-core schedule
BACKWARD = {gb.IPM_TF32X3: 2e-6, gb.IPM_TF32: 5e-3, gb.IPM_BF16: 2e-2}
# decades spanned by D: BF16 updates (unit roundoff 2^-8) break down, with
# perturbed pivots, once the pivots' cancellation exceeds their precision
SPREAD = {gb.IPM_TF32X3: 2.0, gb.IPM_TF32: 2.0, gb.IPM_BF16: 1.0}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _setup(G, prec, seed=5):
    spread = SPREAD[prec]
    lp = gen.grid_lp(G, seed=1)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                        options=gb.default_options(precision=prec, storage_fp64=0))
    info = ctx.kkt_analyze(gen.nd_order_grid3d(G))
    ctx.ipm_set_workspace()
    A = sp.csr_matrix((lp.val, lp.col, lp.rowptr), shape=(lp.m, lp.n))
    mt = lp.m + 2 * lp.n
    D = 10.0 ** gen.uniform(gen.stream_seed(seed, 1), mt, -spread, spread)
    dex = D[lp.m:lp.m + lp.n] + D[lp.m + lp.n:]
    K = (A.T @ sp.diags(D[:lp.m]) @ A + sp.diags(dex + 1e-8)).tocsr()
    ctx.kkt_assemble(dev(lp.val), dev(D), 1e-8)
    st, bad = ctx.kkt_factor(prec)
    assert st == 0 and bad == -1
    assert ctx.ipm_last_perturbed() == 0
    return lp, ctx, info, K


def _factor_csc(ctx, n):
    """All stored entries of L (final numbering) as a scipy CSC matrix."""
    ex = ctx.kkt_symbolic_export()
    sup, srp, sri = ex["super"], ex["srp"], ex["sri"]
    rows_l, cols_l = [], []
    for s in range(len(sup) - 1):
        f, nc = int(sup[s]), int(sup[s + 1] - sup[s])
        below = sri[srp[s]:srp[s + 1]]
        for t in range(nc):
            r = np.concatenate([np.arange(f + t, f + nc, dtype=np.int32), below])
            rows_l.append(r)
            cols_l.append(np.full(r.size, f + t, np.int32))
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    vals = ctx.kkt_factor_entries(rows, cols)
    return sp.csc_matrix((vals, (rows, cols)), shape=(n, n)), ex


@pytest.mark.parametrize("prec", [gb.IPM_TF32X3, gb.IPM_TF32, gb.IPM_BF16],
                         ids=["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("G", [24, 32])
def test_factor_backward_error_at_super_step_schedule(G, prec):
    lp, ctx, info, K = _setup(G, prec)
    # the schedule under test: at least three super-steps on the root front,
    # so the look-ahead stream runs
    assert info.max_ncol > 2 * SUPER
    L, ex = _factor_csc(ctx, lp.n)
    perm = ex["perm"]
    Kp = K[perm][:, perm].tocsr()
    knorm = abs(Kp).sum(axis=1).max()
    # probes: ||(L L^T - P K P^T) z|| / (||K|| ||z||)
    for seed in range(4):
        z = gen.normal(gen.stream_seed(40 + seed, 1), lp.n)
        e = L @ (L.T @ z) - Kp @ z
        eta = np.abs(e).max() / (knorm * np.abs(z).max())
        assert eta <= BACKWARD[prec], (seed, eta)
    # sampled rows of L L^T against K, half of them in the root supernode
    # (the columns the super-steps and the look-ahead compute)
    root0 = int(ex["super"][-2])  # postorder: the root supernode holds the last columns
    assert lp.n - root0 == info.max_ncol
    ex_rows = np.arange(root0, lp.n)
    pick = np.concatenate([ex_rows[gen.splitmix64(61, 24) % np.uint64(ex_rows.size)],
                           gen.splitmix64(62, 24) % np.uint64(lp.n)]).astype(np.int64)
    Lr = L.tocsr()
    worst = 0.0
    for i in pick:
        li = Lr[i].toarray().ravel()
        row = L @ li  # (L L^T)_{:, i} = L (row i of L)^T
        krow = Kp[i].toarray().ravel()
        worst = max(worst, np.abs(row - krow).max() / np.abs(krow).max())
    assert worst <= 20 * BACKWARD[prec], worst


@pytest.mark.parametrize("prec", [gb.IPM_TF32X3, gb.IPM_TF32, gb.IPM_BF16],
                         ids=["tf32x3", "tf32", "bf16"])
def test_unrefined_solve_backward_error_grid40(prec):
    """40^3 (seven super-steps on a 4,720-column root): one solve with the
    factor and no refinement has the normwise backward error of the factor."""
    lp, ctx, info, K = _setup(40, prec, seed=6)
    assert info.max_ncol > 6 * SUPER
    knorm = abs(K).sum(axis=1).max()
    for seed in (1, 2):
        b = gen.normal(gen.stream_seed(70 + seed, 1), lp.n)
        x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_NONE, raise_on_error=False)
        xs = x.cpu().numpy()
        eta = np.abs(K @ xs - b).max() / (knorm * np.abs(xs).max() + np.abs(b).max())
        assert eta <= BACKWARD[prec], (seed, eta)
    # refinement still reaches the FP64 target from this factor
    b = gen.normal(gen.stream_seed(73, 1), lp.n)
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    si = ctx.kkt_solve(dev(b), x, gb.IPM_REFINE_IR)
    r = np.abs(K @ x.cpu().numpy() - b).max() / np.abs(b).max()
    assert si.rel_residual <= 1e-10 and r <= 1e-9


def test_multiple_right_hand_sides_match_single_solves():
    """kkt_solve with nrhs right-hand sides stored one after the other gives
    the same solutions as one call per right-hand side."""
    lp, ctx, info, K = _setup(24, gb.IPM_TF32X3, seed=7)
    B = np.stack([gen.normal(gen.stream_seed(80 + k, 1), lp.n) for k in range(3)])
    Bd = dev(B)
    X = torch.empty_like(Bd)
    si = ctx.kkt_solve(Bd, X, gb.IPM_REFINE_IR)
    assert si.rel_residual <= 1e-10
    for k in range(3):
        x1 = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        ctx.kkt_solve(dev(B[k]), x1, gb.IPM_REFINE_IR)
        np.testing.assert_array_equal(X[k].cpu().numpy(), x1.cpu().numpy())
        r = np.abs(K @ X[k].cpu().numpy() - B[k]).max() / np.abs(B[k]).max()
        assert r <= 1e-9
