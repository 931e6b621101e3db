"""Host-side plan at sizes where the tensor-core schedule uses all its parts
(CPU only: kkt_analyze builds and checks every task list without a GPU).

At these grids the root front has thousands of columns, so the left-looking
factorisation runs in 512-column super-steps with the look-ahead update on a
second stream, and the SYRK and super-step updates are cut into CTA-pair
tiles. kkt_analyze runs the library's own checks of every task (tiles inside
their fronts, K ranges before their columns, assembly tiles covering each
front's lower triangle exactly once, solve phases); a violation is an error."""
import numpy as np
import pytest

import gen
import paper_2508_16094_gb300 as gb


@pytest.mark.parametrize("dims", [(48, 48, 48), (40, 36, 30), (33, 17, 9)])
def test_plan_checks_pass_at_super_step_sizes(dims):
    lp = gen.grid_lp(*dims, seed=5)
    perm = gen.nd_order_grid3d(*dims)
    ctx = gb.IpmContext(lp.n, lp.m, lp.rowptr, lp.col, lp.l, lp.u,
                        options=gb.default_options(precision=gb.IPM_TF32X3, storage_fp64=0))
    info = ctx.kkt_analyze(perm)
    ex = ctx.kkt_symbolic_export()
    ncol = np.diff(ex["super"]).astype(np.int64)
    # the symbolic counts agree with the exported column counts
    assert info.nnz_l == int(ex["colcount"].astype(np.int64).sum())
    assert info.max_ncol == int(ncol.max())
    if dims[0] >= 40:
        assert ncol.max() > 1024  # several super-steps on the root front
    # every supernode lies on one level, levels count up to the root's
    assert int(ex["slevel"].max()) + 1 == info.nlevels
