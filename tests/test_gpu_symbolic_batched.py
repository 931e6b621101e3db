"""Symbolic analysis of a batch of patterns on the GPU (ipm_symbolic_batched)
against the oracle's host analysis, bit for bit: the final numbering, the
elimination tree, the column counts and the fundamental supernodes of every
pattern, on a batch of uneven patterns (batched MPC instances of different
horizons, random LPs and grids, with and without orderings)."""
import numpy as np
import pytest

import gen
import oracle
from tests.test_oracle import _fundamental_starts

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    oracle.build()


def _batch():
    pats, perms = [], []
    mb = gen.mpc_batch(24, seed=3)
    for i in range(24):  # horizons 10..100: uneven sizes
        lp, _ = gen.mpc_instance_qp(*mb.instance(i), u_max=mb.u_max, x_max=mb.x_max)
        pats.append((lp.n, lp.rowptr, lp.col))
        perms.append(np.arange(lp.n, dtype=np.int32))
    for k in range(12):
        lp = gen.random_lp(80 + 37 * k, 40 + 11 * k, 3 + k % 3, seed=100 + k)
        pats.append((lp.n, lp.rowptr, lp.col))
        perms.append(gen.lp_ordering(lp) if k % 2 == 0 else
                     np.argsort(gen.uniform(200 + k, lp.n, 0.0, 1.0)).astype(np.int32))
    for g in (4, 6, 9):
        lp = gen.grid_lp(g, seed=g)
        pats.append((lp.n, lp.rowptr, lp.col))
        perms.append(gen.nd_order_grid3d(g))
    return pats, perms


def test_batched_symbolic_matches_oracle_bit_for_bit():
    pats, perms = _batch()
    (post, parent, cc, sstart), ms = gb.symbolic_batched(pats, perms)
    assert ms > 0
    for b, ((n, rp, cl), pm) in enumerate(zip(pats, perms)):
        S = oracle.analyze(n, len(rp) - 1, rp, cl, pm)
        np.testing.assert_array_equal(post[b], S.perm, err_msg=f"pattern {b}")
        np.testing.assert_array_equal(parent[b], S.parent, err_msg=f"pattern {b}")
        np.testing.assert_array_equal(cc[b], S.colcount, err_msg=f"pattern {b}")
        want = np.zeros(n, np.int32)
        want[_fundamental_starts(S.parent, S.colcount)] = 1
        np.testing.assert_array_equal(sstart[b], want, err_msg=f"pattern {b}")


def test_batched_symbolic_identity_ordering_and_rejection():
    pats, perms = _batch()
    (post, parent, cc, _), _ = gb.symbolic_batched(pats[:5])  # no orderings: identity
    for b in range(5):
        n, rp, cl = pats[b]
        S = oracle.analyze(n, len(rp) - 1, rp, cl, None)
        np.testing.assert_array_equal(parent[b], S.parent)
        np.testing.assert_array_equal(cc[b], S.colcount)
    bad = [p.copy() for p in perms[:5]]
    bad[3][0] = bad[3][1]  # a repeated index: not a permutation
    with pytest.raises(gb.IpmError) as e:
        gb.symbolic_batched(pats[:5], bad)
    assert e.value.status == 1 and "pattern 3" in str(e.value)
