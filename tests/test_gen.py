"""Seeded generators and orderings (inputs of both solvers). CPU only."""
import numpy as np

import gen


def test_splitmix64_reference_values():
    # SplitMix64 with state 0 and increment gamma; first outputs of the published generator
    z = gen.splitmix64(0, 3)
    assert [hex(int(v)) for v in z] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4",
                                        "0x6c45d188009454f"]


def test_streams_deterministic_and_distinct():
    a = gen.normal(7, 1000)
    b = gen.normal(7, 1000)
    c = gen.normal(8, 1000)
    np.testing.assert_array_equal(a, b)
    assert not np.allclose(a, c)
    assert abs(a.mean()) < 0.15 and abs(a.std() - 1) < 0.1
    u = gen.uniform(9, 10000, 2.0, 3.0)
    assert u.min() >= 2.0 and u.max() < 3.0


def test_small_lp_recipe():
    lp = gen.random_lp(2000, 1000, 5, seed=0)
    assert lp.nnz == 5000
    assert np.all(np.diff(lp.rowptr) == 5)
    for i in range(lp.m):
        cs = lp.col[lp.rowptr[i]:lp.rowptr[i + 1]]
        assert len(set(cs.tolist())) == 5 and np.all(np.diff(cs) > 0)
    slack = lp.matvec(lp.x0) - lp.b
    assert slack.min() >= 0.1 and slack.max() < 1.0
    assert lp.x0.min() >= 1.0 and lp.x0.max() < 9.0


def test_grid_lp_recipe():
    g = 5
    lp = gen.grid_lp(g, seed=1)
    assert lp.n == lp.m == g ** 3
    # interior row has 7 entries, a corner row 4
    assert lp.rowptr[1] - lp.rowptr[0] == 4
    mid = (g // 2) * (1 + g + g * g)
    assert lp.rowptr[mid + 1] - lp.rowptr[mid] == 7
    # diagonal carries the +8 boost: mean of diagonal values near 8
    diag = np.array([lp.val[lp.rowptr[i]:lp.rowptr[i + 1]][lp.col[lp.rowptr[i]:lp.rowptr[i + 1]] == i][0]
                     for i in range(lp.n)])
    assert 7.5 < diag.mean() < 8.5


def test_nd_ordering_separates():
    g = 9
    perm = gen.nd_order_grid3d(g, leaf=16)
    assert sorted(perm.tolist()) == list(range(g ** 3))
    # the last block numbered is the top separator: two full planes of the longest side (x)
    sep = perm[-2 * g * g:]
    xs = sep % g
    assert set(xs.tolist()) == {3, 4}


def test_min_degree_is_permutation():
    lp = gen.random_lp(200, 100, 5, seed=3)
    p = gen.min_degree_order(gen.normal_graph(lp))
    assert sorted(p.tolist()) == list(range(200))


def test_sgm10():
    assert abs(gen.sgm10([0.0, 0.0]) - 0.0) < 1e-12
    assert abs(gen.sgm10([90.0, 0.0]) - (np.sqrt(100.0 * 10.0) - 10.0)) < 1e-12
    assert abs(gen.sgm10([5.0]) - 5.0) < 1e-12
