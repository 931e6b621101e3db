"""Pins of the FP64 learned-correction oracle (no GPU).

The learned correction is not in the paper; its definitions (network, probe
loss, Woodbury application, features built from the Eq. (5) diagonal) are
pinned here to facts outside the oracle's own formulas.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import learned as OL


def _theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, OL.NPARAMS)


def _data(seed, n=37, P=3):
    rng = np.random.default_rng(seed)
    feat = rng.normal(0.0, 1.0, (n, OL.NF))
    z = rng.choice([-1.0, 1.0], (P, n))
    w = rng.normal(0.0, 1.0, (P, n)) + 2.0 * z
    return feat, z, w


def test_param_count():
    assert OL.NPARAMS == 32 * 8 + 32 + 32 * 32 + 32 + 17 * 32 + 17 == 1905


def test_gradient_matches_finite_differences():
    """Backpropagation against central differences of the loss, every parameter block."""
    theta = _theta(1)
    feat, z, w = _data(2)
    _, g = OL.probe_loss_grad(theta, feat, z, w)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(np.arange(a, b), 12, replace=False) for a, b in
                          [(0, 256), (256, 288), (288, 1312), (1312, 1344), (1344, 1888),
                           (1888, 1905)]])
    h = 1e-6
    for k in idx:
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd = (OL.probe_loss(tp, feat, z, w) - OL.probe_loss(tm, feat, z, w)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_zero_network_is_identity_correction():
    """All-zero parameters give Delta = 1 and U = 0: the loss is mean ||w - z||^2."""
    theta = np.zeros(OL.NPARAMS)
    feat, z, w = _data(4)
    delta, U, _ = OL.forward(theta, feat)
    assert np.all(delta == 1.0) and np.all(U == 0.0)
    assert OL.probe_loss(theta, feat, z, w) == pytest.approx(np.mean((w - z) ** 2), rel=1e-14)


def test_constant_outputs_match_dense_operator():
    """With only the output biases set, Delta = e^{b0} and every row of U is
    0.1 b[1:]; the loss equals that of the dense matrix e^{b0} I + |u|^2 11^T
    (scaled by e^{-2 b0})."""
    parts = OL.unpack(np.zeros(OL.NPARAMS))
    b3 = np.linspace(-0.5, 0.7, OL.NO)
    parts = {k: v.copy() for k, v in parts.items()}
    parts["b3"] = b3
    theta = OL.pack(parts)
    feat, z, w = _data(5, n=11, P=2)
    n = z.shape[1]
    u = 0.1 * b3[1:]
    M = np.exp(b3[0]) * np.eye(n) + (u @ u) * np.ones((n, n))
    ref = sum(np.sum((w[p] - M @ z[p]) ** 2) for p in range(z.shape[0])) / z.size
    ref /= np.exp(2 * b3[0])  # relative to Delta
    assert OL.probe_loss(theta, feat, z, w) == pytest.approx(ref, rel=1e-12)


def test_woodbury_matches_dense_solve():
    rng = np.random.default_rng(6)
    n = 50
    delta = np.exp(rng.normal(0, 1, n))
    U = rng.normal(0, 0.5, (n, OL.NR))
    v = rng.normal(0, 1, n)
    ref = np.linalg.solve(np.diag(delta) + U @ U.T, v)
    assert np.allclose(OL.woodbury_apply(delta, U, v), ref, rtol=1e-10, atol=1e-12)


def test_features_diagonal_matches_assembled_matrix():
    """k_diagonal equals the diagonal of K assembled by the FP64 oracle (Eq. 5),
    and features of an unchanged iterate are the trivial values."""
    lp = gen.grid_lp(4, 4, 3, seed=7)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, gen.nd_order_grid3d(4, 4, 3))
    rng = np.random.default_rng(8)
    nl, nu = int(np.isfinite(lp.l).sum()), int(np.isfinite(lp.u).sum())
    assert nl == nu == lp.n  # 0 <= x <= 10: rows m..m+n-1 lower, m+n.. upper
    D = np.exp(rng.normal(0, 2, lp.m + nl + nu))
    dextra = D[lp.m:lp.m + lp.n] + D[lp.m + lp.n:]
    kval = oracle.assemble(S, lp.m, lp.rowptr, lp.col, lp.val, D[:lp.m], dextra, 1e-8)
    Kd = oracle.k_dense(S, kval)
    assert np.allclose(OL.k_diagonal(lp, D, 1e-8), np.diag(Kd), rtol=1e-13)
    x = rng.uniform(0, 10, lp.n)
    f = OL.features(lp, D, D, 0.5, 0.5, x, 1e-8, 1e-8)
    assert np.all(f[:, [0, 1, 2, 3, 5]] == 0.0)
    assert np.allclose(f[:, 3], 0.0) and np.allclose(f[:, 7], x / 10)
    assert np.allclose(f[:, 4], np.log10(0.5) / 10)
    # doubling every D doubles diag(K) - delta_p: feature 0 is log 2 up to delta_p
    f2 = OL.features(lp, D, 2 * D, 0.5, 0.25, x, 0.0, 0.0)
    assert np.allclose(f2[:, 0], np.log(2.0), rtol=1e-12)
    assert np.allclose(f2[:, 5], np.log(0.5) / 10)
