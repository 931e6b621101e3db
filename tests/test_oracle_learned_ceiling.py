"""What a diagonal-plus-rank-16 correction of a stale factor can gain at most
(no GPU; FP64 oracle, dense algebra on a 10^3 grid LP).

The learned correction replaces the stale preconditioner L_s L_s^T by
L_s (Delta + U U^T) L_s^T. Here the operator it approximates,
W = L_s^{-1} K_k L_s^{-T}, is formed exactly from the oracle's factor of K at
iterate k0 and the oracle's K at iterate k = k0 + d of the oracle's own
interior-point trajectory, and PCG (relative residual 1e-10, the skip test of
the learned path) is run with corrections that know W exactly:

* E = 0 (the stale factor alone);
* c I for any scalar c: the same PCG iterates, so a training loss that rewards
  matching the scale of W (the bulk of W's change between iterates is a common
  factor mu_k0 / mu_k) buys PCG nothing;
* the exact diagonal of W: the best a per-variable Delta can hope for, it
  gains little;
* the exact diagonal plus the 16 eigenpairs of the diagonally scaled W
  farthest from its bulk: the whole gain of the form (about a third of the
  steps here). Each of those eigenvectors lives on fewer than ten of the
  1000 variables, so a correction that reaches the ceiling has to single out a
  few small coupled groups of variables and their relative signs; a network
  whose U rows
  are one function of each variable's own features has to do that from local
  features alone.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import learned as OL

sl = pytest.importorskip("scipy.linalg")

G, SEED, RANK, TOL = 10, 201, 16, 1e-10


def _pcg_steps(K, minv, b, max_steps=400):
    """Plain preconditioned conjugate gradients; steps to ||r|| <= TOL ||b||."""
    x = np.zeros_like(b)
    r = b.copy()
    z = minv(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for k in range(1, max_steps + 1):
        q = K @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= TOL * nb:
            return k
        z = minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return max_steps


@pytest.fixture(scope="module")
def study():
    oracle.build()
    lp = gen.grid_lp(G, seed=SEED)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, gen.nd_order_grid3d(G))
    lpos, upos = OL.bound_rows(lp)
    traj = []
    for k in range(1, 30):  # iterate k of the oracle's trajectory (deterministic)
        r = oracle.ipm_lp(S, lp, tol=1e-8, max_iter=k)
        traj.append(r)
        if r["status"] == 0:
            break
    assert traj[-1]["status"] == 0 and len(traj) >= 4

    def k_final(r):
        D = OL.scaling(r["s"], r["lam"], 1e-8)
        dx = np.zeros(lp.n)
        for i in range(lp.n):
            dx[i] = sum(D[p] for p in (lpos[i], upos[i]) if p >= 0)
        kval = oracle.assemble(S, lp.m, lp.rowptr, lp.col, lp.val, D[:lp.m], dextra=dx,
                               delta_p=1e-8)
        return kval, oracle.k_dense(S, kval, final=True)

    rng = np.random.default_rng(7)
    rows = []
    for k0 in range(1, len(traj) - 1):
        kval0, _ = k_final(traj[k0])
        lval, bad = oracle.factor(S, kval0)
        assert bad == 0
        Ls = oracle.l_dense(S, lval)
        for d in (1, 2):
            if k0 + d >= len(traj):
                continue
            _, K = k_final(traj[k0 + d])
            X = sl.solve_triangular(Ls, K, lower=True)
            W = sl.solve_triangular(Ls, X.T, lower=True)
            W = 0.5 * (W + W.T)
            b = rng.standard_normal(lp.n)

            def pre(E):
                return lambda v: sl.solve_triangular(
                    Ls.T, E(sl.solve_triangular(Ls, v, lower=True)), lower=False)

            dg = np.diag(W).copy()
            sd = 1.0 / np.sqrt(dg)
            Ws = sd[:, None] * W * sd[None, :]
            ev, V = np.linalg.eigh(Ws)
            med = np.median(ev)
            far = np.argsort(-np.abs(np.log(ev / med)))[:RANK]
            Vr, er = V[:, far], ev[far]
            c = float(np.median(np.linalg.eigvalsh(W)))
            rows.append(dict(
                k0=k0, d=d,
                e0=_pcg_steps(K, pre(lambda y: y), b),
                scalar=_pcg_steps(K, pre(lambda y: y / c), b),
                diag=_pcg_steps(K, pre(lambda y: y / dg), b),
                diag_rank=_pcg_steps(K, pre(lambda y: sd * (sd * y + Vr @ ((med / er - 1.0) * (Vr.T @ (sd * y))))), b),
                spread=float(ev.max() / ev.min()),
                # effective number of variables an eigenvector spreads over
                support=float(np.median(1.0 / np.sum(Vr ** 4, axis=0))),
                support_max=float(np.max(1.0 / np.sum(Vr ** 4, axis=0)))))
    return rows


def test_study_covers_the_trajectory(study):
    assert len(study) >= 5
    for r in study:
        print(r)


def test_scalar_corrections_change_nothing(study):
    """CG with M and c M takes the same iterates: scale is worth no steps."""
    for r in study:
        assert abs(r["scalar"] - r["e0"]) <= 1, r


def test_exact_diagonal_gains_little(study):
    e0 = sum(r["e0"] for r in study)
    diag = sum(r["diag"] for r in study)
    assert diag >= 0.8 * e0, (diag, e0)


def test_exact_diagonal_plus_rank16_is_the_ceiling(study):
    """The form's gain, with W known exactly, is a fraction of the steps, and
    it needs W's global eigenvectors."""
    e0 = sum(r["e0"] for r in study)
    best = sum(r["diag_rank"] for r in study)
    assert 0.4 * e0 <= best <= 0.85 * e0, (best, e0)


def test_the_gain_sits_on_small_groups_of_variables(study):
    """The 16 eigenvectors the ceiling uses each spread over fewer than ten
    variables (participation ratio 1 / sum v^4)."""
    for r in study:
        assert r["support_max"] < 10.0, r
