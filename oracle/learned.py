"""FP64 CPU oracle of the learned stale-factor correction.

TEST INFRASTRUCTURE ONLY: the product never imports this module.

The paper has no learned component; this restates, as plain numpy in FP64,
the definitions the CUDA kernels implement:

  * per-variable features of the change between the condensed matrix that was
    factored (iterate k0) and the current one (iterate k), Eq. (5) diagonals;
  * a two-layer tanh network 8 -> 32 -> 32 -> 17 applied to every variable;
    output 0 is log Delta_j, outputs 1..16 (times 0.1) are row j of U;
  * the probe loss  sum_p ||Delta^{-1} (w_p - Delta z_p - U (U^T z_p))||^2 / (P n)
    with w_p = L_s^{-1} P K_k P^T L_s^{-T} z_p (the error of the correction
    relative to its diagonal, so every variable counts alike whatever the
    scale of its change), and its gradient by backpropagation;
  * (Delta + U U^T)^{-1} v by the Woodbury identity.

Parameter vector layout (shared by the API, defined independently here):
W1 [32 x 8], b1 [32], W2 [32 x 32], b2 [32], W3 [17 x 32], b3 [17], row-major.

Pins (tests/test_oracle_learned.py): central finite differences of the loss,
special cases (zero network -> Delta = 1, U = 0; constant outputs -> a dense
closed form), Woodbury against a dense solve, and the features' diagonal
against the diagonal of the assembled Eq. (5) matrix of the FP64 oracle.
"""
from __future__ import annotations

import numpy as np

NF, NH, NR = 8, 32, 16
NO = 1 + NR
U_SCALE = 0.1
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
         ("W3", (NO, NH)), ("b3", (NO,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    """Split the flat parameter vector into named FP64 arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == NPARAMS
    out, o = {}, 0
    for name, shp in SIZES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in SIZES])


# ---------------------------------------------------------------------------
# Features
# ---------------------------------------------------------------------------
def bound_rows(lp):
    """Rows of g(x) >= 0 in the order A x - b (m rows), x - l (finite l, by
    variable), u - x (finite u, by variable); returns (lpos, upos), -1 = none."""
    n, m = lp.n, lp.m
    lpos = -np.ones(n, np.int64)
    upos = -np.ones(n, np.int64)
    li = np.flatnonzero(np.isfinite(lp.l))
    ui = np.flatnonzero(np.isfinite(lp.u))
    lpos[li] = m + np.arange(li.size)
    upos[ui] = m + li.size + np.arange(ui.size)
    return lpos, upos


def k_diagonal(lp, D, delta_p):
    """diag(K) of Eq. (5) for an LP: sum_r A_ri^2 D_r + D(bound rows of i) + delta_p."""
    n = lp.n
    d = np.full(n, float(delta_p))
    for r in range(lp.m):
        for e in range(lp.rowptr[r], lp.rowptr[r + 1]):
            d[lp.col[e]] += lp.val[e] ** 2 * D[r]
    lpos, upos = bound_rows(lp)
    for i in range(n):
        if lpos[i] >= 0:
            d[i] += D[lpos[i]]
        if upos[i] >= 0:
            d[i] += D[upos[i]]
    return d


def features(lp, D_old, D_new, mu_old, mu_new, x, delta_p_old, delta_p_new):
    """The eight features of every variable (original numbering), FP64.

    0: log(K_new,ii / K_old,ii)                      clamp [-30, 30]
    1: log(bound part new / bound part old) / 10     clamp [-5, 5]
    2: asinh(sum_r (D_new,r - D_old,r) A_ri^2 / K_old,ii)
    3: asinh(sum_r |D_new,r - D_old,r| A_ri^2 / K_old,ii)
    4: log10(mu_new) / 10
    5: log(mu_new / mu_old) / 10                     clamp [-5, 5]
    6: log(bound part new / K_new,ii + 1e-30) / 10   clamp [-7, 1]
    7: x_i / 10
    (the bound part of variable i is the sum of D over its bound rows)"""
    n = lp.n
    kn = k_diagonal(lp, D_new, delta_p_new)
    ko = k_diagonal(lp, D_old, delta_p_old)
    lpos, upos = bound_rows(lp)
    ss = np.zeros(n)
    sa = np.zeros(n)
    for r in range(lp.m):
        for e in range(lp.rowptr[r], lp.rowptr[r + 1]):
            dd = (D_new[r] - D_old[r]) * lp.val[e] ** 2
            ss[lp.col[e]] += dd
            sa[lp.col[e]] += abs(dd)
    bn = np.zeros(n)
    bo = np.zeros(n)
    for i in range(n):
        for pos in (lpos[i], upos[i]):
            if pos >= 0:
                bn[i] += D_new[pos]
                bo[i] += D_old[pos]
    tiny = 1e-300
    mun, muo = max(mu_new, tiny), max(mu_old, tiny)
    f = np.zeros((n, NF))
    f[:, 0] = np.clip(np.log(kn / ko), -30, 30)
    f[:, 1] = np.clip(np.log((bn + tiny) / (bo + tiny)) / 10, -5, 5)
    f[:, 2] = np.arcsinh(ss / ko)
    f[:, 3] = np.arcsinh(sa / ko)
    f[:, 4] = np.log10(mun) / 10
    f[:, 5] = np.clip(np.log(mun / muo) / 10, -5, 5)
    f[:, 6] = np.clip(np.log(bn / kn + 1e-30) / 10, -7, 1)
    f[:, 7] = np.asarray(x, np.float64) / 10
    return f


# ---------------------------------------------------------------------------
# Network, loss, gradient
# ---------------------------------------------------------------------------
def forward(theta, feat):
    """Delta (n,), U (n, 16) and the activations needed by the gradient."""
    p = unpack(theta)
    f = np.asarray(feat, np.float64)
    h1 = np.tanh(f @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    o = h2 @ p["W3"].T + p["b3"]
    delta = np.exp(np.clip(o[:, 0], -20, 20))
    U = U_SCALE * o[:, 1:]
    return delta, U, dict(f=f, h1=h1, h2=h2, o=o)


def probe_loss(theta, feat, z, w):
    """sum_p ||Delta^{-1} (w_p - Delta z_p - U U^T z_p)||^2 / (P n); z, w are (P, n)."""
    delta, U, _ = forward(theta, feat)
    z = np.asarray(z, np.float64)
    w = np.asarray(w, np.float64)
    P, n = z.shape
    r = (w - delta[None, :] * z - (z @ U) @ U.T) / delta[None, :]
    return float(np.sum(r * r) / (P * n))


def probe_loss_grad(theta, feat, z, w):
    """(loss, d loss / d theta) by backpropagation through the network."""
    p = unpack(theta)
    delta, U, a = forward(theta, feat)
    z = np.asarray(z, np.float64)
    w = np.asarray(w, np.float64)
    P, n = z.shape
    t = z @ U                                        # (P, 16): U^T z_p
    r = (w - delta[None, :] * z - t @ U.T) / delta   # (P, n) relative residual
    loss = float(np.sum(r * r) / (P * n))
    q = (r / delta) @ U                              # (P, 16): U^T Delta^{-1} r_p
    s = 1.0 / (P * n)
    # r_j = w_j / Delta_j - z_j - (U t)_j / Delta_j:  d r_j / d Delta_j = -(r_j + z_j) / Delta_j
    g_delta = -2.0 * s * np.sum(r * (r + z), axis=0) / delta
    g_U = -2.0 * s * ((r / delta).T @ t + z.T @ q)   # d loss / d U  (n, 16)
    o = a["o"]
    g_o = np.zeros_like(o)
    inside = (o[:, 0] > -20) & (o[:, 0] < 20)
    g_o[:, 0] = np.where(inside, g_delta * delta, 0.0)
    g_o[:, 1:] = U_SCALE * g_U
    g = {}
    g["W3"] = g_o.T @ a["h2"]
    g["b3"] = g_o.sum(axis=0)
    g_h2 = (g_o @ p["W3"]) * (1 - a["h2"] ** 2)
    g["W2"] = g_h2.T @ a["h1"]
    g["b2"] = g_h2.sum(axis=0)
    g_h1 = (g_h2 @ p["W2"]) * (1 - a["h1"] ** 2)
    g["W1"] = g_h1.T @ a["f"]
    g["b1"] = g_h1.sum(axis=0)
    return loss, pack(g)


def woodbury_apply(delta, U, v):
    """(diag(Delta) + U U^T)^{-1} v via Delta^{-1} v - Delta^{-1} U C^{-1} U^T Delta^{-1} v,
    C = I + U^T Delta^{-1} U."""
    delta = np.asarray(delta, np.float64)
    U = np.asarray(U, np.float64)
    y = np.asarray(v, np.float64) / delta
    C = np.eye(U.shape[1]) + U.T @ (U / delta[:, None])
    return y - (U @ np.linalg.solve(C, U.T @ y)) / delta


def scaling(s, lam, delta_d):
    """D = (delta_d + s / lambda)^{-1}, the row weights of Eq. (5)."""
    return 1.0 / (delta_d + np.asarray(s, np.float64) / np.asarray(lam, np.float64))
