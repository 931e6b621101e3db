"""Training driver of the learned stale-factor correction.

Host orchestration over the C ABI only: the interior-point iterations, the
probe products w = L_s^{-1} P K_k P^T L_s^{-T} z, the features, the network's
forward and backward passes and the Adam updates all run in the library's
kernels (``ipm_solve``, ``ipm_learned_sample``, ``ipm_learned_train``).

Iterates come from the method itself: the trajectory x_k, s_k, lambda_k of an
interior-point run is recorded one iteration at a time (``ipm_solve`` with
max_iter = 1, warm-started from the previous iterate), then for every pair
(k0, k), k0 < k <= k0 + staleness, the factor of iterate k0 is made the held
factor (one more iteration from iterate k0) and iterate k is sampled against it.

The context must have been created with ``learned_probes`` > 0 (the buffers are
sized at ``kkt_analyze``) and a precision whose factor is stored in FP32
(TF32, TF32X3 or FP32).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

N_FEATURES = 8


@dataclass
class Sample:
    k0: int          # iterate whose factor is held
    k: int           # iterate whose matrix K_k is probed
    feat: object     # (n, 8) float32, device, permuted numbering
    z: object        # (P, n) float32 probes, device, permuted numbering
    w: object        # (P, n) float32 = L_s^{-1} P K_k P^T L_s^{-T} z


def probes_of(ctx) -> int:
    return int(min(8, max(1, ctx.options.learned_probes)))


def trajectory(ctx, jv, b, c, k_max: int):
    """Iterates 0..K (K <= k_max; stops early at convergence) of ipm_solve,
    one iteration per call. Returns a list of (x, s, lambda) device tensors."""
    import torch
    n, mt = ctx.n, ctx.m_tot
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.empty(mt, dtype=torch.float64, device="cuda")
    lam = torch.empty(mt, dtype=torch.float64, device="cuda")
    saved = dict(max_iter=ctx.options.max_iter, warm_start=ctx.options.warm_start,
                 learned=ctx.options.learned)
    out = []
    try:
        ctx.ipm_set_options(max_iter=0, warm_start=0, learned=0)
        res = ctx.ipm_solve(jv, b, c, x, s, lam)
        out.append((x.clone(), s.clone(), lam.clone()))
        ctx.ipm_set_options(max_iter=1, warm_start=1)
        for _ in range(k_max):
            if res.kkt <= ctx.options.tol:
                break
            res = ctx.ipm_solve(jv, b, c, x, s, lam)
            if res.status not in (0, 7):  # IPM_OK or IPM_ERR_MAXITER
                break
            out.append((x.clone(), s.clone(), lam.clone()))
    finally:
        ctx.ipm_set_options(**saved)
    return out


def hold_factor(ctx, jv, b, c, state):
    """Make the factor of iterate ``state`` the held one (one iteration from it)."""
    x, s, lam = (t.clone() for t in state)
    saved = dict(max_iter=ctx.options.max_iter, warm_start=ctx.options.warm_start,
                 learned=ctx.options.learned)
    try:
        ctx.ipm_set_options(max_iter=1, warm_start=1, learned=0)
        ctx.ipm_solve(jv, b, c, x, s, lam)
    finally:
        ctx.ipm_set_options(**saved)


def rademacher(P: int, n: int, seed: int):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    return (torch.randint(0, 2, (P, n), generator=g, device="cuda", dtype=torch.int32)
            .to(torch.float32) * 2 - 1).contiguous()


def collect(ctx, jv, b, c, traj, staleness=(1, 2, 3), k_first: int = 1, seed: int = 0):
    """Samples (feat, z, w) for every pair (k0, k0 + d) of the trajectory."""
    import torch
    n, P = ctx.n, probes_of(ctx)
    samples = []
    for k0 in range(k_first, len(traj) - 1):
        ks = [k0 + d for d in staleness if k0 + d < len(traj)]
        if not ks:
            continue
        hold_factor(ctx, jv, b, c, traj[k0])
        for k in ks:
            x, s, lam = traj[k]
            z = rademacher(P, n, seed * 1000003 + k0 * 101 + k)
            feat = torch.empty((n, N_FEATURES), dtype=torch.float32, device="cuda")
            w = torch.empty((P, n), dtype=torch.float32, device="cuda")
            ctx.ipm_learned_sample(jv, x, s, lam, z, feat, w)
            samples.append(Sample(k0, k, feat, z, w))
    return samples


def mean_loss(ctx, samples, weights=None) -> float:
    """Mean probe loss over samples with the given (or the current) weights;
    the current weights are restored afterwards."""
    cur = ctx.ipm_learned_weights()
    if weights is not None:
        ctx.ipm_learned_weights(weights)
    try:
        return float(np.mean([ctx.ipm_learned_loss_grad(sm.feat, sm.z, sm.w)[0]
                              for sm in samples]))
    finally:
        if weights is not None:
            ctx.ipm_learned_weights(cur)


def train(ctx, samples, epochs: int = 20, lr: float = 2e-3, seed: int = 0, steps_per_sample=1):
    """Adam over the samples (shuffled each epoch, one full-batch step per
    sample); returns the mean loss of each epoch as seen during training."""
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        order = rng.permutation(len(samples))
        losses = [ctx.ipm_learned_train(samples[i].feat, samples[i].z, samples[i].w, lr=lr,
                                        steps=steps_per_sample) for i in order]
        hist.append(float(np.mean(losses)))
    return hist
