"""Batched MPC QPs (one persistent launch) against the CPU oracle, instance by
instance, on the first 64 instances of the 4096-instance family; a bounds-free
instance against the LQR closed form; the autotuner; CUDA-graph replay."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_16094_gb300 as gb  # noqa: E402
from tests.test_oracle_qp import lqr_cost  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    oracle.build()


@pytest.fixture(scope="module")
def subset():
    mb = gen.mpc_batch(64, seed=3)
    ref = []
    for i in range(mb.count):
        lp, W = gen.mpc_instance_qp(*mb.instance(i), u_max=mb.u_max, x_max=mb.x_max)
        S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, None, W[0], W[1])
        r = oracle.ipm_lp(S, lp, tol=1e-8, W=W)
        assert r["status"] == 0
        ref.append(r["objective"])
    return mb, np.array(ref)


@pytest.mark.parametrize("prec", [gb.IPM_FP64, gb.IPM_FP32], ids=["fp64", "fp32"])
def test_batched_matches_oracle_per_instance(subset, prec):
    mb, ref = subset
    b = gb.BatchedMPC(mb)
    b.ipm_solve_batched(precision=prec, instances_per_cta=8, tol=1e-8, max_iter=100)
    torch.cuda.synchronize()
    st, obj, kkt = b.status.cpu().numpy(), b.obj.cpu().numpy(), b.kkt.cpu().numpy()
    assert np.all(st == 0), np.flatnonzero(st)
    assert np.all(kkt <= 1e-8)
    np.testing.assert_allclose(obj, ref, rtol=1e-6, atol=0)
    # the returned trajectories respect the input box within the tolerance
    z = b.z.cpu().numpy().reshape(-1, 16)
    assert np.abs(z[:, :4]).max() <= mb.u_max * (1 + 1e-6)
    assert np.abs(z[:, 4:]).max() <= mb.x_max * (1 + 1e-6)


def test_batched_without_active_bounds_is_lqr():
    mb = gen.mpc_batch(8, seed=21, t_min=10, t_max=30)
    mb.u_max = mb.x_max = 1e3
    b = gb.BatchedMPC(mb)
    b.ipm_solve_batched(precision=gb.IPM_FP64, instances_per_cta=4, tol=1e-10, max_iter=100)
    torch.cuda.synchronize()
    obj = b.obj.cpu().numpy()
    for i in range(mb.count):
        want = lqr_cost(*mb.instance(i))
        assert abs(obj[i] - want) <= 1e-6 * max(1.0, abs(want))


def test_autotune_and_graph_replay(subset):
    mb, ref = subset
    b = gb.BatchedMPC(mb)
    cfg, ms = b.ipm_mpc_autotune(precision=gb.IPM_FP32, tol=1e-8)
    assert cfg.instances_per_cta in (2, 4, 8, 16) and cfg.ctas > 0
    assert all(t > 0 for t in ms)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    b.obj.zero_()
    with torch.cuda.graph(g, stream=s):
        b.ipm_solve_batched(precision=gb.IPM_FP32, instances_per_cta=cfg.instances_per_cta,
                            ctas=cfg.ctas, tol=1e-8, stream=s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_allclose(b.obj.cpu().numpy(), ref, rtol=1e-6)
    b.obj.zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_allclose(b.obj.cpu().numpy(), ref, rtol=1e-6)
