"""The benchmark's reference arm (the oracle on the host cores) keeps the JSON
line contract, alone and under torchrun with two ranks (only rank 0 prints).
CPU only: the reference arm never touches a GPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline",
        "e2e"}


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check(line, n_gpus):
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == n_gpus
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 1)


def test_reference_arm_under_torchrun_prints_once():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=900,
                       env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 2)


def test_summary_carries_the_headline_figures():
    """The compact key that ends the own arm's line: every form's time to
    1e-6, the FP64 tensor-core path against the ladder, and the other
    workloads, without the training record."""
    sys.path.insert(0, ROOT)
    import bench
    tti = {"workload": "w", "tf32x3": {"s": 3.67, "iters": 10},
           "tf32_then_tf32x3": {"s": 3.49}, "bf16": {"error": "x"},
           "fp64_tc": {"s": 26.0, "factor_tflops_fp64_equiv": 20.7, "fma_path_s_estimate": 464.5}}
    forms = {"workload": "w", "fp64": {"seconds": 8.06}, "training": {"seconds": 2.7},
             "flops": 1.0}
    nlp = {"workload": "w", "max_iter": 150, "fp64_tc": {"seconds": 7.2}}
    mpc = {"fp64": {"solves_per_s": 33800.0}}
    s = bench.summary(tti, forms, nlp, mpc)
    assert s["tti_1e-6_s"] == {"tf32x3": 3.67, "tf32_then_tf32x3": 3.49, "fp64_tc": 26.0,
                               "fp64_fma_estimate": 464.5}
    assert s["fp64_tc_over_ladder"] == round(26.0 / 3.49, 2)
    assert s["fp64_tc_factor_tflops"] == 20.7
    assert s["forms_48_s"] == {"fp64": 8.06}
    assert s["grid_nlp_s"] == {"fp64_tc": 7.2}
    assert s["mpc_solves_per_s"] == {"fp64": 33800.0}
    assert len(json.dumps(s)) < 1000  # fits the end of the line the driver keeps
