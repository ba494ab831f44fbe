"""bench.py's reference arm on the host (no GPU): one JSON line with the contract's
keys, from rank 0 only when launched as two ranks."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _last_json(out):
    lines = [l for l in out.strip().splitlines() if l.startswith("{")]
    assert lines, out
    return json.loads(lines[-1])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = _last_json(r.stdout)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_reference_arm_two_ranks_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_flops_views_of_the_bench_workload():
    """The three MTTKRP rates of the JSON line: the JK-ALS equivalent of the 300-sample
    leave-one-out workload is 299/300 of the useful rate; the exact form issues ten tensor-core
    products per useful one."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2112_03985_gb300 import workloads as W
    w = W.make_config(2)
    v = bench.flops_views(60.0, "exact_bf16", w.dims[w.n_hat], max(len(D) for D in w.left_out))
    assert v["useful"] == 60.0
    assert abs(v["jk_als_equivalent"] - 60.0 * 299 / 300) < 1e-12
    assert v["issued"] == 600.0
    assert set(bench.ISSUED_PER_USEFUL) == {"fp64", "tf32", "3xtf32", "bf16", "split_bf16", "exact_bf16"}
