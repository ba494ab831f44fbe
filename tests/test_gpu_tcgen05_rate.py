"""Microbenchmark of the tcgen05 MMA rate that the tensor-core MTTKRP's MMA lists
are sized by (tests/gpu_probes/tcgen05_rate.cu, built with nvcc for sm_103a and
run once).  Checked properties of one SM's tensor pipe (cta_group::1, M = 128):

* an MMA of N = 256 runs at the full BF16 rate of 128 x 256 x 16 MACs in 128
  cycles (4096 MACs per clock), and TF32 at half of it;
* every MMA costs 56-62 cycles however narrow (GB300s differ), so MMAs of N < 128
  waste the pipe in proportion (the reason the exact-chain form stacks its B parts
  along N);
* neither the operand row width (64- or 128-byte swizzle) nor writing several
  accumulators in turn changes the rate;
* one stage of the two-step exact-chain kernel (8 stacked MMAs, 704 cycles of
  tensor work) costs 745-772 cycles issued back to back, the per-stage commit
  nothing, and the wait on its (complete) barrier plus the tcgen05 fence ~90."""
import json
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("probe") / "tcgen05_rate")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
                    os.path.join(HERE, "gpu_probes", "tcgen05_rate.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    return json.loads(out.strip().splitlines()[-1])


def test_full_rate_at_n256_and_tf32_at_half(probe):
    row = {r["N"]: r for r in probe["cycles_per_mma"]}
    assert row[256]["bf16_row64"] == pytest.approx(128.0, rel=0.05)
    assert row[256]["tf32_row128"] == pytest.approx(128.0, rel=0.05)   # K = 8: half the MACs
    assert row[128]["bf16_row128"] == pytest.approx(64.0, rel=0.05)


def test_narrow_mmas_cost_nearly_as_much_as_n128(probe):
    """N = 32 and 64 would take 16 and 32 cycles at the full rate; they take most of
    an N = 128 MMA's 64 (56-62 cycles measured on different GB300s)."""
    row = {r["N"]: r for r in probe["cycles_per_mma"]}
    floor = row[128]["bf16_row64"]
    for n in (32, 64):
        assert row[n]["bf16_row64"] >= 0.8 * floor, (n, row[n], floor)
        assert row[n]["bf16_row64"] >= 1.5 * (n / 2), (n, row[n])
    print("\ncycles per MMA:", json.dumps(probe["cycles_per_mma"]))


def test_swizzle_and_accumulator_rotation_do_not_matter(probe):
    for r in probe["cycles_per_mma"]:
        assert r["bf16_row128"] == pytest.approx(r["bf16_row64"], rel=0.05)
        assert r["bf16_row64_rotating_acc"] == pytest.approx(r["bf16_row64"], rel=0.05)


def test_two_step_stage_cost(probe):
    s = probe["stage_cycles"]
    assert probe["wait_errors"] == 0 and probe["cuda"] == "no error"
    assert s["ideal"] <= s["mmas_only"] <= 1.2 * s["ideal"]
    assert s["with_commit"] == pytest.approx(s["mmas_only"], rel=0.03)
    assert s["with_commit_wait_fence"] <= s["mmas_only"] + 200
    print("\nstage cycles:", json.dumps(s))
