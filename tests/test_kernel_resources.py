"""Register budget of every kernel (no GPU): each translation unit is compiled for sm_103a with
ptxas' resource report, and no kernel may spill registers to local memory.  One known
exception is held to its present size: the fused update's generic instantiation for ranks 9-16, in its
per-problem and its grouped (batch) launch."""
import os
import re
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2112_03985_gb300", "csrc")
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"

# mangled-name fragment -> largest allowed spill stores (bytes)
KNOWN_SPILLS = {"update_fused_kernelILi16ELb0E": 108, "update_fused_grouped_kernelILi16ELb0E": 144}


def _report(src, outdir):
    obj = os.path.join(outdir, os.path.basename(src) + ".o")
    cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
           "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stderr


def _spills(text):
    out = {}
    fn = None
    for line in text.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            fn = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and fn is not None:
            out[fn] = int(m.group(1))
            fn = None
    return out


@pytest.fixture(scope="module")
def spills():
    if not os.path.exists(NVCC):
        pytest.skip("nvcc not available")
    srcs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    with tempfile.TemporaryDirectory() as d, ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        texts = list(ex.map(lambda s: _report(s, d), srcs))
    out = {}
    for t in texts:
        out.update(_spills(t))
    return out


def test_every_kernel_was_reported(spills):
    for name in ("mttkrp_tc_kernel", "mttkrp_tts_kernel", "slice_a_kernel", "mttkrp_f64_kernel",
                 "update_fused_kernel", "update_phase_a", "reduce_partials", "align_kernel", "se_kernel"):
        assert any(name in fn for fn in spills), name


def test_no_register_spills(spills):
    for fn, stores in spills.items():
        allowed = next((v for k, v in KNOWN_SPILLS.items() if k in fn), 0)
        assert stores <= allowed, (fn, stores)
