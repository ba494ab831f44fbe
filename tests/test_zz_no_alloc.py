"""The allocation-free MTTKRP entry point (jkcals_mttkrp_f64_noalloc).

Some callers cannot allocate device memory at all: a solver running inside a
memory pool or arena that another framework owns, a step whose memory budget
was fixed up front, or a latency-critical loop where a cudaMalloc would stall
the device.  They cannot create a handle (a handle allocates its tensor copies
and workspace), so the library offers this one call, which allocates nothing
and keeps its split-K partials in a fixed device array.  The test checks it
against the handle's own MTTKRP (jkcals_mttkrp) and against the oracle's
MTTKRP of the same factors, element by element within the 1e-12 tolerance used
for the FP64 MTTKRP everywhere else, on two calls in a row per mode, so that a
second call over the leftovers of the first is covered too.  This file
is collected last so that a run stopping at its first failure has already run
every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu

MTTKRP_RTOL = 1e-12


def test_noalloc_mttkrp_matches_handle_mttkrp_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.make_workload("noalloc 41x33x65 R3", (41, 33, 65), 3, blocks=W.loo_blocks(41, include_full=True),
                        noise=0.01, seed=21)
    with api.from_workload(w) as h:
        U = h.get_factors()
        ref = [h.mttkrp(n) for n in range(3)]
    dev = torch.device("cuda", torch.cuda.current_device())
    Ud = [torch.from_numpy(u).to(dev) for u in U]
    # the unfoldings the caller supplies: columns in Eq. kolda_mapping order
    Tn = [torch.from_numpy(np.ascontiguousarray(O.unfold(w.T, n))).to(dev) for n in range(3)]
    for call in range(2):
        for n in range(3):
            out = torch.full((w.dims[n], w.C), float("nan"), dtype=torch.float64, device=dev)
            # U[n] is not read: pass None for it on the second call
            api.mttkrp_f64_noalloc(Tn[n], [None if (call and k == n) else u for k, u in enumerate(Ud)], n, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            # against the handle's MTTKRP (jkcals_mttkrp) ...
            np.testing.assert_allclose(got, ref[n], rtol=MTTKRP_RTOL, atol=MTTKRP_RTOL * np.abs(ref[n]).max(),
                                       err_msg=f"call {call} mode {n}: vs jkcals_mttkrp")
            # ... and against the oracle's MTTKRP of the same factors (Alg. 3 MTTKRP line)
            ora = O.mttkrp(w.T, U, n)
            np.testing.assert_allclose(got, ora, rtol=MTTKRP_RTOL, atol=MTTKRP_RTOL * np.abs(ora).max(),
                                       err_msg=f"call {call} mode {n}: vs the oracle")


def test_noalloc_rejects_oversized_and_host_buffers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", torch.cuda.current_device())
    # dims[mode] * C = 2^21 + 1 doubles needed > the 2^21 scratch
    U = [torch.zeros((2049, 1024), dtype=torch.float64, device=dev),
         torch.zeros((2, 1024), dtype=torch.float64, device=dev)]
    Tn = torch.zeros((2049, 2), dtype=torch.float64, device=dev)
    out = torch.zeros((2049, 1024), dtype=torch.float64, device=dev)
    with pytest.raises(api.JKError) as ei:
        api.mttkrp_f64_noalloc(Tn, U, 0, out)
    assert ei.value.status == 7
    small = [torch.zeros((4, 3), dtype=torch.float64), torch.zeros((5, 3), dtype=torch.float64)]
    with pytest.raises(api.JKError) as ei:      # host buffers: rejected before any launch
        api.mttkrp_f64_noalloc(torch.zeros((4, 5), dtype=torch.float64), small, 0,
                               torch.zeros((4, 3), dtype=torch.float64))
    assert ei.value.status == 1
