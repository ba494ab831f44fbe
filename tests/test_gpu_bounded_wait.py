"""Failure detection without a GPU fault: the bounded waits of the pipelined
kernels (jkcals_selftest_bounded_wait).  A wait on a barrier phase that nothing
completes gives up after its limit, records its code in the error word and
raises the CTA's abort flag; a second role blocked in a wait with a 64 times
longer limit leaves through that flag.  The kernel returns (no trap, no
fault), and the same process then runs a full parity-checked MTTKRP: the
context is still usable."""
import pytest

from paper_2112_03985_gb300 import _lib, api, workloads as W

from _helpers import compare_mttkrp

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("limit_ms", [5.0, 20.0])
def test_expired_wait_reports_and_aborts_the_other_roles(limit_ms):
    _cuda()
    st, code, left = api.selftest_bounded_wait(limit_ms)
    assert st == 0, _lib.load().jkcals_last_error()
    assert code == 3                      # the timing-out role's code, not the other role's (4)
    assert limit_ms <= left < 8 * limit_ms, left   # far below the second role's own 64x limit
    print(f"\nlimit {limit_ms} ms: the second waiter left after {left:.2f} ms")


def test_context_usable_after_an_expired_wait():
    _cuda()
    st, code, _ = api.selftest_bounded_wait(5.0)
    assert st == 0 and code == 3
    w = W.make_config(1)
    with api.from_workload(w, precision="exact_bf16") as h:
        U = h.get_factors()
        for n in range(w.T.ndim):
            compare_mttkrp(w, h.mttkrp(n), U, n, 1e-8)   # every submodel against the oracle


def test_argument_checks():
    _cuda()
    for bad in (0.0, -1.0, 1000.0):
        st, _, _ = api.selftest_bounded_wait(bad)
        assert st == 1   # JKCALS_ERR_ARG
