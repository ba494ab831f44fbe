"""Argument checks of the entry points that take no handle (no GPU): jkcals_create,
jkcals_batch_create, jkcals_mttkrp_f64_noalloc and jkcals_selftest_bounded_wait reject every
invalid shape, block layout, option or limit with its status and message before the device is
touched."""
import ctypes as ct

import numpy as np
import pytest

from paper_2112_03985_gb300 import _lib as L

ARG, UNSUPPORTED = 1, 7


def _create(N=3, dims=(6, 5, 4), T=True, dtype=1, n_hat=0, ranks=(2, 2), ptr=(0, 1, 2), idx=(0, 3),
            init=True, init_null=None, opt=None, out=True):
    lib = L.load()
    keep = []
    d = np.asarray(dims, dtype=np.int64)
    r = np.asarray(ranks, dtype=np.int32)
    p = np.asarray(ptr, dtype=np.int64)
    i = np.asarray(idx, dtype=np.int64) if idx is not None else None
    Tbuf = np.zeros(4)
    keep += [d, r, p, i, Tbuf]
    inits = (ct.c_void_p * max(N, 1))()
    for k in range(max(N, 1)):
        a = np.zeros(4)
        keep.append(a)
        inits[k] = None if init_null == k else a.ctypes.data
    o = L.Options()
    lib.jkcals_default_options(ct.byref(o))
    for key, val in (opt or {}).items():
        setattr(o, key, val)
    h = ct.c_void_p()
    st = lib.jkcals_create(ct.byref(h) if out else None, N, d.ctypes.data_as(L.I64P),
                           ct.c_void_p(Tbuf.ctypes.data) if T else None, dtype, n_hat, len(r),
                           r.ctypes.data_as(L.I32P), p.ctypes.data_as(L.I64P),
                           i.ctypes.data_as(L.I64P) if i is not None else None,
                           inits if init else None, ct.byref(o), None)
    assert not h.value
    return st, lib.jkcals_last_error().decode()


CASES = [
    ("out NULL", dict(out=False), ARG, "out is NULL"),
    ("one mode", dict(N=1, dims=(6,)), ARG, "N must be"),
    ("nine modes", dict(N=9, dims=(2,) * 9), UNSUPPORTED, "N must be"),
    ("T NULL", dict(T=False), ARG, "NULL argument"),
    ("init NULL", dict(init=False), ARG, "NULL argument"),
    ("bad dtype", dict(dtype=5), ARG, "T_dtype"),
    ("empty mode", dict(dims=(6, 0, 4)), ARG, "dims must be >= 1"),
    ("2^40 elements", dict(dims=(1 << 14, 1 << 14, 1 << 12)), UNSUPPORTED, "2^40"),
    ("mode too long", dict(dims=(8388481, 1, 1)), UNSUPPORTED, "dims must be <="),
    ("sampled mode", dict(n_hat=3), ARG, "sampled_mode"),
    ("no blocks", dict(ranks=(), ptr=(0,), idx=None), ARG, "K must be"),
    ("rank 0", dict(ranks=(2, 0)), ARG, "ranks must be >= 1"),
    ("rank 33", dict(ranks=(2, 33)), UNSUPPORTED, "ranks must be <= 32"),
    ("ptr start", dict(ptr=(1, 1, 2)), ARG, "left_out_ptr[0]"),
    ("ptr order", dict(ptr=(0, 2, 1)), ARG, "non-decreasing"),
    ("idx NULL", dict(idx=None), ARG, "left_out_idx is NULL"),
    ("idx range", dict(idx=(0, 6)), ARG, "out of range"),
    ("idx negative", dict(idx=(-1, 2)), ARG, "out of range"),
    ("duplicate", dict(ptr=(0, 2, 2), idx=(3, 3)), ARG, "duplicate"),
    ("leaves all out", dict(ptr=(0, 6, 6), idx=(0, 1, 2, 3, 4, 5)), ARG, "every sample"),
    ("init[1] NULL", dict(init_null=1), ARG, "init[n] is NULL"),
    ("precision", dict(opt={"precision": 9}), ARG, "precision"),
    ("splits", dict(opt={"splits": -1}), ARG, "splits"),
    ("update mode", dict(opt={"update_mode": 3}), ARG, "update_mode"),
]


@pytest.mark.parametrize("name,kw,status,msg", CASES, ids=[c[0] for c in CASES])
def test_create_rejects(name, kw, status, msg):
    st, err = _create(**kw)
    assert st == status, (st, err)
    assert msg in err, err


def test_too_many_columns_is_unsupported():
    K = 131071
    st, err = _create(ranks=(32,) * K, ptr=(0,) * (K + 1), idx=None)
    assert st == UNSUPPORTED and "sum of ranks" in err, err


def test_batch_create_needs_handles_and_sweeps():
    lib = L.load()
    b = ct.c_void_p()
    hs = (ct.c_void_p * 1)(None)
    assert lib.jkcals_batch_create(None, 1, hs, 10, None) == ARG
    assert lib.jkcals_batch_create(ct.byref(b), 0, hs, 10, None) == ARG
    assert lib.jkcals_batch_create(ct.byref(b), 1, None, 10, None) == ARG
    assert lib.jkcals_batch_create(ct.byref(b), 1, hs, 0, None) == ARG
    assert lib.jkcals_batch_create(ct.byref(b), 1, hs, 10, None) == ARG   # a NULL handle in the list
    assert b.value is None


NOALLOC = [
    ("one mode", dict(N=1), ARG, "N must be"),
    ("NULL dims", dict(dims=None), ARG, "NULL argument"),
    ("mode", dict(mode=3), ARG, "mode out of range"),
    ("no columns", dict(C=0), ARG, "C must be >= 1"),
    ("too many columns", dict(C=65535 * 64 + 1), UNSUPPORTED, "C must be <="),
    ("empty mode", dict(dims=(6, 0, 4)), ARG, "dims must be >= 1"),
    ("2^40 elements", dict(dims=(1 << 14, 1 << 14, 1 << 12)), UNSUPPORTED, "2^40"),
    ("scratch", dict(dims=(70000, 5, 4), C=32), UNSUPPORTED, "static scratch"),
]


@pytest.mark.parametrize("name,kw,status,msg", NOALLOC, ids=[c[0] for c in NOALLOC])
def test_noalloc_rejects(name, kw, status, msg):
    lib = L.load()
    N = kw.get("N", 3)
    dims = kw.get("dims", (6, 5, 4))
    d = np.asarray(dims, dtype=np.int64) if dims is not None else None
    buf = np.zeros(4)
    U = (ct.c_void_p * 3)(buf.ctypes.data, buf.ctypes.data, buf.ctypes.data)
    st = lib.jkcals_mttkrp_f64_noalloc(N, d.ctypes.data_as(L.I64P) if d is not None else None, kw.get("mode", 0),
                                       ct.c_void_p(buf.ctypes.data), U, kw.get("C", 4),
                                       ct.c_void_p(buf.ctypes.data), None)
    err = lib.jkcals_last_error().decode()
    assert st == status, (st, err)
    assert msg in err, err


@pytest.mark.parametrize("limit_ms,code_ok,left_ok", [(0.0, True, True), (-1.0, True, True), (100.5, True, True),
                                                      (float("nan"), True, True), (20.0, False, True),
                                                      (20.0, True, False)])
def test_bounded_wait_selftest_argument_checks(limit_ms, code_ok, left_ok):
    """jkcals_selftest_bounded_wait rejects a limit outside (0, 100] ms or a missing
    output with ERR_ARG before any CUDA call."""
    lib = L.load()
    code = ct.c_int32(-1)
    left = ct.c_double(-1.0)
    st = lib.jkcals_selftest_bounded_wait(limit_ms, ct.byref(code) if code_ok else None,
                                          ct.byref(left) if left_ok else None)
    assert st == ARG
    assert "limit_ms" in lib.jkcals_last_error().decode()
    assert code.value == -1 and left.value == -1.0   # outputs untouched
