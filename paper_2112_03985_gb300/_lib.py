"""ctypes declarations of the C ABI in include/jkcals.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjkcals.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_SPD, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = range(8)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_SPD",
                5: "ERR_TIMEOUT", 6: "ERR_STATE", 7: "ERR_UNSUPPORTED"}
PREC = {"fp64": 0, "tf32": 1, "3xtf32": 2, "bf16": 3, "split_bf16": 4, "exact_bf16": 5}
DTYPE_F32, DTYPE_F64 = 0, 1
BLOCK_NOT_SPD, BLOCK_CONVERGED = 1, 2


class Options(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("normalise", ct.c_int), ("use_graph", ct.c_int),
                ("splits", ct.c_int), ("max_device_bytes", ct.c_int64),
                ("kernel_timing", ct.c_int), ("update_mode", ct.c_int), ("autotune", ct.c_int),
                ("compact", ct.c_int), ("batch_branches", ct.c_int), ("reserved", ct.c_int * 3)]


P = ct.c_void_p
PP = ct.POINTER(ct.c_void_p)
I64P = ct.POINTER(ct.c_int64)
I32P = ct.POINTER(ct.c_int32)

# name -> (restype, argtypes); every symbol declared in include/jkcals.h
SIGNATURES = {
    "jkcals_default_options": (None, [ct.POINTER(Options)]),
    "jkcals_create": (ct.c_int, [ct.POINTER(P), ct.c_int, I64P, P, ct.c_int, ct.c_int, ct.c_int,
                                 I32P, I64P, I64P, PP, ct.POINTER(Options), P]),
    "jkcals_destroy": (None, [P]),
    "jkcals_mttkrp": (ct.c_int, [P, ct.c_int, P]),
    "jkcals_als_sweep": (ct.c_int, [P, ct.c_int, P]),
    "jkcals_als_sweep_async": (ct.c_int, [P, ct.c_int, P]),
    "jkcals_kernel_times": (ct.c_int, [P, ct.POINTER(ct.c_double)]),
    "jkcals_sweep_info": (ct.c_int, [P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "jkcals_jackknife_se": (ct.c_int, [P, ct.c_int, PP, PP, P, PP, ct.POINTER(ct.c_int)]),
    "jkcals_plan_query": (ct.c_int, [ct.c_int, I64P, ct.c_int, I32P, ct.POINTER(Options), ct.c_int, I32P, I32P,
                                     I32P, I32P]),
    "jkcals_mode_plan": (ct.c_int, [P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                    ct.POINTER(ct.c_int)]),
    "jkcals_run": (ct.c_int, [P, ct.c_int, ct.c_double, ct.POINTER(ct.c_int), P]),
    "jkcals_run_block_sweeps": (ct.c_int, [P, I32P]),
    "jkcals_get_factors": (ct.c_int, [P, PP]),
    "jkcals_set_factors": (ct.c_int, [P, PP]),
    "jkcals_get_block_status": (ct.c_int, [P, I32P]),
    "jkcals_grad": (ct.c_int, [P, PP, PP, P]),
    "jkcals_loss_history": (ct.c_int, [P, ct.c_int, P]),
    "jkcals_batch_create": (ct.c_int, [ct.POINTER(P), ct.c_int, PP, ct.c_int, P]),
    "jkcals_batch_sweep": (ct.c_int, [P, ct.c_int]),
    "jkcals_batch_sync": (ct.c_int, [P]),
    "jkcals_batch_destroy": (None, [P]),
    "jkcals_sync": (ct.c_int, [P]),
    "jkcals_selftest_bounded_wait": (ct.c_int, [ct.c_double, I32P, ct.POINTER(ct.c_double)]),
    "jkcals_mttkrp_f64_noalloc": (ct.c_int, [ct.c_int, I64P, ct.c_int, P, PP, ct.c_int, P, P]),
    "jkcals_last_error": (ct.c_char_p, []),
    "jkcals_version": (ct.c_char_p, []),
}

_lib = None


def load():
    """Load libjkcals.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2112_03985_gb300.build` (there is no CPU fallback)")
    lib = ct.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class JKError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = load().jkcals_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def check(status, where):
    if status != OK:
        raise JKError(status, where)
