"""CPU checks of the C ABI: the library builds, loads and exports every entry
point that include/jkcals.h declares; the binding declares each with a signature.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(jkcals_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2112_03985_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("jkcals_create", "jkcals_mttkrp", "jkcals_als_sweep", "jkcals_run", "jkcals_grad",
                     "jkcals_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in sorted(declared_functions()):
        assert hasattr(built_lib, name), name


def test_binding_declares_every_symbol():
    from paper_2112_03985_gb300 import _lib
    assert declared_functions() == set(_lib.SIGNATURES)


def test_binding_loads_without_gpu(built_lib):
    from paper_2112_03985_gb300 import _lib
    lib = _lib.load()
    assert lib.jkcals_version().startswith(b"jkcals")
    opt = _lib.Options()
    lib.jkcals_default_options(ctypes.byref(opt))
    assert opt.precision == 0 and opt.normalise == 1 and opt.use_graph == 1
    assert opt.compact == 1 and opt.batch_branches == 0 and opt.autotune == 0


def header_option_fields():
    text = open(os.path.join(ROOT, "include", "jkcals.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} jkcals_options;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return [(m.group(1), m.group(2), int(m.group(3) or 1))
            for m in re.finditer(r"\b(int|int64_t)\s+(\w+)(?:\[(\d+)\])?\s*;", body)]


def test_options_struct_layout_matches_header():
    from paper_2112_03985_gb300 import _lib
    fields = header_option_fields()
    assert [f[1] for f in fields] == [f[0] for f in _lib.Options._fields_]
    for (ctype, name, count), (pname, ptype) in zip(fields, _lib.Options._fields_):
        base = ctypes.c_int64 if ctype == "int64_t" else ctypes.c_int
        assert ctypes.sizeof(ptype) == ctypes.sizeof(base) * count, name
    # int x 4, int64, int x 8 (with the reserved words) -> 16 + 8 + 32 = 56 bytes, as before
    assert ctypes.sizeof(_lib.Options) == 56


HANDLE_CALLS = ["jkcals_mttkrp", "jkcals_als_sweep", "jkcals_als_sweep_async", "jkcals_kernel_times",
                "jkcals_sweep_info", "jkcals_mode_plan", "jkcals_jackknife_se", "jkcals_run", "jkcals_run_block_sweeps",
                "jkcals_get_factors",
                "jkcals_set_factors", "jkcals_get_block_status", "jkcals_grad", "jkcals_loss_history", "jkcals_sync"]


@pytest.mark.parametrize("name", HANDLE_CALLS)
def test_null_handle_is_an_argument_error(built_lib, name):
    """Every call on a handle checks it first: a NULL handle returns JKCALS_ERR_ARG (no device
    is touched) and leaves a message for jkcals_last_error."""
    from paper_2112_03985_gb300 import _lib
    lib = _lib.load()
    _, argtypes = _lib.SIGNATURES[name]
    args = []
    for t in argtypes:
        if t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64):
            args.append(0)
        elif t is ctypes.c_double:
            args.append(0.0)
        else:
            args.append(None)
    assert getattr(lib, name)(*args) == 1
    assert b"NULL handle" in lib.jkcals_last_error()
