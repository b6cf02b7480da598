"""The C ABI library builds, loads without a GPU and exports every entry
point that include/*.h declares; host-side argument checks need no GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(agipc_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2605_04773_gb300 import build
    try:
        path = build.build()
    except (OSError, RuntimeError) as e:  # no nvcc on this machine
        pytest.skip("cannot build the CUDA library here: %s" % e)
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 8
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    lib.agipc_status_string.restype = ctypes.c_char_p
    for code in range(-7, 1):
        s = lib.agipc_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.agipc_status_string(-99).decode() == "unknown status"


def test_null_context_is_rejected_on_host(lib):
    """Host-side argument checks return INVALID_ARG before touching a GPU."""
    P = ctypes.c_void_p
    lib.agipc_aggregate.argtypes = [P, ctypes.c_int32, ctypes.c_int64, P, P, P, P]
    assert lib.agipc_aggregate(None, 10, 0, None, None, None, None) == -1
    lib.agipc_prolongate.argtypes = [P, ctypes.c_int32, P, P, P]
    assert lib.agipc_prolongate(None, 10, None, None, None) == -1
    lib.agipc_create.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    assert lib.agipc_create(None, None, 1, 1, 1, 1) == -1
    lib.agipc_set_assembly_run.argtypes = [P, ctypes.c_int32]
    assert lib.agipc_set_assembly_run(None, 8) == -1


def test_binding_fails_loudly_without_gpu():
    import torch
    from paper_2605_04773_gb300 import agipc
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        agipc.Context(10, 10, 10, 0)


def test_pcg_options_layout_matches_header():
    # agipc_pcg_options in include/agipc.h: double tol; int32 max_iter,
    # rhs_sign, use_x0, streamed -- 24 bytes, 'streamed' in what was the
    # struct's tail padding.  The binding's ctypes copy must match it field
    # by field, and the header must declare the fields in that order.
    from paper_2605_04773_gb300 import agipc
    O = agipc._PcgOptions
    assert ctypes.sizeof(O) == 24
    assert [(n, getattr(O, n).offset) for n, _ in O._fields_] == [
        ("tol", 0), ("max_iter", 8), ("rhs_sign", 12), ("use_x0", 16), ("streamed", 20)]
    hdr = open(os.path.join(ROOT, "include", "agipc.h")).read()
    body = hdr[hdr.index("typedef struct {", hdr.index("PCG options")):hdr.index("} agipc_pcg_options;")]
    fields = re.findall(r"^\s*(double|int32_t)\s+(\w+);", body, re.M)
    assert fields == [("double", "tol"), ("int32_t", "max_iter"), ("int32_t", "rhs_sign"), ("int32_t", "use_x0"),
                      ("int32_t", "streamed")]
