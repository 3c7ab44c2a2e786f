"""The C ABI on a machine without a GPU: the library loads, exports every function that
include/spx.h declares, the Python binding declares each with the header's argument count,
and the host-only entry points (version, status names, size queries) answer."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spx.h")

spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import abi  # noqa: E402


def declarations():
    """{name: parameter count} of the function declarations in the header."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)                  # comments out
    out = {}
    for m in re.finditer(r"\b(?:spx_status|const char\s*\*|int32_t)\s+(spx_\w+)\s*\(([^;{]*?)\)\s*;", text, re.S):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_header_declares_the_entry_points():
    d = declarations()
    assert len(d) >= 50
    for name in ("spx_spmm", "spx_sddmm", "spx_spmm_t", "spx_csr_transpose", "spx_spgemm_numeric",
                 "spx_spgemm_backward", "spx_cg_batched", "spx_pcg_train", "spx_spadd_numeric", "spx_sptrsv",
                 "spx_spai_update", "spx_spmm_t_noalloc"):
        assert name in d, name


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(abi.LIB_PATH if os.path.exists(abi.LIB_PATH) else abi.lib()._name)
    missing = [n for n in declarations() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header_arity():
    d = declarations()
    host_only = {"spx_last_error", "spx_status_name", "spx_version"}   # restype set apart
    for name, argc in d.items():
        if name in host_only:
            continue
        assert name in abi.SIGNATURES, f"{name} has no binding"
        assert len(abi.SIGNATURES[name]) == argc, f"{name}: header {argc} args, binding {len(abi.SIGNATURES[name])}"


def test_host_only_entry_points():
    lib = abi.lib()
    assert lib.spx_version() == 200
    assert lib.spx_status_name(0) == b"SPX_OK"
    assert lib.spx_status_name(6) == b"SPX_BREAKDOWN"
    sz = ctypes.c_size_t(0)
    assert lib.spx_cg_workspace_size(1000, ctypes.byref(sz)) == 0
    assert sz.value >= 6 * 1000 * 4                                          # six float vectors
    assert lib.spx_spadd_workspace_size(1000, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.spx_cg_workspace_size(-1, ctypes.byref(sz)) == 1                  # SPX_INVALID_ARG
    assert b"bad arguments" in lib.spx_last_error()
