"""CPU-only checks of the C ABI boundary: the library builds, loads without a
GPU, exports every function include/spx.h declares, and the Python binding
declares a signature for each of them.  No compute call is made."""
import os
import re

import pytest

from paper_2103_10116_gb300 import build as spx_build
from paper_2103_10116_gb300 import spx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(spx_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    spx_build.build()
    return spx.load(build_if_missing=False)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("spx_ctx_create", "spx_matrix_create", "spx_spmv", "spx_solve", "spx_batch_solve",
                 "spx_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_a_signature_for_every_symbol():
    missing = [n for n in declared_functions() if n not in spx.SIGNATURES]
    assert not missing, missing


def test_host_only_calls(lib):
    assert spx.spx_version() >= 100
    assert spx.spx_status_str(spx.SPX_ERR_INVALID) == "SPX_ERR_INVALID"
    assert spx.spx_status_str(12345) == "SPX_ERR_UNKNOWN"
    assert isinstance(spx.spx_last_error(), str)


def test_null_arguments_are_rejected_without_a_gpu(lib):
    import ctypes as C
    # argument validation happens before any CUDA call
    assert lib.spx_matrix_get_info(None, None) == spx.SPX_ERR_INVALID
    assert lib.spx_spmv(None, None, None, None) == spx.SPX_ERR_INVALID
    assert lib.spx_ctx_set_grid_sms(None, 0, None) == spx.SPX_ERR_INVALID
    assert lib.spx_server_set_slot_sms(None, 0, None) == spx.SPX_ERR_INVALID
    assert lib.spx_server_set_cluster_rows(None, 0, None) == spx.SPX_ERR_INVALID
    assert "NULL" in spx.spx_last_error()
    out = C.c_void_p()
    assert lib.spx_matrix_create(None, C.byref(out), 0, 0, 1, 1, 0, None, None, None, 0, -1, 0) == spx.SPX_ERR_INVALID


def test_header_constants_match_binding():
    """Every integer #define and enum constant of include/spx.h that the binding
    also names has the same value there."""
    src = open(os.path.join(ROOT, "include", "spx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"^#define\s+(SPX_\w+)\s+(0x[0-9a-fA-F]+|\d+)u?\s*$",
                                                                   src, flags=re.M)}
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"(SPX_\w+)\s*=\s*(-?\d+)", body):
            consts[name] = int(val)
    assert "SPX_SOLVE_ONE_CLUSTER" in consts and "SPX_CG" in consts
    checked = [n for n in consts if hasattr(spx, n)]
    assert len(checked) >= 20
    bad = {n: (consts[n], getattr(spx, n)) for n in checked if getattr(spx, n) != consts[n]}
    assert not bad, bad
