"""CPU checks of the C ABI: the library builds, loads, and exports every
function declared in include/hmg.h (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmg_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_00492_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hmg_build_hierarchy", "hmg_assemble_helmholtz", "hmg_apply", "hmg_vcycle", "hmg_solve",
                     "hmg_theta_grad", "hmg_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_errors_without_gpu(lib):
    lib.hmg_status_string.restype = ctypes.c_char_p
    assert lib.hmg_status_string(0) == b"ok"
    assert lib.hmg_status_string(4) == b"not converged"
    # invalid arguments are rejected before any CUDA call
    import paper_1605_00492_gb300 as hmg
    L = hmg.load_library()
    ctx = ctypes.c_void_p()
    bad = hmg.MeshParams(3, 0, 3, 6.371e6, 1e4)          # nlayers = 0
    assert L.hmg_build_hierarchy(ctypes.byref(bad), ctypes.byref(ctx)) == 1
    assert b"nlayers" in L.hmg_last_error(None)
    bad = hmg.MeshParams(2, 8, 4, 6.371e6, 1e4)          # nlevels > refinement + 1
    assert L.hmg_build_hierarchy(ctypes.byref(bad), ctypes.byref(ctx)) == 1
    assert L.hmg_build_hierarchy(None, ctypes.byref(ctx)) == 1
    assert L.hmg_apply(None, 0, 0, 0, None, None, None) == 1
    assert L.hmg_solve(None, None, None, None, None, None) == 1
    assert L.hmg_destroy(None) == 0
