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


def test_allocator_hook_out_of_memory_without_gpu(lib):
    """A caller allocator that refuses (returns NULL) makes the build fail
    with HMG_ERR_OOM before any device work: the failure is made on the host
    and the build releases what it had taken (nothing here).  NULL callbacks
    are an argument error."""
    import paper_1605_00492_gb300 as hmg
    L = hmg.load_library()
    calls = []

    def refuse(nbytes):
        calls.append(nbytes)
        return None
    released = []
    alloc = hmg.Allocator(refuse, released.append)
    ctx = ctypes.c_void_p()
    p = hmg.MeshParams(2, 8, 2, 6.371e6, 1e4)
    st = L.hmg_build_hierarchy_with_allocator(ctypes.byref(p), alloc.alloc_fn, alloc.release_fn, None,
                                              ctypes.byref(ctx))
    assert st == 3                         # HMG_ERR_OOM
    assert b"allocator returned NULL" in L.hmg_last_error(None)
    assert len(calls) == 1 and calls[0] > 0 and released == [] and not ctx.value
    with pytest.raises(hmg.HMGError) as e:
        hmg.Hierarchy(2, 8, 2, allocator=alloc)
    assert e.value.status == 3
    null_alloc = hmg.ALLOC_FN()
    null_release = hmg.RELEASE_FN()
    assert L.hmg_build_hierarchy_with_allocator(ctypes.byref(p), null_alloc, null_release, None,
                                                ctypes.byref(ctx)) == 1


def test_residual_history_argument_errors_without_gpu(lib):
    import paper_1605_00492_gb300 as hmg
    L = hmg.load_library()
    n = ctypes.c_int()
    assert L.hmg_residual_history(None, None, 0, ctypes.byref(n)) == 1
