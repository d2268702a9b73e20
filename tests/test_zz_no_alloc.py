"""hmg_apply_noalloc: the operator application for callers that may not
allocate device memory at the call (see include/hmg.h), checked through the
C ABI against hmg_apply on two calls in a row.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402

TOL = 1e-13   # the tolerance of the FP64 operator tests


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_apply_matches_apply_twice_in_a_row():
    h = hmg.Hierarchy(3, 16, 3)
    h.assemble()
    lib = hmg.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(21)
    for level in (0, 2):
        n = h.levels[level]["ncells"]
        for _ in range(2):   # two calls in a row: the second must not see the first's contents
            x = torch.tensor(rng.standard_normal(n), device="cuda")
            y_ref = h.apply(x, level=level)
            y = torch.full_like(x, float("nan"))
            st = lib.hmg_apply_noalloc(h._ctx, level, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       stream)
            assert st == 0, lib.hmg_last_error(h._ctx)
            torch.cuda.synchronize()
            assert _rel(y, y_ref) <= TOL
    h.close()


def test_noalloc_apply_rejects_levels_above_its_limit():
    h = hmg.Hierarchy(5, 32, 1)          # 20480 columns x 32 layers = 655360 > 524288 cells
    h.assemble()
    x = torch.ones(h.ncells, dtype=torch.float64, device="cuda")
    with pytest.raises(hmg.HMGError) as e:
        h.apply_noalloc(x, out=torch.empty_like(x))
    assert e.value.name == "HMG_ERR_INVALID_ARG"
    assert "fixed scratch" in str(e.value)
    h.close()
