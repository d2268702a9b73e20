"""The FP64 FMA throughput probe (hmg_measure_fp64_rate), the measured roof
of the FP64 cycle's kernels: it runs, and lands near the rate derived from
the pipe's issue interval (152 SMs x 4 sub-partitions x 32 lanes every 64
cycles x 2 flops at the 2.07 GHz maximum clock = 1.259 TFLOP/s); the bounds
allow for a lower clock under load."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402


def test_fp64_rate_probe():
    h = hmg.Hierarchy(1, 4, 1)
    rate = h.measure_fp64_rate()
    assert 0.5 < rate < 1.5
    h.close()
