"""Host logic of bench.py on CPU: the algorithmic byte model of the timed sweep and the
L2-flush decision of the timing loop."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("prec, planes, B, expect", [
    ("fp32", 4, 1, 41),        # 7-point half planes: 4 coefficients + 6 vectors + mult byte
    ("fp32", 7, 1, 53),        # 7-point full planes
    ("fp32", 14, 1, 81),       # 27-point half planes
    ("fp32", 27, 1, 133),
    ("fp64", 7, 1, 105),
    ("bf16", 7, 1, 39),        # BF16 coefficients, FP32 vectors
    ("fp32", 243, 3, 1045),    # elasticity: 9 blocks of 27 points, 3 components
    ("fp64", 243, 3, 2089),
])
def test_sweep_bytes(prec, planes, B, expect):
    assert bench.sweep_bytes(prec, planes, B) == expect


def test_sweep_flops():
    assert bench.sweep_flops(7) == 20
    assert bench.sweep_flops(27, 3) == 2 * 9 * 27 + 18


class _T:
    """Shape-only stand-in for a tensor (numel, element_size)."""
    def __init__(self, n, size):
        self.n, self.size = n, size

    def numel(self):
        return self.n

    def element_size(self):
        return self.size


class _DP:
    def __init__(self, n, nnz):
        self.rowptr, self.col = _T(n + 1, 8), _T(nnz, 8)
        self.val, self.b = _T(nnz, 8), _T(n, 8)


def test_input_bytes_counts_csr_and_rhs():
    dp = _DP(1000, 7000)
    assert bench.input_bytes(dp) == 8 * 1001 + 16 * 7000 + 8 * 1000


def test_l2_flush_only_when_inputs_fit_in_l2():
    torch = pytest.importorskip("torch")
    big = _DP(29_438_045, 206_070_415)           # the 3D diffusion workload's CSR
    assert bench.input_bytes(big) > bench.L2_BYTES
    assert bench.l2_flush_buffer(big, "cpu") is None
    small = _DP(25_921, 129_609)                 # the 2D Poisson workload's CSR
    buf = bench.l2_flush_buffer(small, "cpu")
    assert isinstance(buf, torch.Tensor)
    assert buf.numel() * buf.element_size() == 2 * bench.L2_BYTES > bench.L2_BYTES


def test_peaks_use_measured_file_or_fallback():
    pk = bench.peaks()
    assert pk["src"] in ("measured", "fallback")
    assert pk["hbm_gbs"] > 1000
    # FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x clock
    assert pk["fp64_tflops"] == pytest.approx(152 * 4 * pk.get("sm_max_mhz", 2070.0) * 1e-6)
