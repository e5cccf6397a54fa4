"""Fifth-generation tensor-core path (tcgen05): one BF16 MMA with an FP32
accumulator in tensor memory per operand layout, against the same integer sums
on the CUDA cores (exact)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2204_13254_gb300 import dd as D

pytestmark = pytest.mark.gpu


def test_tcgen05_kmajor_mma_exact():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mask = D.dd_tc_selftest()
    print(f"tcgen05 self-test mask {mask:#x}")
    assert mask & 1, f"K-major BF16 MMA did not match the CUDA cores (mask {mask:#x})"
