"""The arithmetic-ceiling probe behind the blend's roofline figure."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402


def test_alu_probe_is_plausible():
    r = lfd.measure_alu_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # 128 FP32 lanes per SM at 1-2.5 GHz, within a factor the probe cannot miss
    per_sm = r["fp32_ops_per_s"] / sms
    assert 0.5 * 128e9 < per_sm < 1.2 * 128 * 2.5e9, r
    # the exp2 pipe is far narrower than the FP32 pipe
    assert 0 < r["ex2_per_s"] < r["fp32_ops_per_s"] / 2, r
