"""The measured rates that the rooflines divide by: the vector FMA rates of
the arithmetic roofline, each within a factor of two of the GPU's nominal
rate (GB300: 152 SMs x 128 FP32 lanes x 2 x ~2 GHz ~ 80 TFLOP/s; FP64
1.25 TFLOP/s nominal), and the host-link copy rates of the end-to-end one."""
import pytest

from paper_1207_3392_gb300 import hydro as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1207_3392_gb300 import build
    build.build()


def test_fma_rates_are_plausible():
    fp64 = H.measure_fma_rate(0)
    fp32 = H.measure_fma_rate(1)
    fp32x2 = H.measure_fma_rate(2)
    print(f"FMA rates: FP64 {fp64:.3f}, FP32 {fp32:.1f}, FP32 pairs {fp32x2:.1f} TFLOP/s")
    assert 0.6 < fp64 < 2.5, fp64
    assert 40.0 < fp32 < 160.0, fp32
    assert 40.0 < fp32x2 < 320.0, fp32x2
    with pytest.raises(H.HydroError):
        H.measure_fma_rate(3)


def test_link_rates_are_plausible():
    """The host-link copy rates that the end-to-end roofline divides by: each
    direction between 20 GB/s (slower than any PCIe or NVLink-C2C host link of
    this class) and 1 TB/s, and both directions at once no slower than one."""
    h2d, d2h, both = (H.measure_link_rate(k) for k in range(3))
    print(f"link rates: H2D {h2d:.0f}, D2H {d2h:.0f}, both {both:.0f} GB/s")
    for r in (h2d, d2h):
        assert 20.0 < r < 1000.0, r
    assert 0.9 * max(h2d, d2h) < both < 2000.0, (h2d, d2h, both)
    with pytest.raises(H.HydroError):
        H.measure_link_rate(3)
