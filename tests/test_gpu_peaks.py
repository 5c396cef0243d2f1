"""The measured CUDA-core peaks (tri_alu_peak) that the bench divides the CUDA-core
kernels' throughput by: positive, repeatable, and not above what the SM count and the
maximum SM clock allow (128 FP32 FMA lanes per SM and clock)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    return _lib


def test_alu_peaks_are_plausible(lib):
    props = torch.cuda.get_device_properties(0)
    bound32 = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12     # above the 2070 MHz max clock
    f32a, _ = lib.tri_alu_peak(lib.TRI_F32, 1 << 16)
    f32b, _ = lib.tri_alu_peak(lib.TRI_F32, 1 << 16)
    f64, _ = lib.tri_alu_peak(lib.TRI_F64, 1 << 12)
    assert 0.25 * bound32 < f32a <= bound32 and 0.25 * bound32 < f32b <= bound32
    assert abs(f32a - f32b) <= 0.2 * max(f32a, f32b)
    assert 0.0 < f64 < f32a
    with pytest.raises(lib.TriError):
        lib.tri_alu_peak(lib.TRI_F32_MIXED, 1 << 12)
