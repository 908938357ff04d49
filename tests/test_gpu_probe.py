"""The FMA-rate probe behind the roofline of the FP64-bound kernels: plausible
rates on a GB300 (nominal FP64 1.25 TFLOP/s, FP32 far above it) and argument
errors."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    f64 = dgsl.dgsl_measure_fma_rate(fp64=True)
    f32 = dgsl.dgsl_measure_fma_rate(fp64=False)
    print(f"FMA_RATE fp64 {f64 / 1e12:.3f} TFLOP/s fp32 {f32 / 1e12:.1f} TFLOP/s")
    assert 0.3e12 < f64 < 5e12
    assert f32 > 10 * f64


def test_fma_rate_argument_errors(dgsl_lib):
    import ctypes as C
    from paper_2401_17806_gb300 import dgsl
    v = C.c_double(0.0)
    assert dgsl.load().dgsl_measure_fma_rate(0, 2, C.byref(v)) == dgsl.EINVAL
    assert dgsl.load().dgsl_measure_fma_rate(0, 1, None) == dgsl.EINVAL
