"""The arithmetic-peak probes (mtf_probe_peaks) that the benchmark divides
the assembly kernels' flop rates by: positive, finite rates in the expected
order (the FP32 FMA pipes far wider than FP64 on this GPU) and repeatable to
a few percent between calls."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import _lib
    return _lib


def test_probe_rates_are_plausible_and_repeatable(L):
    a = np.array(L.mtf_probe_peaks())
    b = np.array(L.mtf_probe_peaks())
    assert np.all(np.isfinite(a)) and np.all(a > 0)
    fp32, fp64, sfu = a
    assert fp32 > 5e12 and fp64 > 1e11 and sfu > 1e11, a
    assert fp32 > 10 * fp64, a
    assert np.all(np.abs(a - b) <= 0.1 * np.maximum(a, b)), (a, b)
