"""Numerical calibration of the mixed-precision path on the GPU (through the C ABI).

The SFU exponential that every mixed response value goes through has a small mean relative
error over the exponents of a response profile.  The column normalisation divides out a fixed
value of that bias; this test re-measures it on the device at hand, so a GPU or driver whose SFU
behaves differently shows up here rather than as a drift of the mixed NLL.
"""
import pytest

from paper_1812_05686_gb300 import gsn

pytestmark = pytest.mark.gpu

COMPILED_EX2_BIAS = -2.749454e-8  # the value the column normalisation divides out


def test_sfu_exponential_bias_matches_the_compiled_correction():
    b = gsn.peak_probe(gsn.GSN_PROBE_EX2_BIAS)
    # the correction matters at the 1e-8 level; 3e-9 keeps the residual bias below 10% of it
    assert abs(b - COMPILED_EX2_BIAS) < 3e-9, b
