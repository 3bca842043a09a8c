"""Numerical calibration of the mixed-precision path on the GPU (through the C ABI).

The SFU exponential that every mixed response value goes through has a small mean relative
error over the exponents of a response profile.  A mixed-precision context measures it on its
device when it is created (once per device and process) and divides it out of the column
normalisation.  The probe that measures it must be reproducible, and the bias must be small
enough that dividing it out is a correction rather than a compensation for a broken unit.
"""
import pytest

from paper_1812_05686_gb300 import gsn

pytestmark = pytest.mark.gpu


def test_sfu_exponential_bias_is_small_and_reproducible():
    b1 = gsn.peak_probe(gsn.GSN_PROBE_EX2_BIAS)
    b2 = gsn.peak_probe(gsn.GSN_PROBE_EX2_BIAS)
    # the contexts keep the value rounded to 1e-13: repeated measurements differ by far less
    assert abs(b1 - b2) < 1e-14, (b1, b2)
    # ex2.approx has about 22 correct bits; a mean error beyond 2^-22 would not be rounding
    assert abs(b1) < 2.4e-7, b1
