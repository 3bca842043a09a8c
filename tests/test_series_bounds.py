"""Bounds behind the mixed gamma path's branch-free series (host arithmetic, FP64).

Columns of shape d >= 50 evaluate D(t) = ln(1+t) - t from the odd series in u = t/(2+t),
D = -t u + 2u^3 (1/3 + u^2/5 + ... + u^8/11), truncated after u^11.  The omitted terms have one
sign on each side of the peak, so their effect does not average out over columns; what bounds
it is their effect on a column's mass over its band (the bins where log f(x)/f(mu) >= -20.7).
Here that effect is computed on a fine grid in t for the shapes at the ends of the range the
packed path takes, with the exponent the kernels evaluate, (d-1) D(t) - t, and held to the
bounds the kernels' comments state: 4e-10 at d = 50, 1e-11 at d = 100, 1e-13 at d = 300.  One
more omitted term would break the d = 50 bound (6e-9)."""
import numpy as np
import pytest

CUT = 20.7


def _series_D(t, ncoef):
    u = t / (2.0 + t)
    v = u * u
    p = np.zeros_like(u)
    for k in reversed(range(ncoef)):      # coefficients 1/3, 1/5, ..., 1/(2 ncoef + 1)
        p = p * v + 1.0 / (2 * k + 3)
    return -t * u + 2.0 * u * v * p


def _mass_change(d, ncoef):
    t = np.linspace(-0.999, 3.0, 2_000_001)
    h = (d - 1.0) * (np.log1p(t) - t) - t
    band = h >= -CUT
    f = np.exp(h[band])
    hs = (d - 1.0) * _series_D(t[band], ncoef) - t[band]
    return abs(np.exp(hs).sum() - f.sum()) / f.sum(), np.max(np.abs(t[band] / (2.0 + t[band])))


@pytest.mark.parametrize("d,bound", [(50.0, 4.5e-10), (100.0, 1e-11), (300.0, 1e-13)])
def test_truncated_series_changes_a_column_mass_within_the_stated_bound(d, bound):
    rel, umax = _mass_change(d, 5)       # through u^11
    assert rel < bound, (d, rel)
    assert umax < 0.51                   # |u| inside the band of the packed path


def test_one_more_omitted_term_would_break_the_bound():
    rel, _ = _mass_change(50.0, 4)       # through u^9
    assert rel > 1e-9, rel


def test_mode_offset_series_matches_its_closed_form():
    """The gamma column's exponent offset XM = log2 f(mode)/f(mu), for shape d >= 8, is summed as
    M(d) = (d-1) ln(1 - 1/d) + 1 = sum_k u^k / (k (k+1)), u = 1/d, truncated after u^8 (the column
    prologue's series); held against the closed form evaluated with log1p in FP64."""
    d = np.geomspace(8.0, 1e5, 2000)
    u = 1.0 / d
    m = np.zeros_like(u)
    for k in reversed(range(1, 9)):
        m = (m + 1.0 / (k * (k + 1))) * u
    exact = (d - 1.0) * np.log1p(-1.0 / d) + 1.0
    assert np.max(np.abs(m / exact - 1.0)) < 2e-9


def test_normalisation_exponential_polynomial():
    """exp(y) of the column normalisation, |y| < 0.06 (y = XM ln 2 - Stirling remainder, d >= 8),
    by its degree-6 Taylor polynomial: remainder below 1e-12 relative."""
    y = np.linspace(-0.06, 0.06, 20001)
    p = np.zeros_like(y)
    for k in reversed(range(7)):
        p = p * y + 1.0 / np.prod(np.arange(1, k + 1, dtype=float))
    assert np.max(np.abs(p / np.exp(y) - 1.0)) < 1e-12
    # the argument's range: XM ln 2 - corr for d >= 8
    d = np.geomspace(8.0, 1e5, 2000)
    xm = np.log2(np.e) * ((d - 1.0) * np.log1p(-1.0 / d) + 1.0)
    corr = 1.0 / (12.0 * d) - 1.0 / (360.0 * d ** 3)
    assert np.max(np.abs(xm * np.log(2.0) - corr)) < 0.06
