"""Multivariate slices (section 2.4) on the GPU against the FP64 oracle, through the C ABI.

A second observable splits each histogram into slices with fixed response multipliers and rate
fractions (gsn_set_dataset_factors).  Tolerances as in the other parity tests: FP64 path 1e-10
relative on the NLL and 1e-8 normwise on the gradient; mixed path |dNLL| < 1e-3 and 1e-5.
"""
import numpy as np
import pytest

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import gsn, inputs as I
from tests._helpers import norm_rel

pytestmark = pytest.mark.gpu
FP64, MIXED = gsn.GSN_FP64, gsn.GSN_MIXED


def _data(w, seed):
    mu = [O.expected_counts(w, w["theta0"], d) for d in range(len(w["edges"]))]
    return np.concatenate([I.poisson_counts(m, seed + d) for d, m in enumerate(mu)])


def _check(w, n, p, precision, ctx=None):
    ctx = ctx or gsn.context_from_workload(w, precision, counts=n)
    rc, v, g = ctx.eval_grad(p)
    assert rc == 0, ctx.last_error()
    ref, gref = O.nll(w, p, n), O.nll_grad(w, p, n)
    if precision == FP64:
        assert abs(v - ref) <= 1e-10 * abs(ref), (v, ref)
        assert norm_rel(g, gref) < 1e-8, norm_rel(g, gref)
    else:
        assert abs(v - ref) < 1e-3, (v, ref)
        assert norm_rel(g, gref) < 1e-5, norm_rel(g, gref)
    return ctx


@pytest.fixture(scope="module")
def slices():
    """2 datasets x 3 slices of 120 bins: three response groups of two datasets each."""
    w = I.multivariate_like(seed=5, n_datasets=2, n_slices=3, n_bins=120, n_fine=1500, n_species=6)
    return w, _data(w, 301)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_slices_against_oracle(slices, precision):
    w, n = slices
    for p in I.perturbed_points(w["theta0"], 2, 302):
        _check(w, n, p, precision)


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n_datasets", [4, 5])
def test_datasets_sharing_a_slice_response(precision, n_datasets):
    """4 datasets share each slice's response (one full group of 4), or 5 (groups of 4 + 1)."""
    w = I.multivariate_like(seed=6, n_datasets=n_datasets, n_slices=2, n_bins=80, n_fine=1200, n_species=5)
    n = _data(w, 311)
    _check(w, n, I.perturbed_points(w["theta0"], 1, 312)[0], precision)


def test_256_slices_fp64_and_mixed():
    """The full slice count of the 2-D workload (4 x 64) on short histograms."""
    w = I.multivariate_like(seed=7, n_datasets=4, n_slices=64, n_bins=40, n_fine=400, n_species=4)
    n = _data(w, 321)
    p = I.perturbed_points(w["theta0"], 1, 322)[0]
    for precision in (FP64, MIXED):
        _check(w, n, p, precision)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_factors_with_peak_and_shift_species(precision):
    """Rate fractions and response multipliers on the two-dataset workload (AnaPeak, AnaShift)."""
    w = I.borexino_like(n_bins=260, n_fine=2600)
    rng = np.random.Generator(np.random.PCG64(331))
    S = w["spectra"].shape[0]
    w = dict(w, resp_scale=np.array([[1.03, 1.1, 0.9, 1.0, 1.2], [0.97, 1.0, 1.1, 0.95, 0.8]]),
             rate_factor=rng.uniform(0.3, 1.0, size=(2, S)))
    n = _data(w, 332)
    _check(w, n, I.perturbed_points(w["theta0"], 1, 333)[0], precision)


def test_toy_batch_on_slices(slices):
    w, _ = slices
    mu = [O.expected_counts(w, w["theta0"], d) for d in range(len(w["edges"]))]
    b = I.toy_batch(w, mu, n_toys=6, seed0=340, w_min=60, w_max=120)
    r = {}
    for precision in (FP64, MIXED):
        ctx = gsn.context_from_workload(w, precision)
        rc, nll, g = ctx.eval_grad_batch(b["params"], b["counts"], b["windows"])
        assert rc == 0, ctx.last_error()
        r[precision] = (nll, g)
    for t in (0, 5):
        ref = O.nll(w, b["params"][t], b["counts"][t], b["windows"][t])
        assert abs(r[FP64][0][t] - ref) <= 1e-10 * abs(ref)
    assert np.max(np.abs(r[FP64][0] - r[MIXED][0])) < 1e-3
    for t in range(6):
        assert norm_rel(r[MIXED][1][t], r[FP64][1][t]) < 1e-5


def test_expected_per_species_on_slices(slices):
    """gsn_expected (tensor-core contraction in mixed precision) per slice against the oracle."""
    w, n = slices
    p = I.perturbed_points(w["theta0"], 1, 350)[0]
    for precision, tol in ((FP64, 1e-10), (MIXED, 2e-5)):
        ctx = gsn.context_from_workload(w, precision, counts=n)
        for d in (0, 4):
            got, ref = ctx.expected(p, d), O.expected_per_species(w, p, d)
            big = ref > 1e-6 * ref.max()
            assert np.max(np.abs(got[big] / ref[big] - 1.0)) < tol
        rc, v = ctx.eval(p)
        assert rc == 0 and abs(v - O.nll(w, p, n)) < (1e-10 * abs(v) if precision == FP64 else 1e-3)


def test_factor_arguments_are_validated(slices):
    w, n = slices
    ctx = gsn.context_from_workload(w, FP64, counts=n)
    D, S = len(w["edges"]), w["spectra"].shape[0]
    with pytest.raises(gsn.GsnError):
        ctx.set_dataset_factors(resp_scale=np.zeros((D, 5)))
    with pytest.raises(gsn.GsnError):
        ctx.set_dataset_factors(rate_factor=-np.ones((D, S)))
