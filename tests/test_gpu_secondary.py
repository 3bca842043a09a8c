"""Secondary-observable pieces of the multivariate likelihood (section 2.4) on the GPU.

Against the FP64 oracle through the C ABI: FP64 path 1e-10 relative on the NLL and 1e-8 normwise
on the gradient; mixed path |dNLL| < 1e-3 and the gradient bound 1e-5 read per component on the
statistical scale, |g_i - g_ref,i| <= 1e-5 (|g_ref,i| + sqrt(F_ii)), F the oracle's Fisher diagonal
at theta0 over the evaluated window.  (Near the minimum of these small workloads every gradient
component is small against its statistical spread, and the normwise ratio divides FP32 rounding by
the largest of them.)  The energy slices carry histograms of a second observable whose expectation is built from the species'
expected counts per slice.
"""
import numpy as np
import pytest

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import gsn, inputs as I
from tests._helpers import fisher_rel, norm_rel, oracle_pool_map

pytestmark = pytest.mark.gpu
FP64, MIXED = gsn.GSN_FP64, gsn.GSN_MIXED


def _problem(base, seed, n_slices=6, n_sec=12):
    w = I.with_secondary(base, n_slices=n_slices, n_sec=n_sec)
    D = len(w["edges"])
    mu = [O.expected_counts(w, w["theta0"], d) for d in range(D)]
    ms = np.concatenate([O.secondary_expected(w, w["theta0"], d)[1].ravel()
                         for d in range(D) if w["secondary"][d] is not None])
    return w, mu, ms, I.poisson_counts(np.concatenate(mu + [ms]), seed)


@pytest.fixture(scope="module", params=["gamma", "gauss", "ggamma"])
def problem(request):
    if request.param == "gamma":
        base = I.borexino_like(n_bins=240, n_fine=2400)
    elif request.param == "gauss":
        base = I.single_gauss(n_bins=300, n_fine=600)
    else:
        base = I.with_power(I.borexino_like(n_bins=200, n_fine=2000), 1.4)
    w, mu, ms, n = _problem(base, 601)
    return w, mu, ms, n, O.fisher_diagonal(w, w["theta0"])


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_eval_grad_against_oracle(problem, precision):
    w, mu, ms, n, F = problem
    ctx = gsn.context_from_workload(w, precision, counts=n)
    assert ctx.n_counts() == n.size
    for p in I.perturbed_points(w["theta0"], 2, 602):
        rc, v, g = ctx.eval_grad(p)
        assert rc == 0, ctx.last_error()
        ref, gref = O.nll(w, p, n), O.nll_grad(w, p, n)
        if precision == FP64:
            assert abs(v - ref) <= 1e-10 * abs(ref), (v, ref)
            assert norm_rel(g, gref) < 1e-8, norm_rel(g, gref)
        else:
            assert abs(v - ref) < 1e-3, (v, ref)
            assert fisher_rel(g, gref, F) < 1e-5, (fisher_rel(g, gref, F), norm_rel(g, gref))
        # the value-cache path (per-species shapes of one point)
        rc, v2 = ctx.eval(p)
        assert rc == 0 and abs(v2 - ref) <= (1e-10 * abs(ref) if precision == FP64 else 1e-3)


def test_toy_batch_with_secondary_counts():
    w, mu, ms, _ = _problem(I.borexino_like(n_bins=240, n_fine=2400), 611)
    b = I.toy_batch(w, mu, n_toys=6, seed0=612, w_min=100, w_max=240, mu_sec=ms)
    assert b["counts"].shape[1] == 480 + ms.size
    r = {}
    for precision in (FP64, MIXED):
        ctx = gsn.context_from_workload(w, precision)
        rc, nll, g = ctx.eval_grad_batch(b["params"], b["counts"], b["windows"])
        assert rc == 0, ctx.last_error()
        r[precision] = (nll, g)
    for t in (0, 3, 5):
        ref = O.nll(w, b["params"][t], b["counts"][t], b["windows"][t])
        gref = O.nll_grad(w, b["params"][t], b["counts"][t], b["windows"][t])
        assert abs(r[FP64][0][t] - ref) <= 1e-10 * abs(ref)
        assert norm_rel(r[FP64][1][t], gref) < 1e-8
    assert np.max(np.abs(r[FP64][0] - r[MIXED][0])) < 1e-3
    Fs = oracle_pool_map([("fisher", w, (w["theta0"], b["windows"][t])) for t in range(6)])
    for t in range(6):
        assert fisher_rel(r[MIXED][1][t], r[FP64][1][t], Fs[t]) < 1e-5, (t, norm_rel(r[MIXED][1][t], r[FP64][1][t]))


def test_templates_and_peaks_in_the_secondary_pieces():
    w, mu, ms, n = _problem(I.with_templates(I.borexino_like(n_bins=200, n_fine=1600), 2), 621)
    p = I.perturbed_points(w["theta0"], 1, 622)[0]
    ctx = gsn.context_from_workload(w, FP64, counts=n)
    rc, v, g = ctx.eval_grad(p)
    assert rc == 0, ctx.last_error()
    assert abs(v - O.nll(w, p, n)) <= 1e-10 * abs(v)
    assert norm_rel(g, O.nll_grad(w, p, n)) < 1e-8


def test_secondary_arguments_are_validated():
    w = I.with_secondary(I.borexino_like(n_bins=100, n_fine=800), n_slices=4, n_sec=5)
    ctx = gsn.context_from_workload(w, FP64)
    x = w["secondary"][0]
    with pytest.raises(gsn.GsnError):
        ctx.set_secondary(0, [0, 50, 40, 80, 100], x["shapes"])     # descending boundaries
    with pytest.raises(gsn.GsnError):
        ctx.set_secondary(0, [0, 25, 50, 75, 101], x["shapes"])     # past the last bin
    with pytest.raises(gsn.GsnError):
        ctx.set_secondary(0, x["slice_start"], -np.ones_like(x["shapes"]))
    ctx.set_secondary(1, None, None)
    assert ctx.n_counts() == 200 + 4 * 5
