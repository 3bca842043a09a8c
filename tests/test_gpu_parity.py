"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 path, relative 1e-10 on the NLL and 1e-8 normwise on the
gradient; mixed path, |dNLL| < 1e-3 and normwise gradient error < 1e-5
(||g - g_ref||_inf / max(||g_ref||_inf, 1)).
"""
import numpy as np
import pytest

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import gsn, inputs as I
from tests._helpers import norm_rel, poisson_data

pytestmark = pytest.mark.gpu

FP64, MIXED = gsn.GSN_FP64, gsn.GSN_MIXED


def check_point(work, counts, params, precision, ctx=None, grad=True, windows=None):
    ctx = ctx or gsn.context_from_workload(work, precision, counts=counts)
    ref = O.nll(work, params, counts, windows)
    rc, nll, g = ctx.eval_grad(params)
    assert rc == 0, ctx.last_error()
    if precision == FP64:
        assert abs(nll - ref) <= 1e-10 * max(abs(ref), 1.0), (nll, ref)
    else:
        assert abs(nll - ref) < 1e-3, (nll, ref)
    if grad:
        gref = O.nll_grad(work, params, counts, windows)
        tol = 1e-8 if precision == FP64 else 1e-5
        assert norm_rel(g, gref) < tol, (norm_rel(g, gref), np.c_[g, gref])
    return ctx, nll, g


# ------------------------------------------------------------- small ---------
@pytest.fixture(scope="module")
def small_gauss():
    w = I.single_gauss(n_bins=300, n_fine=700)
    return w, poisson_data(w, 101)


@pytest.fixture(scope="module")
def small_gamma():
    w = I.borexino_like(n_bins=320, n_fine=3000)
    return w, poisson_data(w, 202)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_small_gauss_points(small_gauss, precision):
    w, n = small_gauss
    for p in I.perturbed_points(w["theta0"], 3, 300):
        check_point(w, n, p, precision)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_small_gamma_points(small_gamma, precision):
    w, n = small_gamma
    for p in I.perturbed_points(w["theta0"], 3, 400):
        check_point(w, n, p, precision)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_eval_matches_eval_grad_and_cache(small_gamma, precision):
    w, n = small_gamma
    ctx = gsn.context_from_workload(w, precision, counts=n)
    p = I.perturbed_points(w["theta0"], 1, 500)[0]
    rc, v1 = ctx.eval(p)
    assert rc == 0
    rc, v2, _ = ctx.eval_grad(p)
    ref = O.nll(w, p, n)
    tol = 1e-10 * abs(ref) if precision == FP64 else 1e-3
    assert abs(v1 - ref) < tol and abs(v2 - ref) < tol
    # rate-only change: the response cache is reused and the value still matches the oracle
    q = p.copy(); q[0] *= 1.3; q[5] *= 0.8
    rc, v3 = ctx.eval(q)
    assert rc == 0 and abs(v3 - O.nll(w, q, n)) < (1e-10 * abs(ref) if precision == FP64 else 1e-3)
    rc, v4 = ctx.eval(p)
    assert v4 == v1  # deterministic


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_expected_per_species(small_gamma, precision):
    w, n = small_gamma
    ctx = gsn.context_from_workload(w, precision, counts=n)
    p = I.perturbed_points(w["theta0"], 1, 600)[0]
    for d in range(2):
        got = ctx.expected(p, d)
        ref = O.expected_per_species(w, p, d)
        big = ref > 1e-6 * ref.max()
        rel = np.abs(got[big] / ref[big] - 1.0)
        assert rel.max() < (1e-10 if precision == FP64 else 2e-5), rel.max()
        assert np.all(got[~big] <= 1e-5 * ref.max() + 1e-300)


def test_fd_gradient_of_fp64_path(small_gamma):
    w, n = small_gamma
    ctx = gsn.context_from_workload(w, FP64, counts=n)
    p = I.perturbed_points(w["theta0"], 1, 700)[0]
    rc, v, g = ctx.eval_grad(p)
    fd = np.zeros_like(g)
    for i in range(p.size):
        h = 1e-6 * abs(p[i])
        pp, pm = p.copy(), p.copy(); pp[i] += h; pm[i] -= h
        fd[i] = (ctx.eval_grad(pp)[1] - ctx.eval_grad(pm)[1]) / (2 * h)
    scale = np.abs(g) + 1e-3 * np.max(np.abs(g))
    assert np.max(np.abs(fd - g) / scale) < 1e-4


def test_autograd_function(small_gauss):
    torch = pytest.importorskip("torch")
    w, n = small_gauss
    ctx = gsn.context_from_workload(w, FP64, counts=n)
    F = gsn.make_autograd()
    p = torch.tensor(I.perturbed_points(w["theta0"], 1, 800)[0], requires_grad=True)
    y = F.apply(p, ctx)
    (2.0 * y).backward()
    assert np.allclose(p.grad.numpy(), 2.0 * O.nll_grad(w, p.detach().numpy(), n), rtol=1e-8, atol=1e-9)


# ------------------------------------------------------------ edge cases -----
@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("win", [(0, 1), (319, 320), (0, 320), (0, 37), (250, 320), (100, 100), (7, 8)])
def test_windows(small_gamma, precision, win):
    w, n = small_gamma
    p = I.perturbed_points(w["theta0"], 1, 900)[0]
    T = 1
    wins = np.array([[win, win]], np.int32)
    ctx = gsn.context_from_workload(w, precision, counts=n)
    rc, nll, g = ctx.eval_grad_batch(p[None, :], n[None, :], wins)
    assert rc == 0, ctx.last_error()
    ref = O.nll(w, p, n, [win, win])
    gref = O.nll_grad(w, p, n, [win, win])
    if precision == FP64:
        assert abs(nll[0] - ref) <= 1e-10 * max(abs(ref), 1.0)
        assert norm_rel(g[0], gref) < 1e-8
    else:
        assert abs(nll[0] - ref) < 1e-3
        # A window of a few bins makes the gradient ill-conditioned: it is a sum of
        # w_j = 1 - n_j/mu_j over few bins, and an FP32 relative error eta on mu_j
        # moves w_j by ~eta, i.e. the gradient by ~eta/|w_j| relatively.
        assert norm_rel(g[0], gref) < (1e-5 if win[1] - win[0] >= 20 else 1e-4)


def test_zero_toys_is_noop(small_gauss):
    w, n = small_gauss
    ctx = gsn.context_from_workload(w, FP64, counts=n)
    rc, nll, g = ctx.eval_grad_batch(np.zeros((0, w["n_params"])), np.zeros((0, n.size)), np.zeros((0, 1, 2), np.int32))
    assert rc == 0 and nll.size == 0


def test_nonpositive_mu_and_nonfinite(small_gauss):
    w, n = small_gauss
    ctx = gsn.context_from_workload(w, FP64, counts=n)
    p = w["theta0"].copy()
    for s in range(8):
        p[s] = -abs(p[s])  # negative rates: mu < 0 where counts are positive
    rc, nll, g = ctx.eval_grad(p)
    assert rc == gsn.GSN_ERR_NONPOSITIVE_MU and nll == np.inf
    q = w["theta0"].copy(); q[9] = np.nan
    rc, nll, g = ctx.eval_grad(q)
    assert rc == gsn.GSN_ERR_NONFINITE
    rc, nll, g = ctx.eval_grad(w["theta0"])  # context still usable
    assert rc == 0 and abs(nll - O.nll(w, w["theta0"], n)) < 1e-9 * abs(nll)


# -------------------------------------------------------------- full size ----
@pytest.fixture(scope="module")
def full_gauss():
    w = I.single_gauss()
    return w, poisson_data(w, 1)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_full_single_gauss(full_gauss, precision):
    """900 bins x 2000 fine points, 8 species, at five of the 100 seeded parameter points."""
    w, n = full_gauss
    ctx = gsn.context_from_workload(w, precision, counts=n)
    pts = I.perturbed_points(w["theta0"], 100, 2)
    for i in (0, 17, 42, 77, 99):
        check_point(w, n, pts[i], precision, ctx=ctx, grad=(i in (0, 99)))


@pytest.fixture(scope="module")
def full_gamma():
    w = I.borexino_like()
    return w, poisson_data(w, 3)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_full_borexino_like_nll(full_gamma, precision):
    """2 datasets x 1000 bins x 20000 fine points, 16 species, generalized-gamma response."""
    w, n = full_gamma
    p = I.perturbed_points(w["theta0"], 1, 1001)[0]
    check_point(w, n, p, precision, grad=False)


@pytest.fixture(scope="module")
def toys():
    """Batched pseudo-experiments of the two-dataset workload on a 1200-bin domain."""
    w = I.borexino_like(n_bins=1200)
    mu0 = [O.expected_counts(w, w["theta0"], d) for d in range(2)]
    b = I.toy_batch(w, mu0, n_toys=24, seed0=1000)
    return w, b


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_toy_batch_sampled(toys, precision):
    w, b = toys
    ctx = gsn.context_from_workload(w, precision)
    rc, nll, g = ctx.eval_grad_batch(b["params"], b["counts"], b["windows"])
    assert rc == 0, ctx.last_error()
    for t in (0, 13):
        ref = O.nll(w, b["params"][t], b["counts"][t], b["windows"][t])
        if precision == FP64:
            assert abs(nll[t] - ref) <= 1e-10 * abs(ref)
        else:
            assert abs(nll[t] - ref) < 1e-3
    # batched equals one-toy-at-a-time (FP64: to rounding order; mixed: within the mixed tolerance)
    for t in (5, 23):
        rc1, n1, g1 = ctx.eval_grad_batch(b["params"][t:t + 1], b["counts"][t:t + 1], b["windows"][t:t + 1])
        tol = 1e-12 * abs(n1[0]) if precision == FP64 else 1e-4
        assert abs(n1[0] - nll[t]) < tol
        # one toy alone runs with another split plan (summation order) than the batch
        assert norm_rel(g1[0], g[t]) < (1e-11 if precision == FP64 else 1e-5)


def test_toy_gradient_against_oracle(toys):
    """One toy's full gradient against the oracle (mixed and FP64)."""
    w, b = toys
    t = 7
    gref = O.nll_grad(w, b["params"][t], b["counts"][t], b["windows"][t])
    for precision, tol in ((FP64, 1e-8), (MIXED, 1e-5)):
        ctx = gsn.context_from_workload(w, precision)
        rc, nll, g = ctx.eval_grad_batch(b["params"][t:t + 1], b["counts"][t:t + 1], b["windows"][t:t + 1])
        assert rc == 0
        assert norm_rel(g[0], gref) < tol, (precision, norm_rel(g[0], gref))


def test_mixed_vs_fp64_on_full_toy_batch(toys):
    """|dNLL| < 1e-3 between the mixed and FP64 GPU paths on every toy of the batch."""
    w, b = toys
    r = {}
    for precision in (FP64, MIXED):
        ctx = gsn.context_from_workload(w, precision)
        rc, nll, g = ctx.eval_grad_batch(b["params"], b["counts"], b["windows"])
        assert rc == 0
        r[precision] = (nll, g)
    assert np.max(np.abs(r[FP64][0] - r[MIXED][0])) < 1e-3
    for t in range(len(b["params"])):
        assert norm_rel(r[MIXED][1][t], r[FP64][1][t]) < 1e-5
