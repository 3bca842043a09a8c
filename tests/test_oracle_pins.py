"""Pins of the FP64 oracle against things other than itself (CPU only).

Each pin checks the oracle against a closed form, an independent
arbitrary-precision evaluation (mpmath quadrature / special functions), an
invariant of the mathematics, or brute force on a tiny input.  The mutation
tests at the end plant plausible mistakes in the oracle and check that at least
one pin catches each of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import inputs as I

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40

S0, S1 = I.BIRKS_S0, I.BIRKS_S1


# --------------------------------------------------------------- helpers ----
def tiny_workload(resolution, n_fine=64, n_bins=20, LY=16.0, a=1.0, b=0.5, c=0.01, seed=5):
    """A tiny single-dataset workload (K = 64 fine points, J = 20 bins) for brute force."""
    rng = np.random.Generator(np.random.PCG64(seed))
    E = I.fine_grid(n_fine, 1.0)
    rows = [I.shape_beta(E, 0.8), I.shape_line(E, 0.37), I.shape_expo(E, 0.3), I.shape_flat(E)]
    S = len(rows)
    theta0 = np.concatenate([10.0 ** rng.uniform(1, 3, S), [LY, 0.011, a, b, c]])
    return dict(
        fine_centres=E, spectra=np.array(rows), kind=np.zeros(S, np.int32), shift=np.zeros(S),
        mask=np.ones((S, 1), np.uint8), edges=[I.unit_edges(n_bins)], exposure=np.array([0.7]),
        win_lo=np.array([0]), win_hi=np.array([n_bins]), resolution=resolution,
        birks_s0=S0, birks_s1=S1, n_params=S + 5, slot_map=I._slot_map_shared(S, 1),
        pull_param=np.zeros(0, np.int32), pull_centre=np.zeros(0), pull_width=np.zeros(0),
        theta0=theta0,
    )


def mp_quenched(E, kB):
    """Birks integral by arbitrary-precision quadrature of its defining integrand."""
    E = mpmath.mpf(E)
    return mpmath.quad(lambda t: 1 / (1 + kB * (S0 + S1 / t)), [0, E])


def brute_force_mu(work, params):
    """mu_j by explicit loops in 40-digit arithmetic, independent of the oracle's code."""
    S = work["spectra"].shape[0]
    rates = params[:S]
    LY, kB, a, b, c = params[S:S + 5]
    E = work["fine_centres"]
    f = work["spectra"]
    eps = mpmath.mpf(float(work["exposure"][0]))
    edges = work["edges"][0]
    J = edges.size - 1
    mu = [mpmath.mpf(0)] * J
    norms = [mpmath.fsum(mpmath.mpf(float(v)) for v in f[s]) for s in range(S)]
    for k in range(E.size):
        m = LY * mp_quenched(E[k], kB)
        var = a + b * m + c * m * m
        for j in range(J):
            lo, hi = mpmath.mpf(float(edges[j])), mpmath.mpf(float(edges[j + 1]))
            if work["resolution"] == I.RES_GAUSS:
                sd = mpmath.sqrt(var)
                R = mpmath.ncdf((hi - m) / sd) - mpmath.ncdf((lo - m) / sd)
            else:
                d, s = m * m / var, var / m
                R = mpmath.gammainc(d, lo / s, hi / s, regularized=True)
            for sp in range(S):
                if f[sp][k] != 0:
                    mu[j] += eps * rates[sp] * mpmath.mpf(float(f[sp][k])) / norms[sp] * R
    return np.array([float(v) for v in mu])


def pin_quench_quadrature():
    worst = 0.0
    for kB in (0.005, 0.011, 0.03):
        for E in (1e-4, 0.01, 0.3, 1.0, 1.99):
            ref = integrate.quad(lambda t: 1.0 / (1.0 + kB * (S0 + S1 / t)), 0.0, E,
                                 epsabs=0, epsrel=1e-13, limit=200)[0]
            worst = max(worst, abs(O.quenched_energy(E, kB, S0, S1) / ref - 1.0))
    return worst


def pin_gauss_delta():
    """A one-point spectrum reproduces the Gaussian bin integrals (libm erfc)."""
    w = tiny_workload(I.RES_GAUSS)
    w["spectra"] = np.array([I.shape_line(w["fine_centres"], 0.37)])
    w["kind"] = np.zeros(1, np.int32); w["shift"] = np.zeros(1); w["mask"] = np.ones((1, 1), np.uint8)
    w["slot_map"] = I._slot_map_shared(1, 1); w["n_params"] = 6
    p = np.array([1234.5, 16.0, 0.011, 1.0, 0.5, 0.01])
    mu = O.expected_counts(w, p, 0)
    k = int(np.argmin(np.abs(w["fine_centres"] - 0.37)))
    m = 16.0 * float(mp_quenched(w["fine_centres"][k], 0.011))
    sd = math.sqrt(1.0 + 0.5 * m + 0.01 * m * m)
    ref = np.array([0.7 * 1234.5 * 0.5 * (math.erfc(-(j + 1 - m) / (sd * math.sqrt(2)))
                                          - math.erfc(-(j - m) / (sd * math.sqrt(2)))) for j in range(20)])
    big = ref > 1e-3 * ref.max()
    return float(np.max(np.abs(mu[big] / ref[big] - 1.0)))


def pin_brute_force(resolution):
    w = tiny_workload(resolution)
    p = w["theta0"]
    ref = brute_force_mu(w, p)
    mu = O.expected_counts(w, p, 0)
    big = ref > 1e-12 * ref.max()
    return float(np.max(np.abs(mu[big] / ref[big] - 1.0)))


def pin_rate_identity(work, params, counts):
    """mu is homogeneous of degree 1 in the rates: sum_s r_s dNLL/dr_s = sum_j (mu_j - n_j)."""
    g = O.nll_grad(work, params, counts)
    S = work["spectra"].shape[0]
    sm = np.asarray(work["slot_map"])[:, :S]
    idx = np.unique(sm[sm >= 0])  # the rate parameters, wherever the slot map puts them
    lhs = float(np.dot(params[idx], g[idx]))
    rhs = 0.0
    cs = O._split_counts(work, counts)
    for d in range(len(work["edges"])):
        lo, hi = int(work["win_lo"][d]), int(work["win_hi"][d])
        rhs += float(np.sum(O.expected_counts(work, params, d)[lo:hi] - cs[d][lo:hi]))
    return abs(lhs - rhs) / max(1.0, abs(rhs))


# ------------------------------------------------------------- quenching ----
def test_quench_matches_defining_integral():
    assert pin_quench_quadrature() < 1e-12


def test_quench_kB_zero_is_identity():
    E = np.linspace(0.0, 2.0, 11)
    assert np.array_equal(O.quenched_energy(E, 0.0, S0, S1), E)


def test_quench_slope_is_birks_integrand():
    # dE_q/dE = 1 / (1 + kB S(E)) by arbitrary-precision differentiation of the closed form
    for E in (0.05, 0.5, 1.5):
        slope = mpmath.diff(lambda t: t / (1 + 0.011 * S0) - (0.011 * S1 / (1 + 0.011 * S0) ** 2)
                            * mpmath.log(1 + (1 + 0.011 * S0) * t / (0.011 * S1)), E)
        assert abs(float(slope) * (1 + 0.011 * (S0 + S1 / E)) - 1.0) < 1e-14


def test_quench_dkB_against_mpmath():
    for E in (0.001, 0.2, 1.7):
        for kB in (0.008, 0.011):
            ref = mpmath.diff(lambda k: mp_quenched(E, k), kB)
            assert abs(O.quenched_energy_dkB(E, kB, S0, S1) / float(ref) - 1.0) < 1e-10


# -------------------------------------------------------------- responses ---
def test_gauss_delta_spectrum_reproduces_bin_integrals():
    assert pin_gauss_delta() < 1e-12


def test_gauss_rows_sum_to_one_over_wide_window():
    mu = np.array([50.0, 300.0, 777.7]); sd = np.array([3.0, 17.0, 29.0])
    edges = np.arange(-400.0, 1300.0)
    R = O.response_gauss(edges, mu, sd)
    assert np.max(np.abs(R.sum(axis=0) - 1.0)) < 1e-14


def test_gamma_rows_sum_to_one_from_zero():
    mu = np.array([0.02, 2.0, 50.0, 500.0]); var = 10.0 + 1.1 * mu + 2e-4 * mu * mu
    # the smallest mean has a long exponential tail (scale var/mu ~ 500 p.e.): go far out
    edges = np.concatenate([np.arange(0.0, 3000.0), np.arange(3000.0, 40001.0, 100.0)])
    R = O.response_gamma(edges, mu, var)
    assert np.max(np.abs(R.sum(axis=0) - 1.0)) < 1e-13


@pytest.mark.parametrize("m,var,lo,hi", [
    (0.03, 10.0, 0.0, 1.0), (0.03, 10.0, 1.0, 2.0), (3.0, 13.3, 0.0, 1.0), (3.0, 13.3, 5.0, 6.0),
    (50.0, 65.5, 49.0, 50.0), (50.0, 65.5, 80.0, 81.0), (480.0, 584.0, 470.0, 471.0),
    (480.0, 584.0, 560.0, 561.0), (900.0, 1162.0, 901.0, 902.0)])
def test_gamma_bin_integral_against_mpmath(m, var, lo, hi):
    d, s = m * m / var, var / m
    if lo > 0:  # regular integrand: arbitrary-precision quadrature of the density
        ref = mpmath.quad(lambda x: x ** (d - 1) * mpmath.exp(-x / s) / (s ** d * mpmath.gamma(d)),
                          [lo, (lo + hi) / 2, hi])
    else:  # x^(d-1) singular at 0: mpmath's own incomplete gamma function
        ref = mpmath.gammainc(d, 0, hi / s, regularized=True)
    got = O.response_gamma(np.array([lo, hi]), np.array([m]), np.array([var]))[0, 0]
    assert abs(got / float(ref) - 1.0) < 1e-11


@pytest.mark.parametrize("d,y", [(0.05, 0.01), (0.5, 0.7), (3.0, 2.0), (38.0, 40.0), (410.0, 400.0), (410.0, 460.0)])
def test_gamma_shape_derivative_against_mpmath(d, y):
    ref = mpmath.diff(lambda t: mpmath.gammainc(t, 0, y, regularized=True), d)
    got = float(O._gamma_P_dshape(np.array([d]), np.array([y]))[0])
    assert abs(got - float(ref)) <= 1e-9 * max(abs(float(ref)), 1e-6)


def test_peak_profile_against_libm():
    edges = np.arange(150.0, 260.0)
    prof = O.peak_profile(edges, 201.3, 9.7)
    ref = [0.5 * (math.erfc(-(e1 - 201.3) / (9.7 * math.sqrt(2))) - math.erfc(-(e0 - 201.3) / (9.7 * math.sqrt(2))))
           for e0, e1 in zip(edges[:-1], edges[1:])]
    assert np.max(np.abs(prof - ref)) < 1e-15


def test_shift_moves_normalised_spectrum():
    E = I.fine_grid(2000, 2.0)
    w = dict(fine_centres=E, spectra=np.array([I.shape_beta(E, 0.96)] * 2), kind=np.array([0, 1]),
             shift=np.array([0.0, 1.022]))
    S = O.species_spectra(w)
    assert np.allclose(S[0].sum(), 1.0) and np.allclose(S[1].sum(), 1.0)
    assert np.array_equal(S[1][1022:], S[0][:-1022]) and not S[1][:1022].any()


# ---------------------------------------------------------- brute force -----
def test_brute_force_tiny_gauss():
    assert pin_brute_force(I.RES_GAUSS) < 1e-12


def test_brute_force_tiny_gamma():
    assert pin_brute_force(I.RES_GAMMA) < 1e-11


# ------------------------------------------------------------ likelihood ----
def test_single_bin_by_hand():
    assert O.poisson_term(3.0, 5.0) == pytest.approx(3.0 - 5.0 + 5.0 * math.log(5.0 / 3.0), rel=1e-15)
    assert O.poisson_term(2.5, 0.0) == 2.5
    assert O.poisson_term(0.0, 1.0) == math.inf


@pytest.mark.parametrize("maker", [lambda: I.single_gauss(n_bins=300, n_fine=600),
                                   lambda: I.borexino_like(n_bins=300, n_fine=3000),
                                   lambda: I.template_like(n_bins=300, n_species=6),
                                   lambda: I.with_templates(I.borexino_like(n_bins=200, n_fine=1500), 2)])
def test_asimov_nll_zero_and_gradient_zero(maker):
    w = maker()
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(len(w["edges"]))])
    assert O.nll(w, w["theta0"], mu) == pytest.approx(0.0, abs=1e-9)
    g = O.nll_grad(w, w["theta0"], mu)
    assert np.max(np.abs(g)) < 1e-8
    # and it is a strict minimum: random small moves raise the NLL
    rng = np.random.Generator(np.random.PCG64(9))
    for _ in range(3):
        p = w["theta0"] * (1 + 1e-3 * rng.standard_normal(w["theta0"].size))
        assert O.nll(w, p, mu) > 0.0


def test_rate_homogeneity_identity():
    w = I.borexino_like(n_bins=250, n_fine=2500)
    w["pull_param"] = np.zeros(0, np.int32); w["pull_centre"] = np.zeros(0); w["pull_width"] = np.zeros(0)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    n = I.poisson_counts(mu, 11)
    p = I.perturbed_points(w["theta0"], 1, 12)[0]
    assert pin_rate_identity(w, p, n) < 1e-11


@pytest.mark.parametrize("resolution", [I.RES_GAUSS, I.RES_GAMMA])
def test_analytic_gradient_matches_finite_differences(resolution):
    w = I.borexino_like(n_bins=220, n_fine=1500) if resolution == I.RES_GAMMA else I.single_gauss(n_bins=250, n_fine=500)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(len(w["edges"]))])
    n = I.poisson_counts(mu, 21)
    p = I.perturbed_points(w["theta0"], 1, 22, rel=0.02)[0]
    g = O.nll_grad(w, p, n)
    gf = O.nll_grad_fd(w, p, n, rel=1e-4)
    scale = np.abs(g) + 1e-3 * np.max(np.abs(g))
    assert np.max(np.abs(g - gf) / scale) < 2e-6


def test_synchronised_parameter_gradient_is_sum_over_datasets():
    """Section 2.2: a parameter shared by two datasets gets the sum of their gradients."""
    w = I.borexino_like(n_bins=200, n_fine=1500)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    n = I.poisson_counts(mu, 31)
    p = I.perturbed_points(w["theta0"], 1, 32)[0]
    g_shared = O.nll_grad(w, p, n)
    # unsynchronise LY: dataset 1 gets its own copy as a new parameter P
    w2 = dict(w)
    P = w["n_params"]
    sm = w["slot_map"].copy()
    S = w["spectra"].shape[0]
    sm[1, I.slot_response(S, "LY")] = P
    w2["slot_map"] = sm; w2["n_params"] = P + 1
    p2 = np.concatenate([p, [p[S]]])
    g2 = O.nll_grad(w2, p2, n)
    assert g2[S] + g2[P] == pytest.approx(g_shared[S], rel=1e-12)
    assert O.nll(w2, p2, n) == pytest.approx(O.nll(w, p, n), rel=1e-15)


def test_asimov_fit_recovers_generating_parameters():
    """The NLL of Asimov data is minimised at the generating parameters."""
    w = I.single_gauss(n_bins=1000, n_fine=1000)
    th = w["theta0"].copy()
    mu = O.expected_counts(w, th, 0)
    free = list(range(8)) + [8, 10, 11]  # rates, LY, a, b

    def f(u):
        # logarithmic scale factors keep every trial point at positive rates, light yield and
        # resolution terms, so mu > 0 throughout the search
        x = np.exp(u)
        p = th.copy(); p[free] = th[free] * x
        return O.nll(w, p, mu), O.nll_grad(w, p, mu)[free] * th[free] * x
    u0 = np.log(1.0 + 0.03 * np.sin(np.arange(len(free)) + 1.0))
    res = optimize.minimize(f, u0, jac=True, method="BFGS", options=dict(gtol=1e-11, maxiter=2000))
    res.x = np.exp(res.x)
    assert res.fun < 1e-10
    assert np.max(np.abs(res.x - 1.0)) < 1e-5


# -------------------------------------------------- planted mistakes --------
MUTANTS = {
    "quench drops log term": ("quenched_energy", lambda E, kB, s0, s1: np.asarray(E) / (1 + kB * s0)),
    "gauss cdf sign flip": ("_norm_cdf_diff", lambda lo, hi: (O.special.ndtr(lo) - O.special.ndtr(hi))),
    "gamma scale inverted": ("gamma_shape_scale", lambda mu, var: (mu * mu / var, mu / var)),
    "rate term drops exposure": ("peak_profile", lambda e, m, w: O._norm_cdf_diff((e[:-1] - m) / w, (e[1:] - w) / m)),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(monkeypatch, name):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = []
    try:
        caught.append(pin_quench_quadrature() > 1e-12)
    except Exception:
        caught.append(True)
    for pin in (pin_gauss_delta, lambda: pin_brute_force(I.RES_GAMMA)):
        try:
            caught.append(pin() > 1e-11)
        except Exception:
            caught.append(True)
    try:
        caught.append(abs(float(O.peak_profile(np.arange(150.0, 260.0), 201.3, 9.7).sum()) - 1.0) > 1e-6)
    except Exception:
        caught.append(True)
    assert any(caught), f"no pin caught the planted mistake '{name}'"


# ------------------------------------------- multivariate slices (section 2.4) --------
def _mv_small(unit_response=False):
    w = I.multivariate_like(seed=5, n_datasets=2, n_slices=3, n_bins=90, n_fine=900, n_species=5)
    if unit_response:
        w = dict(w, resp_scale=np.ones_like(w["resp_scale"]))
    return w


def _unsplit(w):
    """The same histograms without the second observable: one dataset per slice group, no factors."""
    Q = w["n_slices"]
    D = len(w["edges"]) // Q
    S = w["spectra"].shape[0]
    one = {k: v for k, v in w.items() if k not in ("resp_scale", "rate_factor")}
    one.update(edges=w["edges"][::Q], exposure=w["exposure"][::Q], mask=np.ones((S, D), np.uint8),
               win_lo=w["win_lo"][::Q], win_hi=w["win_hi"][::Q], slot_map=w["slot_map"][::Q])
    return one


def pin_slices_sum_to_unsplit():
    """Slices with unit response multipliers and rate fractions summing to 1 add up to the unsplit histogram."""
    w = _mv_small(unit_response=True)
    one = _unsplit(w)
    Q = w["n_slices"]
    p = I.perturbed_points(w["theta0"], 1, 7)[0]
    worst = 0.0
    for d in range(len(one["edges"])):
        tot = sum(O.expected_counts(w, p, d * Q + q) for q in range(Q))
        ref = O.expected_counts(one, p, d)
        worst = max(worst, float(np.max(np.abs(tot - ref)) / ref.max()))
    return worst


def pin_multipliers_are_scaled_parameters():
    """A slice's factors act as the scaled parameters would: LY x lambda, a x alpha, rate x fraction."""
    w = _mv_small()
    plain = {k: v for k, v in w.items() if k not in ("resp_scale", "rate_factor")}
    S = w["spectra"].shape[0]
    p = I.perturbed_points(w["theta0"], 1, 8)[0]
    worst = 0.0
    for d in (1, 4):
        q = p.copy()
        q[S] *= w["resp_scale"][d, 0]
        q[S + 2] *= w["resp_scale"][d, 2]
        q[:S] *= w["rate_factor"][d]
        got, ref = O.expected_counts(w, p, d), O.expected_counts(plain, q, d)
        worst = max(worst, float(np.max(np.abs(got - ref)) / ref.max()))
    return worst


def test_slices_sum_to_unsplit_histogram():
    assert pin_slices_sum_to_unsplit() < 1e-12


def test_slice_multipliers_act_as_scaled_parameters():
    assert pin_multipliers_are_scaled_parameters() < 1e-12


def test_multivariate_gradient_matches_finite_differences():
    """Chain rule through the slice multipliers and fractions against Richardson differences."""
    w = _mv_small()
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(len(w["edges"]))])
    n = I.poisson_counts(mu, 23)
    p = I.perturbed_points(w["theta0"], 1, 24, rel=0.02)[0]
    g = O.nll_grad(w, p, n)
    gf = O.nll_grad_fd(w, p, n, rel=1e-4)
    scale = np.abs(g) + 1e-3 * np.max(np.abs(g))
    assert np.max(np.abs(g - gf) / scale) < 2e-6


_factors = O.dataset_factors
FACTOR_MUTANTS = {
    "response multipliers dropped": lambda w, d: (np.ones(5), _factors(w, d)[1]),
    "rate fractions dropped": lambda w, d: (_factors(w, d)[0], np.ones_like(_factors(w, d)[1])),
    "multipliers on the wrong slot": lambda w, d: (np.roll(_factors(w, d)[0], 1), _factors(w, d)[1]),
}


@pytest.mark.parametrize("name", sorted(FACTOR_MUTANTS))
def test_planted_factor_mistake_is_caught(monkeypatch, name):
    monkeypatch.setattr(O, "dataset_factors", FACTOR_MUTANTS[name])
    assert pin_slices_sum_to_unsplit() > 1e-6 or pin_multipliers_are_scaled_parameters() > 1e-6


# --------------------------------------------- Monte Carlo templates (section 3.2) --------
def pin_template_reproduces_smeared_species():
    """A template equal to an Ana species' own expected shape reproduces it: same shape, and a
    total of eps_d f_ds r_s (templates are normalised to unit sum)."""
    w = I.borexino_like(n_bins=150, n_fine=1200)
    p = I.perturbed_points(w["theta0"], 1, 41)[0]
    d, s = 1, 3
    ana = O.expected_per_species(w, p, d)[:, s]
    w2 = dict(w, kind=w["kind"].copy())
    w2["kind"][s] = I.KIND_MC_TEMPLATE
    tpl = [[None] * len(w["edges"]) for _ in range(w["spectra"].shape[0])]
    tpl[s][d] = ana
    w2["templates"] = tpl
    got = O.expected_per_species(w2, p, d)[:, s]
    eps_r = w["exposure"][d] * p[s]
    with np.errstate(invalid="ignore", divide="ignore"):
        v = max(float(np.max(np.abs(got / got.sum() - ana / ana.sum()))), abs(got.sum() / eps_r - 1.0))
    return v if np.isfinite(v) else np.inf


def test_template_reproduces_smeared_species():
    assert pin_template_reproduces_smeared_species() < 1e-13


def test_rate_homogeneity_identity_with_templates():
    w = I.with_templates(I.borexino_like(n_bins=200, n_fine=1500), 3)
    w["pull_param"] = np.zeros(0, np.int32); w["pull_centre"] = np.zeros(0); w["pull_width"] = np.zeros(0)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    n = I.poisson_counts(mu, 42)
    p = I.perturbed_points(w["theta0"], 1, 43)[0]
    assert pin_rate_identity(w, p, n) < 1e-11


def test_template_gradient_matches_finite_differences():
    w = I.with_templates(I.borexino_like(n_bins=160, n_fine=1200), 2)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    n = I.poisson_counts(mu, 44)
    p = I.perturbed_points(w["theta0"], 1, 45, rel=0.02)[0]
    g = O.nll_grad(w, p, n)
    gf = O.nll_grad_fd(w, p, n, rel=1e-4)
    scale = np.abs(g) + 1e-3 * np.max(np.abs(g))
    assert np.max(np.abs(g - gf) / scale) < 2e-6


_template = O.template
TEMPLATE_MUTANTS = {
    "template not normalised": lambda w, s, d: (np.zeros(len(w["edges"][d]) - 1) if w.get("templates") is None
                                                or w["templates"][s][d] is None
                                                else np.asarray(w["templates"][s][d], np.float64)),
    "template of the other dataset": lambda w, s, d: _template(w, s, 1 - d),
}


@pytest.mark.parametrize("name", sorted(TEMPLATE_MUTANTS))
def test_planted_template_mistake_is_caught(monkeypatch, name):
    monkeypatch.setattr(O, "template", TEMPLATE_MUTANTS[name])
    assert pin_template_reproduces_smeared_species() > 1e-6


# ------------------------------------------ profile likelihood (section 4.2) --------
def _counting_experiment(n_obs, b):
    """One bin, a signal and a background template; the background rate is known."""
    w = I.template_like(n_bins=1, n_species=2)
    w["templates"] = [[np.ones(1)], [np.ones(1)]]
    w["exposure"] = np.array([1.0])
    w["edges"] = w["edges"][:1]
    w["mask"] = np.ones((2, 1), np.uint8)
    w["win_lo"], w["win_hi"] = np.zeros(1, np.int32), np.ones(1, np.int32)
    w["slot_map"] = w["slot_map"][:1]
    w["theta0"] = np.array([5.0, b])
    return w, np.array([float(n_obs)])


@pytest.mark.parametrize("n_obs,b", [(30, 12.0), (7, 2.5), (4, 6.0)])
def test_discovery_q0_matches_counting_closed_form(n_obs, b):
    """q0 of a counting experiment with known background b: 2 (n ln(n/b) - (n - b)) for n > b, else 0
    (the asymptotic discovery statistic)."""
    w, n = _counting_experiment(n_obs, b)
    q0, x1, f1, x0, f0 = O.discovery_q0(w, n, w["theta0"], free=[True, False], null_param=0,
                                        lo=[0.0, 0.0], hi=[np.inf, np.inf])
    ref = 2.0 * (n_obs * np.log(n_obs / b) - (n_obs - b)) if n_obs > b else 0.0
    assert abs(q0 - ref) < 1e-8 * max(1.0, ref)
    assert abs(x1[0] - max(n_obs - b, 0.0)) < 1e-6 * max(1.0, n_obs)


def test_oracle_fit_recovers_asimov_minimum():
    """The bounded L-BFGS fit of Asimov data returns the generating rates (templates + smeared species)."""
    w = I.with_templates(I.borexino_like(n_bins=150, n_fine=1000), 2)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    S = w["spectra"].shape[0]
    # rates of species with counts in the histograms (the others leave the NLL unchanged)
    tot = sum(O.expected_per_species(w, w["theta0"], d).sum(axis=0) for d in range(2))
    seen = [s for s in range(S) if tot[s] > 1e-3 * tot.max()]
    rates = np.unique(w["slot_map"][:, seen][w["slot_map"][:, seen] >= 0])
    free = np.zeros(w["n_params"], bool)
    free[rates] = True
    start = w["theta0"] * np.where(free, 1.05, 1.0)
    x, f = O.fit(w, mu, start, free, lo=np.zeros(w["n_params"]))
    assert f < 1e-8
    assert np.max(np.abs(x[rates] / w["theta0"][rates] - 1.0)) < 1e-4


# --------------------- generalized gamma with a free power p (section 2.3) --------
@pytest.mark.parametrize("x", [1e-5, 0.003, 0.5, 3.0, 9.9, 10.0, 57.0, 800.0, 2.0e4])
def test_log_gamma_and_digamma_differences_against_mpmath(x):
    X = mpmath.mpf(x)
    for c in (0.25, 0.4, 1.0, 2.5):
        lg = mpmath.loggamma(X + c) - mpmath.loggamma(X)
        dg = mpmath.digamma(X + c) - mpmath.digamma(X)
        H = mpmath.loggamma(X + 2 * c) + mpmath.loggamma(X) - 2 * mpmath.loggamma(X + c)
        Hx = mpmath.digamma(X + 2 * c) + mpmath.digamma(X) - 2 * mpmath.digamma(X + c)
        assert abs(float(O.lgamma_diff(np.array([x]), c)[0] / lg) - 1.0) < 1e-14
        assert abs(float(O.digamma_diff(np.array([x]), c)[0] / dg) - 1.0) < 1e-14
        assert abs(float(O.ggamma_log_moment_ratio(np.array([x]), c)[0] / H) - 1.0) < 1e-14
        assert abs(float(O.ggamma_log_moment_ratio_dx(np.array([x]), c)[0] / Hx) - 1.0) < 1e-13


def pin_ggamma_moments():
    """Moment matching: the generalized gamma of the returned (d, s, p) has the requested mean and
    variance, its moments E[X^r] = s^r Gamma((d + r)/p) / Gamma(d/p) taken in 40-digit arithmetic."""
    mu = np.array([0.01, 0.3, 1.0, 5.0, 30.0, 200.0, 1000.0, 1.0e4])
    var = 10.0 + 1.1 * mu + 2e-4 * mu * mu
    worst = 0.0
    for p in (0.4, 0.8, 1.0, 1.3, 2.0, 3.5):
        d, s = O.ggamma_shape_scale(mu, var, p)
        for i in range(mu.size):
            D, Sc, Pw = mpmath.mpf(d[i]), mpmath.mpf(s[i]), mpmath.mpf(p)
            m1 = Sc * mpmath.exp(mpmath.loggamma((D + 1) / Pw) - mpmath.loggamma(D / Pw))
            m2 = Sc ** 2 * mpmath.exp(mpmath.loggamma((D + 2) / Pw) - mpmath.loggamma(D / Pw))
            worst = max(worst, abs(float(m1 / mu[i]) - 1.0), abs(float((m2 - m1 ** 2) / var[i]) - 1.0))
    return worst


def test_ggamma_moment_matching_against_mpmath():
    assert pin_ggamma_moments() < 1e-12


def test_ggamma_power_one_is_the_gamma_response():
    mu = np.array([0.02, 2.0, 50.0, 500.0, 1200.0]); var = 10.0 + 1.1 * mu + 2e-4 * mu * mu
    d, s = O.ggamma_shape_scale(mu, var, 1.0)
    assert np.max(np.abs(d / (mu * mu / var) - 1.0)) < 1e-13 and np.max(np.abs(s / (var / mu) - 1.0)) < 1e-13
    edges = np.arange(0.0, 1500.0)
    Rg, Rgg = O.response_gamma(edges, mu, var), O.response_ggamma(edges, mu, var, 1.0)
    assert np.max(np.abs(Rgg - Rg)) < 1e-13


def pin_ggamma_closed_forms():
    """Power 2: shape 1 is the half-normal (CDF erf(x/s)), shape 2 the Rayleigh (CDF 1 - exp(-(x/s)^2))."""
    edges = np.linspace(0.0, 12.0, 41)
    s = np.array([2.7, 4.1])
    half = O.ggamma_bins(edges, np.array([1.0, 1.0]), s, 2.0)
    ray = O.ggamma_bins(edges, np.array([2.0, 2.0]), s, 2.0)
    worst = 0.0
    for k in range(2):
        F1 = np.array([math.erf(e / s[k]) for e in edges])
        F2 = np.array([-math.expm1(-(e / s[k]) ** 2) for e in edges])
        worst = max(worst, float(np.max(np.abs(half[:, k] - np.diff(F1)))), float(np.max(np.abs(ray[:, k] - np.diff(F2)))))
    return worst


def test_ggamma_half_normal_and_rayleigh_closed_forms():
    assert pin_ggamma_closed_forms() < 1e-14


@pytest.mark.parametrize("m,var,p,lo,hi", [
    (3.0, 13.3, 0.7, 0.0, 1.0), (3.0, 13.3, 1.6, 5.0, 6.0), (50.0, 65.5, 0.5, 49.0, 50.0),
    (50.0, 65.5, 2.5, 80.0, 81.0), (480.0, 584.0, 1.3, 470.0, 471.0), (480.0, 584.0, 3.0, 560.0, 561.0)])
def test_ggamma_bin_integral_against_mpmath_quadrature(m, var, p, lo, hi):
    d, s = O.ggamma_shape_scale(np.array([m]), np.array([var]), p)
    D, Sc, Pw = mpmath.mpf(d[0]), mpmath.mpf(s[0]), mpmath.mpf(p)
    norm = Pw / (Sc ** D * mpmath.gamma(D / Pw))
    if lo > 0:
        ref = mpmath.quad(lambda x: norm * x ** (D - 1) * mpmath.exp(-(x / Sc) ** Pw), [lo, (lo + hi) / 2, hi])
    else:
        ref = mpmath.gammainc(D / Pw, 0, (mpmath.mpf(hi) / Sc) ** Pw, regularized=True)
    got = O.ggamma_bins(np.array([lo, hi]), d, s, p)[0, 0]
    assert abs(got / float(ref) - 1.0) < 1e-11


def test_ggamma_rows_sum_to_one_from_zero():
    mu = np.array([0.02, 2.0, 50.0, 500.0]); var = 10.0 + 1.1 * mu + 2e-4 * mu * mu
    edges = np.concatenate([np.arange(0.0, 3000.0), np.arange(3000.0, 200001.0, 100.0)])
    for p in (0.6, 1.5, 2.5):
        R = O.response_ggamma(edges, mu, var, p)
        assert np.max(np.abs(R.sum(axis=0) - 1.0)) < 1e-12


def _gg_small(p=1.4):
    w = I.with_power(I.borexino_like(n_bins=220, n_fine=1500), p)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    return w, I.poisson_counts(mu, 61)


def pin_ggamma_gradient():
    w, n = _gg_small()
    pt = I.perturbed_points(w["theta0"], 1, 62, rel=0.02)[0]
    g = O.nll_grad(w, pt, n)
    gf = O.nll_grad_fd(w, pt, n, rel=1e-4)
    scale = np.abs(g) + 1e-3 * np.max(np.abs(g))
    return float(np.max(np.abs(g - gf) / scale))


def test_ggamma_gradient_matches_finite_differences():
    assert pin_ggamma_gradient() < 2e-6


def test_ggamma_asimov_and_rate_identity():
    w, n = _gg_small(0.8)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    assert O.nll(w, w["theta0"], mu) == pytest.approx(0.0, abs=1e-9)
    assert np.max(np.abs(O.nll_grad(w, w["theta0"], mu))) < 1e-8
    w["pull_param"] = np.zeros(0, np.int32); w["pull_centre"] = np.zeros(0); w["pull_width"] = np.zeros(0)
    assert pin_rate_identity(w, I.perturbed_points(w["theta0"], 1, 63)[0], n) < 1e-11


def test_ggamma_power_one_workload_matches_gamma_workload():
    base = I.borexino_like(n_bins=200, n_fine=1500)
    w = I.with_power(base, 1.0)
    mu = np.concatenate([O.expected_counts(base, base["theta0"], d) for d in range(2)])
    n = I.poisson_counts(mu, 64)
    pt = I.perturbed_points(base["theta0"], 1, 65)[0]
    assert abs(O.nll(w, np.concatenate([pt, [1.0]]), n) / O.nll(base, pt, n) - 1.0) < 1e-12
    g, g0 = O.nll_grad(w, np.concatenate([pt, [1.0]]), n), O.nll_grad(base, pt, n)
    assert np.max(np.abs(g[:-1] - g0)) <= 1e-9 * np.max(np.abs(g0))


GG_MUTANTS = {
    "power dropped from the CDF argument": ("ggamma_bins", lambda e, d, s, p: O._gamma_cdf_diff(
        np.broadcast_to((d / p)[None, :], (len(e) - 1, d.size)),
        np.clip(np.asarray(e)[:-1, None], 0, None) / s[None, :], np.asarray(e)[1:, None] / s[None, :])),
    "moment ratio with a instead of 2a": ("ggamma_log_moment_ratio", lambda x, a: O.lgamma_diff(x, a) - 2.0 * O.lgamma_diff(x, 0.5 * a)),
    "digamma difference sign": ("digamma_diff", lambda x, c: -(O.special.digamma(x + c) - O.special.digamma(x))),
}


@pytest.mark.parametrize("name", sorted(GG_MUTANTS))
def test_planted_ggamma_mistake_is_caught(monkeypatch, name):
    attr, fn = GG_MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = False
    for pin, tol in ((pin_ggamma_moments, 1e-12), (pin_ggamma_closed_forms, 1e-14), (pin_ggamma_gradient, 2e-6)):
        try:
            caught = pin() > tol
        except Exception:
            caught = True
        if caught:
            break
    assert caught, f"no pin caught the planted mistake '{name}'"


# ------------------- secondary observable: the extra likelihood pieces (section 2.4) --------
def _sec_small(n_sec=8):
    w = I.with_secondary(I.borexino_like(n_bins=200, n_fine=800), n_slices=5, n_sec=n_sec)
    mu = [O.expected_counts(w, w["theta0"], d) for d in range(2)]
    ms = np.concatenate([O.secondary_expected(w, w["theta0"], d)[1].ravel() for d in range(2)])
    return w, mu, ms, I.poisson_counts(np.concatenate(mu + [ms]), 71)


def pin_secondary_by_hand():
    """One secondary bin per slice: each slice adds the Poisson term of its total, by hand."""
    w, mu, ms, n = _sec_small(n_sec=1)
    p = I.perturbed_points(w["theta0"], 1, 72)[0]
    J = [len(e) - 1 for e in w["edges"]]
    base = O.nll(dict(w, secondary=None), p, n[:sum(J)])
    extra, o = 0.0, sum(J)
    for d in range(2):
        m = O.expected_counts(w, p, d)
        st = w["secondary"][d]["slice_start"]
        for q in range(len(st) - 1):
            tot, k = float(m[st[q]:st[q + 1]].sum()), n[o]
            extra += tot - k + (k * math.log(k / tot) if k > 0 else 0.0)
            o += 1
    return abs(O.nll(w, p, n) - (base + extra)) / abs(base + extra)


def test_secondary_piece_by_hand():
    assert pin_secondary_by_hand() < 1e-13


def pin_secondary_gradient():
    w, mu, ms, n = _sec_small()
    p = I.perturbed_points(w["theta0"], 1, 73, rel=0.02)[0]
    S = w["spectra"].shape[0]
    # a line, a beta, the peak rate, every response parameter and the peak position and width
    which = [6, 3, 14] + list(range(S, S + 7))
    worst = 0.0
    for win in (None, np.array([[30, 170], [30, 170]])):
        g = O.nll_grad(w, p, n, win)
        gf = O.nll_grad_fd(w, p, n, win, rel=1e-4, which=which)
        worst = max(worst, float(np.max(np.abs(g[which] - gf[which]) / (np.abs(g[which]) + 1e-3 * np.max(np.abs(g))))))
    return worst


def test_secondary_gradient_matches_finite_differences():
    assert pin_secondary_gradient() < 2e-6


def test_secondary_asimov_and_rate_identity():
    w, mu, ms, n = _sec_small()
    asimov = np.concatenate(mu + [ms])
    assert O.nll(w, w["theta0"], asimov) == pytest.approx(0.0, abs=1e-9)
    assert np.max(np.abs(O.nll_grad(w, w["theta0"], asimov))) < 1e-8
    # mu and mu_qm are linear in the rates: sum_s r_s dNLL/dr_s = sum (mu - n) over both pieces
    w2 = dict(w, pull_param=np.zeros(0, np.int32), pull_centre=np.zeros(0), pull_width=np.zeros(0))
    p = I.perturbed_points(w["theta0"], 1, 74)[0]
    g = O.nll_grad(w2, p, n)
    S = w["spectra"].shape[0]
    sm = np.asarray(w["slot_map"])[:, :S]
    idx = np.unique(sm[sm >= 0])
    rhs, o = 0.0, 400
    for d in range(2):
        rhs += float(np.sum(O.expected_counts(w, p, d) - n[200 * d:200 * (d + 1)]))
        mq = O.secondary_expected(w, p, d)[1]
        rhs += float(np.sum(mq - n[o:o + mq.size].reshape(mq.shape)))
        o += mq.size
    assert abs(float(np.dot(p[idx], g[idx])) - rhs) <= 1e-11 * max(1.0, abs(rhs))


def test_secondary_slices_outside_the_window_are_dropped():
    w, mu, ms, n = _sec_small()
    p = I.perturbed_points(w["theta0"], 1, 75)[0]
    st = w["secondary"][0]["slice_start"]
    # a window from the middle of slice 1 to the end of slice 3: slices 2 and 3 only
    win = np.array([[st[1] + 5, st[4]], [st[1] + 5, st[4]]])
    plain = O.nll(dict(w, secondary=None), p, n[:400], win)
    extra, o = 0.0, 400
    for d in range(2):
        mq = O.secondary_expected(w, p, d)[1]
        nq = n[o:o + mq.size].reshape(mq.shape)
        extra += float(np.sum(O.poisson_term(mq[2:4], nq[2:4])))
        o += mq.size
    assert abs(O.nll(w, p, n, win) - (plain + extra)) <= 1e-12 * abs(plain + extra)


SEC_MUTANTS = {
    "shapes not normalised": ("secondary_shapes", lambda work, d: np.asarray(work["secondary"][d]["shapes"], np.float64)),
    "slice includes its upper boundary bin": ("_active_slices", lambda work, d, lo, hi: [
        q for q in range(len(work["secondary"][d]["slice_start"]) - 1)
        if work["secondary"][d]["slice_start"][q] >= lo and work["secondary"][d]["slice_start"][q + 1] <= hi + 1]),
}


@pytest.mark.parametrize("name", sorted(SEC_MUTANTS))
def test_planted_secondary_mistake_is_caught(monkeypatch, name):
    attr, fn = SEC_MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = []
    for pin, tol in ((pin_secondary_by_hand, 1e-13), (pin_secondary_gradient, 2e-6)):
        try:
            caught.append(pin() > tol)
        except Exception:
            caught.append(True)
    try:
        w, mu, ms, n = _sec_small()
        st = w["secondary"][0]["slice_start"]
        win = np.array([[0, st[4] - 1], [0, st[4] - 1]])
        p = w["theta0"]
        got = O.nll(w, p, n, win)
        ref = O.nll(dict(w, secondary=None), p, n[:400], win)
        extra, o = 0.0, 400
        for d in range(2):
            Pn = np.asarray(w["secondary"][d]["shapes"], np.float64)
            Pn = Pn / Pn.sum(axis=2, keepdims=True)
            m = O.expected_per_species(w, p, d)
            for q in range(3):
                Nq = m[st[q]:st[q + 1]].sum(axis=0)
                mq = Nq @ Pn[:, q, :]
                extra += float(np.sum(O.poisson_term(mq, n[o + q * 8:o + q * 8 + 8])))
            o += 5 * 8
        caught.append(abs(got - (ref + extra)) > 1e-10 * abs(ref + extra))
    except Exception:
        caught.append(True)
    assert any(caught), f"no pin caught the planted mistake '{name}'"


# ------------------------- Fisher diagonal (the statistical scale of the gradient) --------
def _asimov_counts(w, theta):
    D = len(w["edges"])
    parts = [O.expected_counts(w, theta, d) for d in range(D)]
    sec = w.get("secondary")
    if sec is not None:
        parts += [O.secondary_expected(w, theta, d)[1].ravel() for d in range(D) if sec[d] is not None]
    return np.concatenate(parts)


@pytest.mark.parametrize("maker", ["gauss", "gamma_window", "secondary"])
def test_fisher_diagonal_is_the_asimov_curvature(maker):
    """With Asimov data n = mu(theta) every w_j = 1 - n_j/mu_j vanishes, so the second derivative
    of the NLL at theta is exactly sum_j (d mu_j / d theta_i)^2 / mu_j (+ 1/sigma^2 for a pull): the
    Fisher diagonal.  Here it is taken by central differences of the oracle's analytic gradient."""
    windows = None
    if maker == "gauss":
        w = I.single_gauss(n_bins=90, n_fine=200)
    elif maker == "gamma_window":
        w = I.borexino_like(n_bins=120, n_fine=500)
        windows = [(10, 100), (25, 120)]
    else:
        w = I.with_secondary(I.borexino_like(n_bins=120, n_fine=500), n_slices=4, n_sec=6)
        windows = [(30, 120), (0, 90)]
    theta = I.perturbed_points(w["theta0"], 1, 71)[0]
    n = _asimov_counts(w, theta)
    F = O.fisher_diagonal(w, theta, windows)
    for i in range(theta.size):
        h = 1e-4 * abs(theta[i])
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        hess = (O.nll_grad(w, tp, n, windows)[i] - O.nll_grad(w, tm, n, windows)[i]) / (2.0 * h)
        assert abs(hess - F[i]) <= 1e-5 * abs(F[i]) + 1e-12, (i, hess, F[i])
