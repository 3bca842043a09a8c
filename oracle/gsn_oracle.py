"""FP64 CPU oracle for the binned Poisson likelihood of a multi-species spectral fit.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only the
tests, the smoke check and the CPU-baseline leg of the benchmark may call it.
It shares no code with the GPU path: it is a plain, slow restatement of what
the method computes, written from the GooStats paper (arXiv:1812.05686):

* section 4.1, Eq. (LL): the binned Poisson log-likelihood plus Gaussian pull
  terms, minimised over the fit parameters;
* section 3.2 (the analytic-fit cost law T = T0 + k1 sum_i N_vis^i N_true^i):
  each species' expected visible spectrum is its fine true-energy spectrum
  convolved with the detector response;
* section 2.3: the analytic response (light yield, non-linear quenching,
  resolution) -- the formulas are stripped from the paper, so the readings
  below are used (they are listed with the design notes);
* section 4.3: species types Ana (smeared fine spectrum), AnaShift (shifted in
  true energy, then smeared) and AnaPeak (a peak with free position and width);
* section 2.2: parameter synchronisation across datasets, expressed as a slot
  map from per-dataset slots to global parameters;
* section 2.4 (multivariate fit): a second observable splits a dataset into
  slices, each a histogram of its own with fixed per-slice factors -- a
  multiplier of each response parameter (LY, kB, a, b, c) and a fraction of
  each species' rate -- expressed here as per-dataset factors: dataset d uses
  resp_scale[d][i] * (slot value) for the response and eps_d f_ds r_s for the
  rates (the workload keys "resp_scale" and "rate_factor"; both default to 1).

Readings (the paper gives no formula for them):
* quenching: Birks' law E_q(E) = int_0^E dE' / (1 + kB S(E')) with the
  two-term stopping power S(E) = s0 + s1/E, integrated in closed form;
* visible mean mu = LY * E_q(E) [p.e.]; variance sigma^2 = a + b mu + c mu^2;
* Gaussian response: the bin integral of N(x; mu, sigma);
* "generalized gamma" response: the gamma density with shape d = mu^2/sigma^2
  and scale s = sigma^2/mu (mean mu, variance sigma^2), bin-integrated with the
  regularised incomplete gamma function;
* generalized gamma with a free power p (resolution 2): Stacy's density
  p x^(d-1) exp(-(x/s)^p) / (s^d Gamma(d/p)) with (d, s) moment-matched to the
  column's mean and variance for the fit parameter p, bin-integrated as
  P(d/p, (x/s)^p); the power sits in the last per-dataset slot;
* spectra are point-sampled at the fine centres and normalised to unit sum;
  AnaShift moves the normalised spectrum up by round(shift / dE) fine bins;
* AnaPeak: a Gaussian of position m and width w directly in p.e.;
* Monte Carlo template species (the template fit of section 3.2): a histogram
  in the dataset's own visible bins ("templates" key: [species][dataset] array
  or None), normalised to unit sum; it enters as eps_d f_ds r_s T_dsj with no
  response;
* multivariate likelihood with a secondary observable (section 2.4, the extra likelihood pieces
  of MultiVariatePdf; workload key "secondary": per dataset None or dict(slice_start (Q+1,),
  shapes (S, Q, M), counts (Q, M))): the dataset's energy bins form Q contiguous slices, each with
  a histogram of a second observable in M bins; species s contributes to slice q its expected
  counts N_sq = sum_{j in q} mu_j^s spread by a fixed shape P_sqm (each (s, q) row normalised to
  unit sum, zero rows allowed); every slice inside the fit window adds
  sum_m [mu_qm - n_qm + n_qm ln(n_qm/mu_qm)], mu_qm = sum_s N_sq P_sqm, to the NLL (an extended
  Poisson piece: its events also populate the energy histogram, as adding likelihood pieces does);
  toy counts append each dataset's secondary counts (slices in order, m inner) after the energy bins;
* NLL = sum_d sum_{j in window} [mu - n + n ln(n/mu)] + 1/2 sum_pulls ((p-c)/sigma)^2,
  i.e. -ln L of Eq. (LL) up to a data-only constant, with the pull term read
  as the usual Gaussian constraint (Eq. (LL) prints its sign/factor garbled).

Parity status of the gradient of the gamma and generalized-gamma responses with
respect to the shape: the derivative of the regularised incomplete gamma function
with respect to its shape has no library routine, so it is taken by fourth-order
central differences in the shape (pinned against arbitrary-precision values in
the tests).  The generalized gamma's moment matching is solved by bracketed
Newton iteration on its defining equation, with the log-gamma differences taken
from their integral forms over the trigamma function where the log-gammas
themselves would cancel (pinned against 40-digit moments).  Everything else is
evaluated from closed forms or library special functions.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

KIND_ANA, KIND_ANA_SHIFT, KIND_ANA_PEAK, KIND_MC_TEMPLATE = 0, 1, 2, 3
RES_GAUSS, RES_GAMMA, RES_GGAMMA = 0, 1, 2
_RESP = ("LY", "kB", "a", "b", "c")


# ------------------------------------------------------------ quenching -----
def quenched_energy(E, kB, s0, s1):
    """Birks-quenched energy E_q(E) = int_0^E dE'/(1 + kB (s0 + s1/E')) (section 2.3, reading).

    With alpha = 1 + kB s0 and beta = kB s1 the integrand is E'/(alpha E' + beta), so
    E_q = E/alpha - (beta/alpha^2) ln(1 + alpha E / beta); kB = 0 gives E_q = E.
    """
    E = np.asarray(E, np.float64)
    alpha = 1.0 + kB * s0
    beta = kB * s1
    if beta == 0.0:
        return E / alpha
    return E / alpha - (beta / alpha**2) * np.log1p(alpha * E / beta)


def quenched_energy_dkB(E, kB, s0, s1):
    """d E_q / d kB of the closed form above (chain rule through alpha and beta)."""
    E = np.asarray(E, np.float64)
    alpha = 1.0 + kB * s0
    beta = kB * s1
    L = np.log1p(alpha * E / beta)
    d_alpha = -E / alpha**2 + 2.0 * beta * L / alpha**3 - E * beta / (alpha**2 * (beta + alpha * E))
    d_beta = -L / alpha**2 + E / (alpha * (beta + alpha * E))
    return s0 * d_alpha + s1 * d_beta


# ------------------------------------------------------------- spectra ------
def species_spectra(work):
    """Normalised (and, for AnaShift, shifted) fine spectra S'[s, k] (section 4.3, reading).

    Rows of AnaPeak and template species are zero (they do not pass through the response).
    """
    E = np.asarray(work["fine_centres"], np.float64)
    f = np.asarray(work["spectra"], np.float64)
    S = np.zeros_like(f)
    dE = (E[-1] - E[0]) / (E.size - 1) if E.size > 1 else 1.0
    for s in range(f.shape[0]):
        kind = int(work["kind"][s])
        if kind in (KIND_ANA_PEAK, KIND_MC_TEMPLATE):
            continue
        tot = f[s].sum()
        row = f[s] / tot if tot > 0 else np.zeros_like(f[s])
        if kind == KIND_ANA_SHIFT:
            n = int(math.floor(work["shift"][s] / dE + 0.5))
            shifted = np.zeros_like(row)
            if n >= 0:
                if n < row.size:
                    shifted[n:] = row[: row.size - n]
            else:
                shifted[: row.size + n] = row[-n:]
            row = shifted
        S[s] = row
    return S


# ------------------------------------------------------------ responses -----
def _norm_cdf_diff(lo, hi):
    """Phi(hi) - Phi(lo), taking upper tails where both points lie above 0."""
    upper = lo >= 0.0
    return np.where(upper, special.ndtr(-lo) - special.ndtr(-hi), special.ndtr(hi) - special.ndtr(lo))


def response_gauss(edges, mu, sigma):
    """R[j, k] = int_{x_j}^{x_{j+1}} N(x; mu_k, sigma_k) dx (section 2.3, reading)."""
    x = np.asarray(edges, np.float64)[:, None]
    z = (x - mu[None, :]) / sigma[None, :]
    return _norm_cdf_diff(z[:-1], z[1:])


def _gamma_cdf_diff(d, lo, hi):
    """P(d, hi) - P(d, lo) with the regularised incomplete gamma, upper tails above the mean."""
    upper = lo >= d
    return np.where(upper, special.gammaincc(d, lo) - special.gammaincc(d, hi),
                    special.gammainc(d, hi) - special.gammainc(d, lo))


def gamma_shape_scale(mu, var):
    """Moment matching: shape d = mu^2/var, scale s = var/mu (mean mu, variance var)."""
    return mu * mu / var, var / mu


def response_gamma(edges, mu, var):
    """R[j, k] = P(d_k, x_{j+1}/s_k) - P(d_k, x_j/s_k), gamma density of mean mu, variance var."""
    d, s = gamma_shape_scale(mu, var)
    y = np.clip(np.asarray(edges, np.float64), 0.0, None)[:, None] / s[None, :]
    dd = np.broadcast_to(d[None, :], y.shape)
    return _gamma_cdf_diff(dd[:-1], y[:-1], y[1:])


def _gamma_P_dshape(d, y):
    """dP(d, y)/dd by fourth-order central differences in d (see module docstring)."""
    h = 2e-3 * np.minimum(d, np.sqrt(np.maximum(d, 1.0)))
    h = np.minimum(h, d / 4.0)
    f = lambda dd: special.gammainc(dd, y)
    return (8.0 * (f(d + h) - f(d - h)) - (f(d + 2 * h) - f(d - 2 * h))) / (12.0 * h)


def _gamma_pdf_times_y(d, y):
    """p(d, y) * y with p the standard gamma density y^(d-1) e^-y / Gamma(d); 0 at y = 0."""
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.exp(d * np.log(y) - y - special.gammaln(d))
    return np.where(y > 0.0, v, 0.0)


# ------------------------------------ generalized gamma with a free power p ----
# Stacy's generalized gamma density, the line shape of the generalized-gamma response the paper cites
# (section 2.3):  f(x; d, s, p) = p x^(d-1) exp(-(x/s)^p) / (s^d Gamma(d/p)),  x > 0,  whose CDF is
# the regularised incomplete gamma P(d/p, (x/s)^p).  Reading: the power p is a fit parameter, and
# every column's (d, s) follow from its mean and variance by moment matching,
#     mu = s Gamma(x + a) / Gamma(x),   mu^2 + var = s^2 Gamma(x + 2a) / Gamma(x),   x = d/p, a = 1/p;
# p = 1 is the gamma reading.  Eliminating s leaves one equation for x,
#     H(x) = lnGamma(x + 2a) + lnGamma(x) - 2 lnGamma(x + a) = ln(1 + var/mu^2).
#
# H and the other differences below are O(1/x) (or O(ln x)) while each log-gamma is O(x ln x), so
# for large x the library log-gammas would cancel.  There they are taken from the textbook integral
# forms of the differences instead (lnGamma' = psi, psi' = psi_1, psi_1' = psi_2):
#     lnGamma(x + c) - lnGamma(x) = int_0^c psi(x + t) dt,
#     psi(x + c) - psi(x)         = int_0^c psi_1(x + t) dt,
#     H(x, a) = int_0^a int_0^a psi_1(x + t + u) du dt = int_0^2a psi_1(x + v) min(v, 2a - v) dv,
#     dH/dx   = int_0^2a psi_2(x + v) min(v, 2a - v) dv,
# with positive, smooth integrands (the nearest pole, at v = -x, lies well outside [0, 2a]),
# integrated by Gauss-Legendre quadrature on [0, a] and [a, 2a] where the kernel is linear.  Below
# _X_DIRECT every term is O(1) and the library differences are used as they stand.
_X_DIRECT = 2.0
_GL_X, _GL_W = np.polynomial.legendre.leggauss(12)


def _trigamma(z):
    return special.polygamma(1, z)


def _tetragamma(z):
    return special.polygamma(2, z)


def _gl(f, x, lo, hi, kernel=None):
    """int_lo^hi f(x + t) k(t) dt for every element of x (Gauss-Legendre; k = 1 if kernel is None)."""
    t = 0.5 * (hi - lo) * _GL_X + 0.5 * (hi + lo)
    w = 0.5 * (hi - lo) * _GL_W * (1.0 if kernel is None else kernel(t))
    return np.sum(f(x[..., None] + t) * w, axis=-1)


def _second_difference(f, x, a):
    """int_0^2a f(x + v) min(v, 2a - v) dv."""
    return _gl(f, x, 0.0, a, lambda t: t) + _gl(f, x, a, 2.0 * a, lambda t: 2.0 * a - t)


def _by_size(x, direct, integral):
    """direct(x) below _X_DIRECT, integral(x) from it on (elementwise)."""
    x = np.asarray(x, np.float64)
    out = np.empty_like(x)
    small = x < _X_DIRECT
    if np.any(small):
        out[small] = direct(x[small])
    if np.any(~small):
        out[~small] = integral(x[~small])
    return out


def lgamma_diff(x, c):
    """lnGamma(x + c) - lnGamma(x) for x > 0, c >= 0."""
    return _by_size(x, lambda v: special.gammaln(v + c) - special.gammaln(v),
                    lambda v: _gl(special.digamma, v, 0.0, c))


def digamma_diff(x, c):
    """psi(x + c) - psi(x) for x > 0, c >= 0."""
    return _by_size(x, lambda v: special.digamma(v + c) - special.digamma(v),
                    lambda v: _gl(_trigamma, v, 0.0, c))


def ggamma_log_moment_ratio(x, a):
    """H(x) = ln[Gamma(x + 2a) Gamma(x) / Gamma(x + a)^2] = ln(E[Y^2a] / E[Y^a]^2), Y ~ Gamma(x, 1)."""
    return _by_size(x, lambda v: special.gammaln(v + 2 * a) + special.gammaln(v) - 2.0 * special.gammaln(v + a),
                    lambda v: _second_difference(_trigamma, v, a))


def ggamma_log_moment_ratio_dx(x, a):
    """dH/dx = psi(x + 2a) - 2 psi(x + a) + psi(x) (negative: H falls as x grows)."""
    return _by_size(x, lambda v: special.digamma(v + 2 * a) - 2.0 * special.digamma(v + a) + special.digamma(v),
                    lambda v: _second_difference(_tetragamma, v, a))


def ggamma_shape_scale(mu, var, p):
    """Moment matching for the generalized gamma of power p: shape d and scale s with mean mu and
    variance var.  H(x) = r, r = ln(1 + var/mu^2), is solved for x = d/p column by column by
    Newton's method in x, safeguarded by a bracket: H falls monotonically from +inf (x -> 0) to 0
    (x -> inf), so every evaluation moves one end of the bracket, and a Newton step that leaves the
    bracket is replaced by its geometric midpoint (or by a factor-4 move while one end is open).
    The start is the large-x limit H ~ a^2/x for r <= 1, else the small-x limit
    H ~ lnGamma(2a) - 2 lnGamma(a) - ln x.  Then s = mu Gamma(x) / Gamma(x + 1/p)."""
    mu = np.asarray(mu, np.float64)
    var = np.asarray(var, np.float64)
    a = 1.0 / p
    r = np.log1p(var / (mu * mu))
    x = np.where(r <= 1.0, a * a / r, np.exp(special.gammaln(2 * a) - 2.0 * special.gammaln(a) - r))
    lo = np.zeros_like(x)
    hi = np.full_like(x, np.inf)
    active = np.ones(x.shape, bool)
    for _ in range(400):
        i = np.nonzero(active)
        xi = x[i]
        h = ggamma_log_moment_ratio(xi, a) - r[i]
        lo[i] = np.where(h > 0.0, xi, lo[i])
        hi[i] = np.where(h <= 0.0, xi, hi[i])
        with np.errstate(divide="ignore", invalid="ignore"):
            step = h / ggamma_log_moment_ratio_dx(xi, a)
        xn = xi - step
        # quadratic convergence: once the Newton step is below 1e-12 x, the point it reaches is at
        # rounding level
        conv = np.abs(step) <= 1e-12 * xi
        inside = (xn > lo[i]) & (xn < hi[i])
        fallback = np.where(np.isinf(hi[i]), 4.0 * xi, np.where(lo[i] > 0.0, np.sqrt(lo[i] * hi[i]), 0.25 * hi[i]))
        x[i] = np.where(inside | conv, xn, fallback)
        active[i] = ~conv
        if not np.any(active):
            break
    else:
        raise FloatingPointError("generalized-gamma moment matching did not converge")
    return p * x, mu * np.exp(-lgamma_diff(x, a))


def ggamma_bins(edges, d, s, p):
    """R[j, k] = P(d_k/p, (x_{j+1}/s_k)^p) - P(d_k/p, (x_j/s_k)^p): bin integrals of the density."""
    y = (np.clip(np.asarray(edges, np.float64), 0.0, None)[:, None] / s[None, :]) ** p
    aa = np.broadcast_to((d / p)[None, :], y.shape)
    return _gamma_cdf_diff(aa[:-1], y[:-1], y[1:])


def response_ggamma(edges, mu, var, p):
    """Generalized-gamma response of power p (moment-matched shape and scale per column)."""
    d, s = ggamma_shape_scale(mu, var, p)
    return ggamma_bins(edges, d, s, p)


def peak_profile(edges, m, w):
    """AnaPeak: int over each bin of N(x; m, w) in p.e. (section 4.3, reading)."""
    z = (np.asarray(edges, np.float64) - m) / w
    return _norm_cdf_diff(z[:-1], z[1:])


def template(work, s, d):
    """Normalised visible-bin template of species s in dataset d (zeros if it has none there)."""
    J = len(work["edges"][d]) - 1
    tpl = work.get("templates")
    h = None if tpl is None else tpl[s][d]
    if h is None:
        return np.zeros(J)
    h = np.asarray(h, np.float64)
    tot = h.sum()
    return h / tot if tot > 0 else np.zeros(J)


# ------------------------------------------------------- parameter map ------
def dataset_values(work, params, d):
    """Per-dataset slot values from the global parameters (section 2.2 synchronisation)."""
    sm = np.asarray(work["slot_map"])[d]
    vals = np.full(sm.size, np.nan)
    used = sm >= 0
    vals[used] = np.asarray(params, np.float64)[sm[used]]
    return vals


def dataset_factors(work, d):
    """Fixed factors of dataset d (section 2.4 slices): response multipliers (5,) and rate fractions (S,)."""
    S = np.asarray(work["spectra"]).shape[0]
    rs = work.get("resp_scale")
    rf = work.get("rate_factor")
    scale = np.ones(5) if rs is None else np.asarray(rs, np.float64)[d]
    frac = np.ones(S) if rf is None else np.asarray(rf, np.float64)[d]
    return scale, frac


def _unpack(work, vals):
    """Slots: S rates, (LY, kB, a, b, c), (m, w) per species, then the generalized-gamma power p."""
    S = np.asarray(work["spectra"]).shape[0]
    rates = vals[:S]
    resp = dict(zip(_RESP, vals[S:S + 5]))
    peaks = vals[S + 5:3 * S + 5].reshape(S, 2)
    if int(work["resolution"]) == RES_GGAMMA:
        resp["p"] = vals[3 * S + 5]
    return rates, resp, peaks


def column_mean_var(work, resp):
    """Per fine column: visible mean mu_k [p.e.] and resolution variance sigma_k^2."""
    E = np.asarray(work["fine_centres"], np.float64)
    Eq = quenched_energy(E, resp["kB"], work["birks_s0"], work["birks_s1"])
    mu = resp["LY"] * Eq
    var = resp["a"] + resp["b"] * mu + resp["c"] * mu * mu
    return Eq, mu, var


def response_matrix(work, edges, resp):
    """Detector response matrix R[j, k] of a dataset (section 2.3 / 2.5 'two-dimensional mesh')."""
    _, mu, var = column_mean_var(work, resp)
    if np.any(var <= 0) or np.any(mu <= 0):
        raise FloatingPointError("non-positive mean or variance")
    if int(work["resolution"]) == RES_GAUSS:
        return response_gauss(edges, mu, np.sqrt(var))
    if int(work["resolution"]) == RES_GGAMMA:
        return response_ggamma(edges, mu, var, resp["p"])
    return response_gamma(edges, mu, var)


# --------------------------------------------------------- expectation ------
def expected_per_species(work, params, d):
    """Expected counts per bin and species of dataset d, shape (J, S) (section 3.1 validation quantity).

    Column s holds eps_d f_ds r_s sum_k R[j,k] S'[s,k] for Ana/AnaShift species,
    eps_d f_ds r_s * peak_j(m_s, w_s) for AnaPeak species and eps_d f_ds r_s T_dsj for
    template species; zero where mask[s, d] = 0.
    R is built from the response slots times the dataset's response multipliers.
    """
    vals = dataset_values(work, params, d)
    rates, resp, peaks = _unpack(work, vals)
    scale, frac = dataset_factors(work, d)
    resp = dict(resp, **{k: resp[k] * scale[i] for i, k in enumerate(_RESP)})
    edges = np.asarray(work["edges"][d], np.float64)
    eps = float(work["exposure"][d])
    Sp = species_spectra(work)
    kinds = np.asarray(work["kind"])
    mask = np.asarray(work["mask"])[:, d].astype(bool)
    R = response_matrix(work, edges, resp) if np.any(mask & (kinds < KIND_ANA_PEAK)) else None
    J, S = edges.size - 1, Sp.shape[0]
    out = np.zeros((J, S))
    for s in range(S):
        if not work["mask"][s][d]:
            continue
        if int(work["kind"][s]) == KIND_ANA_PEAK:
            out[:, s] = eps * frac[s] * rates[s] * peak_profile(edges, peaks[s, 0], peaks[s, 1])
        elif int(work["kind"][s]) == KIND_MC_TEMPLATE:
            out[:, s] = eps * frac[s] * rates[s] * template(work, s, d)
        else:
            out[:, s] = eps * frac[s] * rates[s] * (R @ Sp[s])
    return out


def expected_counts(work, params, d):
    """mu_dj: the rate-weighted sum over species (section 3.2 analytic fit)."""
    return expected_per_species(work, params, d).sum(axis=1)


# ------------------------------------------------------------ likelihood ----
def poisson_term(mu, n):
    """mu - n + n ln(n/mu), i.e. -ln Poisson(n; mu) up to its value at mu = n (Eq. LL)."""
    mu = np.asarray(mu, np.float64)
    n = np.asarray(n, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(n > 0, mu - n + n * np.log(n / mu), mu)
    return np.where((n > 0) & (mu <= 0), np.inf, t)


def pull_term(work, params):
    p = np.asarray(params, np.float64)
    idx = np.asarray(work["pull_param"], np.int64)
    if idx.size == 0:
        return 0.0
    r = (p[idx] - np.asarray(work["pull_centre"])) / np.asarray(work["pull_width"])
    return 0.5 * float(np.sum(r * r))


def _windows(work, windows):
    D = len(work["edges"])
    if windows is None:
        return [(int(work["win_lo"][d]), int(work["win_hi"][d])) for d in range(D)]
    return [(int(windows[d][0]), int(windows[d][1])) for d in range(D)]


def _split_counts(work, counts):
    """Energy counts per dataset (a toy's secondary counts, if any, follow them and are ignored here)."""
    if isinstance(counts, (list, tuple)):
        return [np.asarray(c, np.float64) for c in counts]
    c = np.asarray(counts, np.float64)
    out, o = [], 0
    for e in work["edges"]:
        J = len(e) - 1
        out.append(c[o:o + J]); o += J
    return out


# --------------------------------------------- secondary observable (section 2.4) ----
def secondary_shapes(work, d):
    """Normalised secondary shapes P[s, q, m] of dataset d (rows of zero sum stay zero), or None."""
    sec = work.get("secondary")
    if sec is None or sec[d] is None:
        return None
    P = np.array(sec[d]["shapes"], np.float64, copy=True)
    tot = P.sum(axis=2, keepdims=True)
    return np.divide(P, tot, out=np.zeros_like(P), where=tot > 0)


def _secondary_counts(work, counts):
    """Observed secondary counts per dataset ((Q, M) or None): the tail of a toy's counts row after
    the energy bins when present, else the workload's own."""
    sec = work.get("secondary")
    D = len(work["edges"])
    if sec is None:
        return [None] * D
    flat = None
    if not isinstance(counts, (list, tuple)):
        c = np.asarray(counts, np.float64)
        nE = sum(len(e) - 1 for e in work["edges"])
        if c.size > nE:
            flat, o = c[nE:], 0
    out = []
    for d in range(D):
        if sec[d] is None:
            out.append(None)
            continue
        Q, M = np.asarray(sec[d]["shapes"]).shape[1:]
        if flat is not None:
            out.append(flat[o:o + Q * M].reshape(Q, M)); o += Q * M
        else:
            out.append(np.asarray(sec[d]["counts"], np.float64).reshape(Q, M))
    return out


def _active_slices(work, d, lo, hi):
    st = np.asarray(work["secondary"][d]["slice_start"], np.int64)
    return [q for q in range(st.size - 1) if st[q] >= lo and st[q + 1] <= hi and st[q + 1] > st[q]]


def secondary_expected(work, params, d):
    """N[s, q] (species' expected counts in every slice) and mu[q, m] = sum_s N[s, q] P[s, q, m]."""
    P = secondary_shapes(work, d)
    st = np.asarray(work["secondary"][d]["slice_start"], np.int64)
    per = expected_per_species(work, params, d)
    N = np.stack([per[st[q]:st[q + 1]].sum(axis=0) for q in range(st.size - 1)], axis=1)
    return N, np.einsum("sq,sqm->qm", N, P)


def nll(work, params, counts, windows=None):
    """NLL = sum_d sum_{j in window_d} [mu - n + n ln(n/mu)] + 1/2 sum pulls^2 (section 4.1, Eq. LL)."""
    cs = _split_counts(work, counts)
    sc = _secondary_counts(work, counts)
    total = 0.0
    for d, (lo, hi) in enumerate(_windows(work, windows)):
        if hi <= lo:
            continue
        mu = expected_counts(work, params, d)
        total += float(np.sum(poisson_term(mu[lo:hi], cs[d][lo:hi])))
        if sc[d] is not None:
            act = _active_slices(work, d, lo, hi)
            if act:
                _, mq = secondary_expected(work, params, d)
                total += float(np.sum(poisson_term(mq[act], sc[d][act])))
    return total + pull_term(work, params)


# -------------------------------------------------------------- gradient ----
def nll_grad(work, params, counts, windows=None):
    """Analytic gradient dNLL/dtheta by the chain rule (same readings as nll()).

    dNLL/dmu_dj = 1 - n_dj/mu_dj inside the window; mu_dj depends on the
    rates linearly, on (LY, kB, a, b, c) through every column's mean and
    variance, and on (m, w) of AnaPeak species through the peak profile.
    """
    params = np.asarray(params, np.float64)
    cs = _split_counts(work, counts)
    seccnt = _secondary_counts(work, counts)
    P = int(work["n_params"])
    g = np.zeros(P)
    Sp = species_spectra(work)
    E = np.asarray(work["fine_centres"], np.float64)
    S = Sp.shape[0]
    for d, (lo, hi) in enumerate(_windows(work, windows)):
        if hi <= lo:
            continue
        vals = dataset_values(work, params, d)
        rates, resp, peaks = _unpack(work, vals)
        scale, frac = dataset_factors(work, d)
        resp = dict(resp, **{k: resp[k] * scale[i] for i, k in enumerate(_RESP)})
        edges = np.asarray(work["edges"][d], np.float64)
        eps = float(work["exposure"][d])
        mask = np.asarray(work["mask"])[:, d].astype(bool)
        n = cs[d]
        mu = expected_counts(work, params, d)
        w = np.zeros(edges.size - 1)
        w[lo:hi] = 1.0 - n[lo:hi] / mu[lo:hi]
        # secondary pieces: dNLL/dmu_j^s = v_{s, q(j)} = sum_m (1 - n_qm/mu_qm) P_sqm on the bins of
        # every active slice, on top of the energy weight w_j shared by all species
        V = np.zeros((edges.size - 1, S))
        if seccnt[d] is not None:
            act = _active_slices(work, d, lo, hi)
            if act:
                Psh = secondary_shapes(work, d)
                _, mq = secondary_expected(work, params, d)
                st = np.asarray(work["secondary"][d]["slice_start"], np.int64)
                for q in act:
                    V[st[q]:st[q + 1]] = (1.0 - seccnt[d][q] / mq[q]) @ Psh[:, q, :].T
        gs = np.zeros(vals.size)  # gradient wrt the dataset's slots
        # smeared species and the response parameters (datasets of template / peak species only skip this)
        smeared = mask & (np.asarray(work["kind"]) < KIND_ANA_PEAK)
        base = S
        if smeared.any():
            Eq, mu_k, var_k = column_mean_var(work, resp)
            Ts = eps * (frac * rates)[smeared][:, None] * Sp[smeared]    # per smeared species
            T = Ts.sum(axis=0)
            Vs = V[:, smeared]

            def wsum(dX):
                """sum_j sum_s (w_j + v_sj) dX_jk T_sk: the weighted derivative per column"""
                return (w @ dX) * T + ((Vs.T @ dX) * Ts).sum(axis=0)
            R = response_matrix(work, edges, resp)
            u = w @ R  # u_k = sum_j w_j R_jk
            for s in np.nonzero(smeared)[0]:
                gs[s] += eps * frac[s] * float(Sp[s] @ (u + V[:, s] @ R))
            # response parameters through (mu_k, var_k)
            x = edges[:, None]
            if int(work["resolution"]) == RES_GAUSS:
                sig = np.sqrt(var_k)
                z = (x - mu_k[None, :]) / sig[None, :]
                phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
                dR_dmu = -(phi[1:] - phi[:-1]) / sig[None, :]
                dR_dsig = -(z[1:] * phi[1:] - z[:-1] * phi[:-1]) / sig[None, :]
                g_mu = wsum(dR_dmu)
                g_sig = wsum(dR_dsig)
                g_var = g_sig / (2.0 * sig)
            elif int(work["resolution"]) == RES_GGAMMA:
                pw = resp["p"]
                a = 1.0 / pw
                dsh, sc = ggamma_shape_scale(mu_k, var_k, pw)
                xs = dsh / pw
                ee = np.clip(edges, 0.0, None)[:, None]
                y = (ee / sc[None, :]) ** pw
                aa = np.broadcast_to(xs[None, :], y.shape)
                Pa = _gamma_P_dshape(aa, y)          # dP(a, y)/da at the edges
                py = _gamma_pdf_times_y(aa, y)        # y dP/dy
                with np.errstate(divide="ignore", invalid="ignore"):
                    pyl = np.where(ee > 0.0, py * np.log(ee / sc[None, :]), 0.0)
                # bin-integral derivatives at fixed (d, s, p): a = d/p, y = (x/s)^p
                dR_dd = (Pa[1:] - Pa[:-1]) / pw
                dR_dlns = -pw * (py[1:] - py[:-1])
                dR_dp = -(dsh / pw**2)[None, :] * (Pa[1:] - Pa[:-1]) + (pyl[1:] - pyl[:-1])
                g_d = wsum(dR_dd)
                g_u = wsum(dR_dlns)
                g_pe = wsum(dR_dp)
                # moment matching H(x, a) = ln rho, ln s = ln mu - G(x, a), G = lnGamma(x+a) - lnGamma(x):
                # implicit derivatives of x = d/p and u = ln s with respect to (mu, var, p)
                Hx = ggamma_log_moment_ratio_dx(xs, a)
                Ha = 2.0 * (digamma_diff(xs, 2 * a) - digamma_diff(xs, a))
                Gx = digamma_diff(xs, a)
                Ga = special.digamma(xs + a)
                r_mu = -2.0 * var_k / (mu_k * (mu_k**2 + var_k))
                r_var = 1.0 / (mu_k**2 + var_k)
                x_mu, x_var, x_p = r_mu / Hx, r_var / Hx, Ha / (pw**2 * Hx)
                g_mu = g_d * pw * x_mu + g_u * (1.0 / mu_k - Gx * x_mu)
                g_var = g_d * pw * x_var + g_u * (-Gx * x_var)
                gs[3 * S + 5] += float(np.sum(g_pe + g_d * (xs + pw * x_p) + g_u * (-Gx * x_p + Ga / pw**2)))
            else:
                dsh, sc = gamma_shape_scale(mu_k, var_k)
                y = np.clip(edges, 0.0, None)[:, None] / sc[None, :]
                dd = np.broadcast_to(dsh[None, :], y.shape)
                Pd = _gamma_P_dshape(dd, y)
                py = _gamma_pdf_times_y(dd, y)
                dR_dd = Pd[1:] - Pd[:-1]
                dR_ds = -(py[1:] - py[:-1]) / sc[None, :]
                g_d = wsum(dR_dd)
                g_s = wsum(dR_ds)
                g_mu = g_d * (2.0 * mu_k / var_k) + g_s * (-var_k / mu_k**2)
                g_var = g_d * (-(mu_k**2) / var_k**2) + g_s / mu_k
            g_mu_tot = g_mu + g_var * (resp["b"] + 2.0 * resp["c"] * mu_k)
            gs[base + 0] += float(g_mu_tot @ Eq)
            gs[base + 1] += float(g_mu_tot @ (resp["LY"] * quenched_energy_dkB(E, resp["kB"], work["birks_s0"], work["birks_s1"])))
            gs[base + 2] += float(g_var.sum())
            gs[base + 3] += float(g_var @ mu_k)
            gs[base + 4] += float(g_var @ (mu_k * mu_k))
            # the slots hold the unscaled parameters: d(scale_i p_i)/dp_i = scale_i
            gs[base:base + 5] *= scale
        # template species: mu is linear in the rate
        for s in np.nonzero(mask & (np.asarray(work["kind"]) == KIND_MC_TEMPLATE))[0]:
            gs[s] += eps * frac[s] * float((w + V[:, s]) @ template(work, s, d))
        # peak species
        for s in np.nonzero(mask & (np.asarray(work["kind"]) == KIND_ANA_PEAK))[0]:
            m, wd = peaks[s]
            zz = (edges - m) / wd
            ph = np.exp(-0.5 * zz * zz) / math.sqrt(2.0 * math.pi)
            prof = _norm_cdf_diff(zz[:-1], zz[1:])
            ws = w + V[:, s]
            gs[s] += eps * frac[s] * float(ws @ prof)
            gs[base + 5 + 2 * s] += eps * frac[s] * rates[s] * float(ws @ (-(ph[1:] - ph[:-1]) / wd))
            gs[base + 5 + 2 * s + 1] += eps * frac[s] * rates[s] * float(ws @ (-(zz[1:] * ph[1:] - zz[:-1] * ph[:-1]) / wd))
        sm = np.asarray(work["slot_map"])[d]
        for slot, pidx in enumerate(sm):
            if pidx >= 0:
                g[pidx] += gs[slot]
    idx = np.asarray(work["pull_param"], np.int64)
    for i, p in enumerate(idx):
        g[p] += (params[p] - work["pull_centre"][i]) / work["pull_width"][i] ** 2
    return g


def nll_grad_fd(work, params, counts, windows=None, rel=1e-5, which=None):
    """Richardson-extrapolated central differences of nll() (a self-check of nll_grad)."""
    params = np.asarray(params, np.float64)
    idx = range(params.size) if which is None else which
    g = np.full(params.size, np.nan)
    for i in idx:
        h = rel * (abs(params[i]) if params[i] != 0 else 1e-3)

        def f(t):
            p = params.copy(); p[i] += t
            return nll(work, p, counts, windows)
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
        g[i] = (4.0 * d1 - d2) / 3.0
    return g


def fisher_diagonal(work, params, windows=None, rel=1e-4):
    """Diagonal of the Fisher information of the likelihood (Eq. LL) at params,

        F_ii = sum_d sum_{j in window_d} (d mu_dj / d theta_i)^2 / mu_dj  [+ secondary pieces]
               + 1 / sigma_i^2 for a pulled parameter,

    the variance of dNLL/dtheta_i under Poisson fluctuations of the counts, i.e. the statistical
    scale of each gradient component.  The expected counts are linear in the rates, so a parameter
    that fills only rate slots has d mu / d theta_i = (its species' expected counts) / theta_i; the
    derivatives for the other parameters are central differences with step rel * |theta_i| (a
    scale needs no more precision than that).  Secondary pieces (section 2.4) add
    (d mu_qm / d theta_i)^2 / mu_qm over the slices inside the window.
    """
    params = np.asarray(params, np.float64)
    wins = _windows(work, windows)
    sec = work.get("secondary")
    S = np.asarray(work["spectra"]).shape[0]
    sm = np.asarray(work["slot_map"])

    def per_species(p):
        """expected counts per species over the window bins and active secondary bins: (bins, S)"""
        out = []
        for d, (lo, hi) in enumerate(wins):
            out.append(expected_per_species(work, p, d)[lo:hi])
            if sec is not None and sec[d] is not None:
                act = _active_slices(work, d, lo, hi)
                if act:
                    N, _ = secondary_expected(work, p, d)
                    P = secondary_shapes(work, d)
                    out.append(np.einsum("sq,sqm->qms", N[:, act], P[:, act, :]).reshape(-1, S))
        return out
    base = per_species(params)
    mu = np.concatenate([b.sum(axis=1) for b in base])
    ok = mu > 0
    F = np.zeros(params.size)
    for i in range(params.size):
        slots = np.argwhere(sm == i)
        if slots.size and np.all(slots[:, 1] < S) and params[i] != 0.0:
            # rate: mu is linear in it; blocks follow the datasets, a secondary block after its dataset
            parts, k = [], 0
            for d, (lo, hi) in enumerate(wins):
                rows = [s for dd, s in slots if dd == d]
                for blk in ([0, 1] if (sec is not None and sec[d] is not None and
                                       _active_slices(work, d, lo, hi)) else [0]):
                    b = base[k]; k += 1
                    parts.append(b[:, rows].sum(axis=1) / params[i] if rows else np.zeros(b.shape[0]))
            dm = np.concatenate(parts)
        else:
            h = rel * (abs(params[i]) if params[i] != 0 else 1e-3)
            pp, pm = params.copy(), params.copy()
            pp[i] += h
            pm[i] -= h
            dm = (np.concatenate([b.sum(axis=1) for b in per_species(pp)])
                  - np.concatenate([b.sum(axis=1) for b in per_species(pm)])) / (2.0 * h)
        F[i] = float(np.sum(dm[ok] ** 2 / mu[ok]))
    for k, p in enumerate(np.asarray(work["pull_param"], np.int64)):
        F[p] += 1.0 / work["pull_width"][k] ** 2
    return F


# ----------------------------------------------------------------- batch ----
def nll_batch(work, params, counts, windows):
    """Per-toy NLL for a batch: params (T, P), counts (T, sum J_d), windows (T, D, 2)."""
    return np.array([nll(work, params[t], counts[t], windows[t]) for t in range(len(params))])


def nll_grad_batch(work, params, counts, windows):
    return np.array([nll_grad(work, params[t], counts[t], windows[t]) for t in range(len(params))])


# ------------------------------------------------------- profile likelihood ----
def fit(work, counts, start, free, lo=None, hi=None, windows=None, scale=None):
    """Minimise the NLL over the parameters flagged in `free` (section 4.2 profile likelihood).

    The library minimiser scipy L-BFGS-B is the step; the objective and its gradient are this
    module's nll / nll_grad.  Bounds lo / hi (None = unbounded; rates are usually bounded at 0);
    the search runs in scaled variables u = x / scale (default |start|, 1 where start is 0).
    Returns (x_min, nll_min).
    """
    from scipy import optimize
    x0 = np.asarray(start, np.float64)
    free = np.asarray(free, bool)
    sc = np.where(x0 != 0.0, np.abs(x0), 1.0) if scale is None else np.asarray(scale, np.float64)
    idx = np.nonzero(free)[0]
    if idx.size == 0:
        return x0.copy(), nll(work, x0, counts, windows)

    def full(u):
        x = x0.copy()
        x[idx] = u * sc[idx]
        return x

    def f(u):
        x = full(u)
        return nll(work, x, counts, windows), nll_grad(work, x, counts, windows)[idx] * sc[idx]

    bounds = None
    if lo is not None or hi is not None:
        l = np.full(x0.size, -np.inf) if lo is None else np.asarray(lo, np.float64)
        h = np.full(x0.size, np.inf) if hi is None else np.asarray(hi, np.float64)
        bounds = [(l[i] / sc[i] if np.isfinite(l[i]) else None, h[i] / sc[i] if np.isfinite(h[i]) else None)
                  for i in idx]
    res = optimize.minimize(f, x0[idx] / sc[idx], jac=True, method="L-BFGS-B", bounds=bounds,
                            options=dict(maxiter=5000, ftol=1e-15, gtol=1e-10, maxcor=20))
    x = full(res.x)
    return x, nll(work, x, counts, windows)


def discovery_q0(work, counts, start, free, null_param, lo=None, hi=None, windows=None, scale=None):
    """Discovery test statistic q0 = 2 (min NLL with parameter null_param fixed at 0 - min NLL),
    0 when the free fit prefers a negative-going signal (one-sided, section 4.2)."""
    x1, f1 = fit(work, counts, start, free, lo, hi, windows, scale)
    s0 = np.asarray(start, np.float64).copy()
    s0[null_param] = 0.0
    free0 = np.asarray(free, bool).copy()
    free0[null_param] = False
    x0, f0 = fit(work, counts, s0, free0, lo, hi, windows, scale)
    return max(0.0, 2.0 * (f0 - f1)), x1, f1, x0, f0
