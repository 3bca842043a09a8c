"""Seeded synthetic workloads for the binned spectral-fit likelihood.

This module only *draws inputs*: fine true-energy spectra shaped like the
species of a liquid-scintillator solar-neutrino fit (section 4.3 of the paper:
beta decays, mono-energetic lines, Compton-like shoulders, exponentials, a flat
pile-up-like term, an alpha peak and a positron emitter), bin edges, exposures,
parameter points, fit windows and Poisson counts drawn from a caller-supplied
mean.  It holds none of the likelihood method's arithmetic (no quenching, no
resolution, no convolution, no likelihood): the expected counts that the
Poisson draws need are passed in by the caller.

Both the oracle tests and the GPU path consume the dictionaries built here, so
the integer codes below are interface values, not implementation details.

Workload dictionary keys
------------------------
fine_centres (K,)        ascending fine true-energy centres [MeV]
spectra      (S, K)      unnormalised species shapes at the centres
kind         (S,)        0 = Ana, 1 = AnaShift, 2 = AnaPeak (section 4.3), 3 = Monte Carlo
                         template (section 3.2: a visible-bin histogram per dataset)
shift        (S,)        true-energy shift of AnaShift species [MeV]
mask         (S, D)      1 where species s contributes to dataset d
edges        [D] arrays  visible-energy bin edges [p.e.], ascending
exposure     (D,)        exposure of each dataset (section 4.1)
win_lo/win_hi (D,)       default fit window [lo, hi) in bins
resolution   int         0 = Gaussian, 1 = gamma (generalized gamma of power 1),
                         2 = generalized gamma with a free power p
birks_s0/s1  float       stopping-power model S(E) = s0 + s1/E [MeV/cm, MeV^2/cm]
n_params     int         number of global fit parameters
slot_map     (D, 3S+6)   global parameter index of each per-dataset slot:
                         [rate_0..rate_{S-1}, LY, kB, a, b, c, m_0, w_0, ..., m_{S-1}, w_{S-1}, p]
                         (p: the power of the generalized-gamma response, resolution 2 only)
                         (-1 = unused: peak slots of non-peak species, rates of
                         species absent from the dataset)
pull_param/pull_centre/pull_width   Gaussian pull terms (section 4.1, Eq. LL)
theta0       (P,)        generating parameter point
param_names  list[str]
resp_scale   (D, 5)      optional fixed multipliers of the response slots (LY, kB, a, b, c)
                         of each dataset (section 2.4 slices; default 1)
rate_factor  (D, S)      optional fixed fraction of each species' rate in each dataset
                         (section 2.4 slices; default 1)
templates    [S][D]      optional visible-bin histograms of template species (None elsewhere)
secondary    [D]         optional secondary observable per dataset (section 2.4 multivariate fit):
                         None or dict(slice_start (Q+1,) energy-bin boundaries of the slices,
                         shapes (S, Q, M) per-species distributions of the second observable in
                         every slice (normalised by the consumer), counts (Q, M) observed)
"""
from __future__ import annotations

import numpy as np

KIND_ANA, KIND_ANA_SHIFT, KIND_ANA_PEAK, KIND_MC_TEMPLATE = 0, 1, 2, 3
RES_GAUSS, RES_GAMMA, RES_GGAMMA = 0, 1, 2

# Stopping-power model constants used by every workload (MeV/cm and MeV^2/cm):
# roughly electron dE/dx in a ~0.88 g/cm^3 organic scintillator.
BIRKS_S0 = 1.55
BIRKS_S1 = 0.155


def n_slots(n_species: int) -> int:
    """Per-dataset slot count: S rates, 5 response parameters, 2 peak slots per species, the power."""
    return 3 * n_species + 6


def slot_power(n_species: int) -> int:
    return 3 * n_species + 5


def slot_rate(s: int) -> int:
    return s


def slot_response(n_species: int, which: str) -> int:
    return n_species + ("LY", "kB", "a", "b", "c").index(which)


def slot_peak(n_species: int, s: int, which: str) -> int:
    return n_species + 5 + 2 * s + (0 if which == "m" else 1)


# ----------------------------------------------------------------- shapes ----
def fine_grid(n_fine: int, e_max: float) -> np.ndarray:
    """Centres (k + 1/2) * dE of a uniform fine grid on [0, e_max) MeV."""
    return (np.arange(n_fine, dtype=np.float64) + 0.5) * (e_max / n_fine)


def shape_beta(E, Q):
    """Allowed-beta-like shape E^2 (Q - E)^2 below the endpoint Q."""
    return np.where(E < Q, E * E * (Q - E) ** 2, 0.0)


def shape_line(E, E0):
    """Mono-energetic line: 1 at the fine centre nearest E0 (ties to the lower index)."""
    out = np.zeros_like(E)
    out[int(np.argmin(np.abs(E - E0)))] = 1.0
    return out


def shape_expo(E, tau):
    return np.exp(-E / tau)


def shape_flat(E):
    return np.ones_like(E)


def shape_shoulder(E, edge):
    """Flat up to a Compton-like edge, zero above it."""
    return np.where(E < edge, 1.0, 0.0)


def unit_edges(n_bins: int) -> np.ndarray:
    """Bin edges 0, 1, ..., n_bins p.e. (1 p.e. wide bins)."""
    return np.arange(n_bins + 1, dtype=np.float64)


# -------------------------------------------------------------- workloads ----
def _slot_map_shared(n_species, n_datasets, n_rates_offset=0, peaks=()):
    """Every dataset shares every parameter (full synchronisation, section 2.2).

    Global parameter order: rates 0..S-1, LY, kB, a, b, c, then (m, w) per peak.
    """
    ns = n_slots(n_species)
    sm = -np.ones((n_datasets, ns), dtype=np.int32)
    for d in range(n_datasets):
        for s in range(n_species):
            sm[d, slot_rate(s)] = s
        for i, w in enumerate(("LY", "kB", "a", "b", "c")):
            sm[d, slot_response(n_species, w)] = n_species + i
        for i, s in enumerate(peaks):
            sm[d, slot_peak(n_species, s, "m")] = n_species + 5 + 2 * i
            sm[d, slot_peak(n_species, s, "w")] = n_species + 5 + 2 * i + 1
    return sm


def single_gauss(seed: int = 1, n_bins: int = 900, n_fine: int = 2000, e_max: float = 2.0) -> dict:
    """Plain single-dataset workload: 8 species on a 1 keV grid, Gaussian resolution.

    3 betas (Q ~ U[0.5, 2] MeV), 2 lines (E0 ~ U[0.2, 1.5]), 2 exponentials
    (tau ~ U[0.1, 1]), 1 flat; LY = 500 p.e./MeV, kB = 0.011 cm/MeV,
    sigma^2 = a + b mu with a = 4, b = 1 (c = 0); rates log-uniform in [10, 1e5].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    E = fine_grid(n_fine, e_max)
    rows, names = [], []
    for i in range(3):
        rows.append(shape_beta(E, rng.uniform(0.5, 2.0)))
        names.append(f"beta{i}")
    for i in range(2):
        rows.append(shape_line(E, rng.uniform(0.2, 1.5)))
        names.append(f"line{i}")
    for i in range(2):
        rows.append(shape_expo(E, rng.uniform(0.1, 1.0)))
        names.append(f"expo{i}")
    rows.append(shape_flat(E))
    names.append("flat")
    S = len(rows)
    rates = 10.0 ** rng.uniform(1.0, 5.0, size=S)
    theta0 = np.concatenate([rates, [500.0, 0.011, 4.0, 1.0, 0.0]])
    return dict(
        name=f"single_gauss_{n_bins}x{n_fine}",
        fine_centres=E, spectra=np.array(rows), kind=np.zeros(S, np.int32),
        shift=np.zeros(S), mask=np.ones((S, 1), np.uint8),
        edges=[unit_edges(n_bins)], exposure=np.array([1.0]),
        win_lo=np.array([0], np.int32), win_hi=np.array([n_bins], np.int32),
        resolution=RES_GAUSS, birks_s0=BIRKS_S0, birks_s1=BIRKS_S1,
        n_params=S + 5, slot_map=_slot_map_shared(S, 1),
        pull_param=np.zeros(0, np.int32), pull_centre=np.zeros(0), pull_width=np.zeros(0),
        theta0=theta0, param_names=[f"r_{n}" for n in names] + ["LY", "kB", "a", "b", "c"],
    )


def borexino_like(seed: int = 2, n_bins: int = 1000, n_fine: int = 20000, e_max: float = 2.0) -> dict:
    """Two-dataset (tagged / subtracted) workload with generalized-gamma resolution.

    16 species on a 0.1 keV grid: 6 betas, 2 lines, 2 shoulders, 3
    exponentials, 1 flat, 1 alpha AnaPeak (m ~ 200 p.e., w ~ 10 p.e.), 1
    positron AnaShift (Q = 0.96 MeV shifted by 1.022 MeV, tagged set only).
    Exposures 1.0 and 0.6, resolution sigma^2 = a + b mu + c mu^2 with
    a = 10, b = 1.1, c = 2e-4.  23 parameters: 16 rates, LY, kB, a, b, c, m, w.
    Pulls on kB (0.011 +- 0.002) and on the peak position (200 +- 2 p.e.).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    E = fine_grid(n_fine, e_max)
    rows, names, kinds, shifts = [], [], [], []

    def add(row, name, kind=KIND_ANA, shift=0.0):
        rows.append(row); names.append(name); kinds.append(kind); shifts.append(shift)

    for i in range(6):
        add(shape_beta(E, rng.uniform(0.5, 2.0)), f"beta{i}")
    for i in range(2):
        add(shape_line(E, rng.uniform(0.2, 1.5)), f"line{i}")
    for i in range(2):
        add(shape_shoulder(E, rng.uniform(0.3, 1.2)), f"shoulder{i}")
    for i in range(3):
        add(shape_expo(E, rng.uniform(0.1, 1.0)), f"expo{i}")
    add(shape_flat(E), "flat")
    add(np.zeros_like(E), "alpha", KIND_ANA_PEAK)
    add(shape_beta(E, 0.96), "positron", KIND_ANA_SHIFT, 1.022)
    S = len(rows)
    D = 2
    mask = np.ones((S, D), np.uint8)
    mask[S - 1, 1] = 0  # the positron emitter is present only in the tagged set
    peak_species = (S - 2,)
    rates = 10.0 ** rng.uniform(1.0, 5.0, size=S)
    m0, w0 = 200.0 + rng.uniform(-5, 5), 10.0 + rng.uniform(-1, 1)
    theta0 = np.concatenate([rates, [500.0, 0.011, 10.0, 1.1, 2e-4, m0, w0]])
    P = S + 7
    return dict(
        name=f"borexino_like_2x{n_bins}x{n_fine}",
        fine_centres=E, spectra=np.array(rows), kind=np.array(kinds, np.int32),
        shift=np.array(shifts), mask=mask,
        edges=[unit_edges(n_bins), unit_edges(n_bins)], exposure=np.array([1.0, 0.6]),
        win_lo=np.zeros(D, np.int32), win_hi=np.full(D, n_bins, np.int32),
        resolution=RES_GAMMA, birks_s0=BIRKS_S0, birks_s1=BIRKS_S1,
        n_params=P, slot_map=_slot_map_shared(S, D, peaks=peak_species),
        pull_param=np.array([S + 1, S + 5], np.int32),
        pull_centre=np.array([0.011, m0]), pull_width=np.array([0.002, 2.0]),
        theta0=theta0,
        param_names=[f"r_{n}" for n in names] + ["LY", "kB", "a", "b", "c", "m_alpha", "w_alpha"],
    )


def multivariate_like(seed: int = 5, n_datasets: int = 4, n_slices: int = 64, n_bins: int = 1000,
                      n_fine: int = 50000, n_species: int = 32, e_max: float = 2.0) -> dict:
    """Two-dimensional workload: energy x a second observable (radial / pulse-shape slices).

    Each of n_datasets histograms is split into n_slices slices along the second
    observable (section 2.4); slice q of dataset d is dataset index d * n_slices + q,
    with n_bins energy bins of 1 p.e.  Every species has a seeded slice-fraction
    template f_s(q) (positive, summing to 1 over the slices: a random walk in log
    space, so neighbouring slices are alike), and every slice fixed multipliers of
    the light yield (lambda_q, U[0.95, 1.05]) and of the resolution constant term
    (alpha_q, U[0.8, 1.2]); the free parameters are global.  n_species species on
    a 2 MeV grid of n_fine points (betas, lines, shoulders, exponentials, flats in
    turn), gamma resolution a = 10, b = 1.1, c = 2e-4, exposures 1, 0.8, 0.6, 0.4, ...
    Parameters: n_species rates, LY, kB, a, b, c; a pull on kB.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    E = fine_grid(n_fine, e_max)
    rows, names = [], []
    makers = (lambda: shape_beta(E, rng.uniform(0.3, 2.0)), lambda: shape_line(E, rng.uniform(0.2, 1.6)),
              lambda: shape_shoulder(E, rng.uniform(0.3, 1.4)), lambda: shape_expo(E, rng.uniform(0.1, 1.0)),
              lambda: shape_flat(E))
    tags = ("beta", "line", "shoulder", "expo", "flat")
    for i in range(n_species):
        rows.append(makers[i % 5]())
        names.append(f"{tags[i % 5]}{i // 5}")
    S = n_species
    D = n_datasets * n_slices
    frac = np.empty((S, n_slices))
    for s_ in range(S):
        walk = np.cumsum(rng.normal(0.0, 0.15, size=n_slices))
        f = np.exp(walk - walk.max())
        frac[s_] = f / f.sum()
    lam = rng.uniform(0.95, 1.05, size=n_slices)
    alp = rng.uniform(0.8, 1.2, size=n_slices)
    resp_scale = np.ones((D, 5))
    rate_factor = np.empty((D, S))
    for d in range(n_datasets):
        for q in range(n_slices):
            resp_scale[d * n_slices + q, 0] = lam[q]
            resp_scale[d * n_slices + q, 2] = alp[q]
            rate_factor[d * n_slices + q] = frac[:, q]
    exposure = np.repeat(1.0 - 0.2 * (np.arange(n_datasets) % 5), n_slices)
    rates = 10.0 ** rng.uniform(3.0, 6.0, size=S)
    theta0 = np.concatenate([rates, [500.0, 0.011, 10.0, 1.1, 2e-4]])
    return dict(
        name=f"multivariate_like_{n_datasets}x{n_slices}x{n_bins}x{n_fine}",
        fine_centres=E, spectra=np.array(rows), kind=np.zeros(S, np.int32), shift=np.zeros(S),
        mask=np.ones((S, D), np.uint8), edges=[unit_edges(n_bins) for _ in range(D)], exposure=exposure,
        win_lo=np.zeros(D, np.int32), win_hi=np.full(D, n_bins, np.int32),
        resolution=RES_GAMMA, birks_s0=BIRKS_S0, birks_s1=BIRKS_S1,
        n_params=S + 5, slot_map=_slot_map_shared(S, D),
        pull_param=np.array([S + 1], np.int32), pull_centre=np.array([0.011]), pull_width=np.array([0.002]),
        theta0=theta0, param_names=[f"r_{n}" for n in names] + ["LY", "kB", "a", "b", "c"],
        resp_scale=resp_scale, rate_factor=rate_factor, n_slices=n_slices,
    )


def _visible_shapes(rng, x, n):
    """n smooth positive shapes over visible-bin centres x [p.e.]: exponentials, bumps, betas, flat
    (scales relative to the range: decay lengths 5-30%, bump centres 10-90%, widths 2-6%)."""
    out = []
    xm = max(float(x[-1]), 1.0)
    for i in range(n):
        kind = i % 4
        if kind == 0:
            h = np.exp(-x / (rng.uniform(0.05, 0.3) * xm))
        elif kind == 1:
            h = np.exp(-0.5 * ((x - rng.uniform(0.1, 0.9) * xm) / (rng.uniform(0.02, 0.06) * xm)) ** 2)
        elif kind == 2:
            q = rng.uniform(0.3, 1.0) * xm
            h = np.where(x < q, x * x * (q - x) ** 2, 0.0)
        else:
            h = np.ones_like(x)
        out.append(h / h.max())
    return out


def _template_set(rng, edges_per_dataset, base_shapes):
    """Per-dataset Monte Carlo-like templates of each base shape: a 2% tilt between datasets and 1%
    seeded multiplicative noise (finite simulation statistics)."""
    tpl = []
    for h0 in base_shapes:
        row = []
        for d, e in enumerate(edges_per_dataset):
            x = 0.5 * (np.asarray(e[:-1]) + np.asarray(e[1:]))
            h = h0 * (1.0 + 0.02 * d * (x / x[-1] - 0.5)) * (1.0 + 0.01 * rng.standard_normal(x.size))
            row.append(np.clip(h, 0.0, None))
        tpl.append(row)
    return tpl


def template_like(seed: int = 8, n_bins: int = 1000, n_species: int = 16) -> dict:
    """Monte Carlo template fit (section 3.2): every species is a visible-energy histogram.

    Two datasets (exposures 1.0 and 0.6) of n_bins bins of 1 p.e.; n_species seeded template
    shapes (exponentials, bumps, betas, flat) with per-dataset variations; rates log-uniform in
    [1e3, 1e5].  No response parameters: the slot map leaves LY, kB, a, b, c unused.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    D, S = 2, n_species
    edges = [unit_edges(n_bins) for _ in range(D)]
    x = unit_edges(n_bins)
    shapes = _visible_shapes(rng, 0.5 * (x[:-1] + x[1:]), S)
    sm = -np.ones((D, n_slots(S)), dtype=np.int32)
    for d in range(D):
        sm[d, :S] = np.arange(S)
    rates = 10.0 ** rng.uniform(3.0, 5.0, size=S)
    return dict(
        name=f"template_like_2x{n_bins}x{S}", fine_centres=np.array([0.5e-3, 1.5e-3]), spectra=np.zeros((S, 2)),
        kind=np.full(S, KIND_MC_TEMPLATE, np.int32), shift=np.zeros(S), mask=np.ones((S, D), np.uint8),
        edges=edges, exposure=np.array([1.0, 0.6]), win_lo=np.zeros(D, np.int32),
        win_hi=np.full(D, n_bins, np.int32), resolution=RES_GAMMA, birks_s0=BIRKS_S0, birks_s1=BIRKS_S1,
        n_params=S, slot_map=sm, pull_param=np.zeros(0, np.int32), pull_centre=np.zeros(0),
        pull_width=np.zeros(0), theta0=rates, param_names=[f"r_tpl{i}" for i in range(S)],
        templates=_template_set(rng, edges, shapes),
    )


def with_templates(work: dict, n_templates: int, seed: int = 9) -> dict:
    """A workload plus n_templates Monte Carlo template species (new rate parameters appended)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S0, D, P0 = work["spectra"].shape[0], len(work["edges"]), int(work["n_params"])
    S = S0 + n_templates
    x = np.asarray(work["edges"][0])
    shapes = _visible_shapes(rng, 0.5 * (x[:-1] + x[1:]), n_templates)
    sm = -np.ones((D, n_slots(S)), dtype=np.int32)
    old = np.asarray(work["slot_map"])
    for d in range(D):
        sm[d, :S0] = old[d, :S0]
        sm[d, S:S + 5] = old[d, S0:S0 + 5]
        sm[d, S + 5:S + 5 + 2 * S0] = old[d, S0 + 5:3 * S0 + 5]
        sm[d, slot_power(S)] = old[d, slot_power(S0)]
        sm[d, S0:S] = P0 + np.arange(n_templates)
    tpl = [None] * S0 + _template_set(rng, work["edges"], shapes)
    tpl = [t if t is not None else [None] * D for t in tpl]
    out = dict(work)
    out.update(
        name=work["name"] + f"+{n_templates}tpl",
        spectra=np.vstack([work["spectra"], np.zeros((n_templates, work["spectra"].shape[1]))]),
        kind=np.concatenate([work["kind"], np.full(n_templates, KIND_MC_TEMPLATE, np.int32)]),
        shift=np.concatenate([work["shift"], np.zeros(n_templates)]),
        mask=np.vstack([work["mask"], np.ones((n_templates, D), np.uint8)]),
        n_params=P0 + n_templates, slot_map=sm, templates=tpl,
        theta0=np.concatenate([work["theta0"], 10.0 ** rng.uniform(2.0, 4.0, size=n_templates)]),
        param_names=list(work["param_names"]) + [f"r_tpl{i}" for i in range(n_templates)],
    )
    if work.get("rate_factor") is not None:
        out["rate_factor"] = np.hstack([work["rate_factor"], np.ones((D, n_templates))])
    return out


def perturbed_points(theta0: np.ndarray, n: int, seed0: int, rel: float = 0.01) -> np.ndarray:
    """Parameter points theta0 * (1 + rel * N(0,1)), point i drawn with seed seed0 + i.

    Parameters whose generating value is 0 are perturbed additively by rel * 1e-4.
    """
    out = np.empty((n, theta0.size))
    for i in range(n):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        z = rng.standard_normal(theta0.size)
        out[i] = np.where(theta0 != 0.0, theta0 * (1.0 + rel * z), rel * 1e-4 * np.abs(z))
    return out


def poisson_counts(mu: np.ndarray, seed: int) -> np.ndarray:
    """Poisson draws (as float64) from a caller-supplied mean."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.poisson(np.clip(mu, 0.0, None)).astype(np.float64)


def toy_windows(n_toys: int, n_bins: int, w_min: int, w_max: int, seed: int) -> np.ndarray:
    """Per-toy fit windows [lo, hi): width ~ U{w_min..w_max}, start ~ U{0..n_bins-width}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W = rng.integers(w_min, w_max + 1, size=n_toys)
    lo = np.array([rng.integers(0, n_bins - w + 1) for w in W])
    return np.stack([lo, lo + W], axis=1).astype(np.int32)


def toy_batch(work: dict, mu0: list, n_toys: int, seed0: int = 1000,
              w_min: int = 600, w_max: int = 1200, rel: float = 0.01, mu_sec=None) -> dict:
    """Batched pseudo-experiments of a workload.

    Toy t: counts ~ Poisson(mu0) drawn with seed seed0 + t (all datasets
    concatenated), its own parameter vector theta0 * (1 + rel N(0,1)) (seed
    seed0 + n_toys + t) and one fit window shared by its datasets, width
    U{w_min..w_max} bins.  ``mu0`` holds the expected counts of each dataset at
    theta0, supplied by the caller.
    """
    D = len(work["edges"])
    nb = [len(e) - 1 for e in work["edges"]]
    total = int(sum(nb))
    mu_cat = np.concatenate([np.asarray(m, np.float64) for m in mu0])
    assert mu_cat.size == total
    if mu_sec is not None:  # secondary-observable expectations (datasets, slices, m), appended
        mu_cat = np.concatenate([mu_cat, np.asarray(mu_sec, np.float64).ravel()])
    counts = np.empty((n_toys, mu_cat.size))
    for t in range(n_toys):
        counts[t] = poisson_counts(mu_cat, seed0 + t)
    params = perturbed_points(work["theta0"], n_toys, seed0 + n_toys, rel)
    win = toy_windows(n_toys, min(nb), min(w_min, min(nb)), min(w_max, min(nb)), seed0 + 2 * n_toys)
    windows = np.repeat(win[:, None, :], D, axis=1)  # (T, D, 2)
    return dict(counts=counts, params=params, windows=windows)


def with_power(work: dict, p: float = 1.3, pull_width: float = 0.0) -> dict:
    """The workload with the generalized-gamma response of power p (resolution 2): a new global
    parameter "p" (appended) fills every dataset's power slot; pull_width > 0 adds a pull to p."""
    S, D, P0 = work["spectra"].shape[0], len(work["edges"]), int(work["n_params"])
    sm = np.array(work["slot_map"], dtype=np.int32, copy=True)
    sm[:, slot_power(S)] = P0
    out = dict(work)
    out.update(name=work.get("name", "workload") + f"+ggamma{p:g}", resolution=RES_GGAMMA, slot_map=sm,
               n_params=P0 + 1, theta0=np.concatenate([work["theta0"], [p]]),
               param_names=list(work.get("param_names", [f"p{i}" for i in range(P0)])) + ["p"])
    if pull_width > 0:
        out.update(pull_param=np.concatenate([work["pull_param"], [P0]]).astype(np.int32),
                   pull_centre=np.concatenate([work["pull_centre"], [p]]),
                   pull_width=np.concatenate([work["pull_width"], [pull_width]]))
    return out


def with_secondary(work: dict, n_slices: int = 8, n_sec: int = 16, seed: int = 10, datasets=None) -> dict:
    """A secondary observable for the given datasets (all by default; section 2.4 multivariate fit):
    the energy histogram split into n_slices contiguous slices of equal width, and per species a
    smooth distribution of a pulse-shape-like variable in n_sec bins: a Gaussian bump (centre
    U[0.2, 0.8] of the range, width U[0.08, 0.25]) drifting by up to 5% of the range across the
    slices, on a 2% flat floor.  Observed counts are zeros (tests draw them from an expectation)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    D, S = len(work["edges"]), work["spectra"].shape[0]
    m = (np.arange(n_sec) + 0.5) / n_sec
    sec = []
    for d in range(D):
        if datasets is not None and d not in datasets:
            sec.append(None)
            continue
        J = len(work["edges"][d]) - 1
        start = np.round(np.linspace(0, J, n_slices + 1)).astype(np.int64)
        c = rng.uniform(0.2, 0.8, S)
        wd = rng.uniform(0.08, 0.25, S)
        drift = rng.uniform(-0.05, 0.05, S)
        shapes = np.empty((S, n_slices, n_sec))
        for q in range(n_slices):
            cq = c + drift * (q / max(n_slices - 1, 1) - 0.5)
            shapes[:, q, :] = 0.02 + np.exp(-0.5 * ((m[None, :] - cq[:, None]) / wd[:, None]) ** 2)
        sec.append(dict(slice_start=start, shapes=shapes, counts=np.zeros((n_slices, n_sec))))
    out = dict(work)
    out.update(name=work.get("name", "workload") + f"+sec{n_slices}x{n_sec}", secondary=sec)
    return out
