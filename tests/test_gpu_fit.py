"""Batched minimiser (gsn_minimize_batch_dev) for the profile likelihood of section 4.2.

Checked against a closed form (the discovery statistic of a counting experiment with known
background) and against the oracle's fits (scipy L-BFGS-B on the FP64 oracle NLL): minimum NLL
within 1e-6 (FP64 path; 1e-3 mixed), fitted rates within 1e-3 of their statistical error, and the
discovery statistic q0 = 2 (NLL with the signal rate fixed at 0 - free NLL) within 1e-3.
"""
import numpy as np
import pytest

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import gsn, inputs as I
from tests._helpers import oracle_pool_map

pytestmark = pytest.mark.gpu
FP64, MIXED = gsn.GSN_FP64, gsn.GSN_MIXED


def test_counting_experiment_discovery_statistic():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    b = 12.0
    w = I.template_like(n_bins=1, n_species=2)
    w.update(templates=[[np.ones(1)], [np.ones(1)]], exposure=np.array([1.0]), edges=w["edges"][:1],
             mask=np.ones((2, 1), np.uint8), win_lo=np.zeros(1, np.int32), win_hi=np.ones(1, np.int32),
             slot_map=w["slot_map"][:1])
    n_obs = np.array([3.0, 12.0, 20.0, 30.0, 55.0])
    T = n_obs.size
    ctx = gsn.context_from_workload(w, FP64, counts=n_obs[:1])
    counts = torch.tensor(n_obs[:, None], dtype=torch.float64, device=dev)
    wins = torch.tensor([[[0, 1]]] * T, dtype=torch.int32, device=dev)
    lo, hi = np.zeros(2), np.full(2, np.inf)
    x1 = torch.tensor([[5.0, b]] * T, dtype=torch.float64, device=dev)
    f1, _, s1 = ctx.minimize_batch_dev(x1, counts, wins, free=[1, 0], lo=lo, hi=hi, scale=[3.0, 1.0],
                                       gtol=1e-10, ftol=0.0)
    x0 = torch.tensor([[0.0, b]] * T, dtype=torch.float64, device=dev)
    f0, _, s0 = ctx.minimize_batch_dev(x0, counts, wins, free=[0, 0], lo=lo, hi=hi)
    torch.cuda.synchronize(dev)
    q0 = np.maximum(0.0, 2.0 * (f0.cpu().numpy() - f1.cpu().numpy()))
    ref = np.where(n_obs > b, 2.0 * (n_obs * np.log(n_obs / b) - (n_obs - b)), 0.0)
    assert np.all(s1.cpu().numpy() >= 0) and np.all(s0.cpu().numpy() == 0)
    assert np.max(np.abs(q0 - ref)) < 1e-6 * max(1.0, ref.max())
    assert np.max(np.abs(x1.cpu().numpy()[:, 0] - np.maximum(n_obs - b, 0.0))) < 1e-4


def _rate_fisher(w, species):
    """Fisher diagonal of the rate parameters of the given species at theta0 (d mu / d r = mu_s / r)."""
    fis = np.zeros(w["n_params"])
    for d in range(len(w["edges"])):
        per = O.expected_per_species(w, w["theta0"], d)
        m = per.sum(axis=1)
        for s in species:
            p = w["slot_map"][d, s]
            if p >= 0:
                fis[p] += float(np.sum((per[:, s] / w["theta0"][p]) ** 2 / m))
    return fis


@pytest.fixture(scope="module", params=["smeared", "templates"])
def fit_problem(request):
    """Well-conditioned rate fits: three rates of the smeared workload on two 120-bin datasets
    (beta, exponential, template; Fisher condition number ~60), or the six rates of a pure
    template fit on two 300-bin datasets (~200)."""
    if request.param == "smeared":
        w = I.with_templates(I.borexino_like(n_bins=120, n_fine=600), 2)
        names = ("r_beta3", "r_expo2", "r_tpl0")
        species = [s for s in range(w["spectra"].shape[0])
                   if w["slot_map"][0, s] >= 0 and w["param_names"][w["slot_map"][0, s]] in names]
        nb = 120
    else:
        w = I.template_like(n_bins=300, n_species=6)
        species = list(range(6))
        nb = 300
    mu = [O.expected_counts(w, w["theta0"], d) for d in range(2)]
    b = I.toy_batch(w, mu, n_toys=3, seed0=700, w_min=nb, w_max=nb)
    rates = np.unique(w["slot_map"][:, species][w["slot_map"][:, species] >= 0])
    free = np.zeros(w["n_params"], bool)
    free[rates] = True
    fis = _rate_fisher(w, species)
    scale = np.where(free & (fis > 0), 1.0 / np.sqrt(np.where(fis > 0, fis, 1.0)), 1.0)
    lo = np.where(free, 0.0, -np.inf)
    ref = [O.fit(w, b["counts"][t], w["theta0"], free, lo=lo, scale=scale) for t in range(3)]
    return w, b, free, scale, lo, ref


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_fits_match_oracle(fit_problem, precision):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w, b, free, scale, lo, ref = fit_problem
    ctx = gsn.context_from_workload(w, precision)
    x = torch.tensor(np.repeat(w["theta0"][None, :], 3, axis=0), device=dev)
    counts = torch.tensor(b["counts"], device=dev)
    wins = torch.tensor(b["windows"].astype(np.int32), device=dev)
    nll, evals, status = ctx.minimize_batch_dev(x, counts, wins, free=free, lo=lo, scale=scale, max_evals=400)
    torch.cuda.synchronize(dev)
    nll, x, st = nll.cpu().numpy(), x.cpu().numpy(), status.cpu().numpy()
    tol = 1e-6 if precision == FP64 else 1e-3
    for t in range(3):
        xr, fr = ref[t]
        assert st[t] in (0, 2), (t, st[t], evals.cpu().numpy())
        assert abs(nll[t] - fr) < tol * max(1.0, abs(fr)), (t, nll[t], fr)
        # the NLL at the returned point, evaluated by the oracle, is as low as the oracle's own fit
        assert O.nll(w, x[t], b["counts"][t]) <= fr + tol * max(1.0, abs(fr))
        if precision == FP64:
            assert np.max(np.abs(x[t][free] - xr[free]) / scale[free]) < 1e-3


def test_discovery_statistic_against_oracle(fit_problem):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w, b, free, scale, lo, ref = fit_problem
    # the free species with the fewest counts in the window plays the signal
    fr_idx = np.nonzero(free)[0]
    sig = int(fr_idx[np.argmin(scale[fr_idx] ** -2)])
    ctx = gsn.context_from_workload(w, FP64)
    counts = torch.tensor(b["counts"], device=dev)
    wins = torch.tensor(b["windows"].astype(np.int32), device=dev)
    x1 = torch.tensor(np.repeat(w["theta0"][None, :], 3, axis=0), device=dev)
    f1, _, _ = ctx.minimize_batch_dev(x1, counts, wins, free=free, lo=lo, scale=scale, max_evals=400)
    start0 = w["theta0"].copy()
    start0[sig] = 0.0
    free0 = free.copy()
    free0[sig] = False
    x0 = torch.tensor(np.repeat(start0[None, :], 3, axis=0), device=dev)
    f0, _, _ = ctx.minimize_batch_dev(x0, counts, wins, free=free0, lo=lo, scale=scale, max_evals=400)
    torch.cuda.synchronize(dev)
    q0 = np.maximum(0.0, 2.0 * (f0.cpu().numpy() - f1.cpu().numpy()))
    for t in range(2):
        qr = O.discovery_q0(w, b["counts"][t], w["theta0"], free, sig, lo=lo, scale=scale)[0]
        assert abs(q0[t] - qr) < 1e-3 * max(1.0, qr), (t, q0[t], qr)


# ------------------- toys fitted in windows of their own (uneven fit ranges) --------
def _window_factors_oracle(w, params, windows, max_factor):
    """sqrt(N_whole / N_window) per rate parameter from the oracle's expected counts per species."""
    S = w["spectra"].shape[0]
    sw, sf = np.zeros(w["n_params"]), np.zeros(w["n_params"])
    for d, (lo, hi) in enumerate(windows):
        per = O.expected_per_species(w, params, d)
        for s in range(S):
            p = w["slot_map"][d, s]
            if p >= 0:
                sw[p] += per[lo:hi, s].sum()
                sf[p] += per[:, s].sum()
    f = np.ones(w["n_params"])
    ok = sf > 0
    f[ok] = np.sqrt(sf[ok] / np.maximum(sw[ok], sf[ok] / max_factor ** 2))
    return np.clip(f, 1.0, max_factor), sw, sf


def test_window_scales_against_oracle_counts():
    """Per-toy scales of gsn_window_scales_dev: factor 1 on whole histograms, the oracle's
    sqrt(N_whole / N_window) for rates (the library's counts use a Gaussian response, so within 10%
    where a tenth or more of the species lies inside the window), max_factor for species outside
    it, and untouched non-rate scales."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w = I.with_templates(I.borexino_like(n_bins=240, n_fine=2400), 1)
    P, S = w["n_params"], w["spectra"].shape[0]
    th = w["theta0"]
    wins = np.array([[[0, 240], [0, 240]], [[60, 180], [60, 180]], [[0, 40], [0, 40]]], np.int32)
    T = len(wins)
    ctx = gsn.context_from_workload(w, FP64)
    base = np.linspace(0.5, 2.0, P)
    params = torch.tensor(np.repeat(th[None, :], T, axis=0), device=dev)
    out = ctx.window_scales_dev(params, torch.tensor(wins, device=dev), scale=base, max_factor=50.0)
    torch.cuda.synchronize(dev)
    out = out.cpu().numpy() / base[None, :]
    rates = np.unique(w["slot_map"][:, :S][w["slot_map"][:, :S] >= 0])
    other = np.setdiff1d(np.arange(P), rates)
    assert np.all(out[:, other] == 1.0)
    assert np.max(np.abs(out[0] - 1.0)) < 1e-6
    for t in (1, 2):
        ref, sw, sf = _window_factors_oracle(w, th, wins[t], 50.0)
        inside = rates[sw[rates] >= 0.1 * sf[rates]]
        assert inside.size >= 3
        assert np.max(np.abs(out[t, inside] / ref[inside] - 1.0)) < 0.1, (t, out[t, inside], ref[inside])
        outside = rates[sw[rates] <= 1e-9 * sf[rates]]
        assert np.all(out[t, outside] == 50.0), (t, out[t, outside])


def _ragged_fit_setup(w, T, seed, w_min, w_max, ctx64):
    """All rates free (>= 0) on toys with windows of their own; scales 1/sqrt(Fisher) of the rates over
    the whole histograms at theta0 (expected counts per species from the FP64 context)."""
    S, P, D = w["spectra"].shape[0], w["n_params"], len(w["edges"])
    mu0 = [ctx64.expected(w["theta0"], d).sum(axis=1) for d in range(D)]
    b = I.toy_batch(w, mu0, n_toys=T, seed0=seed, w_min=w_min, w_max=w_max)
    rates = np.unique(w["slot_map"][:, :S][w["slot_map"][:, :S] >= 0])
    free = np.zeros(P, bool)
    free[rates] = True
    fis = np.zeros(P)
    for d in range(D):
        per = ctx64.expected(w["theta0"], d)
        m = per.sum(axis=1)
        ok = m > 0
        for s in range(S):
            p = w["slot_map"][d, s]
            if p >= 0:
                fis[p] += float(np.sum((per[ok, s] / w["theta0"][p]) ** 2 / m[ok]))
    scale = np.where(free & (fis > 0), 1.0 / np.sqrt(np.where(fis > 0, fis, 1.0)), 1.0)
    lo = np.where(free, 0.0, -np.inf)
    return b, free, scale, lo


def test_ragged_window_rate_fits_converge_on_the_toy_workload():
    """The batched pseudo-experiment workload (two datasets on a 1200-bin domain, 16 species on 20000
    fine points, windows of 600..1200 bins) with all 16 rates free (>= 0), fitted by the batched
    Newton rate fit in mixed precision: at least 99% of the fits converge (status 0); the reported
    NLL is the batched path's NLL at the minimum; moving any free rate by a tenth of its statistical
    scale (up, and down where the bound allows) does not lower that NLL; and the minima are no
    higher than those of the window-scaled L-BFGS minimiser on the same toys."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w = I.borexino_like(n_bins=1200)
    ctx64 = gsn.context_from_workload(w, FP64)
    T = 256
    b, free, scale, lo = _ragged_fit_setup(w, T, 5000, 600, 1200, ctx64)
    ctx = gsn.context_from_workload(w, MIXED)
    counts = torch.tensor(b["counts"], device=dev)
    wins = torch.tensor(b["windows"].astype(np.int32), device=dev)
    start = torch.tensor(np.repeat(w["theta0"][None, :], T, axis=0), device=dev)
    x = start.clone()
    nll, iters, status = ctx.fit_rates_batch_dev(x, counts, wins, free=free, lo=lo)
    torch.cuda.synchronize(dev)
    st, nll, xm = status.cpu().numpy(), nll.cpu().numpy(), x.cpu().numpy()
    assert np.mean(st == 0) >= 0.99, (np.unique(st, return_counts=True), iters.cpu().numpy().max())
    rc, n2, _ = ctx.eval_grad_batch(xm, b["counts"], b["windows"])
    assert rc == 0
    ok = st == 0
    bad = np.nonzero(~ok | (np.abs(n2 - nll) >= 1e-3))[0]
    assert np.max(np.abs(n2 - nll)[ok]) < 1e-3, [(int(t), int(st[t]), float(nll[t]), float(n2[t])) for t in bad[:8]]
    for i in np.nonzero(free)[0]:
        for sgn in (1.0, -1.0):
            xp = xm.copy()
            xp[:, i] = np.maximum(lo[i], xm[:, i] + sgn * 0.1 * scale[i])
            rc, n3, _ = ctx.eval_grad_batch(xp, b["counts"], b["windows"], want_grad=False)
            assert rc == 0
            assert np.min((n3 - n2)[ok]) > -1e-3, (w["param_names"][i], sgn, np.min((n3 - n2)[ok]))
    # the window-scaled L-BFGS on the first 64 toys reaches no lower minimum
    sub = slice(0, 64)
    x1 = start[sub].clone()
    sc = ctx.window_scales_dev(x1, wins[sub], scale=scale)
    f1, _, s1 = ctx.minimize_batch_dev(x1, counts[sub], wins[sub], free=free, lo=lo, max_evals=300, scale_dev=sc,
                                       edm=1e-6)
    torch.cuda.synchronize(dev)
    f1 = f1.cpu().numpy()
    assert np.all(nll[sub][ok[sub]] <= f1[ok[sub]] + 1e-3), np.max((nll[sub] - f1)[ok[sub]])


@pytest.fixture(scope="module")
def ragged_problem():
    """A reduced ragged workload (two 160-bin datasets, 1200 fine points, windows of 80..160 bins,
    all 16 rates free) and the oracle's L-BFGS-B fits of two toys."""
    w = I.borexino_like(n_bins=160, n_fine=1200)
    ctx64 = gsn.context_from_workload(w, FP64)
    T = 2
    b, free, scale, lo = _ragged_fit_setup(w, T, 5100, 80, 160, ctx64)
    ref = oracle_pool_map([("fit", w, (b["counts"][t], w["theta0"], free, lo, b["windows"][t], scale))
                           for t in range(T)])
    return w, T, b, free, scale, lo, ref


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_ragged_window_rate_fits_match_oracle(ragged_problem, precision):
    """Minima of the batched Newton rate fits against the oracle's L-BFGS-B fits: NLL within 1e-6
    relative on the FP64 path, 1e-3 mixed; at the FP64 minimum the oracle's own gradient is below
    1e-3 of the statistical spread sqrt(F_ii) of every free rate (F over the toy's window) that is
    not held at 0."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    w, T, b, free, scale, lo, ref = ragged_problem
    ctx = gsn.context_from_workload(w, precision)
    counts = torch.tensor(b["counts"], device=dev)
    wins = torch.tensor(b["windows"].astype(np.int32), device=dev)
    x = torch.tensor(np.repeat(w["theta0"][None, :], T, axis=0), device=dev)
    nll, iters, status = ctx.fit_rates_batch_dev(x, counts, wins, free=free, lo=lo)
    torch.cuda.synchronize(dev)
    nll, x, st = nll.cpu().numpy(), x.cpu().numpy(), status.cpu().numpy()
    tol = 1e-6 if precision == FP64 else 1e-3
    for t in range(T):
        xr, fr = ref[t]
        assert st[t] == 0, (t, st[t], iters.cpu().numpy())
        assert abs(nll[t] - fr) < tol * max(1.0, abs(fr)), (t, nll[t], fr)
        if precision == FP64:
            g = O.nll_grad(w, x[t], b["counts"][t], b["windows"][t])
            F = O.fisher_diagonal(w, x[t], b["windows"][t])
            # rates without information in the window (F ~ 0) have no statistical scale to test against
            moving = free & ~((x[t] <= lo) & (g > 0)) & (F > 1e-12 * F.max())
            assert np.max(np.abs(g[moving]) / np.sqrt(F[moving])) < 1e-3, (t, g[moving] / np.sqrt(F[moving]))


def test_rate_fit_rejects_free_response_parameters():
    w = I.borexino_like(n_bins=100, n_fine=800)
    ctx = gsn.context_from_workload(w, FP64)
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    free = np.zeros(w["n_params"], bool)
    free[w["param_names"].index("LY")] = True
    x = torch.tensor(w["theta0"][None, :], device=dev)
    c = torch.zeros(1, ctx.n_counts(), dtype=torch.float64, device=dev)
    wins = torch.tensor([[[0, 100], [0, 100]]], dtype=torch.int32, device=dev)
    with pytest.raises(gsn.GsnError):
        ctx.fit_rates_batch_dev(x, c, wins, free=free)
