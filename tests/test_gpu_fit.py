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
