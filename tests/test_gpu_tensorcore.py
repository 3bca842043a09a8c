"""The per-species contraction on tcgen05 tensor cores (mixed precision) against the oracle.

gsn_expected and the response cache of gsn_eval run the contraction
M[s][j] = sum_k R_jk S'_sk as split-TF32 products (hi x hi + hi x lo + lo x hi)
with FP32 accumulation in tensor memory, read back every 32 columns into
compensated FP32 sums.  Checked per element against the FP64 oracle: 2e-5
relative where the expected count exceeds 1e-6 of the dataset maximum.  The
accumulation in tensor memory does not round to nearest, so a separate test
bounds the coherent part of the error: the total of every species over the
histogram, against the FP64 GPU path, within 1.5e-7 relative.
"""
import numpy as np
import pytest

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import gsn, inputs as I
from tests._helpers import poisson_data

pytestmark = pytest.mark.gpu


def _workload_20_species(resolution):
    """20 species (two 16-wide MMA chunks, the second padded) on 333 bins (not a multiple of 128)."""
    w = I.borexino_like(n_bins=333, n_fine=4000) if resolution == gsn.GSN_RES_GAMMA else I.single_gauss(n_bins=333, n_fine=1500)
    S = w["spectra"].shape[0]
    rng = np.random.Generator(np.random.PCG64(77))
    extra = [I.shape_beta(w["fine_centres"], q) for q in rng.uniform(0.3, 1.9, 20 - S)]
    D = len(w["edges"])
    spectra = np.vstack([w["spectra"], extra])
    kind = np.concatenate([w["kind"], np.zeros(20 - S, np.int32)])
    shift = np.concatenate([w["shift"], np.zeros(20 - S)])
    mask = np.vstack([w["mask"], np.ones((20 - S, D), np.uint8)])
    # new parameters: rates of the extra species, appended after the existing ones
    P0 = w["n_params"]
    ns_old, ns_new = I.n_slots(S), I.n_slots(20)
    sm = -np.ones((D, ns_new), np.int32)
    for d in range(D):
        old = w["slot_map"][d]
        sm[d, :S] = old[:S]
        sm[d, 20:25] = old[S:S + 5]
        sm[d, 25:25 + 2 * S] = old[S + 5:3 * S + 5]
        sm[d, S:20] = P0 + np.arange(20 - S)
    theta = np.concatenate([w["theta0"], 10.0 ** rng.uniform(2, 4, 20 - S)])
    w2 = dict(w, spectra=spectra, kind=kind, shift=shift, mask=mask, slot_map=sm, n_params=P0 + 20 - S, theta0=theta)
    return w2


@pytest.mark.parametrize("resolution", [gsn.GSN_RES_GAUSS, gsn.GSN_RES_GAMMA])
def test_tensorcore_expected_against_oracle(resolution):
    w = _workload_20_species(resolution)
    n = poisson_data(w, 55)
    ctx = gsn.context_from_workload(w, gsn.GSN_MIXED, counts=n)
    p = I.perturbed_points(w["theta0"], 1, 56)[0]
    for d in range(len(w["edges"])):
        got = ctx.expected(p, d)
        ref = O.expected_per_species(w, p, d)
        big = ref > 1e-6 * ref.max()
        assert np.max(np.abs(got[big] / ref[big] - 1.0)) < 2e-5
        assert np.all(np.abs(got[~big]) <= 2e-6 * ref.max())
    rc, v = ctx.eval(p)
    assert rc == 0 and abs(v - O.nll(w, p, n)) < 1e-3


def test_tensorcore_contraction_has_no_coherent_bias():
    """Species totals over the histogram: the tensor-core path against the FP64 GPU path.

    Random per-element rounding averages out over the bins; a one-sided rounding of the
    accumulator would not, and it would shift the NLL by (bias) x sum(mu - n) far from the data.
    """
    w = I.borexino_like(n_bins=1000, n_fine=20000)
    p = I.perturbed_points(w["theta0"], 1, 58)[0]
    mixed = gsn.context_from_workload(w, gsn.GSN_MIXED)
    fp64 = gsn.context_from_workload(w, gsn.GSN_FP64)
    worst = 0.0
    for d in range(len(w["edges"])):
        a, b = mixed.expected(p, d).sum(axis=0), fp64.expected(p, d).sum(axis=0)
        ok = b > 1e-3 * b.max()
        worst = max(worst, float(np.max(np.abs(a[ok] / b[ok] - 1.0))))
    assert worst < 1.5e-7, worst
