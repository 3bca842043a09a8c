"""Monte Carlo template species (section 3.2 template fit) on the GPU against the FP64 oracle.

Template species enter mu_dj as eps_d f_ds r_s T_dsj with the library-normalised visible-bin
histogram T; a fit of templates only runs no response kernel.  Tolerances as in the other parity
tests: FP64 1e-10 relative on the NLL and 1e-8 normwise on the gradient; mixed |dNLL| < 1e-3, 1e-5.
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
    return mu, np.concatenate([I.poisson_counts(m, seed + d) for d, m in enumerate(mu)])


def _check(w, n, p, precision):
    ctx = gsn.context_from_workload(w, precision, counts=n)
    rc, v, g = ctx.eval_grad(p)
    assert rc == 0, ctx.last_error()
    ref, gref = O.nll(w, p, n), O.nll_grad(w, p, n)
    if precision == FP64:
        assert abs(v - ref) <= 1e-10 * abs(ref), (v, ref)
        assert norm_rel(g, gref) < 1e-8
    else:
        assert abs(v - ref) < 1e-3, (v, ref)
        assert norm_rel(g, gref) < 1e-5
    rc, v2 = ctx.eval(p)
    assert rc == 0 and abs(v2 - ref) <= (1e-10 * abs(ref) if precision == FP64 else 1e-3)
    return ctx


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_pure_template_fit(precision):
    w = I.template_like(n_bins=300, n_species=6)
    mu, n = _data(w, 401)
    ctx = _check(w, n, I.perturbed_points(w["theta0"], 1, 402)[0], precision)
    for d in range(2):
        got, ref = ctx.expected(w["theta0"], d), O.expected_per_species(w, w["theta0"], d)
        assert np.max(np.abs(got - ref)) <= 1e-12 * ref.max()


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_templates_with_smeared_species(precision):
    w = I.with_templates(I.borexino_like(n_bins=240, n_fine=2400), 3)
    mu, n = _data(w, 411)
    _check(w, n, I.perturbed_points(w["theta0"], 1, 412)[0], precision)


def test_template_toy_batch():
    w = I.with_templates(I.borexino_like(n_bins=240, n_fine=2400), 2)
    mu, _ = _data(w, 421)
    b = I.toy_batch(w, mu, n_toys=5, seed0=422, w_min=120, w_max=240)
    for precision in (FP64, MIXED):
        ctx = gsn.context_from_workload(w, precision)
        rc, nll, g = ctx.eval_grad_batch(b["params"], b["counts"], b["windows"])
        assert rc == 0, ctx.last_error()
        for t in (0, 4):
            ref = O.nll(w, b["params"][t], b["counts"][t], b["windows"][t])
            gref = O.nll_grad(w, b["params"][t], b["counts"][t], b["windows"][t])
            if precision == FP64:
                assert abs(nll[t] - ref) <= 1e-10 * abs(ref)
                assert norm_rel(g[t], gref) < 1e-8
            else:
                assert abs(nll[t] - ref) < 1e-3
                assert norm_rel(g[t], gref) < 1e-5


def test_template_removed_and_arguments_validated():
    w = I.template_like(n_bins=120, n_species=4)
    mu, n = _data(w, 431)
    ctx = gsn.context_from_workload(w, FP64, counts=n)
    ctx.set_template(2, 1, None)  # species 2 no longer contributes to dataset 1
    tpl = [list(r) for r in w["templates"]]
    tpl[2][1] = None
    w2 = dict(w, templates=tpl)
    p = I.perturbed_points(w["theta0"], 1, 432)[0]
    rc, v, g = ctx.eval_grad(p)
    assert rc == 0 and abs(v - O.nll(w2, p, n)) <= 1e-10 * abs(v)
    assert norm_rel(g, O.nll_grad(w2, p, n)) < 1e-8
    with pytest.raises(gsn.GsnError):
        ctx.set_template(0, 0, -np.ones(120))
    b = gsn.context_from_workload(I.borexino_like(n_bins=100, n_fine=800), FP64)
    with pytest.raises(gsn.GsnError):
        b.set_template(0, 0, np.ones(100))  # species 0 is not a template species
