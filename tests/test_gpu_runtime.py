"""Launch runtime on the GPU: CUDA-graph replay and the plan autotuner (through the C ABI).

Graph replay must reproduce plain launches bit for bit (same kernels, same plan, same order),
also after another call has reallocated the scratch buffers the graph had recorded.  A tuned
plan only changes how the sums are split, so its results stay within the parity tolerances.
"""
import numpy as np
import pytest

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import gsn, inputs as I

from tests._helpers import norm_rel

pytestmark = pytest.mark.gpu
FP64, MIXED = gsn.GSN_FP64, gsn.GSN_MIXED


@pytest.fixture(scope="module")
def problem():
    w = I.borexino_like(n_bins=400, n_fine=4000)
    mu = [O.expected_counts(w, w["theta0"], d) for d in range(2)]
    n = np.concatenate([I.poisson_counts(m, 71 + d) for d, m in enumerate(mu)])
    b = I.toy_batch(w, mu, n_toys=40, seed0=2000, w_min=200, w_max=400)
    return w, n, b


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_graph_replay_is_bitwise_equal_to_plain_launches(problem, precision):
    w, n, b = problem
    plain = gsn.context_from_workload(w, precision, counts=n, use_graphs=0, autotune=0)
    graph = gsn.context_from_workload(w, precision, counts=n, use_graphs=1, autotune=0)
    pts = I.perturbed_points(w["theta0"], 4, 5100)
    for p in pts:  # the first call records the graph, the others replay it
        r0, v0, g0 = plain.eval_grad(p)
        r1, v1, g1 = graph.eval_grad(p)
        assert r0 == 0 and r1 == 0
        assert v0 == v1 and np.array_equal(g0, g1)
    for rep in range(2):
        r0, n0, g0 = plain.eval_grad_batch(b["params"], b["counts"], b["windows"])
        r1, n1, g1 = graph.eval_grad_batch(b["params"], b["counts"], b["windows"])
        assert r0 == 0 and r1 == 0
        assert np.array_equal(n0, n1) and np.array_equal(g0, g1)
    # the batch grew the scratch buffers: the single-point graph must be recorded again
    r0, v0, g0 = plain.eval_grad(pts[0])
    r1, v1, g1 = graph.eval_grad(pts[0])
    assert v0 == v1 and np.array_equal(g0, g1)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_autotuned_plan_stays_within_parity(problem, precision):
    w, n, b = problem
    ctx = gsn.context_from_workload(w, precision, counts=n, autotune=1)
    h = ctx.plan_info(1, True)
    assert h["tuned"] == 0
    p = I.perturbed_points(w["theta0"], 1, 5200)[0]
    rc, v, g = ctx.eval_grad(p)
    assert rc == 0
    t = ctx.plan_info(1, True)
    assert t["tuned"] == (1 if (h["nsplit"] > 1 or h["bw_bsplit"] > 1) else 0)
    assert 1 <= t["nsplit"] <= 4000 // 256 and t["bw_warps"] in (4, 8) and 1 <= t["bw_bsplit"] <= 16
    ref = O.nll(w, p, n)
    gref = O.nll_grad(w, p, n)
    if precision == FP64:
        assert abs(v - ref) <= 1e-10 * abs(ref)
        assert norm_rel(g, gref) < 1e-8
    else:
        assert abs(v - ref) < 1e-3
        assert norm_rel(g, gref) < 1e-5
    # a second call reuses the tuned plan (and replays its graph): identical results
    rc2, v2, g2 = ctx.eval_grad(p)
    assert rc2 == 0 and v2 == v and np.array_equal(g2, g)
    # a small batch is tuned per toy count
    rc, nll, _ = ctx.eval_grad_batch(b["params"][:3], b["counts"][:3], b["windows"][:3])
    assert rc == 0
    for k in range(3):
        ref = O.nll(w, b["params"][k], b["counts"][k], b["windows"][k])
        tol = 1e-10 * abs(ref) if precision == FP64 else 1e-3
        assert abs(nll[k] - ref) <= tol
