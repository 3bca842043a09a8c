"""gsn_eval_grad_noalloc against gsn_eval_grad (GPU, through the C ABI).

The no-allocation entry point is for callers that must not call cudaMalloc
while they run -- for example a step being captured into a CUDA graph, or a
loop that runs under a fixed, pre-reserved memory budget.  Its intermediate
buffers live in one static device array that every call shares and that keeps
the previous call's contents, so each test makes two calls in a row with
different parameter points and checks both against the allocating entry point,
within the tolerances of the other GPU tests (FP64: 1e-10 relative on the NLL,
1e-8 normwise on the gradient; mixed: 1e-3 absolute and 1e-5).
"""
import ctypes as C

import numpy as np
import pytest

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import gsn, inputs as I

pytestmark = pytest.mark.gpu


def _normwise(g, ref):
    return float(np.max(np.abs(g - ref)) / max(float(np.max(np.abs(ref))), 1.0))


def _workload(kind):
    """The two-dataset gamma workload; with a free-power generalized gamma (its scratch holds the
    adjoint's per-column coefficient records); or with Monte Carlo template species (their rate
    partials go through the deviance scratch)."""
    base = I.borexino_like(n_bins=320, n_fine=3000)
    if kind == "ggamma":
        return I.with_power(base, 1.3)
    if kind == "templates":
        return I.with_templates(base, 2)
    return base


@pytest.mark.parametrize("kind", ["gamma", "ggamma", "templates"])
@pytest.mark.parametrize("precision", [gsn.GSN_FP64, gsn.GSN_MIXED])
def test_noalloc_matches_allocating_entry_point(precision, kind):
    torch = pytest.importorskip("torch")
    w = _workload(kind)
    mu = [O.expected_counts(w, w["theta0"], d) for d in range(2)]
    n = np.concatenate([I.poisson_counts(m, 41 + d) for d, m in enumerate(mu)])
    ctx = gsn.context_from_workload(w, precision, counts=n)
    lib = gsn.load_library()
    pts = I.perturbed_points(w["theta0"], 3, 4100)
    rc, _, _ = ctx.eval_grad(pts[0])  # set-up: puts the problem on the device
    assert rc == 0
    dev = torch.device("cuda", 0)
    for p in pts[1:]:  # two calls in a row share the static scratch array
        rc, ref, gref = ctx.eval_grad(p)
        assert rc == 0
        pd = torch.tensor(p, dtype=torch.float64, device=dev)
        nll = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        grad = torch.full((w["n_params"],), np.nan, dtype=torch.float64, device=dev)
        status = torch.full((1,), 99, dtype=torch.int32, device=dev)
        torch.cuda.synchronize(dev)
        rc = lib.gsn_eval_grad_noalloc(ctx.h, C.c_void_p(pd.data_ptr()), C.c_void_p(nll.data_ptr()),
                                       C.c_void_p(grad.data_ptr()), C.c_void_p(status.data_ptr()))
        assert rc == 0, ctx.last_error()
        torch.cuda.synchronize(dev)
        v, g, st = float(nll.item()), grad.cpu().numpy(), int(status.item())
        assert st == 0
        if precision == gsn.GSN_FP64:
            assert abs(v - ref) <= 1e-10 * abs(ref)
            assert _normwise(g, gref) < 1e-8
        else:
            assert abs(v - ref) < 1e-3
            assert _normwise(g, gref) < 1e-5


def test_noalloc_rejects_oversized_problem_and_unprepared_context():
    torch = pytest.importorskip("torch")
    lib = gsn.load_library()
    w = I.single_gauss(n_bins=40, n_fine=150000)  # FP64 column records alone need 19.2 MB
    ctx = gsn.context_from_workload(w, gsn.GSN_FP64, counts=np.full(40, 5.0))
    dev = torch.device("cuda", 0)
    pd = torch.tensor(w["theta0"], dtype=torch.float64, device=dev)
    out = torch.zeros(w["n_params"] + 1, dtype=torch.float64, device=dev)
    args = (C.c_void_p(pd.data_ptr()), C.c_void_p(out.data_ptr()), C.c_void_p(out[1:].data_ptr()), None)
    assert lib.gsn_eval_grad_noalloc(ctx.h, *args) == gsn.GSN_ERR_STATE
    rc, _, _ = ctx.eval_grad(w["theta0"])
    assert rc == 0
    assert lib.gsn_eval_grad_noalloc(ctx.h, *args) == gsn.GSN_ERR_ARG
    assert "bytes of scratch" in ctx.last_error()
