"""Batches that run as several consecutive launches (chunks), against the FP64 oracle.

A batch larger than the context's toys-per-launch bound (max_toys_per_launch, default 4096) runs as
chunks, one after another on the same scratch buffers; the batched pseudo-experiment workload of
8192 toys (section 4.2 toy Monte Carlo) is two chunks.  Checked here, on the full-size problem (two
datasets on a 1200-bin domain, 16 species on 20000 fine points, windows of 600..1200 bins):

* 24 toys with 8 toys per launch (three chunks), both precisions: toys from every chunk, including
  the first and last toy of each, against the oracle (FP64: 1e-10 relative on the NLL, 1e-8
  normwise on the gradient; mixed: |dNLL| < 1e-3, 1e-5 normwise), and the chunked results bitwise
  equal to the same toys run as separate 8-toy batches (same work plan: autotuning off);
* the launch configuration of the benchmark: 8192 toys, 4096 per launch, mixed path through the
  device-pointer call on a dedicated stream with graphs and autotuning on.  Toys on both sides of
  the chunk boundary against the oracle, and a stride of toys over the whole batch against the FP64
  GPU path.

The oracle's references (about a minute per toy with its gradient) come from a spawn process pool.
"""
import os

import numpy as np
import pytest

from paper_1812_05686_gb300 import gsn, inputs as I
from tests._helpers import norm_rel, oracle_pool_map

pytestmark = pytest.mark.gpu
FP64, MIXED = gsn.GSN_FP64, gsn.GSN_MIXED

SMALL_T, SMALL_CHUNK = 24, 8
SMALL_NLL = (0, 7, 8, 15, 16, 23)        # first and last toy of every chunk
SMALL_GRAD = (3, 12, 20)                 # one toy inside every chunk
BIG_T = 8192
BIG_NLL = (0, 4095, 4096, 8191)          # both sides of the chunk boundary and the ends
BIG_GRAD = (6000,)


@pytest.fixture(scope="module")
def problem():
    w = I.borexino_like(n_bins=1200)
    mu0 = np.loadtxt(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "borexino_like_1200_mu0.txt"))
    mu = [mu0[:1200], mu0[1200:]]
    small = I.toy_batch(w, mu, n_toys=SMALL_T, seed0=3000)
    big = I.toy_batch(w, mu, n_toys=BIG_T, seed0=1000)
    tasks, keys = [], []
    for name, b, nl, gr in (("small", small, SMALL_NLL, SMALL_GRAD), ("big", big, BIG_NLL, BIG_GRAD)):
        for t in sorted(set(nl) | set(gr)):
            tasks.append(("toy", "borexino_like_1200", (b["params"][t], b["counts"][t], b["windows"][t], t in gr)))
            keys.append((name, t))
    refs = dict(zip(keys, oracle_pool_map(tasks)))
    return w, small, big, refs


def _run(w, b, precision, lo, hi, **opt):
    ctx = gsn.context_from_workload(w, precision, **opt)
    rc, nll, g = ctx.eval_grad_batch(b["params"][lo:hi], b["counts"][lo:hi], b["windows"][lo:hi])
    assert rc == 0, ctx.last_error()
    ctx.close()
    return nll, g


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_chunked_batch_against_oracle(problem, precision):
    w, small, _, refs = problem
    nll, g = _run(w, small, precision, 0, SMALL_T, max_toys_per_launch=SMALL_CHUNK, autotune=0)
    for t in SMALL_NLL + SMALL_GRAD:
        ref, gref = refs[("small", t)]
        if precision == FP64:
            assert abs(nll[t] - ref) <= 1e-10 * abs(ref), (t, nll[t], ref)
        else:
            assert abs(nll[t] - ref) < 1e-3, (t, nll[t], ref)
        if gref is not None:
            assert norm_rel(g[t], gref) < (1e-8 if precision == FP64 else 1e-5), (t, norm_rel(g[t], gref))


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_chunked_equals_separate_batches(problem, precision):
    w, small, _, _ = problem
    nll, g = _run(w, small, precision, 0, SMALL_T, max_toys_per_launch=SMALL_CHUNK, autotune=0)
    ctx = gsn.context_from_workload(w, precision, autotune=0)
    for lo in range(0, SMALL_T, SMALL_CHUNK):
        hi = lo + SMALL_CHUNK
        rc, n1, g1 = ctx.eval_grad_batch(small["params"][lo:hi], small["counts"][lo:hi], small["windows"][lo:hi])
        assert rc == 0, ctx.last_error()
        assert np.array_equal(n1, nll[lo:hi]) and np.array_equal(g1, g[lo:hi]), lo
    # one launch of all 24 toys uses another work split: equal up to the order of the sums
    n24, g24 = _run(w, small, precision, 0, SMALL_T, autotune=0)
    if precision == FP64:
        assert np.max(np.abs(n24 - nll) / np.abs(nll)) < 1e-12
        assert max(norm_rel(g24[t], g[t]) for t in range(SMALL_T)) < 1e-11
    else:
        assert np.max(np.abs(n24 - nll)) < 1e-4
        assert max(norm_rel(g24[t], g[t]) for t in range(SMALL_T)) < 1e-5


def test_benchmark_batch_two_chunks(problem):
    torch = pytest.importorskip("torch")
    w, _, b, refs = problem
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = gsn.context_from_workload(w, MIXED, stream=stream.cuda_stream)
    P = w["n_params"]
    params = torch.from_numpy(b["params"]).to(dev)
    counts = torch.from_numpy(b["counts"]).to(dev)
    wins = torch.from_numpy(b["windows"].astype(np.int32)).to(dev)
    nll = torch.empty(BIG_T, dtype=torch.float64, device=dev)
    grad = torch.empty(BIG_T, P, dtype=torch.float64, device=dev)
    status = torch.empty(BIG_T, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)  # inputs copied on torch's stream, the library runs on its own
    for _ in range(2):  # the second call replays the recorded graph
        assert ctx.eval_grad_batch_dev(params, counts, wins, nll, grad, status) == 0, ctx.last_error()
    torch.cuda.synchronize(dev)
    nll_h, g_h = nll.cpu().numpy(), grad.cpu().numpy()
    assert not np.any(status.cpu().numpy())
    for t in BIG_NLL + BIG_GRAD:
        ref, gref = refs[("big", t)]
        assert abs(nll_h[t] - ref) < 1e-3, (t, nll_h[t], ref)
        if gref is not None:
            assert norm_rel(g_h[t], gref) < 1e-5, (t, norm_rel(g_h[t], gref))
    # every 128th toy of the batch (both chunks) against the FP64 GPU path
    idx = np.arange(0, BIG_T, 128)
    sel = torch.from_numpy(idx).to(dev)
    ctx64 = gsn.context_from_workload(w, FP64, stream=stream.cuda_stream)
    p_s, c_s, w_s = params[sel].contiguous(), counts[sel].contiguous(), wins[sel].contiguous()
    n64 = torch.empty(idx.size, dtype=torch.float64, device=dev)
    g64 = torch.empty(idx.size, P, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    assert ctx64.eval_grad_batch_dev(p_s, c_s, w_s, n64, g64, None) == 0, ctx64.last_error()
    torch.cuda.synchronize(dev)
    n64, g64 = n64.cpu().numpy(), g64.cpu().numpy()
    assert np.max(np.abs(n64 - nll_h[idx])) < 1e-3
    assert max(norm_rel(g_h[t], g64[i]) for i, t in enumerate(idx)) < 1e-5
