"""Shared helpers for the GPU parity tests (inputs from the seeded generators, references from the oracle)."""
import numpy as np

from oracle import gsn_oracle as O
from paper_1812_05686_gb300 import inputs as I


def asimov_mu(work, theta=None):
    theta = work["theta0"] if theta is None else theta
    return [O.expected_counts(work, theta, d) for d in range(len(work["edges"]))]


def poisson_data(work, seed, theta=None):
    mu = asimov_mu(work, theta)
    return np.concatenate([I.poisson_counts(m, seed + 17 * d) for d, m in enumerate(mu)])


def norm_rel(g, ref):
    """Normwise gradient error ||g - ref||_inf / max(||ref||_inf, 1)."""
    return float(np.max(np.abs(g - ref)) / max(float(np.max(np.abs(ref))), 1.0))


def default_windows(work):
    return [(int(work["win_lo"][d]), int(work["win_hi"][d])) for d in range(len(work["edges"]))]


# ---------------------------------------------------------------- oracle pool -----
# Oracle references of full-size toys take tens of seconds each; tests that need several of them
# compute them in parallel in a process pool.  The pool is created with the "spawn" start method,
# so the children do not inherit the parent's CUDA context.
_WORKLOADS = {}


def _workload(name):
    if name not in _WORKLOADS:
        if name == "borexino_like_1200":
            _WORKLOADS[name] = I.borexino_like(n_bins=1200)
        else:
            raise KeyError(name)
    return _WORKLOADS[name]


def oracle_task(task):
    """One oracle job of a pool: ("toy", workload, (params, counts, windows, want_grad)) -> (NLL,
    gradient or None); ("fisher", workload, (params, windows)) -> Fisher diagonal; ("fit", workload,
    (counts, start, free, lo, windows, scale)) -> (minimum, NLL there).  The workload is a workload
    dictionary or the name of a full-size one built in the child."""
    kind, w, args = task
    w = _workload(w) if isinstance(w, str) else w
    if kind == "toy":
        params, counts, windows, want_grad = args
        v = O.nll(w, params, counts, windows)
        return v, (O.nll_grad(w, params, counts, windows) if want_grad else None)
    if kind == "fisher":
        params, windows = args
        return O.fisher_diagonal(w, params, windows)
    if kind == "fit":
        counts, start, free, lo, windows, scale = args
        return O.fit(w, counts, start, free, lo=lo, windows=windows, scale=scale)
    raise ValueError(kind)


def oracle_pool_map(tasks):
    """oracle_task over tasks in a spawn process pool of up to one process per core (single-threaded
    BLAS in each), results in task order."""
    import multiprocessing as mp
    import os
    n = max(1, min(len(tasks), len(os.sched_getaffinity(0))))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(oracle_task, tasks, chunksize=1)


def fisher_rel(g, ref, F):
    """Per-component gradient error on the statistical scale:
    max_i |g_i - ref_i| / max(|ref_i| + sqrt(F_ii), 1), F the Fisher diagonal (oracle.fisher_diagonal).
    sqrt(F_ii) is the spread of dNLL/dtheta_i under Poisson fluctuations of the counts; the floor of 1
    (the normwise ratio's max(||ref||, 1)) covers parameters without information in the evaluated
    window (F_ii = 0, e.g. the rate of a species whose counts all lie outside it)."""
    return float(np.max(np.abs(g - ref) / np.maximum(np.abs(ref) + np.sqrt(F), 1.0)))
