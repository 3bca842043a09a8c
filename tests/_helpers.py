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
