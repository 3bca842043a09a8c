"""Write the stored expected counts used to draw the benchmark's toy data.

Calls only the oracle and the seeded input generators:
borexino_like_1200_mu0.txt holds mu_dj at the generating parameters theta0 of
the two-dataset workload on a 1200-bin domain (dataset 0 then dataset 1), the
mean from which every pseudo-experiment's Poisson counts are drawn.
Run: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import gsn_oracle as O  # noqa: E402
from paper_1812_05686_gb300 import inputs as I  # noqa: E402


def main():
    w = I.borexino_like(n_bins=1200)
    mu = np.concatenate([O.expected_counts(w, w["theta0"], d) for d in range(2)])
    hdr = ("expected counts mu_dj at theta0 of inputs.borexino_like(n_bins=1200) "
           "(2 datasets x 1200 bins, dataset 0 first), FP64 oracle; written by make_golden.py")
    np.savetxt(os.path.join(HERE, "borexino_like_1200_mu0.txt"), mu, fmt="%.17g", header=hdr)


if __name__ == "__main__":
    main()
