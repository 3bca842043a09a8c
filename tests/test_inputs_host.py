"""Host-side checks of the seeded workload builders (no GPU, no oracle arithmetic)."""
import numpy as np

from paper_1812_05686_gb300 import inputs as I


def test_with_power_and_with_secondary_layouts():
    """Host-side layout of the free-power and secondary-observable workloads."""
    w = I.borexino_like(n_bins=120, n_fine=400)
    S, P0 = w["spectra"].shape[0], w["n_params"]
    g = I.with_power(w, 1.7, pull_width=0.1)
    assert g["resolution"] == I.RES_GGAMMA and g["n_params"] == P0 + 1
    assert np.all(np.asarray(g["slot_map"])[:, I.slot_power(S)] == P0)
    assert g["theta0"][-1] == 1.7 and g["pull_param"][-1] == P0
    assert np.all(np.asarray(w["slot_map"])[:, I.slot_power(S)] == -1)  # the source is untouched
    x = I.with_secondary(w, n_slices=5, n_sec=7)
    for d in range(2):
        sec = x["secondary"][d]
        st = np.asarray(sec["slice_start"])
        assert st[0] == 0 and st[-1] == 120 and np.all(np.diff(st) > 0) and st.size == 6
        assert np.asarray(sec["shapes"]).shape == (S, 5, 7) and np.all(np.asarray(sec["shapes"]) > 0)
    mu = [np.full(120, 50.0), np.full(120, 30.0)]
    b = I.toy_batch(x, mu, n_toys=3, seed0=9, w_min=60, w_max=120, mu_sec=np.full(2 * 35, 20.0))
    assert b["counts"].shape == (3, 240 + 70)
