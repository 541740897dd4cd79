"""Host logic of the config-4 ensemble experiment: grouping the replica boxes by
(L, tau) and averaging the per-particle VACF sums within a group (CPU only)."""
import math

import numpy as np

from paper_1909_13412_gb300 import experiments as ex
from paper_1909_13412_gb300 import workloads as wl


def test_groups_of_the_68_box_ensemble():
    g = ex.ensemble_groups(wl.ENSEMBLE_68.boxes)
    assert sorted(b for v in g.values() for b in v) == list(range(68))
    assert {k: len(v) for k, v in g.items()} == {
        (64, 0.6): 16, (64, 0.8): 16, (64, 1.0): 16, (96, 0.6): 6, (96, 0.8): 5, (96, 1.0): 5,
        (160, 0.6): 2, (160, 0.8): 1, (160, 1.0): 1}
    for (L, tau), boxes in g.items():
        assert all(wl.ENSEMBLE_68.boxes[b] == (L, L, L, tau) for b in boxes)


def test_group_average_and_tail_amplitude():
    """Per-particle sums with a known shape: particle i of group G has
    C_i(k) = a_i (1 + k)^(-3/2) per pair, so the group's C/C(0) is (1 + k)^(-3/2)
    whatever the a_i, and B over a window is the mean of (t / (1 + t))^(3/2)."""
    w = wl.Ensemble("test", [(8, 8, 8, 0.6), (8, 8, 8, 0.8), (8, 8, 8, 0.6), (12, 12, 12, 0.6)],
                    n_per_box=2)
    K = 50
    k = np.arange(K + 1)
    cnt = (1000 - k).astype(np.int64)
    rng = np.random.default_rng(1)
    a = rng.uniform(0.5, 2.0, w.n_particles)
    cs = a[:, None] * (1.0 + k) ** -1.5 * cnt
    out = ex.ensemble_statistics(w, cs, cnt, (10, 40), lags=(1, 10, 50))
    assert [(g["L"], g["tau"], g["boxes"], g["particles"]) for g in out] == [
        (8, 0.6, 2, 4), (8, 0.8, 1, 2), (12, 0.6, 1, 2)]
    t = np.arange(10, 41)
    for g, rows in zip(out, ([0, 1, 4, 5], [2, 3], [6, 7])):
        assert math.isclose(g["C0"], a[rows].mean(), rel_tol=1e-12)
        for lag in (1, 10, 50):
            assert math.isclose(g["C_over_C0"][str(lag)], (1.0 + lag) ** -1.5, rel_tol=1e-12)
        assert math.isclose(g["B"], float(np.mean((t / (1.0 + t)) ** 1.5)), rel_tol=1e-12)
        assert g["B_se"] < 1e-12  # every particle has the same normalised shape
        assert math.isclose(g["B_paper"], w.M / (12.0 * (math.pi * (g["tau"] - 0.5) / 3.0) ** 1.5))
