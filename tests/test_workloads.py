"""Pins of the seeded input generators that are not covered elsewhere."""

import numpy as np

from workloads import make_workload
from workloads.fields import fibrosis_D, smooth_random_field


def test_smooth_random_field_quantiles_and_determinism():
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 1, size=(2000, 2))
    u = smooth_random_field(pts, 5, 0.1)
    assert u.min() == 0.0 and u.max() == 1.0
    assert np.array_equal(np.sort(u), np.arange(2000) / 1999)  # a rank map: uniform quantiles
    assert np.array_equal(u, smooth_random_field(pts, 5, 0.1))
    assert not np.array_equal(u, smooth_random_field(pts, 6, 0.1))


def test_smooth_random_field_is_spatially_correlated():
    # values at points much closer than the correlation length agree far
    # better than values at points much farther apart
    x = np.linspace(0, 4, 4001)[:, None]
    u = smooth_random_field(x, 3, 0.1)
    near = np.mean(np.abs(u[1:] - u[:-1]))           # spacing 0.001 = corr_len / 100
    far = np.mean(np.abs(u[500:] - u[:-500]))        # spacing 0.5 = 5 corr_len
    assert near < 0.05 * far
    assert 0.25 < far < 0.45  # independent U(0,1) pairs: E|a - b| = 1/3


def test_fibrosis_D_median_split():
    w = make_workload("slab9x5x4_ttp")
    a_l = np.tile(np.array([1.0, 0.0, 0.0]), (w.cells.shape[0], 1))
    D, fib = fibrosis_D(w.coords, w.cells, a_l, 1.33, 0.18, 4, 0.05)
    assert abs(fib.mean() - 0.5) <= 1.0 / fib.size
    assert np.allclose(D[fib][:, 1, 1], 0.0) and np.allclose(D[~fib][:, 1, 1], 0.18)
    assert np.allclose(D[:, 0, 0], 1.33)


def test_cable_workload_matches_sec51_setup():
    w = make_workload("cable_ttp")
    assert w.n == 801 and np.isclose(w.coords[1, 0] - w.coords[0, 0], 0.0025)
    assert np.isclose(w.coords[-1, 0], 2.0)
    assert w.stim_mask.sum() == 61 and w.t_off == 2.0 and w.T == 100.0
