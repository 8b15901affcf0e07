"""The seeded input generators against the recipes they state (CPU): the Gaussian-peak batches and
the scalability appendix's banded workload (grid x_i = i, k = n/10 height-1 Gaussians of width 2
truncated at 5 widths, cost rho |x_i - x_j| below 10 samples, skew-normal mixture targets)."""
import numpy as np

import spectra


def test_sub_batches_reproduce_the_full_batch():
    full = spectra.batch(3, 6, 64, 8, 3)
    part = spectra.batch(3, 2, 64, 8, 3, first=4)
    np.testing.assert_array_equal(part["y"], full["y"][4:6])
    np.testing.assert_array_equal(part["D"], full["D"])
    s_full = spectra.scaling_batch(9, 4, 500)
    s_part = spectra.scaling_batch(9, 1, 500, first=3)
    np.testing.assert_array_equal(s_part["y"][0], s_full["y"][3])


def test_gaussian_dictionary_columns_have_unit_mass():
    d = spectra.batch(3, 2, 256, 16, 3, dtype=np.float64)
    np.testing.assert_allclose(d["D"].sum(axis=0), 1.0, rtol=1e-12)
    assert np.all(d["y"] >= 0)


def test_scaling_dictionary_follows_the_appendix():
    n, k = 1000, 100
    col_ptr, row_idx, val = spectra.scaling_dictionary(n, k)
    assert col_ptr.shape == (k + 1,) and col_ptr[0] == 0 and col_ptr[-1] == row_idx.size == val.size
    for m in range(k):
        rows = row_idx[col_ptr[m]:col_ptr[m + 1]]
        vals = val[col_ptr[m]:col_ptr[m + 1]]
        mu = m * n / k
        # support: every sample within 5 widths (10 samples) of the mean, rows ascending
        expect = np.arange(max(0, int(np.ceil(mu - 10))), min(n - 1, int(np.floor(mu + 10))) + 1)
        np.testing.assert_array_equal(rows, expect)
        np.testing.assert_allclose(vals, np.exp(-0.5 * ((rows - mu) / 2.0) ** 2), rtol=1e-15)
        assert vals.max() == 1.0  # the means fall on the grid (n / k = 10), height 1
    dense = spectra.csc_to_dense(n, col_ptr, row_idx, val)
    assert dense.shape == (n, k) and np.count_nonzero(dense) == val.size


def test_truncated_cost_band_follows_the_appendix():
    n = 50
    Cd, h = spectra.truncated_cost_band(n, rho=0.01, delta=10.0)
    assert h == 9 and Cd.shape == (19, n)
    for d in range(19):
        for i in range(n):
            j = i + d - h
            if 0 <= j < n:
                assert Cd[d, i] == 0.01 * abs(i - j)  # |x_i - x_j| <= 9 < 10: inside the band
            else:
                assert np.isinf(Cd[d, i])
    Cd3, h3 = spectra.truncated_cost_band(n, rho=0.5, delta=3.5)
    assert h3 == 3 and np.isfinite(Cd3[0, 10]) and Cd3[0, 10] == 1.5


def test_scaling_targets_are_nonnegative_mixtures_of_the_stated_size():
    n, k = 4000, 400
    y = spectra.scaling_target(n, k, np.random.default_rng(5))
    assert y.shape == (n,) and np.all(y > 0)  # |noise| > 0 almost surely
    # each skew-normal density has unit mass and each amplitude is |N(1, 0.2)| + 0.01; components
    # near the ends lose part of their mass
    assert 0.8 * k < y.sum() < 1.2 * k + 0.002 * n


def test_ragged_sizes_replay_the_generator():
    """ragged_sizes gives the n, k and eps of ragged() problem by problem (the packed layout of
    the uneven batch is planned from it before the arrays are generated in parallel)."""
    probs = spectra.ragged(4, 12, first=37)
    n, k, eps = spectra.ragged_sizes(4, 12, first=37)
    assert list(n) == [p["n"] for p in probs] and list(k) == [p["k"] for p in probs]
    assert list(eps) == [p["eps"] for p in probs]
