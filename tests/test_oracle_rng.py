"""Pins for the oracle's counter-based start vectors (CPU only)."""
import numpy as np
import scipy.stats as st

import oracle as o
from tests.conftest import golden


def test_splitmix64_reference_outputs():
    g = golden("splitmix64.txt")
    seed = int(g["seed"])
    want = [int(v) for v in g["outputs"].split(",")]
    assert [o.splitmix64_at(seed, c) for c in range(len(want))] == want


def test_rademacher_entries_and_balance():
    x = o.start_vector(11, 20, 10, 3, o.RADEMACHER, 200000)
    assert set(np.unique(x).tolist()) == {-1.0, 1.0}
    assert abs(x.mean()) < 5 / np.sqrt(len(x))


def test_gaussian_entries_are_standard_normal():
    x = o.start_vector(11, 20, 10, 3, o.GAUSS, 200000)
    assert st.kstest(x, "norm").pvalue > 1e-3
    assert abs(x.mean()) < 5 / np.sqrt(len(x))
    assert abs(x.var() - 1) < 0.02


def test_chains_and_sectors_get_distinct_streams():
    a = o.start_vector(1, 16, 8, 0, o.GAUSS, 1000)
    b = o.start_vector(1, 16, 8, 1, o.GAUSS, 1000)
    c = o.start_vector(1, 16, 9, 0, o.GAUSS, 1000)
    d = o.start_vector(2, 16, 8, 0, o.GAUSS, 1000)
    for u, v in ((a, b), (a, c), (a, d)):
        assert abs(np.corrcoef(u, v)[0, 1]) < 0.2
    np.testing.assert_array_equal(a, o.start_vector(1, 16, 8, 0, o.GAUSS, 1000))
