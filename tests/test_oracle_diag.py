"""Pins of the oracle's FP32 diagnostics (oracle/diagnostics.py): the ghost test
of Eq. 25 against closed forms, interlacing and invariances, cluster weights
against the exact spectral measure, and Eq. 22 on a hand example."""
import numpy as np
import pytest

import oracle as o
from oracle import diagnostics as dg
from paper_2605_26261_gb300 import inputs


def test_two_by_two_closed_form():
    a, b, c = 0.3, 0.7, -1.1
    g = dg.ghosts([a, c], [b], c_tau=1.0, u=0.1)
    mid, rad = (a + c) / 2, np.hypot((a - c) / 2, b)
    np.testing.assert_allclose(g["theta"], [mid - rad, mid + rad], rtol=1e-14)
    np.testing.assert_allclose(g["theta1"], [c])  # T^(1) = [c]
    np.testing.assert_allclose(g["ell"], np.abs(np.array([mid - rad, mid + rad]) - c), rtol=1e-13)
    assert g["tau"] == pytest.approx(0.1 * 2 * rad)


def test_decoupled_matrix():
    # beta = 0: T = diag(a), T^(1) = diag(a[1:]); every theta but a_1 repeats an
    # eigenvalue of T^(1) exactly (l = 0); the weight sits on a_1 alone
    a = np.array([0.5, -2.0, 1.0, 3.0])
    g = dg.ghosts(a, np.zeros(3), c_tau=1.0, u=1e-3)
    k1 = int(np.argmin(np.abs(g["theta"] - 0.5)))
    for k in range(4):
        if k == k1:
            assert g["ell"][k] == pytest.approx(0.5) and not g["flags"][k]
        else:
            assert g["ell"][k] == 0.0 and g["flags"][k]
    np.testing.assert_allclose(g["weight"], (np.arange(4) == k1).astype(float), atol=1e-15)


def test_interlacing_and_invariance():
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=40), np.abs(rng.normal(size=39)) + 0.01
    g = dg.ghosts(a, b, c_tau=50.0)
    th, t1 = g["theta"], g["theta1"]
    assert np.all(th[:-1] <= t1 + 1e-12) and np.all(t1 <= th[1:] + 1e-12)  # Cauchy interlacing
    h = dg.ghosts(3.0 * a - 7.0, 3.0 * b, c_tau=50.0)  # T -> 3 T - 7
    np.testing.assert_allclose(h["ell"], 3.0 * g["ell"], rtol=1e-9, atol=1e-12)
    assert np.array_equal(h["flags"], g["flags"]) and np.array_equal(h["cluster"], g["cluster"])
    np.testing.assert_allclose(np.sum(g["cweight"][np.unique(g["cluster"], return_index=True)[1]]), 1.0, rtol=1e-12)


def test_clusters_of_a_decoupled_matrix():
    # T = diag(1, 1 + d, 5, 1 + 2d, 9): all weight on the first diagonal entry;
    # T^(1) = diag(1 + d, 5, 1 + 2d, 9).  With tau = 3 d the three values near 1
    # form one cluster carrying the whole weight, 5 and 9 are singletons of weight 0;
    # l = d for theta = 1 and 0 for the rest, so all five are ghosts.
    d = 1e-3
    a = np.array([1.0, 1.0 + d, 5.0, 1.0 + 2 * d, 9.0])
    g = dg.ghosts(a, np.zeros(4), c_tau=1.0, u=3 * d / 8.0)
    assert g["tau"] == pytest.approx(3 * d)
    np.testing.assert_allclose(g["theta"], [1.0, 1.0 + d, 1.0 + 2 * d, 5.0, 9.0])
    np.testing.assert_allclose(g["ell"], [d, 0, 0, 0, 0], atol=1e-15)
    assert g["count"] == 5
    assert list(g["cluster"]) == [0, 0, 0, 3, 4]
    np.testing.assert_allclose(g["cweight"], [1, 1, 1, 0, 0], atol=1e-15)


def test_ghosts_of_a_long_run():
    # Lanczos run to the sector dimension without reorthogonalization: converged
    # eigenvalues reappear (ghosts at the FP32 threshold), the weights still sum to 1
    N, K = 10, 5
    bonds = inputs.random_graph(N, seed=6)
    b = o.basis(N, K)
    r = inputs.seeded_vector(len(b), 2)
    a, bt, m = o.lanczos(bonds, b, r, 400, 0.0)
    g = dg.ghosts(a, bt, c_tau=1.0, u=2.0**-24)
    assert m == len(b) and g["count"] > 0
    firsts = np.unique(g["cluster"], return_index=True)[1]
    assert np.sum(g["cweight"][firsts]) == pytest.approx(1.0, rel=1e-12)


def test_sigma_emp_hand_example():
    mean, sig = dg.sigma_emp([[1.0, 2.0, 5.0], [3.0, 6.0, 5.0]])
    np.testing.assert_allclose(mean, [2.0, 4.0, 5.0])
    np.testing.assert_allclose(sig, [1.0, 2.0, 0.0])  # 1/N_s, not 1/(N_s - 1)
