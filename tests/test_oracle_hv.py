"""Pins for the oracle's H.v (Eq. 12-14 at s = 1/2), CPU only.

The reference here is an independent construction: the full 2^N-dimensional
Hamiltonian sum_b J_b S_i . S_j built from Kronecker products of 2x2 spin
matrices (scipy.sparse), then restricted to the labels with K up spins.  Nothing
in it shares the oracle's bit manipulation or ladder-coefficient formulas.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as o
from oracle import counting
from paper_2605_26261_gb300 import inputs as I

# Local basis: index 0 = down (bit 0), 1 = up (bit 1).
SZ = np.array([[-0.5, 0.0], [0.0, 0.5]])
SP = np.array([[0.0, 0.0], [1.0, 0.0]])  # S+ |down> = |up>
SM = SP.T


def site_op(N, k, A):
    """A acting on site k of the full space; label bit k is site k."""
    left = sp.identity(2 ** (N - 1 - k), format="csr")
    right = sp.identity(2**k, format="csr")
    return sp.kron(sp.kron(left, sp.csr_matrix(A)), right, format="csr")


def kron_hamiltonian(N, bonds):
    bi, bj, J = bonds
    H = sp.csr_matrix((2**N, 2**N))
    for i, j, Jb in zip(bi, bj, J):
        i, j = int(i), int(j)
        H = H + Jb * (site_op(N, i, SZ) @ site_op(N, j, SZ)
                      + 0.5 * (site_op(N, i, SP) @ site_op(N, j, SM)
                               + site_op(N, i, SM) @ site_op(N, j, SP)))
    return H.toarray()


def sector_block(Hfull, N, K):
    idx = [n for n in range(2**N) if bin(n).count("1") == K]
    return Hfull[np.ix_(idx, idx)]


GRAPHS = {
    "dimer": (2, I.dimer(0.7)),
    "ring8": (8, I.ring(8)),
    "ladder8": (8, I.ladder(8, 0.6, 1.3)),
    "random9": (9, I.random_graph(9, seed=3)),
    "lattice_3x3": (9, I.square_j1j2(3, 3, 1.0, 0.5)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_hv_matches_kronecker_hamiltonian(name):
    N, bonds = GRAPHS[name]
    Hfull = kron_hamiltonian(N, bonds)
    for K in range(N + 1):
        b = o.basis(N, K)
        H = o.dense_h(bonds, b, o.full_lut(N, b))
        np.testing.assert_allclose(H, sector_block(Hfull, N, K), atol=1e-14, rtol=0)
        # without the table (binary-search index map) it is the same matrix
        np.testing.assert_array_equal(H, o.dense_h(bonds, b))


def test_hv_all_ones_is_multiplet_eigenvector():
    # Every sector contains one state of the S = N/2 multiplet, the uniform vector,
    # with energy sum_b J_b / 4; exact in FP64 for dyadic couplings.
    bonds = I.random_graph(12, seed=5)
    bi, bj, J = bonds
    J = np.round(J * 64) / 64  # dyadic couplings
    bonds = (bi, bj, J)
    for K in (0, 3, 6, 11):
        b = o.basis(12, K)
        y = o.hv(bonds, b, np.ones(len(b)))
        assert np.all(y == J.sum() / 4)


def test_spin_flip_maps_sector_k_to_n_minus_k():
    N, bonds = GRAPHS["random9"]
    for K in range(N + 1):
        e1 = np.linalg.eigvalsh(o.dense_h(bonds, o.basis(N, K)))
        e2 = np.linalg.eigvalsh(o.dense_h(bonds, o.basis(N, N - K)))
        np.testing.assert_allclose(e1, e2, atol=1e-12)


def test_ring_translation_commutes():
    N, K = 10, 5
    bonds = I.ring(N, 1.0)
    b = o.basis(N, K)
    lut = o.full_lut(N, b)
    rot = lambda n: ((n << 1) | (n >> (N - 1))) & ((1 << N) - 1)
    P = np.zeros((len(b), len(b)))
    for t, n in enumerate(b):
        P[lut[rot(int(n))], t] = 1.0
    H = o.dense_h(bonds, b, lut)
    np.testing.assert_allclose(P @ H, H @ P, atol=1e-14)


def test_counting_rows_match_full_hv():
    N, K = 16, 7
    bonds = I.random_graph(N, seed=11)
    b = o.basis(N, K)
    x = I.seeded_vector(len(b), 4)
    y = o.hv(bonds, b, x)
    rows = np.random.default_rng(2).integers(0, len(b), size=100)
    yr = counting.hv_rows(N, K, bonds, rows, lambda k: x[k])
    np.testing.assert_allclose(yr, y[rows], rtol=0, atol=1e-12)
