"""Pins for the oracle's sector tables: basis, index maps, CLT arrays (CPU only).

Each check compares the oracle with something other than itself: binomial
coefficients, brute-force counts, the paper's worked CLT example and printed
memory figures, and Table 1's nonzero count.
"""
import math

import numpy as np
import pytest

import oracle as o
from oracle import counting
from paper_2605_26261_gb300 import inputs as I
from tests.conftest import golden


@pytest.mark.parametrize("N", [1, 2, 5, 8, 13, 16])
def test_sector_dims_sum_to_full_space(N):
    # Eq. 17 sectors partition the 2^N labels; each has C(N, K) states.
    dims = [o.enumerate_count(N, K) for K in range(N + 1)]
    assert dims == [math.comb(N, K) for K in range(N + 1)]
    assert sum(dims) == 2**N


@pytest.mark.parametrize("N,K", [(1, 0), (1, 1), (6, 3), (10, 4), (16, 8), (16, 16)])
def test_basis_sorted_and_in_sector(N, K):
    b = o.basis(N, K)
    assert len(b) == math.comb(N, K)
    assert np.all(np.diff(b.astype(np.int64)) > 0)
    assert all(bin(int(n)).count("1") == K for n in b)
    assert int(b[0]) == (1 << K) - 1  # smallest label: K lowest bits set
    assert int(b[-1]) == ((1 << K) - 1) << (N - K)  # largest: K highest bits set


@pytest.mark.parametrize("N,K", [(8, 4), (12, 5), (14, 7)])
def test_lut_bsearch_counting_agree(N, K):
    b = o.basis(N, K)
    lut = o.full_lut(N, b)
    rng = np.random.default_rng(0)
    for n in rng.integers(0, 1 << N, size=400):
        n = int(n)
        ref = int(lut[n])
        assert o.index_bsearch(b, n) == ref
        assert counting.index_of(N, K, n) == ref
    for t in range(len(b)):
        assert lut[b[t]] == t
    for t in rng.integers(0, len(b), size=200):
        assert counting.label_of(N, K, int(t)) == int(b[t])
    assert np.count_nonzero(lut >= 0) == len(b)


def test_counting_large_sector_endpoints():
    # Smallest / largest labels at N = 34, K = 17 have indices 0 and D - 1.
    N, K = 34, 17
    D = math.comb(N, K)
    assert counting.index_of(N, K, (1 << K) - 1) == 0
    assert counting.index_of(N, K, ((1 << K) - 1) << (N - K)) == D - 1
    for t in (0, 1, 12345, D // 2, D - 2, D - 1):
        assert counting.index_of(N, K, counting.label_of(N, K, t)) == t


def test_clt_worked_example():
    g = golden("clt_worked_example.txt")
    offs = [int(v) for v in g["offsets_in_block"].split(",")]
    bidx, Cb_before = 3, 7  # block 3, preceded by 7 in-sector labels
    labels = np.array(sorted(list(range(7)) + [32 * bidx + k for k in offs]), dtype=np.uint64)
    # The example's occupancy is not a Heisenberg sector, so build the arrays of
    # Eq. 18 over a 7-bit label space from this label set directly.
    mask, prefix = o.clt_build(7, labels)
    assert mask[bidx] == int(g["mask_binary"], 2)
    assert prefix[bidx] == Cb_before
    j = int(g["lookup_offset"])
    assert o.clt_lookup(mask, prefix, 32 * bidx + j) == Cb_before + int(g["lookup_local_rank"])
    assert o.clt_lookup(mask, prefix, 32 * bidx + 1) == -1  # occupancy bit clear


@pytest.mark.parametrize("N,K", [(5, 2), (10, 5), (16, 7), (16, 8)])
def test_clt_lookup_equals_index(N, K):
    b = o.basis(N, K)
    mask, prefix = o.clt_build(N, b)
    assert len(mask) == -(-(1 << N) // 32)
    lut = o.full_lut(N, b)
    for n in range(1 << N):
        assert o.clt_lookup(mask, prefix, n) == lut[n]


def test_clt_and_basis_memory_figures():
    g = golden("memory_figures.txt")
    N = int(g["N"])
    D0 = math.comb(N, N // 2)
    clt_bytes = 8 * -(-(1 << N) // 32)  # Eq. 21
    assert round(clt_bytes / 1e6) == int(g["clt_mb"])
    assert round(4 * D0 / 1e6) == int(g["basis_mb"])
    # Table 4 prints the vector budget with D_0 rounded to 1.55e8 (7440 vs 7446).
    assert abs(3 * 4 * D0 * 4 / 1e6 - int(g["vectors_mb_b4"])) < 1e-3 * int(g["vectors_mb_b4"])
    assert 4 / (8 / 32) == int(g["full_over_clt"])


def test_table1_nonzero_count():
    g = golden("table1_icosahedron.txt")
    bonds = I.icosahedron()
    N, K = int(g["N"]), int(g["K"])
    assert len(bonds[0]) == int(g["n_bonds"])
    b = o.basis(N, K)
    assert len(b) == int(g["D0"])
    nnz = len(b) + o.offdiag_terms(bonds, b)
    assert nnz == int(g["N_nz"])
    # Eq. 10 at s = 1/2: D + 2 N_B C(N-2, K-1).
    assert nnz == len(b) + 2 * len(bonds[0]) * math.comb(N - 2, K - 1)
    # The oracle's H.v applies exactly those nonzeros (diagonal + ladder terms).
    H = o.dense_h(bonds, b)
    assert np.count_nonzero(H - np.diag(np.diag(H))) + len(b) == int(g["N_nz"])
