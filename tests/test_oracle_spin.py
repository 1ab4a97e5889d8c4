"""Pins of the general-spin oracle (oracle/spin.py) against the paper and against
mathematics it does not share code with.

  * Table 1: D_0 and N_nz of the s = 1/2 .. 3 icosahedron, M = 0 (Eq. 15, Eq. 10),
    and for s = 1, 3/2 the same counts from the enumerated basis and the H.v rows.
  * Table 2 (s = 2) and Table 4 (s = 3/2, 2): the printed memory budgets from the
    same D_0 and N_nz.
  * Brute-force counting of the base-d labels vs the Eq. 15 recursion.
  * Exact diagonalization: the sector blocks of H built from Kronecker products of
    the spin-s matrices (numpy) have the spectra of the oracle's H.v.
  * The two-spin closed form E = J/2 [S(S+1) - 2 s(s+1)], multiplicity 2S + 1.
  * s = 1/2 through the spin-s code equals the spin-1/2 oracle.
  * FTLM in exact-trace mode equals the partition function from ED.
"""
import math

import numpy as np
import pytest

import oracle as o
from oracle import spin
from paper_2605_26261_gb300 import inputs
from tests.conftest import golden


def test_table1_dimensions_and_nnz():
    g = golden("table1_spin_s.txt")
    N, nb = int(g["N"]), int(g["n_bonds"])
    assert nb == len(inputs.icosahedron()[2])
    for two_s, D0, nnz, mem in zip(g["two_s"].split(","), g["D0"].split(","), g["N_nz"].split(","),
                                   g["memory"].split(",")):
        two_s, D0, nnz = int(two_s), int(D0), int(nnz)
        A = spin.sector_A(N, two_s, 0)
        assert spin.dim(N, two_s, A) == D0
        assert spin.nnz(N, two_s, A, nb) == nnz
        # footnote a: 16 N_nz + 8 (D0 + 1) bytes, at the printed precision
        value, unit = mem.split()
        scale = {"MB": 1e6, "GB": 1e9}[unit]
        digits = len(value.split(".")[1]) if "." in value else 0
        assert round((16 * nnz + 8 * (D0 + 1)) / scale, digits) == float(value)


@pytest.mark.parametrize("two_s", [2, 3])
def test_table1_counts_from_enumeration_and_rows(two_s):
    # the sector enumerated label by label, and N_nz counted from the H.v rows
    N, bonds = 12, inputs.icosahedron()
    A = spin.sector_A(N, two_s, 0)
    b = spin.basis(N, two_s, A)
    assert len(b) == spin.dim(N, two_s, A)
    assert np.all(np.diff(b.astype(np.int64)) > 0)
    assert len(b) + spin.offdiag_terms(N, two_s, bonds, b) == spin.nnz(N, two_s, A, len(bonds[2]))


@pytest.mark.parametrize("N,two_s", [(5, 2), (4, 3), (3, 4), (6, 2), (3, 6)])
def test_dimensions_by_brute_force(N, two_s):
    counts = [spin.enumerate_count(N, two_s, A) for A in range(N * two_s + 1)]
    assert counts == [spin.dim(N, two_s, A) for A in range(N * two_s + 1)]
    assert sum(counts) == (two_s + 1) ** N
    assert counts == counts[::-1]  # A <-> 2sN - A (spin flip)


def spin_matrices(two_s):
    """S^z, S^+, S^- in the basis a = m + s = 0 .. 2s (textbook angular momentum)."""
    s = two_s / 2
    d = two_s + 1
    m = np.arange(d) - s
    Sz = np.diag(m)
    Sp = np.zeros((d, d))
    for a in range(d - 1):  # S^+ |m> = sqrt(s(s+1) - m(m+1)) |m+1>
        Sp[a + 1, a] = math.sqrt(s * (s + 1) - m[a] * (m[a] + 1))
    return Sz, Sp, Sp.T


def kron_h(N, two_s, bonds):
    """Full H = sum_b J_b S_i . S_j on d^N states, site k the k-th least significant
    base-d digit of the state index."""
    Sz, Sp, Sm = spin_matrices(two_s)
    d = two_s + 1

    def site_op(op, k):
        mats = [np.eye(d)] * N
        mats[N - 1 - k] = op  # kron's first factor is the most significant digit
        out = mats[0]
        for m_ in mats[1:]:
            out = np.kron(out, m_)
        return out

    H = np.zeros((d**N, d**N))
    for i, j, J in zip(*bonds):
        H += J * (site_op(Sz, i) @ site_op(Sz, j)
                  + 0.5 * (site_op(Sp, i) @ site_op(Sm, j) + site_op(Sm, i) @ site_op(Sp, j)))
    return H


@pytest.mark.parametrize("N,two_s,seed", [(4, 2, 1), (3, 3, 2), (5, 2, 3), (3, 4, 4), (3, 5, 5), (3, 7, 6)])
def test_sector_spectra_match_kronecker_ed(N, two_s, seed):
    rng = np.random.default_rng(seed)
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
    bonds = (np.array([p[0] for p in pairs], dtype=np.int32), np.array([p[1] for p in pairs], dtype=np.int32),
             rng.uniform(-1.0, 1.5, size=len(pairs)))
    H = kron_h(N, two_s, bonds)
    d = two_s + 1
    digits = np.array([[(n // d**k) % d for k in range(N)] for n in range(d**N)])
    for A in range(N * two_s + 1):
        idx = np.nonzero(digits.sum(1) == A)[0]  # ascending labels of the sector
        b = spin.basis(N, two_s, A)
        assert np.array_equal(b.astype(np.int64), idx)
        Hs = spin.dense_h(N, two_s, bonds, b)
        np.testing.assert_allclose(Hs, H[np.ix_(idx, idx)], atol=1e-12)


@pytest.mark.parametrize("two_s", [2, 3, 4, 5, 6, 7])
def test_two_spin_closed_form(two_s):
    s, J = two_s / 2, 0.8
    bonds = (np.array([0], dtype=np.int32), np.array([1], dtype=np.int32), np.array([J]))
    levels = []
    for A in range(2 * two_s + 1):
        b = spin.basis(2, two_s, A)
        levels += list(np.linalg.eigvalsh(spin.dense_h(2, two_s, bonds, b)))
    want = []
    for S2 in range(0, 2 * two_s + 1, 2):  # total S = 0 .. 2s
        S = S2 / 2
        want += [J / 2 * (S * (S + 1) - 2 * s * (s + 1))] * int(2 * S + 1)
    np.testing.assert_allclose(np.sort(levels), np.sort(want), atol=1e-12)


def test_spin_half_through_spin_code():
    N = 10
    bonds = inputs.random_graph(N, seed=4)
    for K in (5, 7):
        b = o.basis(N, K)
        assert np.array_equal(spin.basis(N, 1, K), b)
        x = inputs.seeded_vector(len(b), 3)
        assert np.array_equal(spin.hv(N, 1, bonds, b, x), o.hv(bonds, b, x))
        assert spin.nnz(N, 1, K, len(bonds[2])) == len(b) + o.offdiag_terms(bonds, b)


def test_hermitian_and_spin_flip():
    N, two_s = 6, 3
    bonds = inputs.random_graph(N, seed=8, dmin=2, dmax=3)
    rng = np.random.default_rng(0)
    for A in (4, 9):
        b = spin.basis(N, two_s, A)
        u, v = rng.standard_normal((2, len(b)))
        assert abs(u @ spin.hv(N, two_s, bonds, b, v) - spin.hv(N, two_s, bonds, b, u) @ v) < 1e-10
        flip = spin.basis(N, two_s, N * two_s - A)
        np.testing.assert_allclose(np.linalg.eigvalsh(spin.dense_h(N, two_s, bonds, b)),
                                   np.linalg.eigvalsh(spin.dense_h(N, two_s, bonds, flip)), atol=1e-10)


@pytest.mark.parametrize("N,two_s", [(4, 2), (3, 3)])
def test_exact_trace_mode_matches_ed(N, two_s):
    bonds = inputs.ring(N, J=1.0) if N > 3 else inputs.random_graph(3, seed=1, dmin=2, dmax=2)
    T = np.array([0.3, 1.0, 4.0])
    res = spin.run_ftlm(N, two_s, bonds, 0, 0, start="unit")
    got = o.thermo(res, T, mirror=True)
    ev_all, Mz_all = [], []
    for two_sz in range(-N * two_s, N * two_s + 1, 2):
        b = spin.basis(N, two_s, spin.sector_A(N, two_s, two_sz))
        ev = np.linalg.eigvalsh(spin.dense_h(N, two_s, bonds, b))
        ev_all += list(ev)
        Mz_all += [two_sz / 2] * len(ev)
    ev_all, Mz_all = np.array(ev_all), np.array(Mz_all)
    for n, t in enumerate(T):
        w = np.exp(-(ev_all - ev_all.min()) / t)
        E = np.sum(w * ev_all) / w.sum()
        C = (np.sum(w * ev_all**2) / w.sum() - E**2) / t**2
        chi = 4.0 / t * np.sum(w * Mz_all**2) / w.sum()
        np.testing.assert_allclose([got["E"][n], got["C"][n], got["chi"][n]], [E, C, chi], rtol=1e-10)


def test_lanczos_quadrature_moments():
    N, two_s = 6, 2
    bonds = inputs.random_graph(N, seed=5, dmin=2, dmax=4)
    A = spin.sector_A(N, two_s, 0)
    b = spin.basis(N, two_s, A)
    r = spin.start_vector(3, N, two_s, A, 0, o.GAUSS, len(b))
    a, bt, m = spin.lanczos(N, two_s, bonds, b, r, 20, spin.tau_of(bonds[2], two_s))
    th, w = o.ritz(a, bt)
    q = r / np.linalg.norm(r)
    Hq = spin.hv(N, two_s, bonds, b, q)
    assert abs(w.sum() - 1) < 1e-12
    assert abs(np.sum(w * th) - q @ Hq) < 1e-10
    assert abs(np.sum(w * th**2) - Hq @ Hq) < 1e-9


def test_table2_and_table4_memory_budgets():
    """The oracle's sector dimension (Eq. 15) and nonzero count (Eq. 10) reproduce
    the memory figures of Table 2 (s = 2) and the icosahedron rows of Table 4, each
    at the precision printed."""
    g = golden("table2_table4_memory.txt")
    N, nb = 12, len(inputs.icosahedron()[2])
    mb = lambda nbytes: nbytes / 1e6

    def close(value, printed):
        digits = len(printed.split(".")[1]) if "." in printed else 0
        return round(value, digits) == float(printed)

    two_s = int(g["t2_two_s"])
    d = two_s + 1
    A = spin.sector_A(N, two_s, 0)
    D0, nnz = spin.dim(N, two_s, A), spin.nnz(N, two_s, A, nb)
    parts = {
        "t2_cs_hamiltonian": mb(16 * nnz + 8 * (D0 + 1)),
        "t2_full_lookup": mb(4 * d**N),
        "t2_clt": mb(8 * -(-(d**N) // 32)),
        "t2_basis": mb(4 * D0),
        "t2_work_fp64": mb(3 * 8 * D0),
        "t2_work_fp32": mb(3 * 4 * D0),
    }
    for k, v in parts.items():
        assert close(v, g[k]), (k, v)
    # the column sums add the printed (rounded) entries
    r = {k: round(v) for k, v in parts.items()}
    assert r["t2_cs_hamiltonian"] + r["t2_work_fp64"] == int(g["t2_sum_cs"])
    assert r["t2_full_lookup"] + r["t2_basis"] + r["t2_work_fp64"] == int(g["t2_sum_full"])
    assert r["t2_clt"] + r["t2_basis"] + r["t2_work_fp64"] == int(g["t2_sum_clt"])

    cols = [g[k].split(",") for k in ("t4_two_s", "t4_clt", "t4_basis", "t4_vectors_b4", "t4_total")]
    for two_s, clt, basis, vec, total in zip(*cols):
        two_s = int(two_s)
        d = two_s + 1
        D0 = spin.dim(N, two_s, spin.sector_A(N, two_s, 0))
        c, bsz, v = mb(8 * -(-(d**N) // 32)), mb(4 * D0), mb(3 * 4 * D0 * 4)
        assert close(c, clt) and close(bsz, basis), (two_s, c, bsz)
        # the vectors column is printed to about three figures (941.3 MB as 940)
        assert close(v, vec) or abs(v - float(vec)) <= 2e-3 * float(vec), (two_s, v)
        # "≈" totals: within the last printed digit of the largest entry
        assert abs(c + bsz + v - float(total)) <= 0.01 * float(total), (two_s, c + bsz + v)
