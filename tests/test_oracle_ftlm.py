"""Pins for the oracle's Lanczos, Ritz step and thermodynamic sums (CPU only).

References: dense exact diagonalization of the Kronecker-product Hamiltonian
(thermodynamics from all eigenvalues, by definition), the two-spin closed form,
the exact-trace mode (R = D unit start vectors, M = D steps), quadrature moment
identities of the tridiagonal T, beta -> 0 limits and high-temperature series.
"""
import math

import numpy as np
import pytest

import oracle as o
from paper_2605_26261_gb300 import inputs as I
from tests.test_oracle_hv import kron_hamiltonian, sector_block


def ed_thermo(N, bonds, T, g=2.0, h=0.0):
    """Thermodynamics from every eigenvalue of every sector (no mirroring)."""
    Hfull = kron_hamiltonian(N, bonds)
    E, Mz = [], []
    for K in range(N + 1):
        ev = np.linalg.eigvalsh(sector_block(Hfull, N, K))
        M = K - N / 2
        E.append(ev - h * M)
        Mz.append(np.full(len(ev), M))
    E, Mz = np.concatenate(E), np.concatenate(Mz)
    E0 = E.min()
    out = {k: np.empty(len(T)) for k in ("E", "C", "chi", "mag")}
    for n, Tn in enumerate(T):
        b = 1.0 / Tn
        p = np.exp(-b * (E - E0))
        Z = p.sum()
        e1 = (p * E).sum() / Z
        e2 = (p * E**2).sum() / Z
        m1 = (p * Mz).sum() / Z
        m2 = (p * Mz**2).sum() / Z
        out["E"][n] = e1
        out["C"][n] = b * b * (e2 - e1 * e1)
        out["chi"][n] = g * g * b * (m2 - m1 * m1)
        out["mag"][n] = m1
    return out


T_GRID = I.log_t_grid(60, 0.05, 20.0)


@pytest.mark.parametrize("name,N,bonds,h", [
    ("ring8", 8, I.ring(8), 0.0),
    ("random9", 9, I.random_graph(9, seed=7), 0.0),
    ("ladder8_field", 8, I.ladder(8, 0.4, 1.1), 0.8),
])
def test_exact_trace_mode_equals_ed(name, N, bonds, h):
    # R = D orthonormal start vectors e_t and M = D make the estimator exact.
    secs = o.run_ftlm(N, bonds, R=0, M=0, start="unit")
    th = o.thermo(secs, T_GRID, g=2.0, h=h)
    ed = ed_thermo(N, bonds, T_GRID, h=h)
    for k in ("E", "C", "chi", "mag"):
        if k == "mag" and h == 0.0:
            assert np.max(np.abs(th[k])) < 1e-12
            continue
        np.testing.assert_allclose(th[k], ed[k], rtol=1e-9, atol=1e-12 * np.max(np.abs(ed[k])))


def test_dimer_closed_form():
    J, g = 1.3, 2.0
    secs = o.run_ftlm(2, I.dimer(J), R=0, M=0, start="unit")
    T = np.array([0.05, 0.3, 1.0, 4.0, 50.0])
    th = o.thermo(secs, T, g=g)
    b = 1.0 / T
    Z = np.exp(0.75 * b * J) + 3 * np.exp(-0.25 * b * J)
    E = (-0.75 * J * np.exp(0.75 * b * J) + 3 * 0.25 * J * np.exp(-0.25 * b * J)) / Z
    # two levels J apart: Var(H) = J^2 p (1 - p), p = triplet probability
    p = 3 * np.exp(-0.25 * b * J) / Z
    C = b**2 * J**2 * p * (1 - p)
    chi = g**2 * b * 2 * np.exp(-0.25 * b * J) / Z
    np.testing.assert_allclose(th["E"], E, rtol=1e-12)
    np.testing.assert_allclose(th["C"], C, rtol=1e-10)
    np.testing.assert_allclose(th["chi"], chi, rtol=1e-12)


def test_mirror_equals_explicit_negative_sectors():
    # Sectors +M and -M have identical spectra (Sec. 2, Model): mirroring the
    # computed M >= 0 sectors equals computing every sector explicitly.
    N, bonds = 9, I.random_graph(9, seed=2)
    T = I.log_t_grid(20, 0.1, 10.0)
    mir = o.thermo(o.run_ftlm(N, bonds, R=0, M=0, start="unit"), T)
    allK = o.run_ftlm(N, bonds, R=0, M=0, start="unit", Ks=range(N + 1))
    full = o.thermo(allK, T, mirror=False)
    for k in ("E", "C", "chi"):
        np.testing.assert_allclose(mir[k], full[k], rtol=1e-10)


def test_quadrature_moments_and_weight_sum():
    # sum_k w_k = 1 (Sec. 2), sum w theta = alpha_1 = <r|H|r>,
    # sum w theta^2 = alpha_1^2 + beta_1^2 = ||H r||^2 (first row of T and T^2).
    N, K = 14, 7
    bonds = I.random_graph(N, seed=9)
    b = o.basis(N, K)
    lut = o.full_lut(N, b)
    r = o.start_vector(1, N, K, 0, o.GAUSS, len(b))
    a, bt, m = o.lanczos(bonds, b, r, 60, o.breakdown_tol(bonds[2]), lut)
    th, w = o.ritz(a, bt)
    q = r / np.linalg.norm(r)
    Hq = o.hv(bonds, b, q, lut)
    assert m == 60
    assert abs(w.sum() - 1.0) < 1e-13
    assert abs((w * th).sum() - a[0]) < 1e-12
    assert abs(a[0] - q @ Hq) < 1e-12
    assert abs((w * th**2).sum() - (a[0] ** 2 + bt[0] ** 2)) < 1e-11
    assert abs((w * th**2).sum() - Hq @ Hq) < 1e-11


def test_lanczos_quadrature_matches_dense_functions():
    # With M at least the Krylov dimension, sum_k w_k f(theta_k) = <r|f(H)|r>.
    N, K = 10, 5
    bonds = I.random_graph(N, seed=4)
    b = o.basis(N, K)
    H = sector_block(kron_hamiltonian(N, bonds), N, K)
    ev, V = np.linalg.eigh(H)
    r = o.start_vector(3, N, K, 1, o.RADEMACHER, len(b))
    q = r / np.linalg.norm(r)
    a, bt, m = o.lanczos(bonds, b, r, len(b), o.breakdown_tol(bonds[2]))
    th, w = o.ritz(a, bt)
    c2 = (V.T @ q) ** 2
    for beta in (0.1, 1.0, 5.0):
        np.testing.assert_allclose((w * np.exp(-beta * th)).sum(),
                                   (c2 * np.exp(-beta * ev)).sum(), rtol=1e-10)
    assert m <= len(b)


def test_breakdown_stops_at_krylov_dimension():
    # One down spin on a ring of 12: the magnon levels depend on cos k, so they are
    # two-fold degenerate except k = 0 and pi; a random start vector spans a
    # 7-dimensional Krylov space and the recurrence must stop there.
    N = 12
    bonds = I.ring(N)
    b = o.basis(N, N - 1)
    r = o.start_vector(5, N, N - 1, 0, o.GAUSS, len(b))
    a, bt, m = o.lanczos(bonds, b, r, 12, o.breakdown_tol(bonds[2]))
    assert m == 7
    th, w = o.ritz(a, bt)
    ev = np.unique(np.round(np.linalg.eigvalsh(o.dense_h(bonds, b)), 10))
    np.testing.assert_allclose(np.sort(th), ev, atol=1e-10)


def test_beta_zero_partition_function_counts_states():
    # Z(beta = 0) = sum_M D_M = 2^N for any start vectors (weights sum to one).
    N = 12
    bonds = I.ring(N)
    secs = o.run_ftlm(N, bonds, R=3, M=20, seed=8)
    th = o.thermo(secs, np.array([np.inf]))
    assert abs(th["Z_shifted"][0] - 2**N) < 1e-9 * 2**N


def test_high_temperature_series():
    # C T^2 -> (3/16) sum J^2, chi T -> g^2 N / 4, E T -> -(3/16) sum J^2.
    N = 10
    bonds = I.random_graph(N, seed=12)
    J2 = float(np.sum(bonds[2] ** 2))
    secs = o.run_ftlm(N, bonds, R=0, M=0, start="unit")
    T = np.array([300.0])
    th = o.thermo(secs, T)
    assert abs(th["C"][0] * T[0] ** 2 / (3 / 16 * J2) - 1) < 1e-2
    assert abs(th["chi"][0] * T[0] / (4 * N / 4) - 1) < 1e-2
    assert abs(th["E"][0] * T[0] / (-3 / 16 * J2) - 1) < 1e-2


def test_stochastic_estimate_within_spread_of_ed():
    # FTLM with R random vectors scatters around the exact result with a spread
    # that falls like 1/sqrt(R) (Sec. 2, Eq. 2-3); check |mean - ED| < 4 sigma/sqrt(Ns).
    N = 12
    bonds = I.ring(N)
    T = np.array([0.3, 1.0, 3.0])
    ed = ed_thermo(N, bonds, T)
    runs = [o.thermo(o.run_ftlm(N, bonds, R=4, M=40, seed=s), T) for s in range(8)]
    for k in ("C", "chi"):
        v = np.array([r[k] for r in runs])
        mean, sig = v.mean(0), v.std(0)
        assert np.all(np.abs(mean - ed[k]) < 4 * sig / math.sqrt(len(runs)) + 1e-12)
