"""General local spin s for the oracle (TEST INFRASTRUCTURE ONLY).

Sec. 2 of the paper states the method for any s: labels with base-d digits,
d = 2s + 1 (Eq. 11), sectors by digit sum A = N s + M (Eq. 17), the Heisenberg row
of Eq. 12 with the ladder coefficients of Eq. 13-14, sector dimensions by the
recursion of Eq. 15 and the number of stored entries N_nz of Eq. 10.  Everything
here is written from those definitions:

  dim(N, two_s, A)           Eq. 15, exact integers
  nnz(N, two_s, A, n_bonds)  Eq. 10, exact integers
  basis(N, two_s, A)         brute force over all d^N labels (C)
  hv(...), offdiag_terms     Eq. 12-14 row by row, sources by binary search (C)
  lanczos(...)               the recurrence of ftlm.lanczos (Paige order, FP64)
  run_ftlm(...)              every sector with M >= 0, R chains, for ftlm.thermo

Spins are passed as two_s = 2s (an integer >= 1).  Start vectors reuse the
spin-1/2 generator with the sector tag (N | two_s << 8, A) in place of (N, K) when
two_s >= 2, so spin-1/2 chains keep their keys.
"""
import numpy as np

from .ftlm import GAUSS, U64, _bonds, _p, breakdown_tol, lib, ritz


def dim(N, two_s, A):
    """D(N, A) of Eq. 15: digit strings of length N, digits 0..2s, digit sum A."""
    if A < 0 or A > N * two_s:
        return 0
    row = [1]  # D(0, .)
    for _ in range(N):
        nxt = [0] * (len(row) + two_s)
        for a, v in enumerate(row):
            for q in range(two_s + 1):
                nxt[a + q] += v
        row = nxt
    return row[A]


def sector_A(N, two_s, two_sz):
    """Digit sum of the sector with 2 S^z = two_sz (Eq. 17: A = N s + M)."""
    twice = N * two_s + two_sz
    if twice % 2:
        raise ValueError("two_sz must have the parity of N * two_s")
    return twice // 2


def nnz(N, two_s, A, n_bonds):
    """N_nz of Eq. 10: D_A(N) diagonal entries plus, per bond and per ladder term,
    the sector states whose two bond sites admit the move (source digits
    a_i in 0..2s-1, a_j in 1..2s for s_i^+ s_j^-, the mirror image for the other
    term), counted on the remaining N - 2 sites."""
    off = 0
    for ai in range(0, two_s):
        for aj in range(1, two_s + 1):
            off += dim(N - 2, two_s, A - ai - aj)
    return dim(N, two_s, A) + 2 * n_bonds * off


def enumerate_count(N, two_s, A):
    return lib().or_spin_basis_enumerate(N, two_s, A, None, 0)


def basis(N, two_s, A):
    D = dim(N, two_s, A)
    out = np.empty(max(D, 1), dtype=np.uint64)
    got = lib().or_spin_basis_enumerate(N, two_s, A, _p(out), D)
    assert got == D
    return out[:D]


def hv_range(N, two_s, bonds, b, x, t0, t1, out=None):
    bi, bj, J = _bonds(bonds)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(t1 - t0) if out is None else out
    lib().or_spin_hv_range(N, two_s, len(J), _p(bi), _p(bj), _p(J), _p(b), len(b), _p(x), _p(y),
                           int(t0), int(t1))
    return y


def hv(N, two_s, bonds, b, x):
    return hv_range(N, two_s, bonds, b, x, 0, len(b))


def offdiag_terms(N, two_s, bonds, b):
    bi, bj, _ = _bonds(bonds)
    return lib().or_spin_offdiag_terms(N, two_s, len(bi), _p(bi), _p(bj), _p(b), len(b))


def dense_h(N, two_s, bonds, b):
    D = len(b)
    H = np.empty((D, D))
    e = np.zeros(D)
    for t in range(D):
        e[t] = 1.0
        H[:, t] = hv(N, two_s, bonds, b, e)
        e[t] = 0.0
    return H


def key_tag(N, two_s):
    """The N argument of the chain key for spin s (see the module docstring)."""
    return N if two_s == 1 else (N | (two_s << 8))


def start_vector(seed, N, two_s, A, r, dist, D):
    out = np.empty(D, dtype=np.float64)
    lib().or_start_vector(int(seed) & (2**64 - 1), key_tag(N, two_s), A, r, dist, D, _p(out))
    return out


def tau_of(J, two_s, u=U64):
    """Breakdown threshold 100 u ||H||_bd, ||H||_bd = s (s + 1) sum_b |J_b|: the
    eigenvalues of S_i . S_j are [S (S + 1) - 2 s (s + 1)] / 2 for S = 0 .. 2s, so
    its norm is s (s + 1) (3/4 at s = 1/2, the bound of ftlm.breakdown_tol)."""
    s = 0.5 * two_s
    return breakdown_tol(J, u) * (s * (s + 1.0)) / 0.75


def lanczos(N, two_s, bonds, b, r, M, tau):
    """Paige-order Lanczos in FP64 (the recurrence of ftlm.lanczos) with the spin-s
    H.v; returns (alpha, beta, m_eff)."""
    D = len(b)
    m_max = min(M, D)
    q = np.asarray(r, dtype=np.float64) / np.sqrt(np.sum(np.asarray(r, dtype=np.float64) ** 2))
    qp = np.zeros(D)
    beta_prev = 0.0
    alpha, beta = [], []
    for j in range(1, m_max + 1):
        y = hv(N, two_s, bonds, b, q) - beta_prev * qp
        a = float(np.sum(q * y))
        alpha.append(a)
        w = y - a * q
        if j == m_max:
            break
        bj = float(np.sqrt(np.sum(w * w)))
        if bj <= tau:
            break
        beta.append(bj)
        qp, q, beta_prev = q, w / bj, bj
    return np.array(alpha), np.array(beta), len(alpha)


def run_ftlm(N, two_s, bonds, R, M, seed=1, dist=GAUSS, u=U64, start="seeded"):
    """Every sector with M >= 0 (mirrored in ftlm.thermo), R chains of M steps;
    start="unit" uses the D unit vectors with M = D (exact trace)."""
    _, _, J = _bonds(bonds)
    tau = tau_of(J, two_s, u)
    out = []
    for two_sz in range((N * two_s) % 2, N * two_s + 1, 2):
        A = sector_A(N, two_s, two_sz)
        b = basis(N, two_s, A)
        D = len(b)
        res = []
        if start == "unit":
            for r in range(D):
                v = np.zeros(D)
                v[r] = 1.0
                a, bt, m = lanczos(N, two_s, bonds, b, v, D, tau)
                res.append(ritz(a, bt))
            Rk = D
        else:
            for r in range(R):
                a, bt, m = lanczos(N, two_s, bonds, b, start_vector(seed, N, two_s, A, r, dist, D), M, tau)
                res.append(ritz(a, bt))
            Rk = R
        out.append({"two_sz": two_sz, "dim": D, "chains": res, "R": Rk})
    return out
