"""Python half of the FTLM oracle (TEST INFRASTRUCTURE ONLY; see oracle/__init__.py).

Wraps the C routines of ftlm_oracle.c and adds the two steps that are plain numpy:

  * ritz():   the N_L x N_L tridiagonal eigenproblem of the Lanczos matrix T,
              solved in FP64 by numpy.linalg.eigh on the dense T (Sec. 2, FTLM
              paragraph: theta_k = eigenvalues, w_k = |s_{k,1}|^2).
  * thermo(): Eq. 6-9 (Z, <H>, <H^2>, C = beta^2 (<H^2> - <H>^2), chi = g^2 beta
              <(S^z)^2>) summed over S^z sectors; sectors -M are mirrors of +M
              (Sec. 2, Model paragraph).  Exponents are shifted by the global
              minimum Ritz value E0, which cancels in every ratio.

Readings where the paper is silent (stated once here, and in the design notes):
  * breakdown:  the recurrence stops after step j when beta_j <= tau with
                tau = 100 u (3/4) sum_b |J_b|, u the unit roundoff of the storage
                type under test (2^-53 for FP64, 2^-24 for FP32).
  * field h:    H_Z = -h S^z, so Ritz values of sector M shift by -h M; with h != 0
                chi is the fluctuation form g^2 beta (<M^2> - <M>^2).
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """The compiled C half of the oracle (built on first use)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        c_i64, c_u64, c_int, c_dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        P = ctypes.c_void_p
        L.or_basis_enumerate.restype = c_i64
        L.or_basis_enumerate.argtypes = [c_int, c_int, P, c_i64]
        L.or_full_lut.restype = None
        L.or_full_lut.argtypes = [c_int, P, c_i64, P]
        L.or_index_bsearch.restype = c_i64
        L.or_index_bsearch.argtypes = [P, c_i64, c_u64]
        L.or_clt_build.restype = None
        L.or_clt_build.argtypes = [c_int, P, c_i64, P, P, c_i64]
        L.or_clt_lookup.restype = c_i64
        L.or_clt_lookup.argtypes = [P, P, c_u64]
        L.or_hv.restype = None
        L.or_hv.argtypes = [c_int, P, P, P, P, c_i64, P, P, P]
        L.or_hv_range.restype = None
        L.or_hv_range.argtypes = [c_int, P, P, P, P, c_i64, P, P, P, c_i64, c_i64]
        L.or_offdiag_terms.restype = c_i64
        L.or_offdiag_terms.argtypes = [c_int, P, P, P, c_i64]
        L.or_splitmix64_at.restype = c_u64
        L.or_splitmix64_at.argtypes = [c_u64, c_u64]
        L.or_chain_key.restype = c_u64
        L.or_chain_key.argtypes = [c_u64, c_int, c_int, ctypes.c_uint32]
        L.or_start_vector.restype = None
        L.or_start_vector.argtypes = [c_u64, c_int, c_int, ctypes.c_uint32, c_int, c_i64, P]
        L.or_lanczos.restype = c_int
        L.or_lanczos.argtypes = [c_int, P, P, P, P, c_i64, P, P, c_int, c_dbl, P, P]
        L.or_num_threads.restype = c_int
        L.or_num_threads.argtypes = []
        L.or_set_num_threads.restype = None
        L.or_set_num_threads.argtypes = [c_int]
        L.or_spin_basis_enumerate.restype = c_i64
        L.or_spin_basis_enumerate.argtypes = [c_int, c_int, c_int, P, c_i64]
        L.or_spin_hv_range.restype = None
        L.or_spin_hv_range.argtypes = [c_int, c_int, c_int, P, P, P, P, c_i64, P, P, c_i64, c_i64]
        L.or_spin_offdiag_terms.restype = c_i64
        L.or_spin_offdiag_terms.argtypes = [c_int, c_int, c_int, P, P, P, c_i64]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _bonds(bonds):
    bi, bj, J = bonds
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    return bi, bj, J


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    """Threads of the oracle's OpenMP loops from now on (n >= 1)."""
    lib().or_set_num_threads(int(n))


# ---------------------------------------------------------------- sector tables
def sector_dim(N, K):
    """D = C(N, K): dimension of the sector with K up spins (Eq. 17: A_tot = K)."""
    return math.comb(N, K) if 0 <= K <= N else 0


def basis(N, K):
    """Sorted sector basis (labels with K set bits), by brute force over 2^N."""
    D = sector_dim(N, K)
    out = np.empty(max(D, 1), dtype=np.uint64)
    got = lib().or_basis_enumerate(N, K, _p(out), D)
    assert got == D
    return out[:D]


def enumerate_count(N, K):
    """Sector dimension counted by the brute-force enumeration itself."""
    return lib().or_basis_enumerate(N, K, None, 0)


def full_lut(N, b):
    lut = np.empty(1 << N, dtype=np.int32)
    lib().or_full_lut(N, _p(b), len(b), _p(lut))
    return lut


def index_bsearch(b, label):
    return lib().or_index_bsearch(_p(b), len(b), int(label))


def clt_build(N, b):
    """CLT arrays (mask M_b, prefix C_b) of Eq. 18 over ceil(2^N / 32) blocks."""
    nblocks = -(-(1 << N) // 32)
    mask = np.empty(nblocks, dtype=np.uint32)
    prefix = np.empty(nblocks, dtype=np.uint32)
    lib().or_clt_build(N, _p(b), len(b), _p(mask), _p(prefix), nblocks)
    return mask, prefix


def clt_lookup(mask, prefix, label):
    mask = np.ascontiguousarray(mask, dtype=np.uint32)
    prefix = np.ascontiguousarray(prefix, dtype=np.uint32)
    return lib().or_clt_lookup(_p(mask), _p(prefix), int(label))


# ----------------------------------------------------------------------- H.v
def hv(bonds, b, x, lut=None):
    """y = H x on the sector (Eq. 12-14, s = 1/2), FP64."""
    bi, bj, J = _bonds(bonds)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    if lut is not None:
        lut = np.ascontiguousarray(lut, dtype=np.int32)
    lib().or_hv(len(J), _p(bi), _p(bj), _p(J), _p(b), len(b), _p(lut), _p(x), _p(y))
    return y


def hv_range(bonds, b, x, t0, t1, lut=None, out=None):
    """Rows t0 .. t1-1 of H x (Eq. 12-14, s = 1/2), FP64."""
    bi, bj, J = _bonds(bonds)
    y = np.empty(t1 - t0) if out is None else out
    if lut is not None:
        lut = np.ascontiguousarray(lut, dtype=np.int32)
    lib().or_hv_range(len(J), _p(bi), _p(bj), _p(J), _p(b), len(b), _p(lut), _p(x), _p(y),
                      int(t0), int(t1))
    return y


def offdiag_terms(bonds, b):
    bi, bj, _ = _bonds(bonds)
    return lib().or_offdiag_terms(len(bi), _p(bi), _p(bj), _p(b), len(b))


def dense_h(bonds, b, lut=None):
    """The sector Hamiltonian as a dense matrix, column t = H e_t (small D only)."""
    D = len(b)
    H = np.empty((D, D))
    e = np.zeros(D)
    for t in range(D):
        e[t] = 1.0
        H[:, t] = hv(bonds, b, e, lut)
        e[t] = 0.0
    return H


# ------------------------------------------------------------- start vectors
def splitmix64_at(key, c):
    return lib().or_splitmix64_at(int(key) & (2**64 - 1), int(c))


def chain_key(seed, N, K, r):
    return lib().or_chain_key(int(seed) & (2**64 - 1), N, K, r)


GAUSS, RADEMACHER = 0, 1


def start_vector(seed, N, K, r, dist, D=None):
    """Un-normalized start vector of chain r of sector (N, K) (see ftlm_oracle.c)."""
    if D is None:
        D = sector_dim(N, K)
    out = np.empty(D, dtype=np.float64)
    lib().or_start_vector(int(seed) & (2**64 - 1), N, K, r, dist, D, _p(out))
    return out


# ------------------------------------------------------------------- Lanczos
U64, U32 = 2.0**-53, 2.0**-24


def breakdown_tol(J, u=U64):
    """tau = 100 u (3/4) sum_b |J_b|  (reading; the paper does not say)."""
    return 100.0 * u * 0.75 * float(np.sum(np.abs(np.asarray(J, dtype=np.float64))))


def lanczos(bonds, b, r, M, tau, lut=None):
    """FP64 Lanczos from start vector r: returns (alpha[m_eff], beta[m_eff-1], m_eff)."""
    bi, bj, J = _bonds(bonds)
    r = np.ascontiguousarray(r, dtype=np.float64)
    alpha = np.zeros(max(M, 1))
    beta = np.zeros(max(M, 1))
    if lut is not None:
        lut = np.ascontiguousarray(lut, dtype=np.int32)
    m = lib().or_lanczos(len(J), _p(bi), _p(bj), _p(J), _p(b), len(b), _p(lut), _p(r), M,
                         float(tau), _p(alpha), _p(beta))
    return alpha[:m].copy(), beta[:max(m - 1, 0)].copy(), m


def ritz(alpha, beta):
    """Eigenvalues theta_k of T and weights w_k = |s_{k,1}|^2 (ascending theta)."""
    m = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    if m > 1:
        off = np.asarray(beta[: m - 1], dtype=np.float64)
        T += np.diag(off, 1) + np.diag(off, -1)
    theta, S = np.linalg.eigh(T)
    return theta, S[0, :] ** 2


# -------------------------------------------------------------------- thermo
def thermo(sectors, T, g=2.0, h=0.0, mirror=True):
    """FTLM observables on a temperature grid (Eq. 6-9).

    sectors: iterable of dicts with keys
        two_sz  2 S^z = 2M of the computed sector (M >= 0 when mirror is set),
        dim     sector dimension D_M,
        chains  list of (theta, weight) arrays, one per random vector (R = len).
    Each sector with M > 0 also stands for -M when mirror is set (same Ritz data).
    Returns dict with E, C, chi, mag (= <S^z>), Z_shifted and E0, all FP64.
    C = beta^2 Var(H) (Eq. 8 moments) and, in a field, chi = g^2 beta Var(S^z); both
    variances are evaluated as central second moments <(X - <X>)^2>.
    """
    E_list, W_list, M_list = [], [], []
    for s in sectors:
        M = s["two_sz"] / 2.0
        R = len(s["chains"])
        images = [M] if (not mirror or M == 0) else [M, -M]
        for Mi in images:
            for theta, w in s["chains"]:
                theta = np.asarray(theta, dtype=np.float64)
                w = np.asarray(w, dtype=np.float64)
                E_list.append(theta - h * Mi)
                W_list.append(w * (s["dim"] / R))
                M_list.append(np.full(len(theta), Mi))
    E = np.concatenate(E_list)
    W = np.concatenate(W_list)
    Mz = np.concatenate(M_list)
    E0 = float(np.min(E))
    out = {k: np.empty(len(T)) for k in ("E", "C", "chi", "mag", "Z_shifted")}
    for n, Tn in enumerate(T):
        beta = 1.0 / Tn
        bw = W * np.exp(-beta * (E - E0))
        Z = np.sum(bw)
        e1 = np.sum(bw * (E - E0)) / Z
        m1 = np.sum(bw * Mz) / Z
        # variances as central second moments: <(X - <X>)^2>
        varE = np.sum(bw * (E - E0 - e1) ** 2) / Z
        out["E"][n] = E0 + e1
        out["C"][n] = beta**2 * varE
        if h == 0.0:
            out["chi"][n] = g**2 * beta * np.sum(bw * Mz**2) / Z  # Eq. 9
        else:
            out["chi"][n] = g**2 * beta * np.sum(bw * (Mz - m1) ** 2) / Z
        out["mag"][n] = m1
        out["Z_shifted"][n] = Z
    out["E0"] = E0
    return out


def log_t_grid(n=200, lo=0.01, hi=10.0):
    """n log-spaced temperatures from lo to hi, both ends included."""
    return np.logspace(math.log10(lo), math.log10(hi), n)


# -------------------------------------------------------------- FTLM driver
def computed_sectors(N):
    """Up-spin counts K of the sectors with M = K - N/2 >= 0 (Sec. 2, Model)."""
    return list(range((N + 1) // 2, N + 1))


def run_ftlm(N, bonds, R, M, seed=1, dist=GAUSS, Ks=None, chains=None, u=U64, start="seeded",
         keep_coeffs=False):
    """Run the FP64 oracle FTLM over sectors Ks (default: all with M >= 0).

    start="seeded": chain r uses start_vector(seed, N, K, r, dist);
    start="unit":   R is ignored and the D unit vectors e_t are used with M = D,
                    which makes the trace exact (the exact-trace mode).
    chains: optional subset of chain indices r to run (default range(R)); the
    thermodynamic sums then average over the chains actually run.
    Returns list of sector dicts for thermo() (plus 'coeffs' when keep_coeffs).
    """
    bi, bj, J = _bonds(bonds)
    tau = breakdown_tol(J, u)
    if Ks is None:
        Ks = computed_sectors(N)
    out = []
    for K in Ks:
        b = basis(N, K)
        D = len(b)
        lut = full_lut(N, b) if N <= 26 else None
        res, coeffs = [], []
        if start == "unit":
            Rk, Mk = D, D
            rs = range(D)
        else:
            Rk, Mk = R, M
            rs = range(R) if chains is None else chains
        for r in rs:
            if start == "unit":
                v = np.zeros(D)
                v[r] = 1.0
            else:
                v = start_vector(seed, N, K, r, dist, D)
            a, bt, m = lanczos((bi, bj, J), b, v, Mk, tau, lut)
            res.append(ritz(a, bt))
            coeffs.append((a, bt, m))
        d = {"two_sz": 2 * K - N, "dim": D, "chains": res, "R": Rk}
        if keep_coeffs:
            d["coeffs"] = coeffs
        out.append(d)
    return out
