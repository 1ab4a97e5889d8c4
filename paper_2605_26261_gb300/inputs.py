"""Seeded synthetic inputs: cluster graphs, couplings, temperature grids, test vectors.

This module holds none of the method's arithmetic.  It only builds the inputs a
user hands to the library (a bond list with couplings J_ij, a temperature grid)
and seeded test vectors.  It is shared by the CUDA path's tests and the oracle's
tests, and imports neither.

Bond lists are returned as (bi, bj, J): int32 site pairs with bi < bj and FP64
couplings, each unordered pair at most once.
"""
import itertools
import math

import numpy as np


def _pack(edges):
    edges = sorted((min(i, j), max(i, j), float(J)) for i, j, J in edges)
    seen = set()
    for i, j, _ in edges:
        if i == j or (i, j) in seen:
            raise ValueError(f"bad or duplicate bond {(i, j)}")
        seen.add((i, j))
    bi = np.array([e[0] for e in edges], dtype=np.int32)
    bj = np.array([e[1] for e in edges], dtype=np.int32)
    J = np.array([e[2] for e in edges], dtype=np.float64)
    return bi, bj, J


def dimer(J=1.0):
    return _pack([(0, 1, J)])


def ring(N, J=1.0):
    """Periodic chain: bonds (k, k+1 mod N)."""
    if N == 2:
        return dimer(J)
    return _pack([(k, (k + 1) % N, J) for k in range(N)])


def square_j1j2(Lx=4, Ly=6, J1=1.0, J2=0.5):
    """Periodic Lx x Ly square lattice, site (x, y) -> Lx*y + x; J1 on the nearest-
    neighbour bonds, J2 on both diagonals (x+1, y+1) and (x+1, y-1)."""
    s = lambda x, y: Lx * (y % Ly) + (x % Lx)
    e = []
    for y in range(Ly):
        for x in range(Lx):
            e.append((s(x, y), s(x + 1, y), J1))
            e.append((s(x, y), s(x, y + 1), J1))
            e.append((s(x, y), s(x + 1, y + 1), J2))
            e.append((s(x, y), s(x + 1, y - 1), J2))
    return _pack(e)


def _icosahedron_vertices():
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a, b in itertools.product((-1.0, 1.0), (-phi, phi)):
        base = (0.0, a, b)
        for c in range(3):
            v.append(tuple(base[(k - c) % 3] for k in range(3)))
    return sorted(v)


def _icosahedron_edges():
    v = _icosahedron_vertices()
    e = []
    for i in range(len(v)):
        for j in range(i + 1, len(v)):
            d = math.dist(v[i], v[j])
            if abs(d - 2.0) < 1e-9:
                e.append((i, j))
    return e


def icosahedron(J=1.0):
    """12 vertices: cyclic permutations of (0, +-1, +-phi), sorted; 30 edges of
    length 2."""
    return _pack([(i, j, J) for i, j in _icosahedron_edges()])


def icosidodecahedron(J=1.0):
    """30 sites at the edge midpoints of the icosahedron (sites numbered by the
    sorted endpoint pairs of the edges); a bond joins two edges of a common
    triangular face: 20 faces x 3 = 60 bonds, 4-regular."""
    edges = _icosahedron_edges()
    idx = {e: k for k, e in enumerate(edges)}
    adj = {i: set() for i in range(12)}
    for i, j in edges:
        adj[i].add(j)
        adj[j].add(i)
    faces = set()
    for i, j in edges:
        for k in adj[i] & adj[j]:
            faces.add(tuple(sorted((i, j, k))))
    bonds = []
    for a, b, c in sorted(faces):
        fe = [idx[(a, b)], idx[(a, c)], idx[(b, c)]]
        for p, q in itertools.combinations(fe, 2):
            bonds.append((p, q, J))
    return _pack(bonds)


def ladder(N, J_rung=1.0, J_leg=1.0):
    """Two-leg ladder with N/2 rungs and periodic legs; leg sites 0..L-1 and
    L..2L-1, rung (k, k+L)."""
    L = N // 2
    if N % 2 or L < 2:
        raise ValueError("ladder needs an even N >= 4")
    e = [(k, k + L, J_rung) for k in range(L)]
    if L == 2:
        e += [(0, 1, J_leg), (2, 3, J_leg)]
    else:
        e += [(k, (k + 1) % L, J_leg) for k in range(L)]
        e += [(L + k, L + (k + 1) % L, J_leg) for k in range(L)]
    return _pack(e)


def random_graph(N, seed, dmin=3, dmax=5, Jlo=0.5, Jhi=1.5, max_tries=100000):
    """Random simple connected graph with every degree in [dmin, dmax]: degrees
    drawn uniformly (even sum), wired by the configuration model, rejected until
    simple and connected; J_ij ~ U[Jlo, Jhi]."""
    rng = np.random.default_rng(seed)
    for _ in range(max_tries):
        deg = rng.integers(dmin, dmax + 1, size=N)
        if deg.sum() % 2:
            continue
        stubs = np.repeat(np.arange(N), deg)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        es = {(min(a, b), max(a, b)) for a, b in pairs}
        if len(es) != len(pairs):
            continue
        seen, stack = {0}, [0]
        nbr = {i: [] for i in range(N)}
        for a, b in es:
            nbr[a].append(b)
            nbr[b].append(a)
        while stack:
            u = stack.pop()
            for w in nbr[u]:
                if w not in seen:
                    seen.add(w)
                    stack.append(w)
        if len(seen) != N:
            continue
        es = sorted(es)
        J = rng.uniform(Jlo, Jhi, size=len(es))
        return _pack([(a, b, j) for (a, b), j in zip(es, J)])
    raise RuntimeError("no graph found")


def cluster_set(n=256, seed=256, sizes=(18, 20, 22)):
    """n independent clusters: N drawn uniformly from `sizes`, each a random_graph
    (degrees 3-5, J ~ U[0.5, 1.5]) with its own seed; returns [(N, bonds)]."""
    rng = np.random.default_rng(seed)
    Ns = rng.choice(np.asarray(sizes), size=n)
    return [(int(N), random_graph(int(N), seed=seed * 100_003 + c)) for c, N in enumerate(Ns)]


def serving_requests(n, rate, seed=4, sizes=(16, 18, 20, 22, 24, 26)):
    """n FTLM requests arriving as a Poisson process of `rate` per second: each a
    ring or a two-leg ladder (equal odds) with N uniform in `sizes`, couplings
    U[0.2, 1.5] (one J for the ring; J_rung and J_leg for the ladder) and field
    h ~ U[0, 2].  Returns ([{"N", "bonds", "h", "kind"}], arrival seconds from 0)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for _ in range(n):
        N = int(rng.choice(np.asarray(sizes)))
        if rng.random() < 0.5:
            reqs.append({"N": N, "bonds": ring(N, J=float(rng.uniform(0.2, 1.5))), "kind": "ring"})
        else:
            reqs.append({"N": N, "bonds": ladder(N, J_rung=float(rng.uniform(0.2, 1.5)),
                                                 J_leg=float(rng.uniform(0.2, 1.5))), "kind": "ladder"})
        reqs[-1]["h"] = float(rng.uniform(0.0, 2.0))
    return reqs, arrivals


def log_t_grid(n=200, lo=0.01, hi=10.0):
    """n log-spaced temperatures T_i = lo (hi/lo)^(i/(n-1)), both ends included."""
    return np.logspace(math.log10(lo), math.log10(hi), n)


def seeded_vector(D, seed, dtype=np.float64):
    """Seeded N(0,1) test vector of length D."""
    return np.random.default_rng(seed).standard_normal(D).astype(dtype)


def hashed_value(k):
    """Deterministic test-vector entry x[k] = (((k * 0x9E3779B1) mod 2^32) >> 22 - 512)
    / 512, a multiple of 2^-9 in [-1, 1) (exact in FP32 and FP64).  Used where a
    vector is too large to build on the host (N = 34)."""
    k = np.asarray(k, dtype=np.uint64)
    h = ((k * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)) >> np.uint64(22)
    return (h.astype(np.float64) - 512.0) / 512.0


def hashed_vector_torch(D, dtype, device, chunk=1 << 26):
    """hashed_value(0..D-1) filled on a torch device, in chunks."""
    import torch

    out = torch.empty(D, dtype=dtype, device=device)
    for s in range(0, D, chunk):
        e = min(D, s + chunk)
        k = torch.arange(s, e, dtype=torch.int64, device=device)
        h = ((k * 0x9E3779B1) & 0xFFFFFFFF) >> 22
        out[s:e] = ((h.to(torch.float64) - 512.0) / 512.0).to(dtype)
    return out
