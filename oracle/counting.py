"""Index <-> label by counting, and single rows of H.v (TEST INFRASTRUCTURE ONLY).

For sectors too large to enumerate (N = 30, 34) the oracle cannot hold a basis
array or a lookup table.  The sector index of a label is then, by definition, the
number of sector labels smaller than it (the basis is sorted by label).  That
number follows from a counting argument: a label u < v with the same digit sum
agrees with v on the bits above some set bit p of v, has 0 at p, and places its
remaining up spins anywhere in the p bits below; there are C(p, K - ones above p)
of those.  Python integers and math.comb make every step exact.

label_of(t) inverts it: walk the bits from the top; if t is at least the number of
completions that put 0 at the current bit, the bit must be 1.
"""
import math


def count_below(N, K, v):
    """Number of labels u < v (u < 2^N) with exactly K set bits."""
    cnt, above = 0, 0
    for p in range(N - 1, -1, -1):
        if (v >> p) & 1:
            need = K - above
            if 0 <= need <= p:
                cnt += math.comb(p, need)
            above += 1
    return cnt


def index_of(N, K, label):
    """Sector index of label, or -1 when the label is not in the sector."""
    if label < 0 or label >= (1 << N) or bin(label).count("1") != K:
        return -1
    return count_below(N, K, label)


def label_of(N, K, t):
    """The t-th label (0-based) of the sector, in increasing label order."""
    if not 0 <= t < math.comb(N, K):
        raise IndexError(t)
    v, need = 0, K
    for p in range(N - 1, -1, -1):
        zeros_here = math.comb(p, need) if need <= p else 0
        if t >= zeros_here:
            v |= 1 << p
            t -= zeros_here
            need -= 1
    return v


def hv_row(N, K, bonds, t, x_at):
    """Row t of y = H x (Eq. 12-14 at s = 1/2, bond-list order, FP64).

    x_at(k) returns x[k] for a sector index k (an array or a generator formula).
    """
    bi, bj, J = bonds
    s, ss1 = 0.5, 0.75
    n = label_of(N, K, t)
    diag, off = 0.0, 0.0
    for i, j, Jb in zip(bi, bj, J):
        i, j, Jb = int(i), int(j), float(Jb)
        mi = ((n >> i) & 1) - s
        mj = ((n >> j) & 1) - s
        diag += Jb * mi * mj
        if mi - 1 >= -s and mj + 1 <= s:
            cp = 0.5 * Jb * math.sqrt(ss1 - mi * (mi - 1)) * math.sqrt(ss1 - mj * (mj + 1))
            off += cp * float(x_at(index_of(N, K, n - (1 << i) + (1 << j))))
        if mi + 1 <= s and mj - 1 >= -s:
            cm = 0.5 * Jb * math.sqrt(ss1 - mi * (mi + 1)) * math.sqrt(ss1 - mj * (mj - 1))
            off += cm * float(x_at(index_of(N, K, n + (1 << i) - (1 << j))))
    return diag * float(x_at(t)) + off


def hv_rows(N, K, bonds, rows, x_at):
    return [hv_row(N, K, bonds, int(t), x_at) for t in rows]
