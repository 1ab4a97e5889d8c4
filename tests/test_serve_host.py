"""Host logic of the request loop (no GPU): grouping policy and the request stream."""
import collections
import math

import numpy as np

from paper_2605_26261_gb300 import inputs, serve


class _J:
    def __init__(self, i, N):
        self.job_id, self.N = i, N


def test_sector_rows():
    for N in (2, 7, 16, 26):
        assert serve.sector_rows(N) == sum(math.comb(N, K) for K in range((N + 1) // 2, N + 1))
    # even N: half of 2^N plus half of the middle sector
    assert serve.sector_rows(16) == (2**16 + math.comb(16, 8)) // 2


def test_take_group_is_fifo_and_bounded():
    q = collections.deque(_J(i, N) for i, N in enumerate([16, 16, 18, 26, 16, 16]))
    g = serve.take_group(q, max_group=8, max_rows=serve.sector_rows(16) * 2 + serve.sector_rows(18))
    assert [j.job_id for j in g] == [0, 1, 2]           # N = 26 does not fit behind them
    g = serve.take_group(q, max_group=8, max_rows=10)    # the head job is always taken
    assert [j.job_id for j in g] == [3]
    g = serve.take_group(q, max_group=1, max_rows=1 << 40)
    assert [j.job_id for j in g] == [4]
    assert [j.job_id for j in q] == [5]


def test_serving_requests_recipe():
    reqs, t = inputs.serving_requests(400, 200.0, seed=4)
    assert t[0] == 0 and np.all(np.diff(t) >= 0)
    assert abs(len(t) / t[-1] - 200.0) < 40.0           # Poisson rate
    assert {r["N"] for r in reqs} == {16, 18, 20, 22, 24, 26}
    assert {r["kind"] for r in reqs} == {"ring", "ladder"}
    for r in reqs:
        bi, bj, J = r["bonds"]
        assert np.all((J >= 0.2) & (J <= 1.5)) and 0.0 <= r["h"] <= 2.0
        assert len(J) == (r["N"] if r["kind"] == "ring" else 3 * r["N"] // 2)
    again, t2 = inputs.serving_requests(400, 200.0, seed=4)
    assert np.array_equal(t, t2) and all(np.array_equal(a["bonds"][2], b["bonds"][2]) for a, b in zip(reqs, again))


def test_cluster_set_recipe():
    cs = inputs.cluster_set(40, seed=3)
    assert {N for N, _ in cs} <= {18, 20, 22}
    for N, (bi, bj, J) in cs:
        deg = np.bincount(np.concatenate([bi, bj]), minlength=N)
        assert deg.min() >= 3 and deg.max() <= 5
        assert np.all((J >= 0.5) & (J <= 1.5))
