"""Host logic of the request loop (no GPU): admission order and the request stream."""
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


def test_admission_is_fifo_by_sector_and_resumes():
    q = serve.AdmissionQueue()
    for i, n in enumerate([3, 2, 4]):
        q.push(_J(i, 2 * n), range(n))
    room = [4]
    started = []

    def try_add(job, k):  # a capacity of `room` sectors
        if room[0] == 0:
            return False
        room[0] -= 1
        return True

    got = q.admit(lambda j: started.append(j.job_id), try_add)
    assert [(j.job_id, k) for j, k in got] == [(0, 0), (0, 1), (0, 2), (1, 0)]
    assert started == [0, 1] and q.in_flight == 2 and len(q) == 2   # job 1 waits for its second sector
    room[0] = 10
    got = q.admit(lambda j: started.append(j.job_id), try_add)
    assert [(j.job_id, k) for j, k in got] == [(1, 1), (2, 0), (2, 1), (2, 2), (2, 3)]
    assert started == [0, 1, 2] and q.in_flight == 3 and len(q) == 0


def test_admission_limits_jobs_in_flight_and_starts_jobs_without_sectors():
    q = serve.AdmissionQueue(max_jobs=1)
    q.push(_J(0, 4), [])        # only small sectors: started, nothing offered
    for i in range(1, 3):
        q.push(_J(i, 4), range(2))
    started = []
    got = q.admit(started.append, lambda j, k: True)
    assert got == [] and [j.job_id for j in started] == [0]     # one job at a time
    q.finished()
    got = q.admit(started.append, lambda j, k: True)
    assert [(j.job_id, k) for j, k in got] == [(1, 0), (1, 1)]
    assert q.admit(started.append, lambda j, k: True) == []
    q.finished()
    got = q.admit(started.append, lambda j, k: True)
    assert [(j.job_id, k) for j, k in got] == [(2, 0), (2, 1)]


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
