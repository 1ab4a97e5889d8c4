"""The request loop on the GPU (chain-level continuous batching): each job's
results are the same alone and in the mix (bit for bit), a served FP64 job matches
the oracle, and a small memory budget serialises the jobs without stalling."""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import inputs, serve

pytestmark = pytest.mark.gpu

T = inputs.log_t_grid(40, 0.05, 10.0)


def make_jobs(n, seed, sizes=(8, 10, 12, 14, 16)):
    reqs, arrivals = inputs.serving_requests(n, 400.0, seed=seed, sizes=sizes)
    jobs = [serve.Job(job_id=i, N=r["N"], bonds=r["bonds"], h=r["h"], seed=500 + i) for i, r in enumerate(reqs)]
    return jobs, arrivals


def engine(dtype=torch.float32, **kw):
    return serve.Engine(R=4, M=30, dtype=dtype, block=4, T=T, **kw)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_results_identical_alone_and_in_mix(cuda_dev, dtype):
    jobs, arrivals = make_jobs(24, seed=7, sizes=(8, 10, 12, 14, 16, 18))
    eng = engine(dtype, memory_budget=1 << 30)
    mix = {j.job_id: j for j in eng.run(jobs, arrivals)}
    assert len(mix) == len(jobs)
    assert eng.stats["max_jobs_in_flight"] > 1, eng.stats   # jobs shared the flow
    eng.close()
    alone_jobs, _ = make_jobs(24, seed=7, sizes=(8, 10, 12, 14, 16, 18))
    eng1 = engine(dtype, memory_budget=1 << 30, max_jobs=1)
    alone = eng1.run(alone_jobs)
    assert eng1.stats["max_jobs_in_flight"] == 1
    eng1.close()
    for j in alone:
        assert np.array_equal(j.result, mix[j.job_id].result), j.job_id
        assert j.updates == mix[j.job_id].updates
        assert np.all(np.isfinite(j.result))
    lat = [j.latency for j in mix.values()]
    assert min(lat) > 0


def test_served_job_matches_oracle(cuda_dev):
    # ladder N = 10 in a field, FP64: E, C, chi and <S^z> vs the oracle's FTLM with
    # the same start vectors (chain keys by seed, N, K, r)
    bonds = inputs.ladder(10, 0.7, 1.1)
    job = serve.Job(job_id=100, N=10, bonds=bonds, h=0.6, seed=77)
    filler, _ = make_jobs(6, seed=3, sizes=(8, 10, 12))
    eng = engine(torch.float64, memory_budget=1 << 28)
    done = eng.run([job] + filler)
    eng.close()
    got = next(j for j in done if j.job_id == 100).result
    ref = o.thermo(o.run_ftlm(10, bonds, 4, 30, seed=77, dist=o.GAUSS), T, g=2.0, h=0.6)
    for row, k in enumerate(("E", "C", "chi", "mag")):
        want = ref[k]
        scale = np.max(np.abs(want))
        np.testing.assert_allclose(got[row], want, rtol=1e-9, atol=1e-12 * scale)


def test_small_budget_serialises_without_stalling(cuda_dev):
    # N = 18 jobs: their two sectors above 32768 rows join the flow (1.6 and 1.4 MB
    # of units at R = 4 in FP32), the rest run in each job's persistent batch; a
    # flow workspace of 4 MB (with the coefficient rows of 64 units) holds about one
    # job's large sectors, so later sectors wait for room
    jobs, arrivals = make_jobs(8, seed=11, sizes=(18,))
    eng = engine(memory_budget=4 << 20, max_units=64)
    done = eng.run(jobs, arrivals)
    eng.close()
    assert len(done) == len(jobs)
    assert eng.stats["refusals"] > 0 and eng.stats["flow_sectors"] == 2 * len(jobs)
    assert all(np.all(np.isfinite(j.result)) for j in done)
