"""The request loop on the GPU: each job's results are the same alone and in the
mix (bit for bit), a served FP64 job matches the oracle, and admission by memory
budget serialises groups without stalling."""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs, serve

pytestmark = pytest.mark.gpu

T = inputs.log_t_grid(40, 0.05, 10.0)


def make_jobs(n, seed, sizes=(8, 10, 12, 14, 16)):
    reqs, arrivals = inputs.serving_requests(n, 400.0, seed=seed, sizes=sizes)
    jobs = [serve.Job(job_id=i, N=r["N"], bonds=r["bonds"], h=r["h"], seed=500 + i) for i, r in enumerate(reqs)]
    return jobs, arrivals


def engine(slots, max_group, dtype=torch.float32, **kw):
    return serve.Engine(slots=slots, R=4, M=30, dtype=dtype, block=4, streams=2, T=T, max_group=max_group, **kw)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_results_identical_alone_and_in_mix(cuda_dev, dtype):
    jobs, arrivals = make_jobs(24, seed=7, sizes=(8, 10, 12, 14, 16, 18))
    eng = engine(3, 4, dtype)
    mix = {j.job_id: j for j in eng.run(jobs, arrivals)}
    assert len(mix) == len(jobs)
    assert eng.stats["max_group"] > 1, eng.stats   # some jobs shared a batch
    assert eng.stats["max_busy"] > 1, eng.stats    # some groups ran concurrently
    alone_jobs, _ = make_jobs(24, seed=7, sizes=(8, 10, 12, 14, 16, 18))
    alone = engine(1, 1, dtype).run(alone_jobs)
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
    job = serve.Job(job_id=0, N=10, bonds=bonds, h=0.6, seed=77)
    filler, _ = make_jobs(6, seed=3, sizes=(8, 10, 12))
    done = engine(2, 4, torch.float64).run([job] + filler)
    got = next(j for j in done if j.job_id == 0).result
    ref = o.thermo(o.run_ftlm(10, bonds, 4, 30, seed=77, dist=o.GAUSS), T, g=2.0, h=0.6)
    for row, k in enumerate(("E", "C", "chi", "mag")):
        want = ref[k]
        scale = np.max(np.abs(want))
        np.testing.assert_allclose(got[row], want, rtol=1e-9, atol=1e-12 * scale)


def test_memory_budget_serialises_groups(cuda_dev):
    jobs, arrivals = make_jobs(8, seed=11)
    eng = engine(3, 2, memory_budget=1)  # every group is over budget: one at a time
    done = eng.run(jobs, arrivals)
    assert len(done) == len(jobs)
    assert eng.stats["max_busy"] == 1
    assert eng.in_use == 0
