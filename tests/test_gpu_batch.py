"""Batched chains of many sectors (ftlm_batch_*) against per-sector ftlm_lanczos
and against the oracle.

Per-sector comparison: the same chains (same seed and chain indices), so Ritz data
agree up to the summation order of the dot products; compared through spectral
sums sum_k w_k exp(-b theta_k), which are insensitive to how near-degenerate
(ghost) Ritz pairs split their weight: 1e-10 relative in FP64, 1e-5 in FP32.
"""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu

BETAS = (0.2, 1.0, 5.0)


def spectral_sums(theta, weight, m):
    th, w = theta.cpu().numpy(), weight.cpu().numpy()
    out = []
    for r in range(th.shape[0]):
        k = int(m[r])
        out.append([np.sum(w[r, :k] * np.exp(-b * (th[r, :k] - th[r, 0]))) for b in BETAS] + [th[r, 0]])
    return np.array(out)


def clusters():
    return [(10, inputs.random_graph(10, seed=1)), (12, inputs.random_graph(12, seed=2)),
            (13, inputs.random_graph(13, seed=3)), (16, inputs.ring(16))]


@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-10), (torch.float32, 1e-5)])
@pytest.mark.parametrize("block", [1, 4, 8, 16])
def test_batch_matches_per_sector_lanczos(cuda_dev, dtype, rtol, block):
    M, R, seed = 40, 6, 11
    bases = []
    for N, bonds in clusters():
        for tz in ftlm.computed_two_sz(N):
            bases.append(ftlm.Basis(N, tz, bonds, ftlm.RANK_CR if N % 2 else ftlm.RANK_CLT))
    entries = [(b, R, seed + i, 3 * i) for i, b in enumerate(bases)]
    with ftlm.Batch(entries, M, ftlm.GAUSS, dtype, block) as batch:
        res = batch.run()
        torch.cuda.synchronize()
        for (b, R_, s, c0), got in zip(entries, res):
            # reference: the same chains through ftlm_lanczos, one sector at a time
            ref = ftlm.lanczos(b, R + c0, M, seed=s, dist=ftlm.GAUSS, dtype=dtype)
            torch.cuda.synchronize()
            m_ref = ref["m_eff"][c0:].cpu().numpy()
            assert np.array_equal(got["m_eff"].cpu().numpy(), m_ref), (b.N, b.two_sz)
            a = spectral_sums(got["theta"], got["weight"], m_ref)
            e = spectral_sums(ref["theta"][c0:], ref["weight"][c0:], m_ref)
            np.testing.assert_allclose(a, e, rtol=rtol, atol=rtol * 1e-3)
    for b in bases:
        b.close()


def test_batch_mixes_small_and_large_sectors(cuda_dev):
    # D = C(18, 9) = 48620 runs through the grid-wide path, the rest inside CTAs.
    M, R = 30, 5
    bonds = inputs.ring(18)
    bases = [ftlm.Basis(18, tz, bonds) for tz in (0, 2, 10, 18)]
    entries = [(b, R, 4, 0) for b in bases]
    with ftlm.Batch(entries, M, ftlm.RADEMACHER, torch.float64) as batch:
        res = batch.run()
        torch.cuda.synchronize()
        for b, got in zip(bases, res):
            ref = ftlm.lanczos(b, R, M, seed=4, dist=ftlm.RADEMACHER, dtype=torch.float64)
            torch.cuda.synchronize()
            np.testing.assert_allclose(spectral_sums(got["theta"], got["weight"], got["m_eff"]),
                                       spectral_sums(ref["theta"], ref["weight"], ref["m_eff"]), rtol=1e-10)
    for b in bases:
        b.close()


def test_batch_run_captured_in_cuda_graph(cuda_dev):
    M, R = 30, 8
    bases = [ftlm.Basis(12, tz, inputs.random_graph(12, seed=9)) for tz in (0, 2, 4)]
    entries = [(b, R, 1, 0) for b in bases]
    with ftlm.Batch(entries, M, ftlm.GAUSS, torch.float32, 8) as batch:
        direct = [{k: v.clone() for k, v in r.items()} for r in batch.run()]
        torch.cuda.synchronize()
        for r in batch.results:
            for v in r.values():
                v.zero_()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            batch.run(stream=s)
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(direct, batch.results):
            for k in ("theta", "weight", "m_eff"):
                assert torch.equal(a[k], b[k]), k
    for b in bases:
        b.close()


def test_batch_ftlm_matches_oracle(cuda_dev):
    # Two random clusters, every S^z >= 0 sector, FP64: thermodynamics vs the oracle.
    M, R = 40, 5
    T = inputs.log_t_grid(60, 0.05, 10.0)
    for N, seed in ((11, 21), (12, 22)):
        bonds = inputs.random_graph(N, seed=seed)
        bases = [ftlm.Basis(N, tz, bonds) for tz in ftlm.computed_two_sz(N)]
        with ftlm.Batch([(b, R, 7, 0) for b in bases], M, ftlm.GAUSS, torch.float64, 4) as batch:
            res = batch.run()
            obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)],
                              torch.as_tensor(T, device=cuda_dev), R, M)
        ref = o.thermo(o.run_ftlm(N, bonds, R, M, seed=7), T)
        for k in ("E", "C", "chi"):
            got, want = obs[k].cpu().numpy(), ref[k]
            scale = np.max(np.abs(want))
            np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12 * scale)
        for b in bases:
            b.close()


def test_batch_rejects_bad_items(cuda_dev):
    with ftlm.Basis(8, 0, inputs.ring(8)) as b:
        with pytest.raises(ftlm.FtlmError):
            ftlm.Batch([(b, 0, 1, 0)], 10)
        with pytest.raises(ftlm.FtlmError):
            ftlm.Batch([(b, 2, 1, 0)], 10, block=3)


def _mid_sector_bases():
    # three spin-1/2 sectors above 32768 states (ring 18: K = 9, 10; random N = 19:
    # K = 10), run by the multi-sector path, and two small ones for the persistent
    # kernel
    b18 = inputs.ring(18)
    b19 = inputs.random_graph(19, seed=31)
    return [ftlm.Basis(18, 0, b18), ftlm.Basis(18, 2, b18), ftlm.Basis(19, 1, b19),
            ftlm.Basis(18, 8, b18), ftlm.Basis(19, 11, b19)]


@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-10), (torch.float32, 1e-5)])
@pytest.mark.parametrize("block", [1, 4, 16])
def test_multi_sector_path_matches_per_sector_lanczos(cuda_dev, dtype, rtol, block):
    # R = 6 leaves a partial last unit (nact < block) for block 4 and 16
    M, R = 30, 6
    bases = _mid_sector_bases()
    entries = [(b, R, 40 + i, 2 * i) for i, b in enumerate(bases)]
    with ftlm.Batch(entries, M, ftlm.GAUSS, dtype, block) as batch:
        res = batch.run()
        torch.cuda.synchronize()
        for (b, _, s, c0), got in zip(entries, res):
            ref = ftlm.lanczos(b, R + c0, M, seed=s, dist=ftlm.GAUSS, dtype=dtype)
            torch.cuda.synchronize()
            m_ref = ref["m_eff"][c0:].cpu().numpy()
            assert np.array_equal(got["m_eff"].cpu().numpy(), m_ref), (b.N, b.two_sz)
            np.testing.assert_allclose(spectral_sums(got["theta"], got["weight"], m_ref),
                                       spectral_sums(ref["theta"][c0:], ref["weight"][c0:], m_ref),
                                       rtol=rtol, atol=rtol * 1e-3)
    for b in bases:
        b.close()


def test_multi_sector_results_independent_of_the_mix(cuda_dev):
    # a unit's arithmetic depends only on its own tiles: bit-identical alone and
    # together with other sectors
    M, R = 25, 8
    bases = _mid_sector_bases()
    with ftlm.Batch([(bases[0], R, 5, 0)], M, ftlm.RADEMACHER, torch.float32, 8) as alone:
        a = {k: v.clone() for k, v in alone.run()[0].items()}
    with ftlm.Batch([(b, R, 5 if i == 0 else 9 + i, 0) for i, b in enumerate(bases)], M, ftlm.RADEMACHER,
                    torch.float32, 8) as mix:
        m = mix.run()[0]
        torch.cuda.synchronize()
        for k in ("theta", "weight", "m_eff"):
            assert torch.equal(a[k], m[k]), k
    for b in bases:
        b.close()


def test_multi_sector_path_matches_oracle(cuda_dev):
    # every S^z >= 0 sector of a random N = 18 cluster (D up to 48620), FP64
    N, M, R = 18, 30, 5
    T = inputs.log_t_grid(50, 0.05, 10.0)
    bonds = inputs.random_graph(N, seed=44)
    bases = [ftlm.Basis(N, tz, bonds) for tz in ftlm.computed_two_sz(N)]
    with ftlm.Batch([(b, R, 7, 0) for b in bases], M, ftlm.GAUSS, torch.float64, 4) as batch:
        res = batch.run()
        obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)], torch.as_tensor(T, device=cuda_dev),
                          R, M)
    ref = o.thermo(o.run_ftlm(N, bonds, R, M, seed=7), T)
    for k in ("E", "C", "chi"):
        want = ref[k]
        np.testing.assert_allclose(obs[k].cpu().numpy(), want, rtol=1e-9, atol=1e-12 * np.max(np.abs(want)))
    for b in bases:
        b.close()


def test_multi_sector_cr_path_matches_oracle(cuda_dev):
    # the same N = 18 cluster with every sector in CR (digit-block ranks): the two
    # largest sectors on the multi-sector kernels, the rest in the persistent kernel
    N, M, R = 18, 30, 5
    T = inputs.log_t_grid(50, 0.05, 10.0)
    bonds = inputs.random_graph(N, seed=44)
    bases = [ftlm.Basis(N, tz, bonds, ftlm.RANK_CR) for tz in ftlm.computed_two_sz(N)]
    with ftlm.Batch([(b, R, 7, 0) for b in bases], M, ftlm.GAUSS, torch.float64, 4) as batch:
        res = batch.run()
        obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)], torch.as_tensor(T, device=cuda_dev),
                          R, M)
    ref = o.thermo(o.run_ftlm(N, bonds, R, M, seed=7), T)
    for k in ("E", "C", "chi"):
        want = ref[k]
        np.testing.assert_allclose(obs[k].cpu().numpy(), want, rtol=1e-9, atol=1e-12 * np.max(np.abs(want)))
    for b in bases:
        b.close()


def _n33_bases():
    # N = 33 ring sectors above 32768 states (K = 29: 40920, K = 28: 237336): the
    # launch sequence of ftlm_lanczos on side streams; K = 30 (5456) is small
    bonds = inputs.ring(33)
    return [ftlm.Basis(33, 2 * K - 33, bonds) for K in (29, 28, 30)]


@pytest.mark.parametrize("block", [4, 8])
def test_side_streams_do_not_change_results(cuda_dev, block):
    # Sectors with N > 32 run ftlm_lanczos's launch sequence with blocks of `block`
    # chains on side streams: bit-identical for any number of side streams, and
    # equal to ftlm_lanczos with the same block width on the caller's stream.
    M, R = 25, 8
    bases = _n33_bases()
    entries = [(b, R, 40 + i, 0) for i, b in enumerate(bases)]
    runs = []
    for streams in (1, 3, 8):
        with ftlm.Batch(entries, M, ftlm.GAUSS, torch.float32, block, streams) as batch:
            runs.append([{k: v.clone() for k, v in r.items()} for r in batch.run()])
            torch.cuda.synchronize()
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            for k in ("theta", "weight", "m_eff"):
                assert torch.equal(a[k], b[k]), k
    ftlm.ftlm_lanczos_set_block(block)
    try:
        for i, b in enumerate(bases[:2]):  # the side-stream sectors
            ref = ftlm.lanczos(b, R, M, seed=40 + i, dist=ftlm.GAUSS, dtype=torch.float32)
            torch.cuda.synchronize()
            for k in ("theta", "weight", "m_eff"):
                assert torch.equal(ref[k], runs[0][i][k]), (i, k)
    finally:
        ftlm.ftlm_lanczos_set_block(0)
    for b in bases:
        b.close()


def test_graph_capture_with_all_paths(cuda_dev):
    # persistent kernel, multi-sector path (spin 1/2 and spin 1) and side streams in
    # one captured run
    M, R = 20, 8
    bases = _mid_sector_bases() + [ftlm.Basis(8, 0, inputs.ring(8), two_s=2)] + _n33_bases()[:1]
    with ftlm.Batch([(b, R, 3, 0) for b in bases], M, ftlm.RADEMACHER, torch.float32, 8, 3) as batch:
        direct = [{k: v.clone() for k, v in r.items()} for r in batch.run()]
        torch.cuda.synchronize()
        for r in batch.results:
            for v in r.values():
                v.zero_()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            batch.run(stream=s)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        for a, b in zip(direct, batch.results):
            for k in ("theta", "weight", "m_eff"):
                assert torch.equal(a[k], b[k]), k
    for b in bases:
        b.close()


@pytest.mark.parametrize("side_items", [False, True])
def test_autotune_picks_a_timed_candidate(cuda_dev, side_items):
    M, R = 15, 16
    bases = _mid_sector_bases()
    if side_items:
        bases.append(_n33_bases()[0])
    entries = [(b, R, 1, 0) for b in bases]
    block, streams, times = ftlm.autotune(entries, M, ftlm.GAUSS, torch.float32)
    assert (block, streams) in times
    assert len(times) == (12 if side_items else 3)  # stream counts only with side-stream items
    assert times[(block, streams)] == min(times.values())
    # a plan with the tuned parameters runs and agrees with the default plan
    with ftlm.Batch(entries, M, ftlm.GAUSS, torch.float32, block, streams) as tuned:
        a = [{k: v.clone() for k, v in r.items()} for r in tuned.run()]
    with ftlm.Batch(entries, M, ftlm.GAUSS, torch.float32, 16) as ref:
        e = ref.run()
        torch.cuda.synchronize()
        for x, y in zip(a, e):
            assert torch.equal(x["m_eff"], y["m_eff"])
            np.testing.assert_allclose(spectral_sums(x["theta"], x["weight"], x["m_eff"]),
                                       spectral_sums(y["theta"], y["weight"], y["m_eff"]), rtol=1e-5)
    for b in bases:
        b.close()


def test_plan_autotune_tunes_tiles_and_plans_agree(cuda_dev):
    """ftlm_batch_autotune_plan times block widths, then H.v and streaming tile rows
    of the multi-sector path; every plan gives the same chains up to the summation
    order of the per-tile sums, and the fastest candidate is the one returned."""
    M, R = 15, 8
    bases = _mid_sector_bases()
    entries = [(b, R, 1, 0) for b in bases]
    best, tried = ftlm.autotune_plan(entries, M, ftlm.GAUSS, torch.float32)
    assert len(tried) == 3 + 2 + 2  # blocks, then tile rows, then streaming tile rows
    assert {t[2] for t, _ in tried} >= {1024, 2048, 4096} and {t[3] for t, _ in tried} >= {8192, 16384, 32768}
    assert best.as_tuple() == min(tried, key=lambda kv: kv[1])[0]
    with ftlm.Batch(entries, M, ftlm.GAUSS, torch.float32, plan=best) as tuned:
        a = [{k: v.clone() for k, v in r.items()} for r in tuned.run()]
    odd = ftlm.BatchPlan(4, 1, 512, 1024)  # small tiles: many partial sums per unit
    with ftlm.Batch(entries, M, ftlm.GAUSS, torch.float32, plan=odd) as other:
        e = other.run()
        torch.cuda.synchronize()
        for x, y in zip(a, e):
            assert torch.equal(x["m_eff"], y["m_eff"])
            np.testing.assert_allclose(spectral_sums(x["theta"], x["weight"], x["m_eff"]),
                                       spectral_sums(y["theta"], y["weight"], y["m_eff"]), rtol=1e-5)
    with pytest.raises(ftlm.FtlmError):
        ftlm.Batch(entries, M, ftlm.GAUSS, torch.float32, plan=ftlm.BatchPlan(8, 1, 1000, 0))
    for b in bases:
        b.close()
