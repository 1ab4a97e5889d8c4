"""The continuous Lanczos flow (ftlm_flow_*): sectors that join at different
Lanczos steps share launches, and each sector's results are bit-identical to the
same sector alone, to the batch's multi-sector path, and (FP64) match the oracle."""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu


def _run(flow, steps_before, bases, R, seeds):
    """Add bases[i] after steps_before[i] flow steps; step until every sector is done."""
    pending = sorted(range(len(bases)), key=lambda i: steps_before[i])
    tickets, outs, step = {}, {}, 0
    while pending or len(outs) < len(bases):
        while pending and steps_before[pending[0]] <= step:
            i = pending.pop(0)
            t = flow.add(bases[i], R, seeds[i], 0, owner=i)
            assert t is not None
            tickets[t] = i
        flow.step(1)
        step += 1
        for t, out, i in flow.done():
            outs[i] = out
        assert step < 2000
    torch.cuda.synchronize()
    return [outs[i] for i in range(len(bases))]


def _mid_bases():
    b18, b19 = inputs.ring(18), inputs.random_graph(19, seed=31)
    return [ftlm.Basis(18, 0, b18), ftlm.Basis(18, 2, b18), ftlm.Basis(19, 1, b19), ftlm.Basis(19, 11, b19),
            ftlm.Basis(12, 0, inputs.random_graph(12, seed=2)), ftlm.Basis(8, 0, inputs.ring(8), two_s=2)]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_flow_results_do_not_depend_on_the_mix_or_the_start_step(cuda_dev, dtype):
    M, R = 30, 8
    bases = _mid_bases()
    seeds = [11 + i for i in range(len(bases))]
    with ftlm.Flow(M, ftlm.GAUSS, dtype, 8, 64, 1 << 30) as flow:
        mix = _run(flow, [0, 0, 7, 13, 3, 20], bases, R, seeds)
    for i, b in enumerate(bases):
        with ftlm.Flow(M, ftlm.GAUSS, dtype, 8, 8, 1 << 28) as flow:
            alone = _run(flow, [0], [b], R, [seeds[i]])[0]
        for k in ("theta", "weight", "m_eff"):
            assert torch.equal(mix[i][k], alone[k]), (i, k)
    for b in bases:
        b.close()


def test_flow_equals_batch_multi_sector_path(cuda_dev):
    # sectors above 32768 rows run on the batch's multi-sector path: same units,
    # tiles and reductions
    M, R = 25, 8
    bases = _mid_bases()[:3]
    with ftlm.Batch([(b, R, 5, 0) for b in bases], M, ftlm.RADEMACHER, torch.float32, 8) as batch:
        ref = [{k: v.clone() for k, v in r.items()} for r in batch.run()]
    with ftlm.Flow(M, ftlm.RADEMACHER, torch.float32, 8, 16, 1 << 30) as flow:
        got = _run(flow, [0, 4, 9], bases, R, [5, 5, 5])
    for a, b in zip(got, ref):
        for k in ("theta", "weight", "m_eff"):
            assert torch.equal(a[k], b[k]), k
    for b in bases:
        b.close()


def test_flow_fp64_matches_oracle(cuda_dev):
    N, M, R, seed = 12, 30, 5, 7
    T = inputs.log_t_grid(50, 0.05, 10.0)
    bonds = inputs.random_graph(N, seed=22)
    bases = [ftlm.Basis(N, tz, bonds) for tz in ftlm.computed_two_sz(N)]
    with ftlm.Flow(M, ftlm.GAUSS, torch.float64, 4, 64, 1 << 28) as flow:
        res = _run(flow, list(range(len(bases))), bases, R, [seed] * len(bases))
        obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)], torch.as_tensor(T, device=cuda_dev),
                          R, M)
    ref = o.thermo(o.run_ftlm(N, bonds, R, M, seed=seed), T)
    for k in ("E", "C", "chi"):
        want = ref[k]
        np.testing.assert_allclose(obs[k].cpu().numpy(), want, rtol=1e-9, atol=1e-12 * np.max(np.abs(want)))
    for b in bases:
        b.close()


@pytest.mark.parametrize("mode", [ftlm.RANK_CR, ftlm.RANK_CLT])
def test_flow_fp64_matches_oracle_in_both_rank_modes(cuda_dev, mode):
    # every S^z >= 0 sector of a random N = 16 cluster, every rank computed the one
    # way: the multi-sector kernels in CR (digit-block ranks) and in CLT, FP64
    N, M, R, seed = 16, 25, 4, 9
    T = inputs.log_t_grid(40, 0.05, 10.0)
    bonds = inputs.random_graph(N, seed=23)
    bases = [ftlm.Basis(N, tz, bonds, mode) for tz in ftlm.computed_two_sz(N)]
    with ftlm.Flow(M, ftlm.GAUSS, torch.float64, 4, 64, 1 << 28) as flow:
        res = _run(flow, list(range(len(bases))), bases, R, [seed] * len(bases))
        obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)], torch.as_tensor(T, device=cuda_dev),
                          R, M)
    ref = o.thermo(o.run_ftlm(N, bonds, R, M, seed=seed), T)
    for k in ("E", "C", "chi"):
        want = ref[k]
        np.testing.assert_allclose(obs[k].cpu().numpy(), want, rtol=1e-9, atol=1e-12 * np.max(np.abs(want)))
    for b in bases:
        b.close()


def test_flow_refuses_what_does_not_fit(cuda_dev):
    with ftlm.Basis(18, 0, inputs.ring(18)) as big, ftlm.Basis(10, 0, inputs.ring(10)) as small:
        need = ftlm.ftlm_flow_unit_bytes(big.handle, torch.float32, 8)
        with ftlm.Flow(10, ftlm.GAUSS, torch.float32, 8, 4, need + (1 << 20)) as flow:
            assert flow.add(big, 8, 1) is not None
            assert flow.add(big, 8, 2) is None          # no room for a second one
            assert flow.status()["units"] == 1
            flow.step(12)
            done = flow.done()
            assert len(done) == 1
            assert flow.add(big, 8, 2) is not None      # its region was freed
            assert flow.add(small, 4, 3) is not None
            assert flow.status()["units"] == 2
            flow.step(12)
            assert len(flow.done()) == 2
            torch.cuda.synchronize()


def test_flow_reuses_coefficient_rows_after_the_ritz_launch(cuda_dev):
    """One unit of coefficient rows: a sector added right after another finished
    waits for that sector's Ritz launch (on the flow's own stream) before taking its
    rows; both results equal the sectors run alone."""
    M, R = 20, 8
    with ftlm.Basis(16, 0, inputs.ring(16)) as b1, ftlm.Basis(16, 2, inputs.ladder(16, 1.0, 0.7)) as b2:
        alone = []
        for b, seed in ((b1, 3), (b2, 4)):
            with ftlm.Flow(M, ftlm.GAUSS, torch.float32, 8, 1, 1 << 28) as flow:
                alone.append(_run(flow, [0], [b], R, [seed])[0])
        with ftlm.Flow(M, ftlm.GAUSS, torch.float32, 8, 1, 1 << 28) as flow:
            assert flow.add(b1, R, 3, owner=0) is not None
            flow.step(M)
            (t1, out1, _), = flow.done()
            assert flow.add(b2, R, 4, owner=1) is not None   # rows of b1 held by its Ritz launch
            flow.step(M)
            (t2, out2, _), = flow.done()
            torch.cuda.synchronize()
        for got, want in ((out1, alone[0]), (out2, alone[1])):
            for k in ("theta", "weight", "m_eff"):
                assert torch.equal(got[k], want[k]), k


def test_flow_wave_streams_do_not_change_results(cuda_dev):
    """Sectors of 2.7 M rows (173 MB of vectors per unit) fill several 256 MB waves,
    spread over 3 wave streams; every sector's results equal those of the flow with
    all waves on one stream."""
    M, R = 12, 8
    r24, l24 = inputs.ring(24), inputs.ladder(24, 0.8, 1.2)
    bases = [ftlm.Basis(24, 0, r24), ftlm.Basis(24, 0, l24), ftlm.Basis(24, 2, r24), ftlm.Basis(24, 4, l24),
             ftlm.Basis(18, 0, inputs.ring(18)), ftlm.Basis(20, 2, inputs.random_graph(20, seed=5))]
    seeds = [21 + i for i in range(len(bases))]
    res = {}
    for streams in (1, 3):
        with ftlm.Flow(M, ftlm.GAUSS, torch.float32, 8, 64, 4 << 30, streams=streams) as flow:
            res[streams] = _run(flow, [0, 0, 2, 3, 0, 5], bases, R, seeds)
    for a, b in zip(res[1], res[3]):
        for k in ("theta", "weight", "m_eff"):
            assert torch.equal(a[k], b[k]), k
    for b in bases:
        b.close()


def test_flow_set_streams_rejects_bad_counts(cuda_dev):
    with ftlm.Flow(10, ftlm.GAUSS, torch.float32, 8, 4, 1 << 24) as flow:
        for n in (0, 5):
            with pytest.raises(ftlm.FtlmError):
                ftlm._check(ftlm.lib().ftlm_flow_set_streams(flow.handle, n))
