"""Stream-ordered sector tables, the launch counter and the bandwidth probes.

Tables live in one block of the library's device memory pool: a release queued on a
stream (ftlm_basis_destroy_async) must not disturb work still queued before it, and
memory it frees is reused without corrupting later sectors.
"""
import numpy as np
import pytest
import torch

from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu


def test_async_release_behind_queued_work(cuda_dev):
    N, M, R = 20, 40, 8
    bonds = inputs.random_graph(N, seed=12)
    with ftlm.Basis(N, 0, bonds) as b:
        ref = ftlm.lanczos(b, R, M, seed=2, dtype=torch.float32)
        torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            b = ftlm.Basis(N, 0, bonds, stream=s)
            got = ftlm.lanczos(b, R, M, seed=2, dtype=torch.float32, stream=s)
            b.release(s)  # queued behind the chains, no wait
            # a new sector right away may reuse the block once the release completes
            other = ftlm.Basis(N, 2, bonds, stream=s)
            ftlm.lanczos(other, R, M, seed=3, dtype=torch.float32, stream=s)
            other.release(s)
            s.synchronize()
            for k in ("theta", "weight", "m_eff"):
                assert torch.equal(got[k], ref[k]), k


def test_batch_release_async(cuda_dev):
    bonds = inputs.ring(14)
    bases = [ftlm.Basis(14, tz, bonds) for tz in (0, 2, 4)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch = ftlm.Batch([(b, 4, 1, 0) for b in bases], 20, ftlm.GAUSS, torch.float64, 4, stream=s)
        res = batch.run(s)
        batch.release(s)
        s.synchronize()
    assert all(int(r["m_eff"].min()) > 0 for r in res)
    for b in bases:
        b.close()


def test_launch_counter(cuda_dev):
    N, M, R = 12, 10, 8
    bonds = inputs.ring(N)
    c0 = ftlm.ftlm_launch_count()
    b = ftlm.Basis(N, 0, bonds, ftlm.RANK_CR)  # coarse index build: 1 kernel
    assert ftlm.ftlm_launch_count() - c0 == 1
    x = torch.ones(b.dim, dtype=torch.float64, device=cuda_dev)
    y = torch.empty_like(x)
    c1 = ftlm.ftlm_launch_count()
    ftlm.ftlm_hv(b.handle, x, y)
    assert ftlm.ftlm_launch_count() - c1 == 1
    c2 = ftlm.ftlm_launch_count()
    # one block of 8: start, M x (H.v + tile alpha sums + update), m_eff copy, Ritz
    ftlm.lanczos(b, R, M, dtype=torch.float32)
    assert ftlm.ftlm_launch_count() - c2 == 1 + 3 * M + 1 + 1
    torch.cuda.synchronize()
    b.close()
    with ftlm.Basis(N, 0, bonds, ftlm.RANK_CLT) as b:  # CLT: the H.v launch finishes alpha itself
        c3 = ftlm.ftlm_launch_count()
        ftlm.lanczos(b, R, M, dtype=torch.float32)
        assert ftlm.ftlm_launch_count() - c3 == 1 + 2 * M + 1 + 1
        torch.cuda.synchronize()


def test_bandwidth_probes(cuda_dev):
    """The read probes behind the rooflines: coalesced, scattered 32-byte rows and
    1 KB runs over an L2-sized buffer return positive rates; a scattered read is no
    faster than a coalesced one; bad arguments are refused."""
    buf = torch.zeros(64 << 20, dtype=torch.uint8, device=cuda_dev)
    coalesced = ftlm.ftlm_probe_read_bandwidth(buf, 4)
    rows = ftlm.ftlm_probe_gather_bandwidth(buf, 1, 4)
    runs = ftlm.ftlm_probe_gather_bandwidth(buf, 32, 4)
    assert coalesced > 0 and rows > 0 and runs > 0
    assert rows <= 1.1 * coalesced
    with pytest.raises(ftlm.FtlmError):
        ftlm.ftlm_probe_gather_bandwidth(buf, 7, 4)
    with pytest.raises(ftlm.FtlmError):
        ftlm.ftlm_probe_gather_bandwidth(buf[:16], 32, 4)
