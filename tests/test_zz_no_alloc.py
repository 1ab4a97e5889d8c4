"""ftlm_lanczos_noalloc: the Lanczos entry point for callers that cannot allocate
device memory -- a host application that owns every device allocation and forbids
new ones after start-up, or code that must not risk the device synchronization
that cudaMalloc/cudaFree can cause.  It keeps its scratch in a static device array
inside the library.  These checks call it through the C ABI twice in a row (the
second call starts from the first call's leftovers in that array) and compare with
ftlm_lanczos, which runs the same launch sequence in a caller workspace: the
results must be bit-identical, for single chains and for blocks of 4 and 8.  The
size limit follows the workspace of the call (ftlm_lanczos_workspace_bytes), which
grows with the block width of the chains."""
import pytest
import torch

from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu


def _outputs(dev, R, M):
    return (torch.full((R, M), float("nan"), dtype=torch.float64, device=dev),
            torch.full((R, M), float("nan"), dtype=torch.float64, device=dev),
            torch.full((R,), -1, dtype=torch.int32, device=dev),
            torch.full((R, M), float("nan"), dtype=torch.float64, device=dev),
            torch.full((R, M), float("nan"), dtype=torch.float64, device=dev))


@pytest.mark.parametrize("R", [3, 8])  # single chains; blocks of 4 (FP64) or 8 (FP32)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("two_sz", [0, 2])  # D = 12870, 11440
def test_noalloc_matches_workspace_entry_point(cuda_dev, dtype, R, two_sz):
    N, M, seed = 16, 60, 21
    with ftlm.Basis(N, two_sz, inputs.ring(N)) as b:
        ref = ftlm.lanczos(b, R, M, seed=seed, dist=ftlm.GAUSS, dtype=dtype, keep_coeffs=True)
        torch.cuda.synchronize()
        for _ in range(2):
            th, w, m, a, bt = _outputs(cuda_dev, R, M)
            ftlm.ftlm_lanczos_noalloc(b.handle, R, M, seed, ftlm.GAUSS, dtype, th, w, m, a, bt)
            torch.cuda.synchronize()
            assert torch.equal(m, ref["m_eff"])
            for got, want in ((th, ref["theta"]), (w, ref["weight"]), (a, ref["alpha"]), (bt, ref["beta"])):
                assert torch.equal(got, want)


def test_noalloc_limit_follows_the_block_width(cuda_dev):
    """D = 705432 fits the 32 MiB scratch with single FP64 chains but not with a
    block of 4 (two interleaved blocks of 4 vectors are 45 MB)."""
    N = 22
    with ftlm.Basis(N, 0, inputs.ring(N)) as b:
        assert b.dim == 705432
        assert ftlm.ftlm_lanczos_workspace_bytes(b.handle, 1, 10, torch.float64) <= 32 << 20
        assert ftlm.ftlm_lanczos_workspace_bytes(b.handle, 8, 10, torch.float64) > 32 << 20
        th, w, m, a, bt = _outputs(cuda_dev, 1, 10)
        ftlm.ftlm_lanczos_noalloc(b.handle, 1, 10, 5, ftlm.GAUSS, torch.float64, th, w, m, a, bt)
        ref = ftlm.lanczos(b, 1, 10, seed=5, dist=ftlm.GAUSS, dtype=torch.float64, keep_coeffs=True)
        torch.cuda.synchronize()
        assert torch.equal(a, ref["alpha"]) and torch.equal(bt, ref["beta"])
        th, w, m, _, _ = _outputs(cuda_dev, 8, 10)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_lanczos_noalloc(b.handle, 8, 10, 5, ftlm.GAUSS, torch.float64, th, w, m)
        assert e.value.status == ftlm.FTLM_EUNSUPPORTED
        assert "static scratch" in str(e.value)


def test_noalloc_rejects_sectors_beyond_its_scratch(cuda_dev):
    with ftlm.Basis(24, 0, inputs.square_j1j2()) as b:  # D = 2704156: 43 MB of FP64 vectors
        th, w, m, _, _ = _outputs(cuda_dev, 1, 10)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_lanczos_noalloc(b.handle, 1, 10, 1, ftlm.GAUSS, torch.float64, th, w, m)
        assert e.value.status == ftlm.FTLM_EUNSUPPORTED
        assert "static scratch" in str(e.value)
