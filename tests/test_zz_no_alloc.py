"""ftlm_lanczos_noalloc: the Lanczos entry point for callers that cannot allocate
device memory (a host application that owns every allocation, or code that must
not risk the device synchronization cudaMalloc/cudaFree can cause).  It keeps its
scratch in a static device array inside the library; these checks call it through
the C ABI twice in a row and compare with ftlm_lanczos, which uses a caller
workspace, within the tolerances the other Lanczos tests use (1e-9 relative with
FP64 vectors, 1e-4 with FP32)."""
import numpy as np
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


@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-9), (torch.float32, 1e-4)])
def test_noalloc_matches_workspace_entry_point(cuda_dev, dtype, rtol):
    N, R, M, seed = 16, 3, 60, 21
    with ftlm.Basis(N, 2, inputs.ring(N)) as b:  # S^z = 1, D = 11440
        ref = ftlm.lanczos(b, R, M, seed=seed, dist=ftlm.GAUSS, dtype=dtype, keep_coeffs=True)
        torch.cuda.synchronize()
        for _ in range(2):  # the second call starts from the first call's leftovers
            th, w, m, a, bt = _outputs(cuda_dev, R, M)
            ftlm.ftlm_lanczos_noalloc(b.handle, R, M, seed, ftlm.GAUSS, dtype, th, w, m, a, bt)
            torch.cuda.synchronize()
            assert torch.equal(m, ref["m_eff"])
            for got, want in ((th, ref["theta"]), (w, ref["weight"]), (a, ref["alpha"]), (bt, ref["beta"])):
                np.testing.assert_allclose(got.cpu().numpy(), want.cpu().numpy(), rtol=rtol, atol=1e-12)


def test_noalloc_rejects_sectors_beyond_its_scratch(cuda_dev):
    with ftlm.Basis(24, 0, inputs.square_j1j2()) as b:  # D = 2704156: 43 MB of FP64 vectors
        th, w, m, _, _ = _outputs(cuda_dev, 1, 10)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_lanczos_noalloc(b.handle, 1, 10, 1, ftlm.GAUSS, torch.float64, th, w, m)
        assert e.value.status == ftlm.FTLM_EUNSUPPORTED
        assert "static scratch" in str(e.value)
