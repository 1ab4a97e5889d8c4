"""Full-size sectors, in the launch configuration the benchmark times.

  * icosidodecahedron, N = 30, S^z = 0 (D = 155 117 520), CLT and CR;
  * ring, N = 34, S^z = 0 (D = 2 333 606 220), CR.
The oracle cannot enumerate these sectors, so it computes sampled output rows one
by one (index <-> label by counting); the whole vectors are checked through
properties that hold at any size: the uniform vector is an exact eigenvector, and
the fused Lanczos launch reproduces alpha_1 = <q, Hq> and beta_1^2 = ||Hq||^2 -
alpha_1^2 computed from a separate H.v.
"""
import math

import numpy as np
import pytest
import torch

from oracle import counting
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu

ICOSIDODECA = (30, inputs.icosidodecahedron())
RING34 = (34, inputs.ring(34))


def sample_rows(D, n, seed):
    rng = np.random.default_rng(seed)
    rows = np.concatenate([[0, 1, D // 2, D - 2, D - 1], rng.integers(0, D, size=n)])
    return np.unique(rows)


def check_sampled_rows(dev, N, bonds, mode, dtype, nrows):
    K = N // 2
    with ftlm.Basis(N, 0, bonds, mode) as b:
        assert b.dim == math.comb(N, K)
        x = inputs.hashed_vector_torch(b.dim, dtype, dev)
        y = torch.empty_like(x)
        ftlm.ftlm_hv(b.handle, x, y)
        rows = sample_rows(b.dim, nrows, 17)
        got = y[torch.as_tensor(rows, device=dev)].double().cpu().numpy()
        del x, y
    ref = np.array(counting.hv_rows(N, K, bonds, rows, lambda k: float(inputs.hashed_value(k))))
    # entries of x are multiples of 2^-9 and J = 1: every partial sum is exact
    # in FP64, and exact in FP32 while below 2^15.
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_icosidodecahedron_sampled_rows(cuda_dev, mode, dtype):
    check_sampled_rows(cuda_dev, *ICOSIDODECA, mode, dtype, 3000)


def test_ring34_sampled_rows(cuda_dev):
    check_sampled_rows(cuda_dev, *RING34, ftlm.RANK_CR, torch.float32, 3000)


@pytest.mark.parametrize("N,bonds,mode", [(*ICOSIDODECA, ftlm.RANK_CLT), (*ICOSIDODECA, ftlm.RANK_CR),
                                          (*RING34, ftlm.RANK_CR)])
def test_uniform_vector_exact_at_full_size(cuda_dev, N, bonds, mode):
    with ftlm.Basis(N, 0, bonds, mode) as b:
        x = torch.ones(b.dim, dtype=torch.float32, device=cuda_dev)
        y = torch.empty_like(x)
        ftlm.ftlm_hv(b.handle, x, y)
        assert torch.all(y == float(bonds[2].sum()) / 4).item()


@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
def test_fused_lanczos_launch_at_full_size(cuda_dev, mode):
    N, bonds = ICOSIDODECA
    with ftlm.Basis(N, 0, bonds, mode) as b:
        res = ftlm.lanczos(b, 1, 2, seed=1, dist=ftlm.RADEMACHER, dtype=torch.float32, keep_coeffs=True)
        # the same start vector, rebuilt here: Rademacher signs of the seeded chain
        a1, b1 = res["alpha"][0, 0].item(), res["beta"][0, 0].item()
        del res
        torch.cuda.empty_cache()
        # <q, Hq> and ||Hq||^2 through the separate H.v launch on the start vector
        # taken from a 1-step run (work vector 0 holds u_1 after the run)
        nbytes = ftlm.ftlm_lanczos_workspace_bytes(b.handle, 1, 1, torch.float32)
        work = torch.empty(nbytes, dtype=torch.uint8, device=cuda_dev)
        out = ftlm.lanczos(b, 1, 1, seed=1, dist=ftlm.RADEMACHER, dtype=torch.float32, work=work)
        torch.cuda.synchronize()
        q = work[: 4 * b.dim].view(torch.float32).clone()
        del work, out
        q = q / torch.linalg.vector_norm(q.double()).float()
        hq = torch.empty_like(q)
        ftlm.ftlm_hv(b.handle, q, hq)
        alpha = torch.dot(q.double(), hq.double()).item()
        beta2 = torch.dot(hq.double(), hq.double()).item() - alpha**2
    assert abs(a1 - alpha) <= 1e-5 * (abs(alpha) + 1)
    assert abs(b1**2 - beta2) <= 1e-4 * beta2


def test_split_lanczos_at_full_size(cuda_dev):
    """The benchmark's H.v schedule at full size: 8 FP32 chains as one block on the
    N = 30 sector take the split (blocked walk A + transposed walk B) under AUTO.
    alpha_1 and beta_1 of every chain must match <q, Hq> and ||Hq||^2 - alpha_1^2
    computed through the one-walk H.v launch (whose rows are checked against the
    oracle above) on the same start vectors."""
    N, bonds = ICOSIDODECA
    R = 8
    with ftlm.Basis(N, 0, bonds, ftlm.RANK_CR) as b:
        assert ftlm.ftlm_basis_hv_schedule(b.handle, R, torch.float32) == ftlm.HV_SPLIT
        res = ftlm.lanczos(b, R, 2, seed=3, dist=ftlm.RADEMACHER, dtype=torch.float32, keep_coeffs=True)
        a1 = res["alpha"][:, 0].cpu().numpy()
        b1 = res["beta"][:, 0].cpu().numpy()
        del res
        torch.cuda.empty_cache()
        # the start block (work vector 0 after a 1-step run), then the one-walk H.v
        nbytes = ftlm.ftlm_lanczos_workspace_bytes(b.handle, R, 1, torch.float32)
        work = torch.empty(nbytes, dtype=torch.uint8, device=cuda_dev)
        out = ftlm.lanczos(b, R, 1, seed=3, dist=ftlm.RADEMACHER, dtype=torch.float32, work=work)
        torch.cuda.synchronize()
        q = work[: 4 * R * b.dim].view(torch.float32).view(b.dim, R).clone()
        del work, out
        torch.cuda.empty_cache()
        q = q / torch.linalg.vector_norm(q.double(), dim=0).float()
        hq = torch.empty_like(q)
        ftlm.ftlm_hv_block(b.handle, R, q, hq)
        alpha = (q.double() * hq.double()).sum(dim=0).cpu().numpy()
        beta2 = (hq.double() ** 2).sum(dim=0).cpu().numpy() - alpha**2
    np.testing.assert_allclose(a1, alpha, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(b1**2, beta2, rtol=1e-4)
