"""H.v on the GPU (CLT and CR, FP32 and FP64) vs the oracle, element by element.

Tolerance: every output row is a sum of at most n_bonds + 1 terms of magnitude at
most (sum_b |J_b|) max|x|, so rounding in the storage type u (2^-24 FP32, 2^-53
FP64) bounds the difference to the FP64 oracle by (n_bonds + 2) u sum|J| max|x|.
"""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu

U = {torch.float32: 2.0**-24, torch.float64: 2.0**-53}

GRAPHS = {
    "dimer": (2, inputs.dimer(0.8)),
    "ring16": (16, inputs.ring(16)),
    "icosahedron": (12, inputs.icosahedron()),
    "random18": (18, inputs.random_graph(18, seed=2)),
    "ladder20": (20, inputs.ladder(20, 0.7, 1.2)),
    "lattice4x6": (24, inputs.square_j1j2()),
}


def tol(bonds, x, dtype):
    return (len(bonds[2]) + 2) * U[dtype] * np.sum(np.abs(bonds[2])) * np.max(np.abs(x))


def run_hv(dev, N, K, bonds, x, mode, dtype):
    with ftlm.Basis(N, 2 * K - N, bonds, mode) as b:
        xd = torch.as_tensor(x, device=dev).to(dtype)
        yd = torch.full_like(xd, float("nan"))
        ftlm.ftlm_hv(b.handle, xd, yd)
        return yd.double().cpu().numpy(), xd.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_hv_matches_oracle(cuda_dev, name, mode, dtype):
    N, bonds = GRAPHS[name]
    Ks = sorted({N // 2, max(0, N // 2 - 3), N - 1, N}) if N > 2 else [0, 1, 2]
    for K in Ks:
        ref_b = o.basis(N, K)
        x = inputs.seeded_vector(len(ref_b), 100 + K)
        y, xr = run_hv(cuda_dev, N, K, bonds, x, mode, dtype)
        # the oracle sees the same (dtype-rounded) input vector
        y_ref = o.hv(bonds, ref_b, xr, o.full_lut(N, ref_b))
        err = np.max(np.abs(y - y_ref))
        assert err <= tol(bonds, xr, dtype), (K, err)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
def test_all_ones_is_exact_eigenvector(cuda_dev, mode, dtype):
    # The uniform vector of a sector is an S = N/2 state: H 1 = (sum J / 4) 1,
    # exactly for dyadic couplings.
    N = 20
    bi, bj, J = inputs.random_graph(N, seed=8)
    J = np.round(J * 16) / 16
    for K in (3, 10, 19):
        with ftlm.Basis(N, 2 * K - N, (bi, bj, J), mode) as b:
            x = torch.ones(b.dim, dtype=dtype, device=cuda_dev)
            y = torch.empty_like(x)
            ftlm.ftlm_hv(b.handle, x, y)
            assert torch.all(y == J.sum() / 4).item()


@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
def test_hv_is_symmetric(cuda_dev, mode):
    N, K = 24, 12
    bonds = inputs.square_j1j2()
    with ftlm.Basis(N, 0, bonds, mode) as b:
        g = torch.Generator(device="cpu").manual_seed(3)
        u = torch.randn(b.dim, generator=g, dtype=torch.float64).to(cuda_dev)
        v = torch.randn(b.dim, generator=g, dtype=torch.float64).to(cuda_dev)
        hu, hv = torch.empty_like(u), torch.empty_like(v)
        ftlm.ftlm_hv(b.handle, u, hu)
        ftlm.ftlm_hv(b.handle, v, hv)
        a, c = torch.dot(v, hu).item(), torch.dot(hv, u).item()
        assert abs(a - c) <= 1e-11 * abs(a)


def test_clt_and_cr_agree_bitwise_in_fp64_on_ring(cuda_dev):
    # Same bonds, same per-row term set; only the summation order of the bond loop
    # can differ, and on a ring with J = 1 every partial sum is exact.
    N, K = 20, 10
    bonds = inputs.ring(N)
    x = torch.as_tensor(np.round(inputs.seeded_vector(184756, 1) * 1024) / 1024, device=cuda_dev)
    ys = []
    for mode in (ftlm.RANK_CLT, ftlm.RANK_CR):
        with ftlm.Basis(N, 0, bonds, mode) as b:
            y = torch.empty_like(x)
            ftlm.ftlm_hv(b.handle, x, y)
            ys.append(y)
    assert torch.equal(ys[0], ys[1])


def test_hv_rejects_bad_vectors(cuda_dev):
    with ftlm.Basis(8, 0, inputs.ring(8)) as b:
        x = torch.ones(b.dim + 1, dtype=torch.float64, device=cuda_dev)
        with pytest.raises(ftlm.FtlmError):
            ftlm.ftlm_hv(b.handle, x, x)  # in place not allowed
        with pytest.raises(ftlm.FtlmError):
            ftlm.ftlm_hv(b.handle, x[1:], x[:-1].clone())  # misaligned input


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
@pytest.mark.parametrize("B", [4, 8, 16])
def test_block_hv_columns_equal_single_hv(cuda_dev, mode, dtype, B):
    # Interleaved block of B vectors: each column is bit-identical to ftlm_hv.
    N, K = 18, 8
    bonds = inputs.random_graph(N, seed=21)
    with ftlm.Basis(N, 2 * K - N, bonds, mode) as b:
        g = torch.Generator(device="cpu").manual_seed(B)
        X = torch.randn((b.dim, B), generator=g, dtype=torch.float64).to(dtype).to(cuda_dev)
        Y = torch.full_like(X, float("nan"))
        ftlm.ftlm_hv_block(b.handle, B, X, Y)
        for r in range(B):
            x = X[:, r].contiguous()
            y = torch.empty_like(x)
            ftlm.ftlm_hv(b.handle, x, y)
            assert torch.equal(Y[:, r], y), r


def test_block_hv_rejects_other_widths(cuda_dev):
    with ftlm.Basis(8, 0, inputs.ring(8)) as b:
        X = torch.ones((b.dim, 3), dtype=torch.float32, device=cuda_dev)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_hv_block(b.handle, 3, X, X.clone())
        assert e.value.status == ftlm.FTLM_EINVAL
