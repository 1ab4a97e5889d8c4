"""Sector setup on the GPU vs the oracle: basis enumeration, rank (CLT and CR)
and the CLT arrays of Eq. 18 must be bit-exact."""
import math

import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu

CASES = [(1, 0), (1, 1), (2, 1), (4, 2), (5, 0), (5, 5), (10, 5), (13, 4), (16, 8), (16, 3),
         (20, 10), (22, 11), (24, 12), (24, 20)]
MODES = [ftlm.RANK_CLT, ftlm.RANK_CR]


def ring_or_empty(N):
    return inputs.ring(N) if N >= 2 else (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("N,K", CASES)
def test_labels_bit_exact(cuda_dev, N, K, mode):
    ref = o.basis(N, K)
    with ftlm.Basis(N, 2 * K - N, ring_or_empty(N), mode) as b:
        assert b.dim == len(ref) == math.comb(N, K)
        lab = torch.empty(b.dim, dtype=torch.int64, device=cuda_dev)
        ftlm.ftlm_basis_labels(b.handle, 0, b.dim, lab)
        np.testing.assert_array_equal(lab.cpu().numpy().astype(np.uint64), ref)
        # a ragged window in the middle
        if b.dim > 10:
            f, c = b.dim // 3, b.dim // 3 + 1
            part = torch.empty(c, dtype=torch.int64, device=cuda_dev)
            ftlm.ftlm_basis_labels(b.handle, f, c, part)
            np.testing.assert_array_equal(part.cpu().numpy().astype(np.uint64), ref[f:f + c])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("N,K", [(4, 2), (10, 5), (16, 8), (16, 3), (22, 11), (24, 12)])
def test_rank_bit_exact(cuda_dev, N, K, mode):
    ref = o.basis(N, K)
    lut = o.full_lut(N, ref)
    rng = np.random.default_rng(N * 100 + K)
    labels = np.concatenate([
        ref[rng.integers(0, len(ref), size=min(len(ref), 20000))].astype(np.int64),
        rng.integers(0, 1 << N, size=20000),            # mostly outside the sector
        np.array([(1 << N), (1 << N) + 5, (1 << (N + 3)) - 1], dtype=np.int64),  # beyond 2^N
    ])
    want = np.where(labels < (1 << N), lut[np.minimum(labels, (1 << N) - 1)], -1)
    with ftlm.Basis(N, 2 * K - N, ring_or_empty(N), mode) as b:
        ld = torch.as_tensor(labels, device=cuda_dev)
        idx = torch.empty_like(ld)
        ftlm.ftlm_basis_rank(b.handle, ld, idx)
        np.testing.assert_array_equal(idx.cpu().numpy(), want)


@pytest.mark.parametrize("N,K", [(1, 1), (4, 2), (5, 2), (12, 6), (16, 8), (20, 7), (24, 12)])
def test_clt_arrays_match_eq18(cuda_dev, N, K):
    ref = o.basis(N, K)
    mask_ref, prefix_ref = o.clt_build(N, ref)
    with ftlm.Basis(N, 2 * K - N, ring_or_empty(N), ftlm.RANK_CLT) as b:
        nb = len(mask_ref)
        m = torch.empty(nb, dtype=torch.int32, device=cuda_dev)
        p = torch.empty(nb, dtype=torch.int32, device=cuda_dev)
        ftlm.ftlm_basis_clt(b.handle, m, p)
        np.testing.assert_array_equal(m.cpu().numpy().view(np.uint32), mask_ref)
        np.testing.assert_array_equal(p.cpu().numpy().view(np.uint32), prefix_ref)
        assert b.table_bytes >= 8 * nb + 4 * len(ref)  # Eq. 21 plus the basis array


def test_clt_export_rejected_in_cr_mode(cuda_dev):
    with ftlm.Basis(8, 0, inputs.ring(8), ftlm.RANK_CR) as b:
        m = torch.empty(8, dtype=torch.int32, device=cuda_dev)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_basis_clt(b.handle, m, m)
        assert e.value.status == ftlm.FTLM_EUNSUPPORTED


def test_labels_beyond_dimension_rejected(cuda_dev):
    with ftlm.Basis(8, 0, inputs.ring(8)) as b:
        lab = torch.empty(2, dtype=torch.int64, device=cuda_dev)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_basis_labels(b.handle, b.dim - 1, 2, lab)
        assert e.value.status == ftlm.FTLM_EINVAL


@pytest.mark.parametrize("name,N,K,bonds", [
    ("icosahedron", 12, 6, inputs.icosahedron()),
    ("lattice", 24, 12, inputs.square_j1j2()),
    ("random", 18, 7, inputs.random_graph(18, seed=1)),
])
def test_update_count_matches_eq10(cuda_dev, name, N, K, bonds):
    ref = o.basis(N, K)
    with ftlm.Basis(N, 2 * K - N, bonds) as b:
        assert b.updates == len(ref) + o.offdiag_terms(bonds, ref)
        # AUTO: CLT below 2^20 rows (its small tables fit), CR from there up
        assert b.mode == (ftlm.RANK_CLT if len(ref) < 1 << 20 else ftlm.RANK_CR)


def test_auto_mode_picks_cr_when_clt_cannot_be_built(cuda_dev):
    with ftlm.Basis(34, 32, inputs.ring(34)) as b:  # N > 32: no CLT
        assert b.mode == ftlm.RANK_CR


@pytest.mark.parametrize("wait", [True, False])
@pytest.mark.parametrize("two_s, N", [(1, 16), (2, 8)])
def test_create_sectors_equals_one_by_one(cuda_dev, two_s, N, wait):
    """ftlm_basis_create_sectors (one wait for all tables, or none: the uses below
    follow the builds on the same stream) builds the same sectors as single
    creations: dimensions, update counts, labels and Lanczos coefficients."""
    bonds = inputs.random_graph(N, seed=17)
    two_sz = ftlm.computed_two_sz(N, two_s)
    many = ftlm.Basis.sectors(N, two_sz, bonds, two_s=two_s, wait=wait)
    for tz, b in zip(two_sz, many):
        with ftlm.Basis(N, tz, bonds, two_s=two_s) as one:
            assert (b.dim, b.updates, b.mode) == (one.dim, one.updates, one.mode)
            n = min(b.dim, 4096)
            la, lb = (torch.empty(n, dtype=torch.int64, device=cuda_dev) for _ in range(2))
            ftlm.ftlm_basis_labels(b.handle, 0, n, la)
            ftlm.ftlm_basis_labels(one.handle, 0, n, lb)
            assert torch.equal(la, lb)
            if b.dim >= 2:
                m = min(10, b.dim)
                r1 = ftlm.lanczos(b, 4, m, seed=3, dtype=torch.float64, keep_coeffs=True)
                r2 = ftlm.lanczos(one, 4, m, seed=3, dtype=torch.float64, keep_coeffs=True)
                for k in ("alpha", "beta", "theta", "weight", "m_eff"):
                    assert torch.equal(r1[k], r2[k]), k
        b.close()


def test_create_sectors_rejects_bad_input_and_keeps_nothing(cuda_dev):
    bonds = inputs.ring(10)
    with pytest.raises(ftlm.FtlmError):
        ftlm.ftlm_basis_create_sectors(10, 1, [0, 2, 3], *bonds)   # 2 S^z = 3 has the wrong parity
    with pytest.raises(ftlm.FtlmError):
        ftlm.ftlm_basis_create_sectors(10, 1, [], *bonds)
