"""The split Lanczos H.v against the oracle.

The split runs each Lanczos step's H.v as two walks (walk A: the lo-lo and cross
bonds in tiles of 32 low-pattern columns x a run of high patterns; walk B: the
high-high bonds in the transposed order).  FP64 chains fed the oracle's own start
vectors must reproduce the oracle's Lanczos coefficients (Paige's ordering) to
1e-10 relative before orthogonality is lost, for every block width and on sectors
whose column chunks are ragged, whose popcount classes hold fewer high patterns
than one run, and whose low popcount range stops at the edge of the low block; the
FP32 chains agree to 1e-4 (the FP32 tolerance of the coefficients).
"""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu

# (sites, 2 S^z, bonds), each with high-high bonds: a random cluster at S^z = 0; a
# deeper sector of another (K = 8 of 20); an odd ring (K = 9 of 17: 3 high sites,
# runs cut short); a ladder with few up spins (K = 5 of 20: low popcounts 0 .. 5
# only); the N = 16 ring at K = 13 (2 high sites, low popcounts 11 .. 13).
CASES = [
    (18, 0, inputs.random_graph(18, seed=14)),
    (20, -4, inputs.random_graph(20, seed=12)),
    (17, 1, inputs.ring(17)),
    (20, -10, inputs.ladder(20, 0.7, 1.2)),
    (16, 10, inputs.ring(16)),
]


def oracle_coeffs(N, K, bonds, starts, M, u=o.U64):
    b = o.basis(N, K)
    lut = o.full_lut(N, b)
    return [o.lanczos(bonds, b, s, M, o.breakdown_tol(bonds[2], u), lut) for s in starts]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("block", [1, 4, 8, 16])
def test_split_fp64_matches_oracle(cuda_dev, case, block):
    N, tz, bonds = CASES[case]
    K = (N + tz) // 2
    M, R = 30, max(block, 2)
    D = len(o.basis(N, K))
    starts = np.stack([inputs.seeded_vector(D, 300 + r) for r in range(R)])
    ftlm.ftlm_lanczos_set_block(block)
    try:
        with ftlm.Basis(N, tz, bonds, ftlm.RANK_CR) as b:
            b.set_schedule(ftlm.HV_SPLIT)
            assert ftlm.ftlm_basis_hv_schedule(b.handle, block, ftlm.F64) == ftlm.HV_SPLIT
            res = ftlm.lanczos(b, R, M, dtype=torch.float64, start=torch.as_tensor(starts, device=cuda_dev),
                               keep_coeffs=True)
            torch.cuda.synchronize()
    finally:
        ftlm.ftlm_lanczos_set_block(0)
    for r, (a, bt, m) in enumerate(oracle_coeffs(N, K, bonds, starts[:R], M)):
        k = min(m, 15)  # the first steps precede any loss of orthogonality
        assert int(res["m_eff"][r]) == m
        np.testing.assert_allclose(res["alpha"][r, :k].cpu().numpy(), a[:k], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(res["beta"][r, :k - 1].cpu().numpy(), bt[:k - 1], rtol=1e-10)


@pytest.mark.parametrize("case", [0, 2, 3])
@pytest.mark.parametrize("block", [8, 16])
def test_split_fp32_matches_oracle(cuda_dev, case, block):
    N, tz, bonds = CASES[case]
    K = (N + tz) // 2
    M, R, seed = 12, block, 21
    ftlm.ftlm_lanczos_set_block(block)
    try:
        with ftlm.Basis(N, tz, bonds, ftlm.RANK_CR) as b:
            b.set_schedule(ftlm.HV_SPLIT)
            res = ftlm.lanczos(b, R, M, seed=seed, dist=ftlm.RADEMACHER, dtype=torch.float32, keep_coeffs=True)
            torch.cuda.synchronize()
    finally:
        ftlm.ftlm_lanczos_set_block(0)
    D = len(o.basis(N, K))
    starts = [o.start_vector(seed, N, K, r, o.RADEMACHER, D) for r in range(2)]
    for r, (a, bt, m) in enumerate(oracle_coeffs(N, K, bonds, starts, M, o.U32)):
        k = min(m, M)
        np.testing.assert_allclose(res["alpha"][r, :k].cpu().numpy(), a[:k], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(res["beta"][r, :k - 1].cpu().numpy(), bt[:k - 1], rtol=1e-4)


def test_split_and_one_walk_agree_with_walk_b_tile_sizes(cuda_dev):
    """FP64 blocks of 4 on one sector: the one walk, and the split with 1, 8 and 32
    high patterns per walk-B tile, give the same coefficients to rounding."""
    N, tz, bonds = CASES[1]
    R, M = 4, 25
    out = []
    for sched, rows in ((ftlm.HV_ONE_WALK, 0), (ftlm.HV_SPLIT, 1), (ftlm.HV_SPLIT, 8), (ftlm.HV_SPLIT, 32)):
        with ftlm.Basis(N, tz, bonds, ftlm.RANK_CR) as b:
            b.set_schedule(sched, rows)
            res = ftlm.lanczos(b, R, M, seed=5, dist=ftlm.GAUSS, dtype=torch.float64, keep_coeffs=True)
            torch.cuda.synchronize()
        out.append((res["alpha"][:, :15].cpu().numpy(), res["beta"][:, :14].cpu().numpy()))
    for a, bt in out[1:]:
        np.testing.assert_allclose(a, out[0][0], rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(bt, out[0][1], rtol=1e-11)
