"""FP32 vector storage (FP64 reductions) against the FP64 oracle, on the paths the
FP32 benchmarks run: the CR Lanczos H.v with blocks of 8 chains on a large sector
(one walk and the split walk), the batch paths (persistent small-sector kernel and
multi-sector step kernels), and a served job.

Tolerances (the FP32 reading of the observables' tolerance form): relative 1e-4
where |O| >= 1e-6 max_T |O|, absolute 1e-4 max_T |O| below; Lanczos coefficients
1e-4 relative over the steps before orthogonality is lost.  The oracle's breakdown
threshold uses the FP32 unit roundoff, as the library does for FP32 vectors.
"""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs, serve

pytestmark = pytest.mark.gpu

RTOL32 = 1e-4


def assert_observable_close(got, want, rtol=RTOL32, what=""):
    scale = np.max(np.abs(want))
    band = np.abs(want) >= 1e-6 * scale
    err_rel = np.abs(got[band] - want[band]) / np.abs(want[band])
    err_abs = np.abs(got[~band] - want[~band])
    assert np.all(err_rel <= rtol), (what, float(err_rel.max()))
    assert np.all(err_abs <= rtol * scale), (what, float(err_abs.max()) if err_abs.size else 0.0)


# --------------------------------------------------------------------------
# The 4 x 6 J1-J2 lattice, S^z = 0: D = 2 704 156, 96 bonds, CR with blocks of 8.
J1J2_N, J1J2_K, J1J2_M, J1J2_SEED = 24, 12, 12, 1


@pytest.fixture(scope="module")
def j1j2_oracle_chains():
    """The oracle's FP64 coefficients of chains 0 and 1 (Rademacher, seed 1)."""
    bonds = inputs.square_j1j2(4, 6, 1.0, 0.5)
    b = o.basis(J1J2_N, J1J2_K)
    lut = o.full_lut(J1J2_N, b)
    tau = o.breakdown_tol(bonds[2], o.U32)
    out = []
    for r in range(2):
        v = o.start_vector(J1J2_SEED, J1J2_N, J1J2_K, r, o.RADEMACHER, len(b))
        out.append(o.lanczos(bonds, b, v, J1J2_M, tau, lut))
    return bonds, out


@pytest.mark.parametrize("schedule", [ftlm.HV_ONE_WALK, ftlm.HV_SPLIT])
def test_j1j2_sz0_fp32_block8_matches_oracle(cuda_dev, j1j2_oracle_chains, schedule):
    bonds, chains = j1j2_oracle_chains
    with ftlm.Basis(J1J2_N, 0, bonds, ftlm.RANK_CR) as b:
        assert b.dim == 2704156
        b.set_schedule(schedule)
        res = ftlm.lanczos(b, 8, J1J2_M, seed=J1J2_SEED, dist=ftlm.RADEMACHER, dtype=torch.float32,
                           keep_coeffs=True)
        torch.cuda.synchronize()
    for r, (a, bt, m) in enumerate(chains):
        assert m == J1J2_M and int(res["m_eff"][r]) == J1J2_M
        np.testing.assert_allclose(res["alpha"][r, :m].cpu().numpy(), a, rtol=RTOL32, atol=1e-5)
        np.testing.assert_allclose(res["beta"][r, :m - 1].cpu().numpy(), bt, rtol=RTOL32)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("block", [4, 8])
def test_fp32_batch_paths_match_oracle(cuda_dev, block):
    """Every S^z >= 0 sector of a random N = 18 cluster in one FP32 batch: the two
    largest (D = 48620, 43758) run on the multi-sector step kernels, the rest in the
    persistent small-sector kernel; E, C, chi vs the FP64 oracle."""
    N, M, R, seed = 18, 30, 5, 7
    T = inputs.log_t_grid(50, 0.05, 10.0)
    bonds = inputs.random_graph(N, seed=44)
    bases = [ftlm.Basis(N, tz, bonds) for tz in ftlm.computed_two_sz(N)]
    assert max(b.dim for b in bases) > 32768 and min(b.dim for b in bases) <= 32768
    with ftlm.Batch([(b, R, seed, 0) for b in bases], M, ftlm.GAUSS, torch.float32, block) as batch:
        res = batch.run()
        obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)], torch.as_tensor(T, device=cuda_dev),
                          R, M)
        torch.cuda.synchronize()
    ref = o.thermo(o.run_ftlm(N, bonds, R, M, seed=seed, u=o.U32), T)
    for k in ("E", "C", "chi"):
        assert_observable_close(obs[k].cpu().numpy(), ref[k], what=k)
    for b in bases:
        b.close()


def test_fp32_multi_sector_kernels_match_oracle_coefficients(cuda_dev):
    """The multi-sector step kernels in FP32 (one unit of 8 chains of the D = 48620
    sector): Ritz moments sum_k w theta^p, p = 0, 1, 2, which the Lanczos recurrence
    fixes from alpha_1 and beta_1, vs the oracle's chains."""
    N, K, M, R, seed = 18, 9, 20, 8, 3
    bonds = inputs.random_graph(N, seed=44)
    with ftlm.Basis(N, 0, bonds) as b:
        with ftlm.Batch([(b, R, seed, 0)], M, ftlm.RADEMACHER, torch.float32, 8) as batch:
            got = batch.run()[0]
            torch.cuda.synchronize()
            th, w = got["theta"].cpu().numpy(), got["weight"].cpu().numpy()
            m_got = got["m_eff"].cpu().numpy()
    bo = o.basis(N, K)
    lut = o.full_lut(N, bo)
    for r in range(R):
        a, bt, m = o.lanczos(bonds, bo, o.start_vector(seed, N, K, r, o.RADEMACHER, len(bo)), M,
                             o.breakdown_tol(bonds[2], o.U32), lut)
        assert m_got[r] == m
        k = m
        np.testing.assert_allclose(w[r, :k].sum(), 1.0, atol=1e-12)
        np.testing.assert_allclose((w[r, :k] * th[r, :k]).sum(), a[0], rtol=RTOL32)
        np.testing.assert_allclose((w[r, :k] * th[r, :k] ** 2).sum(), a[0] ** 2 + bt[0] ** 2, rtol=RTOL32)


# --------------------------------------------------------------------------
def test_served_fp32_job_matches_oracle(cuda_dev):
    """A ladder N = 18 in a field, served in FP32 next to other jobs: E, C, chi and
    <S^z> vs the oracle's FP64 FTLM from the same start vectors."""
    T = inputs.log_t_grid(40, 0.05, 10.0)
    bonds = inputs.ladder(18, 0.7, 1.1)
    job = serve.Job(job_id=0, N=18, bonds=bonds, h=0.6, seed=77)
    reqs, _ = inputs.serving_requests(5, 400.0, seed=3, sizes=(8, 10, 12, 14))
    filler = [serve.Job(job_id=1 + i, N=r["N"], bonds=r["bonds"], h=r["h"], seed=600 + i) for i, r in enumerate(reqs)]
    eng = serve.Engine(R=4, M=30, dtype=torch.float32, block=4, T=T, memory_budget=1 << 30)
    done = eng.run([job] + filler)
    eng.close()
    got = next(j for j in done if j.job_id == 0).result
    ref = o.thermo(o.run_ftlm(18, bonds, 4, 30, seed=77, dist=o.GAUSS, u=o.U32), T, g=2.0, h=0.6)
    for row, k in enumerate(("E", "C", "chi", "mag")):
        assert_observable_close(got[row], ref[k], what=k)
