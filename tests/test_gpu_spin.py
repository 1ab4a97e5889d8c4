"""General local spin s on the GPU (ftlm_basis_create_spin) against the spin-s
oracle: base-d labels and ranks bit-exact, H.v to FP64 rounding, N_nz of Eq. 10
(Table 1), Lanczos coefficients from shared and from seeded start vectors, and the
FTLM observables."""
import numpy as np
import pytest
import torch

import oracle as o
from oracle import spin
from paper_2605_26261_gb300 import ftlm, inputs
from tests.conftest import golden

pytestmark = pytest.mark.gpu

CASES = [  # (N, two_s, two_sz, bonds)
    (12, 2, 0, inputs.icosahedron()),
    (8, 3, 2, inputs.random_graph(8, seed=3, dmin=2, dmax=4)),
    (6, 6, 0, inputs.ring(6, J=0.9)),
    (10, 2, 4, inputs.ladder(10, 0.7, 1.2)),
    (5, 5, -3, inputs.random_graph(5, seed=7, dmin=2, dmax=3)),
    (16, 2, 14, inputs.ring(16)),
    (7, 7, 1, inputs.ring(7, J=1.1)),       # s = 7/2, the largest local spin
    (4, 7, 26, inputs.ring(4)),             # one flipped quantum: D = 4
    (4, 7, 28, inputs.ring(4)),             # fully polarized: D = 1, diagonal only
]


def ids(c):
    return f"N{c[0]}_2s{c[1]}_2sz{c[2]}"


@pytest.mark.parametrize("case", CASES, ids=[ids(c) for c in CASES])
def test_labels_and_ranks_bit_exact(cuda_dev, case):
    N, two_s, two_sz, bonds = case
    A = spin.sector_A(N, two_s, two_sz)
    ref = spin.basis(N, two_s, A)
    with ftlm.Basis(N, two_sz, bonds, two_s=two_s) as b:
        assert b.dim == len(ref) and b.mode == ftlm.RANK_CR
        assert b.updates == spin.nnz(N, two_s, A, len(bonds[2]))
        lab = torch.empty(b.dim, dtype=torch.int64, device=cuda_dev)
        ftlm.ftlm_basis_labels(b.handle, 0, b.dim, lab)
        assert np.array_equal(lab.cpu().numpy().astype(np.uint64), ref)
        idx = torch.empty_like(lab)
        ftlm.ftlm_basis_rank(b.handle, lab, idx)
        assert np.array_equal(idx.cpu().numpy(), np.arange(b.dim))
        # labels outside the sector: other digit sums, and >= d^N
        d = two_s + 1
        rng = np.random.default_rng(1)
        cand = rng.integers(0, d**N, size=2000, dtype=np.int64)
        cand = np.concatenate([cand, [d**N, d**N + 5]])
        got = torch.empty(len(cand), dtype=torch.int64, device=cuda_dev)
        ftlm.ftlm_basis_rank(b.handle, torch.as_tensor(cand, device=cuda_dev), got)
        want = np.array([np.searchsorted(ref, c) if (c < d**N and np.searchsorted(ref, c) < len(ref)
                                                     and ref[np.searchsorted(ref, c)] == c) else -1
                         for c in cand.astype(np.uint64)])
        assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("case", CASES, ids=[ids(c) for c in CASES])
def test_hv_matches_oracle(cuda_dev, case):
    N, two_s, two_sz, bonds = case
    A = spin.sector_A(N, two_s, two_sz)
    ref_b = spin.basis(N, two_s, A)
    x = inputs.seeded_vector(len(ref_b), 11)
    want = spin.hv(N, two_s, bonds, ref_b, x)
    scale = np.max(np.abs(want))
    with ftlm.Basis(N, two_sz, bonds, two_s=two_s) as b:
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-6)):
            xd = torch.as_tensor(x, dtype=dt, device=cuda_dev)
            yd = torch.empty_like(xd)
            ftlm.ftlm_hv(b.handle, xd, yd)
            np.testing.assert_allclose(yd.cpu().numpy(), want, rtol=0, atol=tol * scale * 10)


@pytest.mark.parametrize("B", [4, 8, 16])
def test_block_columns_equal_single_vectors(cuda_dev, B):
    N, two_s, two_sz, bonds = CASES[0]
    with ftlm.Basis(N, two_sz, bonds, two_s=two_s) as b:
        for dt in (torch.float32, torch.float64):
            X = inputs.hashed_vector_torch(b.dim * B, dt, cuda_dev).view(b.dim, B)
            Y = torch.empty_like(X)
            ftlm.ftlm_hv_block(b.handle, B, X, Y)
            for r in range(B):
                y = torch.empty(b.dim, dtype=dt, device=cuda_dev)
                ftlm.ftlm_hv(b.handle, X[:, r].contiguous(), y)
                assert torch.equal(Y[:, r], y), (dt, r)


def test_table1_spin2_sector_and_sampled_rows(cuda_dev):
    # s = 2 icosahedron, M = 0: D_0 and N_nz of Table 1, and 40 960 sampled rows of
    # H.v (FP64) against the oracle's rows
    g = golden("table1_spin_s.txt")
    bonds = inputs.icosahedron()
    N, two_s = 12, 4
    with ftlm.Basis(N, 0, bonds, two_s=two_s) as b:
        assert b.dim == int(g["D0"].split(",")[3])
        assert b.updates == int(g["N_nz"].split(",")[3])
        ref_b = spin.basis(N, two_s, spin.sector_A(N, two_s, 0))
        x = inputs.hashed_value(np.arange(b.dim))
        xd = torch.as_tensor(x, device=cuda_dev)
        yd = torch.empty_like(xd)
        ftlm.ftlm_hv(b.handle, xd, yd)
        y = yd.cpu().numpy()
        for t0 in np.linspace(0, b.dim - 1024, 40).astype(np.int64):
            want = spin.hv_range(N, two_s, bonds, ref_b, x, int(t0), int(t0) + 1024)
            np.testing.assert_allclose(y[t0:t0 + 1024], want, rtol=1e-13, atol=1e-13)


def test_lanczos_coefficients(cuda_dev):
    N, two_s, two_sz, bonds = CASES[1]
    A = spin.sector_A(N, two_s, two_sz)
    ref_b = spin.basis(N, two_s, A)
    D, M, R = len(ref_b), 40, 3
    tau = spin.tau_of(bonds[2], two_s)
    with ftlm.Basis(N, two_sz, bonds, two_s=two_s) as b:
        # from the oracle's own start vectors, and from the seeded generator
        starts = np.stack([inputs.seeded_vector(D, 60 + r) for r in range(R)])
        got = ftlm.lanczos(b, R, M, dtype=torch.float64, start=torch.as_tensor(starts, device=cuda_dev),
                           keep_coeffs=True)
        seeded = ftlm.lanczos(b, R, M, seed=5, dist=ftlm.GAUSS, dtype=torch.float64, keep_coeffs=True)
        torch.cuda.synchronize()
        for r in range(R):
            for res, v in ((got, starts[r]), (seeded, spin.start_vector(5, N, two_s, A, r, o.GAUSS, D))):
                a, bt, m = spin.lanczos(N, two_s, bonds, ref_b, v, M, tau)
                np.testing.assert_allclose(res["alpha"][r, :15].cpu().numpy(), a[:15], rtol=1e-10, atol=1e-12)
                np.testing.assert_allclose(res["beta"][r, :15].cpu().numpy(), bt[:15], rtol=1e-10)


@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-9), (torch.float32, 1e-4)])
def test_ftlm_observables_match_oracle(cuda_dev, dtype, rtol):
    N, two_s, R, M, seed = 6, 2, 4, 30, 9
    bonds = inputs.random_graph(N, seed=2, dmin=2, dmax=4)
    T = inputs.log_t_grid(40, 0.1, 10.0)
    sectors = []
    for tz in ftlm.computed_two_sz(N, two_s):
        b = ftlm.Basis(N, tz, bonds, two_s=two_s)
        sectors.append((tz, b.dim, ftlm.lanczos(b, R, M, seed=seed, dist=ftlm.GAUSS, dtype=dtype)))
        torch.cuda.synchronize()
        b.close()
    for h in (0.0, 0.7):
        obs = ftlm.thermo(sectors, torch.as_tensor(T, device=cuda_dev), R, M, h=h)
        ref = o.thermo(spin.run_ftlm(N, two_s, bonds, R, M, seed=seed, dist=o.GAUSS,
                                     u=o.U64 if dtype == torch.float64 else o.U32), T, h=h)
        for k in ("E", "C", "chi", "mag"):
            want = ref[k]
            scale = max(np.max(np.abs(want)), 1.0)  # <S^z> vanishes at h = 0 up to roundoff
            np.testing.assert_allclose(obs[k].cpu().numpy(), want, rtol=rtol, atol=rtol * scale)


def test_spin3_icosahedron_symmetric_at_full_size(cuda_dev):
    # s = 3, M = 0: D_0 = 786 588 243 (Table 1); <u, H v> = <H u, v> over the
    # whole sector with FP64 vectors (6.3 GB each)
    g = golden("table1_spin_s.txt")
    with ftlm.Basis(12, 0, inputs.icosahedron(), two_s=6) as b:
        assert b.dim == int(g["D0"].split(",")[5]) and b.updates == int(g["N_nz"].split(",")[5])
        u = inputs.hashed_vector_torch(b.dim, torch.float64, cuda_dev)
        v = torch.roll(u, 12345)
        hu, hv = torch.empty_like(u), torch.empty_like(u)
        ftlm.ftlm_hv(b.handle, u, hu)
        ftlm.ftlm_hv(b.handle, v, hv)
        a, c = torch.dot(u, hv).item(), torch.dot(hu, v).item()
        assert abs(a - c) <= 1e-11 * abs(a)
        del u, v, hu, hv
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-10), (torch.float32, 1e-5)])
def test_batch_runs_spin_sectors(cuda_dev, dtype, rtol):
    # every sector of a spin-1 ring N = 10 (D up to 8953) through the multi-sector
    # path of a batch, against per-sector ftlm_lanczos (same chains), and the
    # thermodynamics against the oracle
    N, two_s, R, M = 10, 2, 6, 25
    bonds = inputs.ring(N, J=0.8)
    bases = [ftlm.Basis(N, tz, bonds, two_s=two_s) for tz in ftlm.computed_two_sz(N, two_s)]
    with ftlm.Batch([(b, R, 3, 0) for b in bases], M, ftlm.GAUSS, dtype, 4) as batch:
        res = batch.run()
        torch.cuda.synchronize()
        for b, got in zip(bases, res):
            ref = ftlm.lanczos(b, R, M, seed=3, dist=ftlm.GAUSS, dtype=dtype)
            torch.cuda.synchronize()
            assert torch.equal(got["m_eff"], ref["m_eff"])
            for r in range(R):
                m = int(got["m_eff"][r])
                for beta in (0.3, 1.0, 3.0):
                    a = (got["weight"][r, :m] * torch.exp(-beta * (got["theta"][r, :m] - got["theta"][r, 0]))).sum()
                    e = (ref["weight"][r, :m] * torch.exp(-beta * (ref["theta"][r, :m] - got["theta"][r, 0]))).sum()
                    assert abs(a.item() - e.item()) <= rtol * abs(e.item())
        if dtype == torch.float64:
            T = inputs.log_t_grid(30, 0.1, 10.0)
            obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)],
                              torch.as_tensor(T, device=cuda_dev), R, M)
            ref = o.thermo(spin.run_ftlm(N, two_s, bonds, R, M, seed=3, dist=o.GAUSS), T)
            for k in ("E", "C", "chi"):
                np.testing.assert_allclose(obs[k].cpu().numpy(), ref[k], rtol=1e-9,
                                           atol=1e-12 * np.max(np.abs(ref[k])))
    for b in bases:
        b.close()


def test_create_rejects_bad_spin_arguments(cuda_dev):
    bonds = inputs.ring(6)
    for args, status in (((6, 2, 1), ftlm.FTLM_EINVAL),      # parity of two_sz
                         ((6, 2, 14), ftlm.FTLM_EINVAL),     # |two_sz| > N two_s
                         ((6, 8, 0), ftlm.FTLM_EUNSUPPORTED),  # s = 4
                         ((17, 2, 0), ftlm.FTLM_EUNSUPPORTED)):  # N > 16
        N, two_s, two_sz = args
        bb = inputs.ring(N) if N != 6 else bonds
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.Basis(N, two_sz, bb, two_s=two_s)
        assert e.value.status == status
