"""Lanczos chains and the Ritz step on the GPU vs the oracle.

FP64 chains fed the oracle's own start vectors must reproduce the oracle's
Lanczos coefficients to 1e-10 relative before orthogonality is lost; seeded chains
regenerate the same start vectors on the device (same counter-based generator,
separately implemented).  FP32 storage agrees to 1e-4 over the first steps.
"""
import numpy as np
import pytest
import torch

import oracle as o
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu


def oracle_chain(bonds, N, K, start, M, u=o.U64):
    b = o.basis(N, K)
    return o.lanczos(bonds, b, start, M, o.breakdown_tol(bonds[2], u), o.full_lut(N, b))


@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
def test_fp64_coefficients_from_given_start(cuda_dev, mode):
    N, K, M, R = 18, 9, 40, 3
    bonds = inputs.random_graph(N, seed=5)
    D = len(o.basis(N, K))
    starts = np.stack([inputs.seeded_vector(D, 50 + r) for r in range(R)])
    with ftlm.Basis(N, 0, bonds, mode) as b:
        res = ftlm.lanczos(b, R, M, dtype=torch.float64, start=torch.as_tensor(starts, device=cuda_dev),
                           keep_coeffs=True)
        torch.cuda.synchronize()
    for r in range(R):
        a, bt, m = oracle_chain(bonds, N, K, starts[r], M)
        assert int(res["m_eff"][r]) == m == M
        # the first 15 steps precede any loss of orthogonality
        np.testing.assert_allclose(res["alpha"][r, :15].cpu().numpy(), a[:15], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(res["beta"][r, :15].cpu().numpy(), bt[:15], rtol=1e-10)


@pytest.mark.parametrize("R", [4, 8, 13])  # blocks of 4 / 8 / 8 + 4 + 1 chains
@pytest.mark.parametrize("dist", [ftlm.GAUSS, ftlm.RADEMACHER])
def test_seeded_start_vectors_match_oracle_generator(cuda_dev, dist, R):
    N, K, M, seed = 16, 8, 12, 1234
    bonds = inputs.ring(N)
    with ftlm.Basis(N, 0, bonds) as b:
        res = ftlm.lanczos(b, R, M, seed=seed, dist=dist, dtype=torch.float64, keep_coeffs=True)
        torch.cuda.synchronize()
    for r in range(R):
        v = o.start_vector(seed, N, K, r, dist)
        a, bt, m = oracle_chain(bonds, N, K, v, M)
        np.testing.assert_allclose(res["alpha"][r, :m].cpu().numpy(), a, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(res["beta"][r, :m - 1].cpu().numpy(), bt, rtol=1e-10)


@pytest.mark.parametrize("R", [2, 8])  # single chains / one block of 8
@pytest.mark.parametrize("mode", [ftlm.RANK_CLT, ftlm.RANK_CR])
def test_fp32_coefficients_close_to_fp64_oracle(cuda_dev, mode, R):
    N, K, M = 20, 10, 20
    bonds = inputs.ladder(20, 0.6, 1.0)
    with ftlm.Basis(N, 0, bonds, mode) as b:
        res = ftlm.lanczos(b, R, M, seed=9, dtype=torch.float32, keep_coeffs=True)
        torch.cuda.synchronize()
    for r in range(R):
        v = o.start_vector(9, N, K, r, o.GAUSS)
        a, bt, m = oracle_chain(bonds, N, K, v, M, o.U32)
        np.testing.assert_allclose(res["alpha"][r, :m].cpu().numpy(), a, rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(res["beta"][r, :m - 1].cpu().numpy(), bt, rtol=1e-4)


@pytest.mark.parametrize("R", [3, 8])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_breakdown_at_krylov_dimension(cuda_dev, dtype, R):
    # One down spin on a 12-ring: 7 distinct levels, the chain must stop after 7.
    N = 12
    bonds = inputs.ring(N)
    with ftlm.Basis(N, N - 2, bonds) as b:
        res = ftlm.lanczos(b, R, 12, seed=5, dtype=dtype)
        torch.cuda.synchronize()
        assert res["m_eff"].tolist() == [7] * R
        th = res["theta"][0, :7].cpu().numpy()
        ev = np.unique(np.round(np.linalg.eigvalsh(o.dense_h(bonds, o.basis(N, N - 1))), 8))
        np.testing.assert_allclose(np.sort(th), ev, atol=1e-9 if dtype == torch.float64 else 1e-5)
        w = res["weight"].cpu().numpy()
        np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-12)
        assert np.all(w[:, 7:] == 0) and np.all(res["theta"][:, 7:].cpu().numpy() == 0)


def test_dimension_one_and_two_sectors(cuda_dev):
    N = 10
    bonds = inputs.random_graph(N, seed=3)
    with ftlm.Basis(N, N, bonds) as b:  # all up: D = 1
        res = ftlm.lanczos(b, 2, 50, dtype=torch.float64)
        torch.cuda.synchronize()
        assert res["m_eff"].tolist() == [1, 1]
        np.testing.assert_allclose(res["theta"][:, 0].cpu().numpy(), bonds[2].sum() / 4, rtol=1e-14)
        np.testing.assert_array_equal(res["weight"][:, 0].cpu().numpy(), 1.0)
    with ftlm.Basis(2, 0, inputs.dimer(1.0)) as b:  # D = 2: singlet and triplet
        res = ftlm.lanczos(b, 1, 10, dtype=torch.float64)
        torch.cuda.synchronize()
        assert int(res["m_eff"][0]) == 2
        np.testing.assert_allclose(res["theta"][0, :2].cpu().numpy(), [-0.75, 0.25], atol=1e-14)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("R", [2, 4, 8])
def test_zero_start_vector_gives_empty_chain(cuda_dev, R, dtype):
    # A zero start vector ends its chain at once without disturbing the other
    # chains of its block.
    N, K = 10, 5
    bonds = inputs.ring(N)
    with ftlm.Basis(N, 0, bonds) as b:
        start = torch.as_tensor(np.stack([inputs.seeded_vector(b.dim, 70 + r) for r in range(R)]), device=cuda_dev)
        start[0].zero_()
        res = ftlm.lanczos(b, R, 10, dtype=dtype, start=start, keep_coeffs=True)
        torch.cuda.synchronize()
        assert int(res["m_eff"][0]) == 0
        assert torch.all(res["weight"][0] == 0).item()
        for r in range(1, R):
            a, bt, m = oracle_chain(bonds, N, K, start[r].cpu().numpy(), 10,
                                    o.U64 if dtype == torch.float64 else o.U32)
            assert int(res["m_eff"][r]) == m
            rtol = 1e-10 if dtype == torch.float64 else 1e-4
            np.testing.assert_allclose(res["alpha"][r, :m].cpu().numpy(), a, rtol=rtol, atol=10 * rtol)


def test_workspace_too_small_is_rejected(cuda_dev):
    with ftlm.Basis(8, 0, inputs.ring(8)) as b:
        need = ftlm.ftlm_lanczos_workspace_bytes(b.handle, 2, 10, torch.float64)
        work = torch.empty(need - 256, dtype=torch.uint8, device=cuda_dev)
        out = [torch.empty((2, 10), dtype=torch.float64, device=cuda_dev) for _ in range(2)]
        me = torch.empty(2, dtype=torch.int32, device=cuda_dev)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_lanczos(b.handle, 2, 10, 1, 0, torch.float64, work, out[0], out[1], me)
        assert e.value.status == ftlm.FTLM_ENOMEM


@pytest.mark.parametrize("N,bonds,mode,R,M", [
    (16, inputs.ring(16), ftlm.RANK_AUTO, 2, 30),
    # CR H.v launches take their 32-row tiles from a counter (2.7 M rows: far more
    # tiles than warps, so which warp takes which tile varies from run to run);
    # the per-tile alpha sums keep the coefficients bit-identical
    (24, inputs.square_j1j2(), ftlm.RANK_CR, 9, 12),
    (24, inputs.square_j1j2(), ftlm.RANK_CR, 1, 12),
])
def test_repeated_runs_are_bit_identical(cuda_dev, N, bonds, mode, R, M):
    with ftlm.Basis(N, 0, bonds, mode) as b:
        runs = [ftlm.lanczos(b, R, M, seed=4, dtype=torch.float32, keep_coeffs=True) for _ in range(3)]
        torch.cuda.synchronize()
        for r in runs[1:]:
            for k in ("alpha", "beta", "theta", "weight", "m_eff"):
                assert torch.equal(runs[0][k], r[k]), k


def random_tridiagonals(n, M, seed):
    rng = np.random.default_rng(seed)
    m = rng.integers(1, M + 1, size=n)
    m[0], m[1] = M, 1
    a = rng.normal(size=(n, M))
    b = np.abs(rng.normal(size=(n, M))) + 0.1
    return a, b, m.astype(np.int32)


@pytest.mark.parametrize("M", [1, 2, 7, 100, 300])
def test_ritz_matches_dense_eigh(cuda_dev, M):
    n = 16
    a, b, m = random_tridiagonals(n, M, M)
    th = torch.empty((n, M), dtype=torch.float64, device=cuda_dev)
    w = torch.empty_like(th)
    ftlm.ftlm_ritz(n, M, torch.as_tensor(a, device=cuda_dev), torch.as_tensor(b, device=cuda_dev),
                   torch.as_tensor(m, device=cuda_dev), th, w)
    th, w = th.cpu().numpy(), w.cpu().numpy()
    for c in range(n):
        k = m[c]
        T = np.diag(a[c, :k]) + np.diag(b[c, :k - 1], 1) + np.diag(b[c, :k - 1], -1)
        ev, S = np.linalg.eigh(T)
        np.testing.assert_allclose(th[c, :k], ev, atol=1e-12 * max(1, np.abs(ev).max()))
        # weights through smooth spectral functions (insensitive to near-degenerate splits)
        for beta in (0.3, 1.0):
            np.testing.assert_allclose((w[c, :k] * np.exp(-beta * th[c, :k])).sum(),
                                       (S[0] ** 2 * np.exp(-beta * ev)).sum(), rtol=1e-11)
        assert abs(w[c, :k].sum() - 1) < 1e-12
        assert np.all(th[c, k:] == 0) and np.all(w[c, k:] == 0)


def test_ritz_reports_non_convergence(cuda_dev):
    """A sweep limit far below what implicit QR needs leaves every chain with m > 1
    unconverged: its theta and weight rows are NaN, ftlm_ritz_status counts it and
    returns FTLM_ENOCONV; with the default limit the same input converges."""
    n, M = 6, 40
    a, b, _ = random_tridiagonals(n, M, M)
    m = np.array([1, 40, 40, 30, 20, 10], dtype=np.int32)  # a 1 x 1 problem needs no sweep
    args = [torch.as_tensor(v, device=cuda_dev) for v in (a, b, m)]
    th = torch.empty((n, M), dtype=torch.float64, device=cuda_dev)
    w = torch.empty_like(th)
    ftlm.ftlm_ritz_status()  # start from a clear count
    try:
        ftlm.ftlm_ritz_set_max_sweeps(1)
        ftlm.ftlm_ritz(n, M, *args, th, w)
        with pytest.raises(ftlm.FtlmError) as e:
            ftlm.ftlm_ritz_status()
        assert e.value.status == ftlm.FTLM_ENOCONV and e.value.unconverged == n - 1
    finally:
        ftlm.ftlm_ritz_set_max_sweeps(0)
    th_h, w_h = th.cpu().numpy(), w.cpu().numpy()
    assert np.isfinite(th_h[0, 0]) and th_h[0, 0] == a[0, 0] and w_h[0, 0] == 1.0
    for c in range(1, n):
        assert np.all(np.isnan(th_h[c, :m[c]])) and np.all(np.isnan(w_h[c, :m[c]]))
        assert np.all(th_h[c, m[c]:] == 0)
    ftlm.ftlm_ritz(n, M, *args, th, w)
    assert ftlm.ftlm_ritz_status() == 0
    assert np.all(np.isfinite(th.cpu().numpy()))


@pytest.mark.parametrize("R", [1, 8])
def test_fp32_dot_products_accumulate_to_fp64_accuracy(cuda_dev, R):
    # FP32 vectors, FP64-class reductions: with dyadic start entries and J = 1 the
    # FP32 H.v is exact, so alpha_1 = sum_t q_t y_t can be rebuilt on the host from
    # the same FP32 roundings (q = fl(x / s), y = fl((Hx) / s)) and summed in FP64.
    # A plain FP32 accumulation over 184756 rows would miss it by ~1e-6 relative.
    N, K = 20, 10
    bonds = inputs.ring(N)
    b_or = o.basis(N, K)
    D = len(b_or)
    xs = np.stack([inputs.hashed_value(np.arange(D) + 7919 * r) for r in range(R)])
    with ftlm.Basis(N, 0, bonds) as b:
        res = ftlm.lanczos(b, R, 1, dtype=torch.float32, start=torch.as_tensor(xs, device=cuda_dev),
                           keep_coeffs=True)
        torch.cuda.synchronize()
    for r in range(R):
        x = xs[r]
        hx = o.hv(bonds, b_or, x)  # exact: dyadic entries, J = 1
        s = np.sqrt(np.sum(x * x))
        inv_s = np.float32(1.0 / s)
        q = (x.astype(np.float32) * inv_s).astype(np.float64)
        y = (hx.astype(np.float32) * inv_s).astype(np.float64)
        ref = float(np.sum(q * y))
        got = float(res["alpha"][r, 0])
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)


@pytest.mark.parametrize("two_s", [1, 2])
def test_no_bonds_gives_zero_hamiltonian(cuda_dev, two_s):
    # H = 0: H.v is zero, every chain breaks down after one step with theta = 0
    empty = (np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    N = 8
    with ftlm.Basis(N, 0, empty, two_s=two_s) as b:
        assert b.updates == b.dim
        x = torch.ones(b.dim, dtype=torch.float64, device=cuda_dev)
        y = torch.empty_like(x)
        ftlm.ftlm_hv(b.handle, x, y)
        assert torch.count_nonzero(y).item() == 0
        res = ftlm.lanczos(b, 4, 10, dtype=torch.float32)
        torch.cuda.synchronize()
        assert res["m_eff"].tolist() == [1] * 4
        assert torch.all(res["theta"] == 0).item()
        assert torch.all(res["weight"][:, 0] == 1).item()
