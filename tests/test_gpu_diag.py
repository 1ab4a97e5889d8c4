"""FP32 diagnostics on the GPU (ftlm_ghosts, ftlm_sigma_emp, ftlm_partition)
against the oracle's definitions (oracle/diagnostics.py, oracle.thermo)."""
import numpy as np
import pytest
import torch

import oracle as o
from oracle import diagnostics as dg
from paper_2605_26261_gb300 import ftlm, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_ghosts_match_oracle_on_lanczos_data(cuda_dev, dtype):
    # spin-1 icosahedron, S^z = 0 (D = 73 789): 4 chains of 100 steps (Fig. 4's
    # setting), the device test on the chains' own alpha, beta, theta, w
    R, M = 4, 100
    with ftlm.Basis(12, 0, inputs.icosahedron(), two_s=2) as b:
        res = ftlm.lanczos(b, R, M, seed=3, dist=ftlm.GAUSS, dtype=dtype, keep_coeffs=True)
        for c_tau in (1.0, 10.0):
            g = ftlm.ghosts(res, c_tau=c_tau)
            torch.cuda.synchronize()
            for r in range(R):
                m = int(res["m_eff"][r])
                a = res["alpha"][r, :m].cpu().numpy()
                bt = res["beta"][r, :m - 1].cpu().numpy()
                ref = dg.ghosts(a, bt, c_tau=c_tau, u=2.0**-24)
                W = ref["theta"][-1] - ref["theta"][0]
                np.testing.assert_allclose(g["ell"][r, :m].cpu().numpy(), ref["ell"], rtol=0, atol=1e-11 * W)
                far = np.abs(ref["ell"] - ref["tau"]) > 1e-6 * ref["tau"]  # decisions away from the threshold
                flags = g["flags"][r, :m].cpu().numpy().astype(bool)
                assert np.array_equal(flags[far], ref["flags"][far])
                assert int(g["count"][r]) == int(flags.sum())
                assert np.array_equal(g["cluster"][r, :m].cpu().numpy(), ref["cluster"])
                np.testing.assert_allclose(g["cweight"][r, :m].cpu().numpy(), ref["cweight"], rtol=1e-9, atol=1e-13)
                assert np.all(g["cluster"][r, m:].cpu().numpy() == -1)


def test_sigma_emp_kernel(cuda_dev):
    obs = np.random.default_rng(2).normal(size=(7, 33))
    mean = torch.empty(33, dtype=torch.float64, device=cuda_dev)
    sig = torch.empty_like(mean)
    ftlm.ftlm_sigma_emp(torch.as_tensor(obs, device=cuda_dev), mean, sig)
    m_ref, s_ref = dg.sigma_emp(obs)
    np.testing.assert_allclose(mean.cpu().numpy(), m_ref, rtol=1e-14)
    np.testing.assert_allclose(sig.cpu().numpy(), s_ref, rtol=1e-12)


def test_partition_matches_oracle(cuda_dev):
    N, R, M = 10, 3, 20
    bonds = inputs.random_graph(N, seed=8)
    T = inputs.log_t_grid(25, 0.05, 10.0)
    Td = torch.as_tensor(T, device=cuda_dev)
    secs = []
    for tz in ftlm.computed_two_sz(N):
        with ftlm.Basis(N, tz, bonds) as b:
            secs.append((tz, b.dim, ftlm.lanczos(b, R, M, seed=4, dist=ftlm.GAUSS, dtype=torch.float64)))
    for h in (0.0, 0.4):
        Z = torch.empty_like(Td)
        E0 = torch.empty_like(Td)
        ftlm.ftlm_partition([s[0] for s in secs], [s[1] for s in secs], R, M, [s[2]["theta"] for s in secs],
                            [s[2]["weight"] for s in secs], [s[2]["m_eff"] for s in secs], True, h, Td, Z, E0)
        ref = o.thermo(o.run_ftlm(N, bonds, R, M, seed=4), T, h=h)
        np.testing.assert_allclose(Z.cpu().numpy(), ref["Z_shifted"], rtol=1e-9)
        np.testing.assert_allclose(E0.cpu().numpy(), ref["E0"], rtol=1e-10)
        # Z_eff(T -> infinity) = sum of all sector dimensions = 2^N
    Zhot = torch.empty(1, dtype=torch.float64, device=cuda_dev)
    ftlm.ftlm_partition([s[0] for s in secs], [s[1] for s in secs], R, M, [s[2]["theta"] for s in secs],
                        [s[2]["weight"] for s in secs], [s[2]["m_eff"] for s in secs], True, 0.0,
                        torch.tensor([1e12], dtype=torch.float64, device=cuda_dev), Zhot)
    assert Zhot.item() == pytest.approx(2.0**N, rel=1e-9)
