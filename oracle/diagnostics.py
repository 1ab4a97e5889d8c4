"""FP32 diagnostics of the oracle (TEST INFRASTRUCTURE ONLY; see oracle/__init__.py).

Written from Sec. 3.1-3.2 of the paper:
  ghosts()     Cullum-Willoughby test, Eq. 25: eigenvalues theta_k of the Lanczos
               matrix T and theta^(1)_j of T without its first row and column
               (numpy eigh / eigvalsh on the dense matrices), l_k = min_j
               |theta_k - theta^(1)_j|, ghost when l_k < tau = C_tau u W_T with
               W_T = theta_max - theta_min; clusters join ascending Ritz values
               closer than tau (transitively), with their total weight.
  sigma_emp()  Eq. 22 with the printed 1/N_s.
"""
import numpy as np


def tridiag(alpha, beta):
    m = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    if m > 1:
        off = np.asarray(beta[: m - 1], dtype=np.float64)
        T += np.diag(off, 1) + np.diag(off, -1)
    return T


def ghosts(alpha, beta, c_tau=1.0, u=2.0**-24):
    """Returns dict theta, weight, theta1, ell, flags, cluster, cweight, count, tau."""
    T = tridiag(alpha, beta)
    m = T.shape[0]
    theta, S = np.linalg.eigh(T)
    weight = S[0, :] ** 2
    theta1 = np.linalg.eigvalsh(T[1:, 1:]) if m > 1 else np.zeros(0)
    tau = c_tau * u * (theta[-1] - theta[0]) if m > 0 else 0.0
    ell = np.array([np.min(np.abs(t - theta1)) if m > 1 else np.inf for t in theta])
    flags = ell < tau
    cluster = np.zeros(m, dtype=np.int64)
    cweight = np.zeros(m)
    start = 0
    for k in range(1, m + 1):
        if k == m or theta[k] - theta[k - 1] > tau:
            cluster[start:k] = start
            cweight[start:k] = weight[start:k].sum()
            start = k
    return {"theta": theta, "weight": weight, "theta1": theta1, "ell": ell, "flags": flags,
            "cluster": cluster, "cweight": cweight, "count": int(flags.sum()), "tau": tau}


def sigma_emp(obs):
    """Eq. 22: obs has one row per seed; returns (mean, sigma) over the rows."""
    obs = np.asarray(obs, dtype=np.float64)
    mean = obs.mean(axis=0)
    return mean, np.sqrt(np.sum((obs - mean) ** 2, axis=0) / obs.shape[0])

