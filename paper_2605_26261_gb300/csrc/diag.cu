// FP32 diagnostics of Sec. 3.1-3.2: Cullum-Willoughby ghost flags with cluster
// weights (Eq. 25), and the empirical standard deviation over seeds (Eq. 22).
//
// Ghosts.  For each chain, T is its m x m Lanczos matrix (theta_k, w_k from the
// Ritz step) and T^(1) the matrix with the first row and column removed.  Its
// eigenvalues theta^(1)_j come from the same implicit QR as the Ritz step; with
// both spectra ascending, l_k = min_j |theta_k - theta^(1)_j| (Eq. 25) is found by
// one merge.  theta_k is a ghost when l_k < tau = C_tau u W_T, W_T = theta_max -
// theta_min.  Clusters: consecutive ascending theta closer than tau (|theta_k -
// theta_l| <= tau, closed transitively) share one cluster, whose total weight is
// reported for every member.  One thread per chain, many chains per CTA.
#include <cmath>

#include "ftlm_internal.cuh"
#include "tridiag.cuh"

namespace ftlm {

namespace {

// T^(1) problems that did not converge (read and cleared by ftlm_ritz_status).
__device__ unsigned long long g_ghost_unconverged;

__global__ void ghost_kernel(int n, int M, const double *__restrict__ alpha, const double *__restrict__ beta,
                             const int *__restrict__ mv, const double *__restrict__ theta,
                             const double *__restrict__ weight, double c_tau, double u, double *ell, int *cluster,
                             double *cweight, int *flags, int *count, int max_sweeps)
{
    extern __shared__ double sh[];
    const int T = blockDim.x, i = threadIdx.x;
    const int c = blockIdx.x * T + i;
    if (c >= n) return;
    Strided d{sh + i, T}, e{sh + (size_t)M * T + i, T}, z{sh + (size_t)2 * M * T + i, T};
    int m = mv[c];
    m = m < 0 ? 0 : (m > M ? M : m);
    const double *th = theta + (size_t)c * M, *w = weight + (size_t)c * M;
    const size_t o = (size_t)c * M;
    // T^(1): diagonal alpha_2 .. alpha_m, off-diagonal beta_2 .. beta_{m-1}
    const int m1 = m - 1;
    for (int k = 0; k < m1; ++k) {
        d[k] = alpha[o + 1 + k];
        e[k] = k + 1 < m1 ? beta[o + 1 + k] : 0.0;
        z[k] = 0.0;
    }
    bool ok = true;
    if (m1 > 1) {
        ok = tridiag_qr(d, e, z, m1, max_sweeps);
        if (ok) sort_ascending(d, z, m1);
        else atomicAdd(&g_ghost_unconverged, 1ull);
    }
    const double tau = m > 0 ? c_tau * u * (th[m - 1] - th[0]) : 0.0;
    int ghosts = 0, j = 0, start = 0;
    double acc = 0.0;
    for (int k = 0; k <= m; ++k) {
        if (k < m) {
            double l = INFINITY;
            if (m1 > 0) {  // nearest theta^(1): advance while the next one is not farther
                while (j + 1 < m1 && fabs(d[j + 1] - th[k]) <= fabs(d[j] - th[k])) ++j;
                l = fabs(d[j] - th[k]);
            }
            if (!ok) l = NAN;  // no spectrum of T^(1): no ghost test
            const bool ghost = l < tau;
            ghosts += ghost;
            ell[o + k] = l;
            flags[o + k] = ghost ? 1 : 0;
        }
        // close the running cluster at the end or at a gap above tau
        if (k == m || (k > 0 && th[k] - th[k - 1] > tau)) {
            for (int q = start; q < k; ++q) {
                cluster[o + q] = start;
                cweight[o + q] = acc;
            }
            start = k;
            acc = 0.0;
        }
        if (k < m) acc += w[k];
    }
    for (int k = m; k < M; ++k) {
        ell[o + k] = 0.0;
        flags[o + k] = 0;
        cluster[o + k] = -1;
        cweight[o + k] = 0.0;
    }
    count[c] = ghosts;
}

// Eq. 22 over the N_s rows of obs (N_s x nT): mean and sigma with 1/N_s.
__global__ void sigma_kernel(int ns, int nT, const double *__restrict__ obs, double *mean, double *sigma)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < ns; ++k) s += obs[(size_t)k * nT + t];
        const double mu = s / ns;
        double v = 0.0;
        for (int k = 0; k < ns; ++k) {
            const double dv = obs[(size_t)k * nT + t] - mu;
            v += dv * dv;
        }
        if (mean) mean[t] = mu;
        sigma[t] = sqrt(v / ns);
    }
}

}  // namespace

ftlm_status ghost_unconverged_take(cudaStream_t stream, uint64_t *count)
{
    unsigned long long v = 0, zero = 0;
    FTLM_CUDA(cudaMemcpyFromSymbolAsync(&v, g_ghost_unconverged, sizeof(v), 0, cudaMemcpyDeviceToHost, stream));
    FTLM_CUDA(cudaMemcpyToSymbolAsync(g_ghost_unconverged, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));
    *count = v;
    return FTLM_OK;
}

}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_ghosts(int n, int M, const double *alpha_dev, const double *beta_dev, const int *m_dev,
                                   const double *theta_dev, const double *weight_dev, double c_tau, double u,
                                   double *ell_dev, int *cluster_dev, double *cweight_dev, int *flags_dev,
                                   int *count_dev, void *stream)
{
    if (n < 0 || M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "n or M out of range");
    if (!(c_tau >= 0.0) || !(u >= 0.0)) return fail(FTLM_EINVAL, "c_tau and u must be >= 0");
    if (n == 0) return FTLM_OK;
    if (!alpha_dev || !beta_dev || !m_dev || !theta_dev || !weight_dev || !ell_dev || !cluster_dev || !cweight_dev ||
        !flags_dev || !count_dev)
        return fail(FTLM_EINVAL, "NULL device pointer");
    constexpr size_t kSmemMax = 96 * 1024;
    int occ = 1;
    FTLM_CUDA(kernel_occupancy((const void *)ghost_kernel, 32, kSmemMax, true, &occ));
    const size_t per_chain = 3 * (size_t)M * sizeof(double);
    int T = (int)(kSmemMax / per_chain);
    T = T < 1 ? 1 : (T > 32 ? 32 : T);
    if (T > n) T = n;
    ghost_kernel<<<(n + T - 1) / T, T, per_chain * T, (cudaStream_t)stream>>>(
        n, M, alpha_dev, beta_dev, m_dev, theta_dev, weight_dev, c_tau, u, ell_dev, cluster_dev, cweight_dev,
        flags_dev, count_dev, ritz_max_sweeps());
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_sigma_emp(int ns, int nT, const double *obs_dev, double *mean_dev, double *sigma_dev,
                                      void *stream)
{
    if (ns < 1 || nT < 0) return fail(FTLM_EINVAL, "ns < 1 or nT < 0");
    if (nT == 0) return FTLM_OK;
    if (!obs_dev || !sigma_dev) return fail(FTLM_EINVAL, "NULL device pointer");
    sigma_kernel<<<(nT + 127) / 128, 128, 0, (cudaStream_t)stream>>>(ns, nT, obs_dev, mean_dev, sigma_dev);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}
